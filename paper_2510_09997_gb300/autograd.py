"""torch.autograd binding of the rasterizer: forward through clod_preprocess /
clod_bin_sort / clod_render_fwd, backward through clod_render_bwd (both in
libclod's CUDA kernels; this module only marshals arguments)."""
from __future__ import annotations

import ctypes
from typing import Sequence

import torch

from . import abi
from . import clod as C


def _scene_struct(means, scales, quats, opacity, sh, decay) -> abi.clod_scene:
    n = int(means.shape[0])
    k = sh.shape[1]
    deg = int(round(k ** 0.5)) - 1
    return abi.clod_scene(n, deg, 0, means.data_ptr(), scales.data_ptr(), quats.data_ptr(), opacity.data_ptr(),
                          sh.data_ptr(), decay.data_ptr())


class _Scene:
    """Minimal stand-in for clod.DeviceScene over existing tensors."""

    def __init__(self, tensors):
        self.tensors = tensors
        self.c = _scene_struct(*tensors)
        self.n = int(tensors[0].shape[0])


class CLoDRender(torch.autograd.Function):
    """Inputs: activated means (n,3), scales (n,3), quats (n,4), opacity (n,),
    sh (n,K,3), decay (n,), plus the views.  Outputs: packed image, alpha''
    (V, n), mask M (V, n, not differentiable), counts (V, 2: sum M, rendered)."""

    @staticmethod
    def forward(ctx, means, scales, quats, opacity, sh, decay, views):
        ts = [t.detach().contiguous() for t in (means, scales, quats, opacity, sh, decay)]
        sc = _Scene(ts)
        fr = C.render(sc, views, want_keys=False)
        ctx.sc = sc
        ctx.fr = fr
        ctx.mark_non_differentiable(fr.mask, fr.counts)
        return fr.image, fr.alpha_eff, fr.mask, fr.counts

    @staticmethod
    def backward(ctx, g_img, g_alpha, g_mask, g_counts):
        sc, fr = ctx.sc, ctx.fr
        means, scales, quats, opacity, sh, decay = sc.tensors
        grads = [torch.zeros_like(t) for t in sc.tensors]
        V = len(fr.views)
        nb = ctypes.c_size_t()
        C.check("clod_backward_workspace_size", C.lib().clod_backward_workspace_size(sc.n, V, ctypes.byref(nb)))
        bws = torch.empty(max(int(nb.value), 1), dtype=torch.uint8, device="cuda")
        gi = (g_img if g_img is not None else torch.zeros_like(fr.image)).contiguous()
        ga = g_alpha.contiguous() if g_alpha is not None else None
        C.check("clod_render_bwd", C.lib().clod_render_bwd(
            ctypes.byref(sc.c), C._ptr(fr.ws), C._ptr(fr.vals), C._ptr(fr.ranges), C._ptr(fr.T_final),
            C._ptr(fr.n_contrib), C._ptr(gi), C._ptr(ga), None, C._ptr(bws), bws.numel(),
            *[C._ptr(g) for g in grads], C._stream(None)))
        return (*grads, None)


def render(means, scales, quats, opacity, sh, decay, views: Sequence):
    """Differentiable render of ``views``; returns (list of (3,H,W) images,
    alpha'' (V,n), mask (V,n), counts (V,2))."""
    img, alpha, mask, counts = CLoDRender.apply(means, scales, quats, opacity, sh, decay, list(views))
    out, b = [], 0
    for v in views:
        p = v.width * v.height
        out.append(img[3 * b: 3 * (b + p)].view(3, v.height, v.width))
        b += p
    return out, alpha, mask, counts


class L1Loss(torch.autograd.Function):
    """mean |image - target| by clod_l1_loss (value and gradient in one kernel)."""

    @staticmethod
    def forward(ctx, image, target):
        image = image.contiguous()
        target = target.contiguous()
        loss = torch.zeros(1, dtype=torch.float32, device=image.device)
        grad = torch.empty_like(image)
        C.check("clod_l1_loss", C.lib().clod_l1_loss(C._ptr(image), C._ptr(target), image.numel(), 1.0,
                                                     C._ptr(loss), C._ptr(grad), C._stream(None)))
        ctx.save_for_backward(grad)
        return loss[0]

    @staticmethod
    def backward(ctx, g):
        (grad,) = ctx.saved_tensors
        return grad * g, None


class RenderLoss(torch.autograd.Function):
    """(1 - w) L1 + w (1 - SSIM) by clod_render_loss (value and gradient)."""

    @staticmethod
    def forward(ctx, image, target, dssim_weight: float = 0.2):
        image = image.contiguous()
        target = target.contiguous()
        Cc, H, W = image.shape
        loss = torch.zeros(1, dtype=torch.float32, device=image.device)
        grad = torch.empty_like(image)
        nb = ctypes.c_size_t()
        C.check("clod_render_loss_workspace_size", C.lib().clod_render_loss_workspace_size(Cc, H, W, ctypes.byref(nb)))
        ws = torch.empty(int(nb.value), dtype=torch.uint8, device=image.device)
        C.check("clod_render_loss", C.lib().clod_render_loss(C._ptr(image), C._ptr(target), Cc, H, W,
                                                             float(dssim_weight), 1.0, C._ptr(ws), ws.numel(),
                                                             C._ptr(loss), C._ptr(grad), C._stream(None)))
        ctx.save_for_backward(grad)
        return loss[0]

    @staticmethod
    def backward(ctx, g):
        (grad,) = ctx.saved_tensors
        return grad * g, None, None

