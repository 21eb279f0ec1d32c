"""Virtual-distance-scaling training step of CLoD-GS (Sec. 3.3).

Per view a virtual scale s_v is drawn (log-uniform on [1, s_max] by default;
the paper's example is uniform on [1, 10]), the view is rendered with that
s_v, and the objective is

    L_total = w_s (L_render + lambda_reg L_reg)                     (Eq. 5)
    w_s     = (1 - 0.5 s_v / s_max)^2
    L_reg   = (s_v - 1)^2 ReLU(eta_actual - eta_target)^2           (Eq. 4)
    eta_target = s_v^-1.5                                            (Eq. 3)
    eta_actual = sum_i M_i / N_total

averaged over the step's views.  L_render = (1 - w) L1 + w D-SSIM (w = 0.2
as in the 3DGS training the paper builds on; w = 0 gives L1 alone).
eta_actual is a count of the binary mask; its gradient is taken straight
through, dM_i/dalpha''_i := 1, so every alpha'' of view v receives
2 w_v lambda (s_v - 1)^2 ReLU(eta_a - eta_t) / N, one scalar per view that the
rasterizer's backward carries on to alpha, sigma_d and the means.

Every step runs in libclod's kernels: the forward (clod_preprocess,
clod_bin_sort, clod_render_fwd), the loss and its image gradient
(clod_render_loss, written straight into the packed gradient), L_reg, the
total and the per-view straight-through scalars (clod_lreg_grad), the
backward (clod_render_bwd_set, which overwrites the gradients) and Adam
fused with the parameter activations (clod_adam_step: raw log-scales and
opacity logits, exp / sigmoid; keep_grads, as the next backward refills
them).  Python
only allocates the buffers once and passes pointers.  sigma_d has learning
rate 1e-2 and lambda_reg = 1 (Sec. 4.1).
"""
from __future__ import annotations

import ctypes
import math
from typing import List, Optional, Sequence

import numpy as np
import torch

from . import abi
from . import clod as C

LR_NAMES = ("means", "log_scales", "quats", "opacity_logit", "sh", "decay")


def eta_target(s_v: float) -> float:
    return s_v ** -1.5


class GaussianModel:
    """Raw parameters (what Adam updates) and the activated scales and
    opacities the rasterizer reads.  At construction the activated copies are
    the scene's values themselves; afterwards clod_adam_step rewrites them."""

    def __init__(self, scene, device="cuda"):
        t = lambda a: torch.tensor(np.ascontiguousarray(a, np.float32), device=device)
        self.means = t(scene.means)
        self.log_scales = t(np.log(np.asarray(scene.scales, np.float64)))
        self.quats = t(scene.quats)
        op = np.clip(np.asarray(scene.opacity, np.float64), 1e-6, 1 - 1e-6)
        self.opacity_logit = t(np.log(op / (1 - op)))
        self.sh = t(scene.sh)
        self.decay = t(scene.decay)
        self.scales = t(scene.scales)
        self.opacity = t(scene.opacity)
        self.sh_degree = int(round(self.sh.shape[1] ** 0.5)) - 1

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    def activated(self):
        return (self.means, self.scales, self.quats, self.opacity, self.sh, self.decay)

    def raw(self):
        return (self.means, self.log_scales, self.quats, self.opacity_logit, self.sh, self.decay)

    def scene(self) -> C.DeviceScene:
        return C.DeviceScene.from_tensors(*self.activated())


class TrainStep:
    """One optimisation step over a batch of views."""

    def __init__(self, model: GaussianModel, s_max: float = 16.0, lam_reg: float = 1.0, sampler: str = "log",
                 seed: int = 0, extent: float = 1.0, dssim_weight: float = 0.2, betas=(0.9, 0.999),
                 eps: float = 1e-15):
        self.model = model
        self.dssim = float(dssim_weight)
        self.s_max = float(s_max)
        self.lam = float(lam_reg)
        self.sampler = sampler
        self.rng = np.random.default_rng(seed)
        self.lr = [1.6e-4 * extent, 5e-3, 1e-3, 5e-2, 2.5e-3, 1e-2]
        self.betas = (float(betas[0]), float(betas[1]))
        self.eps = float(eps)
        self.t = 0
        dev = model.means.device
        ne = ctypes.c_int64()
        C.check("clod_adam_state_size", C.lib().clod_adam_state_size(model.n, model.sh_degree, ctypes.byref(ne)))
        self.m = torch.zeros(ne.value, dtype=torch.float32, device=dev)
        self.v = torch.zeros(ne.value, dtype=torch.float32, device=dev)
        self.grads = [torch.zeros_like(p) for p in model.activated()]
        self.total = torch.zeros(1, dtype=torch.float32, device=dev)
        self.lrender = torch.zeros(C.MAX_VIEWS, dtype=torch.float32, device=dev)
        self.lreg = torch.zeros(C.MAX_VIEWS, dtype=torch.float32, device=dev)
        self.dalpha = torch.zeros(C.MAX_VIEWS, dtype=torch.float32, device=dev)
        self._bws = None
        self._lws = None
        self.scene = model.scene()

    def sample_scale(self) -> float:
        if self.s_max <= 1.0:
            return 1.0
        if self.sampler == "uniform":
            s = self.rng.uniform(1.0, self.s_max)
        else:
            s = math.exp(self.rng.uniform(0.0, math.log(self.s_max)))
        return float(np.float32(s))

    def _workspace(self, attr, nbytes):
        buf = getattr(self, attr)
        if buf is None or buf.numel() < nbytes:
            buf = torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=self.model.means.device)
            setattr(self, attr, buf)
        return buf

    def forward_backward(self, views: Sequence, targets: Sequence[torch.Tensor], scales: Optional[List[float]] = None):
        """Forward, loss, L_reg, backward: the six activated-parameter
        gradients of this call overwrite self.grads.  Returns (frame, per-view
        info)."""
        if scales is None:
            scales = [self.sample_scale() for _ in views]
        views = [v.replace(s_v=s) for v, s in zip(views, scales)]
        V = len(views)
        L = C.lib()
        st = C._stream(None)
        fr = C.render(self.scene, views, want_keys=False)
        dimg = torch.empty_like(fr.image)
        s_arr = (ctypes.c_float * V)(*scales)
        w_arr = (ctypes.c_float * V)()
        C.check("clod_step_weights", L.clod_step_weights(s_arr, V, self.s_max, w_arr))
        weights = list(w_arr)
        self.lrender[:V].zero_()
        for k, v in enumerate(views):
            b = 3 * fr.pix_base[k]
            img = fr.image[b:b + 3 * v.width * v.height]
            ws = None
            nbytes = 0
            if self.dssim > 0:
                nb = ctypes.c_size_t()
                C.check("clod_render_loss_workspace_size",
                        L.clod_render_loss_workspace_size(3, v.height, v.width, ctypes.byref(nb)))
                ws = self._workspace("_lws", nb.value)
                nbytes = ws.numel()
            C.check("clod_render_loss", L.clod_render_loss(
                C._ptr(img), C._ptr(targets[k]), 3, v.height, v.width, self.dssim, weights[k],
                C._ptr(ws) if ws is not None else None, nbytes, C._ptr(self.lrender[k:]),
                C._ptr(dimg[b:]), st))
        C.check("clod_lreg_grad", L.clod_lreg_grad(C._ptr(fr.counts), self.model.n, V, s_arr, w_arr, self.lam,
                                                   C._ptr(self.lrender), C._ptr(self.dalpha), C._ptr(self.total),
                                                   C._ptr(self.lreg), st))
        nb = ctypes.c_size_t()
        C.check("clod_backward_workspace_size", L.clod_backward_workspace_size(self.model.n, V, ctypes.byref(nb)))
        bws = self._workspace("_bws", nb.value)
        C.check("clod_render_bwd_set", L.clod_render_bwd_set(
            ctypes.byref(self.scene.c), C._ptr(fr.ws), C._ptr(fr.vals), C._ptr(fr.ranges), C._ptr(fr.T_final),
            C._ptr(fr.n_contrib), C._ptr(dimg), None, C._ptr(self.dalpha), C._ptr(bws), bws.numel(),
            *[C._ptr(g) for g in self.grads], st))
        info = dict(views=views, n=self.model.n, scales=list(scales), w_s=[w * V for w in weights],
                    eta_target=[eta_target(s) for s in scales], counts=fr.counts, l_render=self.lrender[:V],
                    l_reg=self.lreg[:V])
        self.last = dict(frame=fr, dimage=dimg, **info)
        return fr, info

    def loss(self, views, targets, scales=None):
        """L_total (device scalar) and per-view diagnostics, without the update
        (this call's gradients are left in self.grads)."""
        fr, info = self.forward_backward(views, targets, scales)
        return self.total, info

    def step(self, views: Sequence, targets: Sequence[torch.Tensor], scales: Optional[List[float]] = None):
        """Forward + backward + Adam.  Returns (L_total as a device scalar
        tensor, per-view diagnostics as device tensors)."""
        fr, info = self.forward_backward(views, targets, scales)
        self.t += 1
        cfg = abi.clod_adam_cfg()
        for k in range(6):
            cfg.lr[k] = self.lr[k]
        cfg.beta1, cfg.beta2, cfg.eps, cfg.step = self.betas[0], self.betas[1], self.eps, self.t
        cfg.keep_grads = 1     # the next step's backward overwrites them
        P = ctypes.c_void_p * 6
        raw = P(*[C._ptr(p) for p in self.model.raw()])
        grads = P(*[C._ptr(g) for g in self.grads])
        C.check("clod_adam_step", C.lib().clod_adam_step(ctypes.byref(cfg), self.model.n, self.model.sh_degree, raw,
                                                         grads, C._ptr(self.model.scales),
                                                         C._ptr(self.model.opacity), C._ptr(self.m), C._ptr(self.v),
                                                         C._stream(None)))
        return self.total, info


def per_view_info(info) -> List[dict]:
    """Host copy of a step's diagnostics (synchronises)."""
    cnt = info["counts"].cpu().numpy()
    lr = info["l_render"].cpu().numpy()
    lg = info["l_reg"].cpu().numpy()
    out = []
    for k, s in enumerate(info["scales"]):
        out.append(dict(s_v=s, l_render=float(lr[k]), l_reg=float(lg[k]), eta_actual=float(cnt[k, 0]) / info["n"],
                        eta_target=info["eta_target"][k], w_s=info["w_s"][k], rendered=int(cnt[k, 1])))
    return out
