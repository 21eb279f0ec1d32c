"""FP64 reference gradients for the CLoD-GS rasterizer (plain PyTorch CPU ops).

TEST INFRASTRUCTURE ONLY (see ``clod_oracle.c``).  This is a second, vectorised
FP64 statement of the forward function -- attenuated opacity (Sec. 3.2, Eq. 2),
EWA projection and SH colour (Sec. 3.1), and front-to-back blending (Eq. 1) --
written with differentiable torch ops, so that reverse-mode autograd gives the
exact gradient of the FP64 image.  The discrete decisions are frozen and taken
from the C oracle's FP32 decision arithmetic:

* the view-frustum argmax j* of the distance (so d_max = d_{j*}); the gradient
  of d_max reaches only mu_{j*} (ties go to the lowest index);
* the survivor set (mask, near plane, det > 0, non-empty tile rectangle);
* the ordered list of (pixel, Gaussian) pairs that contributed to each pixel
  (the alpha skip, the transmittance stop and the depth order).

Everything else (the 0.99 opacity clamp, ReLU of sigma_d, the clamp of the
projected direction to 1.3 x the half field of view, the colour clamp at 0) is
part of the differentiated function.
"""
from __future__ import annotations

from typing import Dict, Optional, Sequence

import numpy as np
import torch

from . import oracle as O

F64 = torch.float64


def _basis(x, y, z, deg):
    b = [torch.full_like(x, 0.28209479177387814)]
    if deg >= 1:
        c1 = 0.4886025119029199
        b += [-c1 * y, c1 * z, -c1 * x]
    if deg >= 2:
        xx, yy, zz = x * x, y * y, z * z
        b += [1.0925484305920792 * x * y, -1.0925484305920792 * y * z,
              0.31539156525252005 * (2.0 * zz - xx - yy), -1.0925484305920792 * x * z,
              0.5462742152960396 * (xx - yy)]
    if deg >= 3:
        b += [-0.5900435899266435 * y * (3.0 * xx - yy), 2.890611442640554 * x * y * z,
              -0.4570457994644658 * y * (4.0 * zz - xx - yy),
              0.3731763325901154 * z * (2.0 * zz - 3.0 * xx - 3.0 * yy),
              -0.4570457994644658 * x * (4.0 * zz - xx - yy), 1.445305721320277 * z * (xx - yy),
              -0.5900435899266435 * x * (xx - 3.0 * yy)]
    return torch.stack(b, dim=1)


def _rotation(q):
    q = q / torch.linalg.norm(q, dim=1, keepdim=True)
    w, x, y, z = q.unbind(1)
    R = torch.stack([
        1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y),
        2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
        2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], dim=1)
    return R.reshape(-1, 3, 3)


def view_forward(P: Dict[str, torch.Tensor], view, frozen) -> Dict[str, torch.Tensor]:
    """FP64 forward for one view.  ``P`` holds f64 tensors means (n,3),
    scales (n,3), quats (n,4), opacity (n,), sh (n,K,3), decay (n,).
    ``frozen``: dict with argmax (int), survive (n,) bool, contrib_pix,
    contrib_gid (blending order).  Returns image (3,H,W), alpha_eff (n,)."""
    means, scales, quats, opacity, sh, decay = (P[k] for k in ("means", "scales", "quats", "opacity", "sh", "decay"))
    n = means.shape[0]
    deg = int(round(np.sqrt(sh.shape[1]))) - 1
    vm = torch.tensor(np.asarray(view.viewmat, np.float32).reshape(3, 4), dtype=F64)
    Rv, tv = vm[:, :3], vm[:, 3]
    c = torch.tensor(np.asarray(view.campos, np.float32), dtype=F64)
    fx, fy, cx, cy = (float(np.float32(a)) for a in (view.fx, view.fy, view.cx, view.cy))
    W, H = view.width, view.height
    s = float(np.float32(view.s_v))
    eps = float(np.float32(view.eps))

    e = means - c
    d = torch.sqrt((e * e).sum(1))
    if view.flags & O.LOD_OFF:
        a2 = opacity
    else:
        j = int(frozen["argmax"])
        if view.flags & O.NO_NORMALIZE:
            dn = d
        elif j >= 0:
            dn = d / d[j]
        else:
            dn = torch.zeros_like(d)
        sr = torch.relu(decay)
        q = dn * s
        a2 = opacity * torch.exp(-(q * q) / (2.0 * sr * sr + eps))

    idx = torch.nonzero(torch.as_tensor(frozen["survive"]).bool()).flatten()
    mu = means[idx]
    t = mu @ Rv.T + tv
    tx, ty, tz = t.unbind(1)
    u = fx * (tx / tz) + cx
    v = fy * (ty / tz) + cy
    R = _rotation(quats[idx])
    M = R * scales[idx][:, None, :]
    Sig = M @ M.transpose(1, 2)
    limx = 1.3 * (0.5 * W / fx)
    limy = 1.3 * (0.5 * H / fy)
    txc = torch.clamp(tx / tz, -limx, limx) * tz
    tyc = torch.clamp(ty / tz, -limy, limy) * tz
    zero = torch.zeros_like(tz)
    J = torch.stack([fx / tz, zero, -fx * txc / (tz * tz), zero, fy / tz, -fy * tyc / (tz * tz)], 1).reshape(-1, 2, 3)
    T = J @ Rv
    cov = T @ Sig @ T.transpose(1, 2)
    a = cov[:, 0, 0] + 0.3
    b = cov[:, 0, 1]
    cc = cov[:, 1, 1] + 0.3
    det = a * cc - b * b
    A, B, C = cc / det, -b / det, a / det
    dirs = e[idx] / d[idx][:, None]
    basis = _basis(dirs[:, 0], dirs[:, 1], dirs[:, 2], deg)
    rgb = torch.clamp_min(torch.einsum("nk,nkc->nc", basis, sh[idx]) + 0.5, 0.0)

    # blend over the frozen contributor lists
    pos = torch.full((n,), -1, dtype=torch.long)
    pos[idx] = torch.arange(idx.numel())
    pix = torch.as_tensor(np.asarray(frozen["contrib_pix"], np.int64))
    gid = torch.as_tensor(np.asarray(frozen["contrib_gid"], np.int64))
    r = pos[gid]
    assert bool((r >= 0).all()), "contributor that is not a survivor"
    px = (pix % W).to(F64) + 0.5
    py = (pix // W).to(F64) + 0.5
    dx = u[r] - px
    dy = v[r] - py
    power = -0.5 * (A[r] * dx * dx + C[r] * dy * dy) - B[r] * dx * dy
    alpha = torch.clamp_max(a2[gid] * torch.exp(power), 0.99)
    lg = torch.log1p(-alpha)
    m = pix.numel()
    if m:
        start = torch.ones(m, dtype=torch.bool)
        start[1:] = pix[1:] != pix[:-1]
        seg = torch.cumsum(start.long(), 0) - 1
        excl = torch.cumsum(lg, 0) - lg
        seg_first = torch.nonzero(start).flatten()
        Tk = torch.exp(excl - excl[seg_first][seg])
        w = alpha * Tk
        img = torch.zeros(3, H * W, dtype=F64)
        img = img.index_add(1, pix, (rgb[r] * w[:, None]).T)
        logT = torch.zeros(H * W, dtype=F64).index_add(0, pix, lg)
    else:
        img = torch.zeros(3, H * W, dtype=F64)
        logT = torch.zeros(H * W, dtype=F64)
    Tf = torch.exp(logT)
    bg = torch.tensor(np.asarray(view.bg, np.float32), dtype=F64)
    img = img + Tf[None, :] * bg[:, None]
    return dict(image=img.reshape(3, H, W), T=Tf.reshape(H, W), alpha_eff=a2)


def params_f64(scene, requires_grad=True) -> Dict[str, torch.Tensor]:
    out = {}
    for k in ("means", "scales", "quats", "opacity", "sh", "decay"):
        out[k] = torch.tensor(np.asarray(getattr(scene, k), np.float32), dtype=F64, requires_grad=requires_grad)
    return out


def frozen_from_oracle(scene, view):
    s1 = O.stage1(scene, view)
    img = O.render(scene, view, s1, O.stage1_f64(scene, view, s1), contrib=True)
    return dict(argmax=int(s1["argmax"][0]), survive=s1["survive"].astype(bool),
                contrib_pix=img["contrib_pix"], contrib_gid=img["contrib_gid"]), s1, img


def reference_gradients(scene, views: Sequence, dL_dimage: Sequence[np.ndarray],
                        dL_dalpha: Optional[Sequence[Optional[np.ndarray]]] = None,
                        frozen: Optional[Sequence] = None):
    """Gradient of sum_v <image_v, dL_dimage_v> + <alpha''_v, dL_dalpha_v>
    with respect to the six activated parameter groups (FP64 numpy arrays)."""
    P = params_f64(scene)
    total = 0.0
    for vi, v in enumerate(views):
        fr = frozen[vi] if frozen is not None else frozen_from_oracle(scene, v)[0]
        out = view_forward(P, v, fr)
        total = total + (out["image"] * torch.as_tensor(np.asarray(dL_dimage[vi], np.float64))).sum()
        if dL_dalpha is not None and dL_dalpha[vi] is not None:
            total = total + (out["alpha_eff"] * torch.as_tensor(np.asarray(dL_dalpha[vi], np.float64))).sum()
    total.backward()
    return {k: (t.grad.numpy().copy() if t.grad is not None else np.zeros(tuple(t.shape)))
            for k, t in P.items()}


def frozen_on_tiles(scene, view, tiles, s1=None):
    """Frozen decisions of one view with the contributor lists of the listed
    tiles only (the other pixels get no contributors), and its Stage I."""
    s1 = O.stage1(scene, view) if s1 is None else s1
    img = O.render(scene, view, s1, None, tiles=tiles, contrib=True)
    return dict(argmax=int(s1["argmax"][0]), survive=s1["survive"].astype(bool),
                contrib_pix=img["contrib_pix"], contrib_gid=img["contrib_gid"]), s1


def reference_gradients_sparse(scene, views: Sequence, frozen: Sequence, dL_dimage: Sequence[np.ndarray],
                               dL_dalpha: Optional[Sequence[Optional[np.ndarray]]] = None):
    """reference_gradients for a loss whose image gradient is non-zero only
    on pixels that have contributors in ``frozen`` and whose alpha''
    gradient is non-zero only on a few Gaussians.  Every other Gaussian's
    gradient is exactly zero, so the same FP64 statement is evaluated on the
    sub-scene of the contributors, the Gaussians with an alpha'' gradient and
    each view's farthest in-view Gaussian (which carries d_max), and the
    result is scattered back into full-size arrays."""
    n = scene.n
    keep = np.zeros(n, bool)
    for vi, fr in enumerate(frozen):
        keep[np.asarray(fr["contrib_gid"], np.int64)] = True
        if fr["argmax"] >= 0:
            keep[fr["argmax"]] = True
        if dL_dalpha is not None and dL_dalpha[vi] is not None:
            keep[np.nonzero(np.asarray(dL_dalpha[vi]))[0]] = True
    idx = np.nonzero(keep)[0]
    new = np.full(n, -1, np.int64)
    new[idx] = np.arange(idx.size)
    sub = scene.subset(idx)
    fsub = [dict(argmax=int(new[fr["argmax"]]) if fr["argmax"] >= 0 else -1, survive=fr["survive"][idx],
                 contrib_pix=fr["contrib_pix"], contrib_gid=new[np.asarray(fr["contrib_gid"], np.int64)])
            for fr in frozen]
    da = None if dL_dalpha is None else [None if a is None else np.asarray(a)[idx] for a in dL_dalpha]
    r = reference_gradients(sub, views, dL_dimage, da, frozen=fsub)
    out = {}
    for k, g in r.items():
        full = np.zeros((n,) + g.shape[1:], np.float64)
        full[idx] = g
        out[k] = full
    return out
