"""Naive FP64 renderer used only to pin the oracle (no sort, no tiles lists).

Written independently of ``oracle/``: numpy matrices for the projection, SciPy's
spherical harmonics for colour (real basis built from the complex one), and
for every pixel a repeated O(N^2) selection of the nearest remaining candidate
(depth, then index).  All decisions are taken in FP64.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import sph_harm_y


def real_sh_basis(dirs: np.ndarray, deg: int) -> np.ndarray:
    """Real SH basis (n, (deg+1)^2) in the 3DGS ordering and signs, built from
    SciPy's complex harmonics: for m > 0 sqrt(2) (-1)^m Re Y_l^m, for m < 0
    sqrt(2) (-1)^m Im Y_l^|m|, m = 0 the real Y_l^0; each band ordered
    m = -l..l, and the functions of odd m negated (the colour model's signs)."""
    x, y, z = dirs[:, 0], dirs[:, 1], dirs[:, 2]
    theta = np.arccos(np.clip(z, -1.0, 1.0))
    phi = np.arctan2(y, x)
    cols = []
    for l in range(deg + 1):
        for m in range(-l, l + 1):
            Y = sph_harm_y(l, abs(m), theta, phi)
            if m > 0:
                v = math.sqrt(2.0) * (-1) ** m * Y.real
            elif m < 0:
                v = math.sqrt(2.0) * (-1) ** m * Y.imag
            else:
                v = Y.real
            cols.append(v * (-1) ** (m % 2))
    return np.stack(cols, axis=1)


def _project(scene, view):
    """FP64 distances, Eq. 2 opacity and mask, projection, conic and 3-sigma
    tile rectangles of every Gaussian; ``keep`` marks the ones rendered."""
    n = scene.means.shape[0]
    vm = np.asarray(view.viewmat, np.float32).astype(np.float64).reshape(3, 4)
    R, t0 = vm[:, :3], vm[:, 3]
    c = np.asarray(view.campos, np.float32).astype(np.float64)
    W, H = view.width, view.height
    fx, fy, cx, cy = (float(np.float32(a)) for a in (view.fx, view.fy, view.cx, view.cy))
    mu = scene.means.astype(np.float64)
    t = mu @ R.T + t0
    d = np.linalg.norm(mu - c, axis=1)
    with np.errstate(divide="ignore", invalid="ignore"):
        u = fx * t[:, 0] / t[:, 2] + cx
        v = fy * t[:, 1] / t[:, 2] + cy
    near = float(np.float32(view.near))
    inview = (t[:, 2] > near) & (u >= 0) & (u <= W) & (v >= 0) & (v <= H)
    dmax = d[inview].max() if inview.any() else 0.0
    s = float(np.float32(view.s_v))
    if view.flags & 1:
        a2 = scene.opacity.astype(np.float64)
        keep = np.ones(n, bool)
    else:
        dn = d / dmax if dmax > 0 else np.zeros(n)
        sig = np.maximum(scene.decay.astype(np.float64), 0.0)
        a2 = scene.opacity * np.exp(-(dn * s) ** 2 / (2 * sig ** 2 + float(np.float32(view.eps))))
        keep = a2 > float(np.float32(view.tau)) * s
    keep &= t[:, 2] > near

    q = scene.quats.astype(np.float64)
    q = q / np.linalg.norm(q, axis=1, keepdims=True)
    w_, x_, y_, z_ = q.T
    Rq = np.stack([
        np.stack([1 - 2 * (y_ ** 2 + z_ ** 2), 2 * (x_ * y_ - w_ * z_), 2 * (x_ * z_ + w_ * y_)], -1),
        np.stack([2 * (x_ * y_ + w_ * z_), 1 - 2 * (x_ ** 2 + z_ ** 2), 2 * (y_ * z_ - w_ * x_)], -1),
        np.stack([2 * (x_ * z_ - w_ * y_), 2 * (y_ * z_ + w_ * x_), 1 - 2 * (x_ ** 2 + y_ ** 2)], -1)], 1)
    S = np.einsum("nij,nj,nkj->nik", Rq, scene.scales.astype(np.float64) ** 2, Rq)
    limx, limy = 1.3 * 0.5 * W / fx, 1.3 * 0.5 * H / fy
    tz = t[:, 2]
    txc = np.clip(t[:, 0] / tz, -limx, limx) * tz
    tyc = np.clip(t[:, 1] / tz, -limy, limy) * tz
    J = np.zeros((n, 2, 3))
    J[:, 0, 0] = fx / tz
    J[:, 0, 2] = -fx * txc / tz ** 2
    J[:, 1, 1] = fy / tz
    J[:, 1, 2] = -fy * tyc / tz ** 2
    T = J @ R
    cov = T @ S @ np.transpose(T, (0, 2, 1)) + 0.3 * np.eye(2)
    det = cov[:, 0, 0] * cov[:, 1, 1] - cov[:, 0, 1] ** 2
    keep &= det > 0
    inv = np.linalg.inv(cov[keep]) if keep.any() else np.zeros((0, 2, 2))
    conic = np.zeros((n, 2, 2))
    conic[keep] = inv
    mid = 0.5 * (cov[:, 0, 0] + cov[:, 1, 1])
    lam = mid + np.sqrt(np.maximum(0.1, mid ** 2 - det))
    rad = np.ceil(3.0 * np.sqrt(np.maximum(lam, 0)))
    TX, TY = (W + 15) // 16, (H + 15) // 16
    x0 = np.floor((u - rad) / 16)
    x1 = np.floor((u + rad) / 16)
    y0 = np.floor((v - rad) / 16)
    y1 = np.floor((v + rad) / 16)
    keep &= ~((x1 < 0) | (x0 > TX - 1) | (y1 < 0) | (y0 > TY - 1))
    return dict(keep=keep, u=u, v=v, tz=tz, conic=conic, a2=a2, x0=x0, x1=x1, y0=y0, y1=y1, mu=mu, c=c, d=d)


def tile_lists_brute(scene, view):
    """Per tile (row-major over the view's tile grid), the rendered Gaussians
    whose 3-sigma rectangle covers the tile, nearest first (camera depth,
    then index): each tile checked against every Gaussian."""
    P = _project(scene, view)
    TX, TY = (view.width + 15) // 16, (view.height + 15) // 16
    ids = np.nonzero(P["keep"])[0]
    out = []
    for ty_ in range(TY):
        for tx_ in range(TX):
            cand = [i for i in ids if P["x0"][i] <= tx_ <= P["x1"][i] and P["y0"][i] <= ty_ <= P["y1"][i]]
            out.append(sorted(cand, key=lambda i: (P["tz"][i], i)))
    return out, P


def render_brute(scene, view, sh_signs=None):
    """FP64 image (3, H, W), transmittance and contributor counts."""
    deg = int(round(math.sqrt(scene.sh.shape[1]))) - 1
    W, H = view.width, view.height
    P = _project(scene, view)
    keep, u, v, tz, conic, a2 = (P[k] for k in ("keep", "u", "v", "tz", "conic", "a2"))
    x0, x1, y0, y1, mu, c, d = (P[k] for k in ("x0", "x1", "y0", "y1", "mu", "c", "d"))
    dirs = (mu - c) / d[:, None]
    B = real_sh_basis(dirs, deg)
    rgb = np.maximum(np.einsum("nk,nkc->nc", B, scene.sh.astype(np.float64)) + 0.5, 0.0)

    img = np.zeros((3, H, W))
    Tf = np.ones((H, W))
    nc = np.zeros((H, W), np.int64)
    ids = np.nonzero(keep)[0]
    bg = np.asarray(view.bg, np.float32).astype(np.float64)
    for py in range(H):
        for px in range(W):
            tx_, ty_ = px // 16, py // 16
            cand = [i for i in ids if x0[i] <= tx_ <= x1[i] and y0[i] <= ty_ <= y1[i]]
            Tt = 1.0
            col = np.zeros(3)
            last = 0
            pos = 0
            remaining = list(cand)
            while remaining:
                best = min(remaining, key=lambda i: (tz[i], i))
                remaining.remove(best)
                pos += 1
                dx, dy = u[best] - (px + 0.5), v[best] - (py + 0.5)
                A, Bc, C = conic[best, 0, 0], conic[best, 0, 1], conic[best, 1, 1]
                power = -0.5 * (A * dx * dx + C * dy * dy) - Bc * dx * dy
                if power > 0:
                    continue
                al = min(0.99, a2[best] * math.exp(power))
                if al < 1.0 / 255.0:
                    continue
                tt = Tt * (1 - al)
                if tt < 1e-4:
                    break
                col += rgb[best] * al * Tt
                Tt = tt
                last = pos
            img[:, py, px] = col + Tt * bg
            Tf[py, px] = Tt
            nc[py, px] = last
    return img, Tf, nc
