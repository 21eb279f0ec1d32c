"""Comparison of a rendered image with the oracle's FP64-decision outcomes.

The oracle's FP64-decision pass (``oracle.render_f64dec``) gives, per pixel,
the outcome of Eq. 1 with every decision taken in FP64 (the main path) and one
more outcome for every decision that lay within its band of a threshold.  A
finite-precision render is accepted at a pixel when it lies within the
tolerance of one of those outcomes.
"""
from __future__ import annotations

import numpy as np


def match_fp64_branches(img, T, nc, dec, sel=None, tol: float = 2e-4):
    """Best outcome per pixel of ``img`` (3, H, W) among the FP64-decision
    outcomes ``dec``, on the pixels of ``sel`` (H, W bool; all if None).

    Returns a dict: max_err (the largest, over pixels, of the smallest
    per-channel max-abs error over the pixel's outcomes), bad (pixels whose
    best outcome is beyond ``tol``), flagged (pixels with more than one
    outcome), multi (more than two), capped (flags not followed), alt_best
    (pixels that only an outcome other than the main path brings within
    ``tol``), nc_differs (pixels where no outcome within ``tol`` has the
    contributor count ``nc``), T_err (transmittance error of the best
    outcome) and pixels (compared)."""
    img = np.asarray(img, np.float64)
    H, W = img.shape[1:]
    if sel is None:
        sel = np.ones((H, W), bool)
    flat_sel = sel.reshape(-1)
    main = dec["img"].reshape(3, -1)
    g = img.reshape(3, -1)
    err_main = np.abs(g - main).max(axis=0)
    best = err_main.copy()
    best_nc = dec["ncontrib"].reshape(-1).astype(np.int64).copy()
    best_T = dec["T"].reshape(-1).copy()
    ncg = None if nc is None else np.asarray(nc).reshape(-1).astype(np.int64)
    same_nc = None if ncg is None else (err_main <= tol) & (best_nc == ncg)
    pix = dec["alt_pix"]
    if pix.size:
        ea = np.abs(g[:, pix].T - dec["alt_val"][:, :3]).max(axis=1)
        if ncg is not None:
            hit = (ea <= tol) & (dec["alt_nc"].astype(np.int64) == ncg[pix])
            same_nc[pix[hit]] = True
        order = np.argsort(ea, kind="stable")[::-1]     # smallest error written last
        for k in order:
            p = pix[k]
            if ea[k] < best[p]:
                best[p] = ea[k]
                best_nc[p] = int(dec["alt_nc"][k])
                best_T[p] = dec["alt_val"][k, 3]
    npaths = dec["n_paths"].reshape(-1)
    s = flat_sel
    out = dict(
        pixels=int(s.sum()),
        max_err=float(best[s].max()) if s.any() else 0.0,
        bad=int((best[s] > tol).sum()),
        flagged=int((npaths[s] > 1).sum()),
        multi=int((npaths[s] > 2).sum()),
        capped=int((dec["n_capped"].reshape(-1)[s] > 0).sum()),
        alt_best=int(((err_main > tol) & (best <= tol) & s).sum()),
    )
    if ncg is not None:
        out["nc_differs"] = int((~same_nc[s]).sum())
    if T is not None:
        out["T_err"] = float(np.abs(np.asarray(T, np.float64).reshape(-1)[s] - best_T[s]).max()) if s.any() else 0.0
    return out


def tile_mask(width: int, height: int, tiles):
    """(H, W) bool of the pixels of the listed 16x16 tiles."""
    tx = (width + 15) // 16
    sel = np.zeros((height, width), bool)
    for t in tiles:
        x0, y0 = (int(t) % tx) * 16, (int(t) // tx) * 16
        sel[y0:y0 + 16, x0:x0 + 16] = True
    return sel
