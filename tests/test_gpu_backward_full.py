"""Backward parity at the training workload's size (Sec. 3.2-3.3, Eq. 1-2
differentiated): the 3M-Gaussian outdoor scene (SH degree 3), one batch of 4
views at 1920x1080 with virtual scales 1, 2.5, 5 and 9 (within the training
sampler's [1, 16]).

The image gradient is non-zero on sampled tiles of every view: the 3x3 block
around the tile with the longest list (so that wide Gaussians receive the
block-reduced atomics of many warps), the four longest lists and four random
tiles.  An external alpha'' gradient sits on 4000 random Gaussians per view.
The oracle's FP64 reference gradients are taken on the frozen contributor
lists of those tiles (only the Gaussians they reach, plus the alpha''-sampled
ones and each view's farthest in-view Gaussian, have non-zero gradients).
Criterion, per parameter group: ||g_gpu - g_ref||_2 / ||g_ref||_2 <= 1e-3.
"""
import numpy as np
import pytest
import torch

from branches import tile_mask
from gpu_helpers import GRAD_NAMES, gpu_grads, rel_errors, tile_list_lengths
from oracle import grad64 as G
from oracle import oracle as O
from paper_2510_09997_gb300 import synth as S

pytestmark = pytest.mark.gpu


def sampled_tiles(lens, view, rng, n_random=4):
    """The 3x3 block around the longest list, the four longest lists and
    n_random random tiles of one view (row-major tile indices)."""
    tx, ty = O.tiles_of(view)
    top = int(np.argmax(lens))
    cy, cx = divmod(top, tx)
    block = [y * tx + x for y in range(max(0, cy - 1), min(ty, cy + 2)) for x in range(max(0, cx - 1), min(tx, cx + 2))]
    longest = [int(t) for t in np.argsort(lens)[-4:]]
    rand = [int(t) for t in rng.choice(tx * ty, n_random, replace=False)]
    return sorted(set(block + longest + rand))


def sparse_check(A, sc, views, seed, s1s=None, n_alpha=4000, tol=1e-3):
    """GPU gradients against the oracle's FP64 gradients on sampled tiles
    and an alpha''-sampled Gaussian subset; returns the per-group errors and
    the longest list among the sampled tiles."""
    rng = np.random.default_rng(seed)
    frozen, gimgs, galphas = [], [], []
    longest = 0
    for vi, v in enumerate(views):
        s1 = O.stage1(sc, v) if s1s is None else s1s[vi]
        lens = tile_list_lengths(s1, v)
        tiles = sampled_tiles(lens, v, rng)
        longest = max(longest, int(lens[tiles].max()))
        fr, _ = G.frozen_on_tiles(sc, v, tiles, s1)
        frozen.append(fr)
        sel = tile_mask(v.width, v.height, tiles)
        gimgs.append(rng.normal(size=(3, v.height, v.width)) * sel[None])
        ga = np.zeros(sc.n)
        pick = rng.choice(sc.n, n_alpha, replace=False)
        ga[pick] = rng.normal(size=n_alpha) * 1e-2
        galphas.append(ga)
    g = gpu_grads(A, sc, views, gimgs, galphas)
    torch.cuda.empty_cache()
    r = G.reference_gradients_sparse(sc, views, frozen, gimgs, galphas)
    err = rel_errors(g, r)
    print("relative errors per group:", {k: float("%.3g" % e) for k, e in err.items()},
          "longest sampled list:", longest)
    for k in GRAD_NAMES:
        assert np.linalg.norm(r[k]) > 0, k
        assert err[k] <= tol, err
    return err, longest


@pytest.mark.parametrize("flags", [0, S.FLAG_FAST_EXP], ids=["exact", "fast_exp"])
def test_outdoor_3m_four_views_1080p(flags):
    """With CLOD_FAST_EXP (the training bench's setting) the blends' decisions
    may move near a threshold against the oracle's frozen FP32 ones; the
    1e-3 criterion stands."""
    from paper_2510_09997_gb300 import autograd, clod
    clod.require_cuda()
    sc = S.outdoor_scene(3_000_000)
    cams = S.orbit_cameras(16, 1920, 1080, d_min=9.0, d_max=16.0, elev_deg=25.0, seed=2)
    views = [cams[k].replace(s_v=s, flags=flags) for k, s in zip((0, 5, 10, 15), (1.0, 2.5, 5.0, 9.0))]
    _, longest = sparse_check(autograd, sc, views, seed=11)
    assert longest > 1000
