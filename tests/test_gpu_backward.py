"""GPU backward pass against the oracle's FP64 reference gradients.

The reference is reverse-mode autodiff of the oracle's FP64 statement of the
forward function with the discrete decisions frozen (pinned against central
differences in test_oracle_pins).  Criterion: per parameter group,
||g_gpu - g_ref||_2 / ||g_ref||_2 <= 1e-3.
"""
import numpy as np
import pytest
import torch

from oracle import grad64 as G
from paper_2510_09997_gb300 import synth as S

from gpu_helpers import gpu_grads, rel_errors

pytestmark = pytest.mark.gpu
NAMES = ("means", "scales", "quats", "opacity", "sh", "decay")


@pytest.fixture(scope="module")
def A():
    from paper_2510_09997_gb300 import autograd, clod
    clod.require_cuda()
    return autograd


def check(A, sc, views, seed=0, with_alpha=True, tol=1e-3):
    rng = np.random.default_rng(seed)
    gimgs = [rng.normal(size=(3, v.height, v.width)) for v in views]
    galphas = [rng.normal(size=sc.n) * 1e-2 for _ in views] if with_alpha else None
    g = gpu_grads(A, sc, views, gimgs, galphas)
    r = G.reference_gradients(sc, views, gimgs, galphas)
    err = rel_errors(g, r)
    for k in NAMES:
        assert np.linalg.norm(r[k]) > 0, k
        assert err[k] <= tol, err
    return err


def test_small_scene_sh3(A):
    sc = S.small_scene(n=200, seed=3, sh_degree=3)
    check(A, sc, [S.look_at((0.4, -1.8, 1.2), (0, 0, 0), 48, 40, s_v=2.0, bg=(0.2, 0.1, 0.0))])


def test_tiny_scene_two_views_decay_and_dmax(A):
    """Two views in one launch; the external alpha'' gradient exercises the
    sigma_d and d_max terms for culled Gaussians too."""
    sc = S.tiny_scene(n=3000, seed=30, sh_degree=1)
    views = [S.tiny_view(1.5).replace(width=96, height=80, cx=48.0, cy=40.0),
             S.look_at((2.0, 1.5, 1.0), (0, 0, 0), 64, 64, s_v=3.0, bg=(0.5, 0.5, 0.5))]
    check(A, sc, views, seed=1)


def test_lod_off_and_no_normalize(A):
    sc = S.small_scene(n=300, seed=31, sh_degree=2)
    views = [S.look_at((0.3, 1.9, 0.8), (0, 0, 0), 40, 40, flags=S.FLAG_LOD_OFF),
             S.look_at((-1.2, -1.2, 1.4), (0, 0, 0), 40, 40, s_v=1.2, flags=S.FLAG_NO_NORMALIZE, tau=0.0)]
    check(A, sc, views, seed=2)


def test_clamped_projection_and_opacity_clamp(A):
    """Wide Gaussians off screen (the 1.3 x tan(fov/2) clamp of the Jacobian)
    and opaque ones (the 0.99 opacity clamp)."""
    sc = S.small_scene(n=200, seed=32, sh_degree=0, extent=1.2, log_scale_mean=-2.2)
    sc.opacity[:80] = 0.999
    check(A, sc, [S.look_at((0.0, -1.6, 0.4), (0, 0, 0), 48, 48, s_v=1.0, fovy_deg=40.0)], seed=3)


def test_l1_loss_kernel(A):
    rng = np.random.default_rng(4)
    a = torch.tensor(rng.normal(size=(3, 37, 29)), device="cuda", dtype=torch.float32, requires_grad=True)
    b = torch.tensor(rng.normal(size=(3, 37, 29)), device="cuda", dtype=torch.float32)
    loss = A.L1Loss.apply(a, b)
    loss.backward()
    ref = (a.detach() - b).abs().mean()
    assert abs(float(loss) - float(ref)) < 1e-5 * float(ref)
    assert torch.allclose(a.grad, torch.sign(a.detach() - b) / a.numel())


def test_gpu_gradients_match_central_differences_200_32x32(A):
    """The 200-Gaussian 32x32 finite-difference subcase of the training
    workload: GPU gradients (with an external dL/dalpha'') against central
    FP64 differences of the oracle's forward statement with its decisions
    frozen, on sampled entries of all six groups."""
    sc = S.small_scene(n=200, seed=3, sh_degree=3)
    v = S.look_at((0.4, -1.8, 1.2), (0, 0, 0), 32, 32, s_v=2.0, bg=(0.2, 0.1, 0.0))
    fr, s1, _ = G.frozen_from_oracle(sc, v)
    rng = np.random.default_rng(5)
    gimg = rng.normal(size=(3, 32, 32))
    galpha = rng.normal(size=sc.n) * 0.1
    g = gpu_grads(A, sc, [v], [gimg], [galpha])

    def loss(P):
        out = G.view_forward(P, v, fr)
        return float((out["image"].detach().numpy() * gimg).sum() + (out["alpha_eff"].detach().numpy() * galpha).sum())

    P0 = G.params_f64(sc, requires_grad=False)
    live = np.nonzero(s1["survive"])[0]
    assert live.size > 20
    pick = rng.choice(live, size=10, replace=False)
    for name in NAMES:
        flat = P0[name].reshape(-1)
        per = flat.numel() // sc.n
        fd, gg = [], []
        for i in pick:
            for j in range(min(per, 4)):
                k = int(i) * per + j
                x0 = float(flat[k])
                h = 1e-6 * max(1.0, abs(x0))
                flat[k] = x0 + h
                lp = loss(P0)
                flat[k] = x0 - h
                lm = loss(P0)
                flat[k] = x0
                fd.append((lp - lm) / (2 * h))
                gg.append(g[name].reshape(-1)[k])
        fd, gg = np.array(fd), np.array(gg)
        assert np.linalg.norm(fd) > 0, name
        assert np.linalg.norm(gg - fd) <= 2e-3 * np.linalg.norm(fd), (name, np.linalg.norm(gg - fd) / np.linalg.norm(fd))


def test_fast_exp_gradients(A):
    """Forward and backward blends under CLOD_FAST_EXP against the FP64
    reference gradients (decisions frozen from the FP32 specification; the
    fast exponential may move a near-threshold decision, which the 1e-3
    criterion absorbs)."""
    sc = S.tiny_scene(n=3000, seed=30, sh_degree=1)
    views = [S.tiny_view(1.5).replace(width=96, height=80, cx=48.0, cy=40.0, flags=S.FLAG_FAST_EXP),
             S.look_at((2.0, 1.5, 1.0), (0, 0, 0), 64, 64, s_v=3.0, bg=(0.5, 0.5, 0.5), flags=S.FLAG_FAST_EXP)]
    check(A, sc, views, seed=1)
