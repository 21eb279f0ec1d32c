"""GPU parity of the two level-of-detail controls beyond the threshold mask.

* Primitive budget (Sec. 4.2): the mask keeps the B Gaussians of highest
  alpha'' (equal alpha'' in index order).  Mask, Stage I, pairs and images are
  compared with the oracle bit for bit; a budget equal to the threshold
  count reproduces the threshold render.
* Regional views (Sec. 4.4, vertical bands of one frame at different s_v):
  every band equals, bit for bit, the same pixels of the full-frame render at
  its s_v (image, transmittance and contributor count), and the full frames
  match the oracle.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2510_09997_gb300 import synth as S

from gpu_helpers import frame_stage1, run_and_compare, u32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def C():
    from paper_2510_09997_gb300 import clod
    clod.require_cuda()
    return clod


@pytest.mark.parametrize("B", [1, 777, 19999, 20000, 50000])
def test_budget_bit_exact(C, B):
    """20,000 Gaussians: budgets of one, a few hundred, n - 1, n and above n."""
    fr, ref, _ = run_and_compare(C, S.tiny_scene(), [S.tiny_view(4.0, budget=B)])
    assert int(fr.counts[0][0]) == min(B, 20000)


def test_budget_equal_to_threshold_count_gives_threshold_render(C):
    sc = S.tiny_scene(n=20000, seed=81)
    ds = C.DeviceScene.from_scene(sc)
    a = C.render(ds, [S.tiny_view(6.0)])
    B = int(a.counts[0][0])
    assert 0 < B < sc.n
    b = C.render(ds, [S.tiny_view(6.0, budget=B)])
    torch.cuda.synchronize()
    assert torch.equal(a.mask, b.mask)
    assert torch.equal(a.image, b.image) and torch.equal(a.T_final, b.T_final)


def test_budget_ties_and_mixed_batch(C):
    """Equal alpha'' (level of detail off, two opacity levels): ties go to the
    lower indices.  One launch mixes threshold, budget, budget >= n and
    level-of-detail-off views."""
    sc = S.tiny_scene(n=12000, seed=82)
    op = np.where(np.arange(sc.n) % 3 == 0, 0.9, 0.5).astype(np.float32)
    sc = S.Scene(sc.means, sc.scales, sc.quats, op, sc.sh, sc.decay)
    views = [S.tiny_view(2.0),
             S.tiny_view(4.0, flags=S.FLAG_LOD_OFF, budget=5000),
             S.look_at((2.5, -1.0, 1.0), (0, 0, 0), 250, 130, s_v=3.0, budget=3001),
             S.look_at((-1.5, 2.0, -1.0), (0.1, 0, 0), 97, 161, s_v=2.0, budget=10 ** 6)]
    fr, ref, _ = run_and_compare(C, sc, views)
    m = fr.mask[1].cpu().numpy().astype(bool)
    hi = np.flatnonzero(op == np.float32(0.9))
    lo = np.flatnonzero(op == np.float32(0.5))
    assert np.array_equal(np.flatnonzero(m), np.sort(np.concatenate([hi, lo[:5000 - hi.size]])))


def test_budget_full_size_mask(C):
    """1M Gaussians at 1080p: the budget mask equals the oracle's Stage I mask."""
    sc = S.object_scene()
    v = S.orbit_cameras(64, 1920, 1080)[20].replace(s_v=2.0, budget=300000)
    ds = C.DeviceScene.from_scene(sc)
    fr = C.render(ds, [v], want_keys=False)
    torch.cuda.synchronize()
    s1 = O.stage1(sc, v)
    assert np.array_equal(fr.mask[0].cpu().numpy(), s1["mask"])
    assert np.array_equal(u32(fr.alpha_eff[0].cpu().numpy()), u32(s1["alpha_eff"]))
    assert int(fr.counts[0][0]) == 300000
    assert int(fr.counts[0][1]) == int(s1["survive"].sum())


def _crop(fr, k, x0, y0, w, h):
    img = fr.view_image(k)[:, y0:y0 + h, x0:x0 + w]
    T = fr.view_T(k)[y0:y0 + h, x0:x0 + w]
    nc = fr.view_ncontrib(k)[y0:y0 + h, x0:x0 + w]
    return img, T, nc


def test_band_views_equal_full_frame_crops(C):
    """Four vertical bands of a ragged 250 x 130 frame at s_v = 8, 4, 2, 1 in one
    launch: each band equals the full-frame render at its s_v."""
    sc = S.tiny_scene(n=20000, seed=83, sh_degree=2)
    full = S.look_at((2.5, -1.0, 1.0), (0, 0, 0), 250, 130, s_v=1.0, bg=(0.2, 0.3, 0.4))
    svals = [8.0, 4.0, 2.0, 1.0]
    bands = C.band_views(full, [0, 64, 128, 176, 250], svals)
    fulls = [full.replace(s_v=s) for s in svals]
    ds = C.DeviceScene.from_scene(sc)
    fb = C.render(ds, bands)
    ff = C.render(ds, fulls)
    torch.cuda.synchronize()
    for k, b in enumerate(bands):
        img, T, nc = _crop(ff, k, b.region_x, 0, b.width, b.height)
        assert torch.equal(fb.view_image(k), img), k
        assert torch.equal(fb.view_T(k), T), k
        assert torch.equal(fb.view_ncontrib(k), nc), k
    # the full frames (and so the bands) against the oracle
    run_and_compare(C, sc, fulls, with64=False)
    # every band sees the full frame's d_max
    g = frame_stage1(fb, sc.n)
    h = frame_stage1(ff, sc.n)
    for k in range(4):
        assert int(g[k]["dmax_bits"]) == int(h[k]["dmax_bits"])
        assert np.array_equal(u32(g[k]["alpha"]), u32(h[k]["alpha"]))


def test_window_with_vertical_offset_and_budget(C):
    """A 96 x 48 window at (32, 64) of a 250 x 130 frame, also under a budget."""
    sc = S.tiny_scene(n=20000, seed=84)
    full = S.look_at((-1.5, 2.0, -1.0), (0.1, 0, 0), 250, 130, s_v=2.0)
    ds = C.DeviceScene.from_scene(sc)
    for budget in (0, 4000):
        f = full.replace(budget=budget)
        win = f.replace(width=96, height=48, region_x=32, region_y=64, full_width=250, full_height=130)
        fw = C.render(ds, [win])
        ff = C.render(ds, [f])
        torch.cuda.synchronize()
        img, T, nc = _crop(ff, 0, 32, 64, 96, 48)
        assert torch.equal(fw.view_image(0), img)
        assert torch.equal(fw.view_T(0), T)
        assert torch.equal(fw.view_ncontrib(0), nc)


def test_band_backward_matches_full_frame(C):
    """Gradients of a band render equal those of the full-frame render whose
    image gradient is zero outside the band (same pixels contribute; only the
    order of the atomic sums differs)."""
    from paper_2510_09997_gb300 import autograd as A
    sc = S.small_scene(n=400, seed=85, sh_degree=2)
    full = S.look_at((0.4, -1.8, 1.2), (0, 0, 0), 80, 64, s_v=2.0)
    band = full.replace(width=32, region_x=32, full_width=80, full_height=64)
    names = ("means", "scales", "quats", "opacity", "sh", "decay")
    rng = np.random.default_rng(3)
    gimg = rng.normal(size=(3, 64, 80)).astype(np.float32)
    grads = []
    for v, g in ((band, gimg[:, :, 32:64]), (full, np.where((np.arange(80) >= 32) & (np.arange(80) < 64), gimg, 0))):
        ps = [torch.tensor(np.asarray(getattr(sc, k), np.float32), device="cuda", requires_grad=True) for k in names]
        imgs, _, _, _ = A.render(*ps, [v])
        (imgs[0] * torch.tensor(np.ascontiguousarray(g, np.float32), device="cuda")).sum().backward()
        grads.append([p.grad.detach().cpu().numpy().astype(np.float64) for p in ps])
    for k, a, b in zip(names, *grads):
        den = max(np.linalg.norm(b), 1e-12)
        assert np.linalg.norm(a - b) / den < 1e-5, k
