"""Large-scene stress at full size: 6M Gaussians (city-block planes + volume
noise, SH degree 3), 8 views per launch at 3840x2160, s_v in {1, 4, 16, 64}.

Every Stage I output of every view is compared with the oracle bit for bit;
per view, sampled tiles (the longest lists and random ones) are compared bit
for bit (image, T, contributor counts), against the FP64 image and against
the outcomes of the FP64 decisions, and the
tile list lengths of all tiles against the oracle's rectangles.  The backward
pass runs at full size: checked for its structure (finite, zero wherever a
Gaussian neither contributes nor receives an external gradient) and against
the oracle's FP64 gradients on sampled tiles.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2510_09997_gb300 import synth as S

from gpu_helpers import assert_image_matches, assert_stage1_equal, frame_stage1

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def city():
    from paper_2510_09997_gb300 import clod as C
    C.require_cuda()
    sc = S.city_scene()
    views = S.city_views()
    ds = C.DeviceScene.from_scene(sc)
    fr = C.render(ds, views, want_keys=False)
    torch.cuda.synchronize()
    return C, sc, views, ds, fr


@pytest.fixture(scope="module")
def city_stage1(city):
    """The oracle's Stage I of every city view (shared by the tests)."""
    C, sc, views, ds, fr = city
    return [O.stage1(sc, view) for view in views]


def test_city_8x4k_stage1_and_sampled_tiles(city, city_stage1):
    C, sc, views, ds, fr = city
    g = frame_stage1(fr, sc.n)
    ranges = fr.ranges.cpu().numpy().view(np.uint32).astype(np.int64)
    base = 0
    rng = np.random.default_rng(7)
    culled = []
    for v, view in enumerate(views):
        s1 = city_stage1[v]
        assert_stage1_equal(g[v], s1)
        culled.append(1.0 - s1["mask"].mean())
        tx, ty = O.tiles_of(view)
        T = tx * ty
        # tile list lengths of every tile from the oracle's rectangles
        lens = np.zeros((ty + 1, tx + 1), np.int64)
        r = s1["rect"][s1["survive"].astype(bool)]
        np.add.at(lens, (r[:, 1], r[:, 0]), 1)
        np.add.at(lens, (r[:, 1], r[:, 2]), -1)
        np.add.at(lens, (r[:, 3], r[:, 0]), -1)
        np.add.at(lens, (r[:, 3], r[:, 2]), 1)
        lens = lens.cumsum(0).cumsum(1)[:ty, :tx].reshape(-1)
        got = ranges[base:base + T, 1] - ranges[base:base + T, 0]
        assert np.array_equal(got, lens)
        tiles = list(np.argsort(lens)[-3:]) + list(rng.choice(T, 5, replace=False))
        r64 = O.stage1_f64(sc, view, s1)
        ref = O.render(sc, view, s1, r64, tiles=tiles)
        ref["dec64"] = O.render_f64dec(view, s1, r64, tiles)
        assert_image_matches(fr, v, ref, tiles)
        base += T
    assert culled[3] > culled[0]          # s_v = 64 culls more than s_v = 1


def test_city_8x4k_backward_structure(city):
    C, sc, views, ds, fr = city
    from paper_2510_09997_gb300 import autograd as A
    ps = [torch.tensor(np.asarray(getattr(sc, k), np.float32), device="cuda", requires_grad=True)
          for k in ("means", "scales", "quats", "opacity", "sh", "decay")]
    imgs, alpha, mask, counts = A.render(*ps, views)
    loss = sum(im.mean() for im in imgs)
    loss.backward()
    torch.cuda.synchronize()
    for p in ps:
        assert torch.isfinite(p.grad).all()
    # a Gaussian rendered in no view gets no gradient from the image
    rendered_any = torch.zeros(sc.n, dtype=torch.bool, device="cuda")
    lay = fr.layout
    V = len(views)
    rect = fr.ws_array("rect", torch.int32, 2 * V * sc.n).view(V, sc.n, 2)
    for v in range(V):
        rendered_any |= (rect[v, :, 1] != 0)
    idle = ~rendered_any
    assert idle.any() and rendered_any.any()
    assert float(ps[4].grad[idle].abs().max()) == 0.0
    assert float(ps[3].grad[idle].abs().max()) == 0.0
    # means of idle Gaussians: zero except the farthest in-view Gaussian of a
    # view, which carries d_max (Eq. 2 normalisation)
    key = fr.ws_array("dmax_key", torch.int64, V).cpu().numpy().view(np.uint64)
    far = [0xFFFFFFFF - (int(k) & 0xFFFFFFFF) for k in key if int(k)]
    idle_m = idle.clone()
    idle_m[far] = False
    assert float(ps[0].grad[idle_m].abs().max()) == 0.0
    assert float(ps[4].grad[rendered_any].abs().sum()) > 0.0


def test_city_8x4k_backward_parity_on_sampled_tiles(city, city_stage1):
    """The backward at full size against the oracle's FP64 gradients: image
    gradient on sampled tiles of all eight 4K views (the 3x3 block around the
    longest list, the four longest lists, four random tiles), an alpha''
    gradient on 4000 random Gaussians per view; relative error <= 1e-3 per
    parameter group."""
    from paper_2510_09997_gb300 import autograd as A
    from test_gpu_backward_full import sparse_check
    C, sc, views, ds, fr = city
    _, longest = sparse_check(A, sc, views, seed=12, s1s=city_stage1)
    assert longest > 1000


def test_city_8x4k_whole_sorted_list(city, city_stage1):
    """The whole sorted pair list of the 8 x 4K launch (all ~38 M values and
    every tile range) bit for bit against the oracle's emission of every
    survivor's tiles in index order and its stable sort by (tile, depth)."""
    C, sc, views, ds, fr = city
    keys, vals, base = [], [], 0
    for v, view in enumerate(views):
        k, val = O.emit_pairs(view, city_stage1[v], base)
        keys.append(k)
        vals.append(val)
        tx, ty = O.tiles_of(view)
        base += tx * ty
    sk, sv = O.stable_sort(np.concatenate(keys), np.concatenate(vals))
    del keys, vals
    assert int(fr.n_pairs) == len(sv)
    assert np.array_equal(fr.vals[:len(sv)].cpu().numpy().view(np.uint32), sv)
    assert np.array_equal(fr.ranges.cpu().numpy().view(np.uint32), O.ranges(sk, base))
