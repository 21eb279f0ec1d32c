"""Pins of the CPU oracle against closed forms, library routines, invariants and
an independent FP64 brute force (CPU only).

Each test names what fixes the expected value; none re-derives it from the
oracle's own code.
"""
import math

import numpy as np
import pytest
import scipy.stats

from oracle import oracle as O
from oracle import losses as L
from paper_2510_09997_gb300 import synth as S

F32 = np.float32
ONE255 = F32(1) / F32(255)


def axis_view(W=128, H=128, f=200.0, cx=None, cy=None, **kw):
    """Camera at the origin looking along +z (camera axes = world axes)."""
    vm = np.zeros((3, 4), np.float32)
    vm[:, :3] = np.eye(3)
    return S.View(width=W, height=H, viewmat=vm, fx=f, fy=f, cx=W / 2 if cx is None else cx,
                  cy=H / 2 if cy is None else cy, campos=np.zeros(3, np.float32), **kw)


def one_gaussian(mu, scales, quat=(1, 0, 0, 0), opacity=0.8, fdc=(0.5, -0.3, 0.2), decay=1.0):
    sh = np.zeros((1, 1, 3), np.float32)
    sh[0, 0] = fdc
    return S.Scene(np.array([mu], np.float32), np.array([scales], np.float32), np.array([quat], np.float32),
                   np.array([opacity], np.float32), sh, np.array([decay], np.float32))


def stack(scenes):
    return S.Scene(*(np.concatenate([getattr(s, k) for s in scenes]) for k in
                     ("means", "scales", "quats", "opacity", "sh", "decay")))


# ---------------------------------------------------------------------------
# exp_spec
# ---------------------------------------------------------------------------
def test_exp_spec_special_values():
    assert O.exp_spec(0.0)[0] == 1.0
    assert O.exp_spec(-0.0)[0] == 1.0
    assert O.exp_spec(np.nan)[0] == 0.0
    assert O.exp_spec(-80.5)[0] == 0.0
    # the blend's early cutoff: for power < -5.6 the opacity is below 1/255 for any alpha'' <= 1
    assert O.exp_spec(-5.6)[0] < ONE255


def test_exp_spec_accuracy_vs_libm():
    x = np.concatenate([-np.random.default_rng(0).uniform(0, 80, 400_000),
                        -np.linspace(0, 6, 200_000)]).astype(np.float32)
    y = O.exp_spec(x).astype(np.float64)
    ref = np.exp(x.astype(np.float64))
    ulp = np.spacing(ref.astype(np.float32)).astype(np.float64)
    err = np.abs(y - ref) / ulp
    # within the blend range: faithful to ~1 ulp; elsewhere the 2-cap costs
    # at most |k| * 6.9e-8 relative (L2E rounded up), k <= 116
    assert err[400_000:].max() < 2.0
    rel = np.abs(y - ref) / ref
    assert rel.max() < 116 * 7e-8 + 3e-7


@pytest.mark.slow
def test_exp_spec_monotone_exhaustive():
    """P4 rests on this: every float in [-80, 0], in order."""
    bad, first = O.exp_spec_monotone_violations(-80.0, -0.0)
    assert bad == 0, first


# ---------------------------------------------------------------------------
# Eq. 2 and the mask (Sec. 3.2)
# ---------------------------------------------------------------------------
def test_attenuation_is_gaussian_falloff_in_normalised_distance():
    """alpha''/alpha is a zero-mean Gaussian in d' s_v with variance
    sigma^2 + eps/2 (library density), d' = d / max over the view frustum."""
    sc = S.tiny_scene(n=3000, seed=11)
    seen = []
    for s in (1.0, 2.5, 7.0):
        v = S.tiny_view(s)
        s1 = O.stage1(sc, v)
        d = np.linalg.norm(sc.means.astype(np.float64) - v.campos, axis=1)
        dn = d / d[s1["argmax"][0]]
        sd = np.sqrt(np.maximum(sc.decay.astype(np.float64), 0) ** 2 + v.eps / 2)
        fall = scipy.stats.norm.pdf(dn * s, scale=sd) / scipy.stats.norm.pdf(0.0, scale=sd)
        expect = sc.opacity * fall
        got = s1["alpha_eff"].astype(np.float64)
        # FP32 rounding of the exponent x (a few ulp) is scaled by x through exp;
        # exp_spec flushes exponents below -80 to zero
        x = (dn * s) ** 2 / (2 * sd ** 2)
        expect = np.where(x > 80.0, 0.0, expect)
        clear = np.abs(x - 80.0) > 1e-3
        tol = (1e-6 + 6e-7 * x) * expect
        assert np.all((np.abs(got - expect) <= tol)[clear])
        seen.append(x)
    seen = np.concatenate(seen)
    assert (seen > 80).any() and (seen < 1).any()


def test_dmax_is_max_over_view_frustum():
    sc = S.tiny_scene(n=2000, seed=12)
    v = S.tiny_view(1.0).replace(width=128, height=64, cx=64.0, cy=32.0)
    s1 = O.stage1(sc, v)
    mu = sc.means.astype(np.float64)
    vm = np.asarray(v.viewmat, np.float64)
    t = mu @ vm[:, :3].T + vm[:, 3]
    u = v.fx * t[:, 0] / t[:, 2] + v.cx
    w = v.fy * t[:, 1] / t[:, 2] + v.cy
    inside = (t[:, 2] > v.near) & (u >= 0) & (u <= v.width) & (w >= 0) & (w <= v.height)
    assert 0 < inside.sum() < sc.n            # the frustum really excludes points
    d = np.linalg.norm(mu - v.campos, axis=1)
    j = np.argmax(np.where(inside, d, -1))
    assert s1["argmax"][0] == j
    assert s1["dmax"][0] == np.float32(np.sqrt(np.float32(d[j] ** 2)))  or abs(s1["dmax"][0] - d[j]) < 1e-6


def test_farthest_in_view_has_unit_normalised_distance():
    """P6: d'_{j*} = x/x = 1 exactly, so alpha'' there depends on s_v and sigma only."""
    sc = S.tiny_scene(n=500, seed=13)
    for s in (1.0, 3.0):
        v = S.tiny_view(s)
        s1 = O.stage1(sc, v)
        j = s1["argmax"][0]
        sig = max(float(sc.decay[j]), 0.0)
        expect = float(sc.opacity[j]) * math.exp(-s * s / (2 * sig * sig + v.eps))
        assert abs(s1["alpha_eff"][j] - expect) <= 4e-7 * expect + 1e-37


def test_scale_invariance_of_normalised_distance():
    """Sec. 3.2 normalises d so the decay is consistent across scene scale:
    scaling the scene and the camera by 4 (exact in binary) changes nothing."""
    sc = S.tiny_scene(n=3000, seed=14)
    v = S.tiny_view(3.0)
    sc4 = S.Scene(sc.means * 4, sc.scales * 4, sc.quats, sc.opacity, sc.sh, sc.decay)
    vm = np.array(v.viewmat)
    vm[:, 3] *= 4
    v4 = v.replace(viewmat=vm, campos=v.campos * 4, near=v.near * 4)
    a, b = O.stage1(sc, v), O.stage1(sc4, v4)
    assert np.array_equal(a["alpha_eff"], b["alpha_eff"])
    assert np.array_equal(a["mask"], b["mask"])
    assert np.array_equal(a["rect"], b["rect"])


def test_monotone_in_virtual_scale():
    """P4: alpha'' non-increasing and the survivor count non-increasing in s_v,
    bit-exactly (the threshold tau s_v grows while alpha'' falls)."""
    sc = S.tiny_scene(n=4000, seed=15)
    prev_a, prev_n = None, None
    for s in np.geomspace(1, 64, 25).astype(np.float32):
        s1 = O.stage1(sc, S.tiny_view(float(s)))
        if prev_a is not None:
            assert np.all(s1["alpha_eff"] <= prev_a)
            assert s1["mask"].sum() <= prev_n
        prev_a, prev_n = s1["alpha_eff"], s1["mask"].sum()
    assert prev_n < 4000 // 4


def test_monotone_in_distance():
    """P4: for equal alpha and sigma_d, alpha'' is non-increasing in d."""
    n = 2000
    z = np.linspace(0.5, 30.0, n).astype(np.float32)
    sc = S.Scene(np.stack([np.zeros(n), np.zeros(n), z], 1).astype(np.float32),
                 np.full((n, 3), 0.01, np.float32), np.tile(np.array([1, 0, 0, 0], np.float32), (n, 1)),
                 np.full(n, 0.7, np.float32), np.zeros((n, 1, 3), np.float32), np.full(n, 0.4, np.float32))
    s1 = O.stage1(sc, axis_view(s_v=2.0))
    assert np.all(np.diff(s1["alpha_eff"]) <= 0)
    assert s1["alpha_eff"][-1] < s1["alpha_eff"][0]


def test_lod_off_equals_plain_3dgs():
    """P3 (reading of "zero decay"): level of detail off gives alpha'' = alpha
    and keeps every Gaussian; sigma_d = +inf with tau = 0 is bit-identical."""
    sc = S.tiny_scene(n=3000, seed=16)
    off = O.stage1(sc, S.tiny_view(4.0, flags=O.LOD_OFF))
    assert np.array_equal(off["alpha_eff"], sc.opacity)
    assert off["mask"].all()
    inf = S.Scene(sc.means, sc.scales, sc.quats, sc.opacity, sc.sh, np.full(sc.n, np.inf, np.float32))
    on = O.stage1(inf, S.tiny_view(4.0, tau=0.0))
    for k in ("alpha_eff", "mask", "survive", "rec", "rect"):
        assert np.array_equal(off[k], on[k]), k
    zero_s = O.stage1(sc, S.tiny_view(0.0, tau=0.0))
    assert np.array_equal(zero_s["alpha_eff"], sc.opacity)


def test_nonpositive_decay_culls_beyond_closed_form_radius():
    """ReLU(sigma_d) = 0: alpha'' = alpha exp(-(d's)^2/eps) falls under tau s
    exactly when d's > sqrt(eps ln(alpha / (tau s)))."""
    sc = S.tiny_scene(n=3000, seed=17)
    sc = S.Scene(sc.means, sc.scales, sc.quats, sc.opacity, sc.sh, -np.abs(sc.decay))
    v = S.tiny_view(1.0, eps=1e-2)
    s1 = O.stage1(sc, v)
    d = np.linalg.norm(sc.means.astype(np.float64) - v.campos, axis=1)
    x = d / d[s1["argmax"][0]] * v.s_v
    lim = np.sqrt(v.eps * np.log(sc.opacity / (v.tau * v.s_v)))
    clear = np.abs(x - lim) > 1e-4
    assert np.array_equal(s1["mask"][clear].astype(bool), (x < lim)[clear])


# ---------------------------------------------------------------------------
# Projection and blending closed forms (Sec. 3.1, Eq. 1)
# ---------------------------------------------------------------------------
SH_C0 = 1.0 / (2.0 * math.sqrt(math.pi))   # Y_0^0 of the real SH basis


def test_lone_isotropic_gaussian_profile():
    """P1: an isotropic Gaussian on the optical axis renders
    rgb * min(0.99, a exp(-r^2 / (2 (sigma_px^2 + 0.3)))) over the background."""
    z, s3, f = 2.0, 0.05, 200.0
    fdc = (0.5, -0.3, 0.2)
    g = one_gaussian((0, 0, z), (s3, s3, s3), opacity=0.8, fdc=fdc)
    v = axis_view(f=f, flags=O.LOD_OFF, bg=(0.1, 0.2, 0.3))
    s1 = O.stage1(g, v)
    assert s1["survive"][0] == 1
    out = O.render(g, v, s1, O.stage1_f64(g, v, s1))
    r32 = lambda a: np.asarray(a, np.float32).astype(np.float64)   # inputs as the oracle sees them
    var = (f * r32(s3) / r32(z)) ** 2 + 0.3
    yy, xx = np.mgrid[0:128, 0:128] + 0.5
    r2 = (xx - 64) ** 2 + (yy - 64) ** 2
    a = np.minimum(0.99, r32(0.8) * np.exp(-r2 / (2 * var)))
    rgb = SH_C0 * r32(fdc) + 0.5
    x0, y0, x1, y1 = s1["rect"][0]
    in_rect = np.zeros((128, 128), bool)
    in_rect[y0 * 16:y1 * 16, x0 * 16:x1 * 16] = True
    on = in_rect & (a >= 1 / 255.0)
    # every pixel within 3 sigma lies in the tile rectangle
    assert in_rect[r2 <= 9 * var].all()
    bg = r32(v.bg)[:, None, None]
    expect = np.where(on[None], rgb[:, None, None] * a[None] + (1 - a[None]) * bg, bg)
    assert np.abs(out["img64"] - expect).max() < 1e-9
    assert np.abs(out["img32"] - expect).max() < 2e-6
    assert np.array_equal(out["ncontrib"], on.astype(np.uint32))


@pytest.mark.parametrize("theta", [0.0, 30.0, 90.0])
def test_rotated_anisotropic_covariance(theta):
    """Sigma = R S^2 R^T with q = (cos t/2, 0, 0, sin t/2) a rotation by t about
    +z; on the optical axis J = f/z I, so cov2D = (f/z)^2 Rz diag(a^2,b^2) Rz^T + 0.3 I."""
    z, f, a, b = 2.0, 200.0, 0.06, 0.02
    t = math.radians(theta)
    g = one_gaussian((0, 0, z), (a, b, 0.01), quat=(math.cos(t / 2), 0, 0, math.sin(t / 2)))
    v = axis_view(f=f, flags=O.LOD_OFF)
    s1 = O.stage1(g, v)
    Rz = np.array([[math.cos(t), -math.sin(t)], [math.sin(t), math.cos(t)]])
    cov = (f / z) ** 2 * Rz @ np.diag([a * a, b * b]) @ Rz.T + 0.3 * np.eye(2)
    inv = np.linalg.inv(cov)
    rec = s1["rec"][0].astype(np.float64)
    got = np.array([-2 * rec[4], -rec[5], -2 * rec[6]])
    want = np.array([inv[0, 0], inv[0, 1], inv[1, 1]])
    assert np.abs(got - want).max() < 2e-5 * np.abs(want).max()
    assert abs(rec[11] - np.linalg.det(cov)) < 2e-5 * np.linalg.det(cov)


@pytest.mark.parametrize("x0,s3", [(0.3, 0.03), (0.9, 0.12)])
def test_perspective_jacobian_off_axis(x0, s3):
    """Off-axis point (x0, 0, z): cov2D = s^2 J J^T + 0.3 I with J the
    perspective Jacobian, x/z clamped to 1.3 tan(fov_x / 2) (the second case
    has its centre off screen, x/z = 0.45 > 0.416, and a footprint on it)."""
    z, f, W = 2.0, 200.0, 128
    g = one_gaussian((x0, 0, z), (s3, s3, s3))
    v = axis_view(W=W, f=f, flags=O.LOD_OFF)
    s1 = O.stage1(g, v)
    lim = 1.3 * (W / 2) / f
    xc = min(lim, x0 / z) * z
    s3 = float(np.float32(s3))
    J = np.array([[f / z, 0, -f * xc / z ** 2], [0, f / z, 0]])
    cov = s3 ** 2 * J @ J.T + 0.3 * np.eye(2)
    inv = np.linalg.inv(cov)
    rec = s1["rec"][0].astype(np.float64)
    assert s1["survive"][0] == 1
    assert abs(rec[0] - (f * x0 / z + W / 2)) < 1e-4
    got = np.array([-2 * rec[4], -rec[5], -2 * rec[6]])
    want = np.array([inv[0, 0], inv[0, 1], inv[1, 1]])
    assert np.abs(got - want).max() < 2e-5 * np.abs(want).max()


def test_constant_layers_transmittance_and_stop():
    """P2: n co-located Gaussians of opacity a at a pixel centre: colour
    sum_k c_k a (1-a)^(k-1) over the first k* = floor(ln 1e-4 / ln(1-a))
    (the next one would push T under 1e-4 and is excluded); ties in depth
    are taken in index order."""
    a, n = 0.3, 40
    rng = np.random.default_rng(5)
    fdcs = rng.uniform(-1, 1, size=(n, 3))
    g = stack([one_gaussian((0, 0, 2.0), (0.05, 0.05, 0.05), opacity=a, fdc=tuple(fd)) for fd in fdcs])
    v = axis_view(W=64, H=64, cx=32.5, cy=32.5, flags=O.LOD_OFF)
    s1 = O.stage1(g, v)
    out = O.render(g, v, s1, O.stage1_f64(g, v, s1))
    kstar = math.floor(math.log(1e-4) / math.log(1 - a))
    assert kstar == 25
    a = float(np.float32(a))
    cols = SH_C0 * fdcs.astype(np.float32).astype(np.float64) + 0.5
    expect = sum(cols[k] * a * (1 - a) ** k for k in range(kstar))
    assert out["ncontrib"][32, 32] == kstar
    assert np.abs(out["img64"][:, 32, 32] - expect).max() < 1e-12
    assert abs(out["T64"][32, 32] - (1 - a) ** kstar) < 1e-15
    assert np.abs(out["img32"][:, 32, 32] - expect).max() < 2e-6
    # reversed depths: order follows depth, not index
    g2 = stack([one_gaussian((0, 0, 2.0 + 0.001 * (n - k)), (0.05, 0.05, 0.05), opacity=a, fdc=tuple(fdcs[k]))
                for k in range(n)])
    s2 = O.stage1(g2, v)
    out2 = O.render(g2, v, s2, O.stage1_f64(g2, v, s2))
    order = list(range(n))[::-1]
    expect2 = sum(cols[order[k]] * a * (1 - a) ** k for k in range(kstar))
    assert np.abs(out2["img64"][:, 32, 32] - expect2).max() < 1e-6


def test_lossless_cull_at_unit_scale():
    """P5: at s_v = 1 and tau = 1/255 every culled Gaussian has alpha'' <= 1/255,
    so every per-pixel alpha would be skipped anyway: the image with the cull
    equals the image without it (tau = 0)."""
    sc = S.tiny_scene(n=6000, seed=18)
    v = S.tiny_view(1.0).replace(width=96, height=96, cx=48.0, cy=48.0)
    a = O.stage1(sc, v)
    b = O.stage1(sc, v.replace(tau=0.0))
    assert a["mask"].sum() < b["mask"].sum()
    ia, ib = O.render(sc, v, a), O.render(sc, v.replace(tau=0.0), b)
    assert np.array_equal(ia["img32"], ib["img32"])
    assert np.array_equal(ia["T32"], ib["T32"])


def test_sh_basis_orthonormal_and_axis_values():
    """P9: the real basis is orthonormal on the sphere (Gauss-Legendre x
    uniform quadrature) and along +-z only the m = 0 functions are non-zero."""
    ct, wt = np.polynomial.legendre.leggauss(24)
    ph = np.linspace(0, 2 * np.pi, 48, endpoint=False)
    CT, PH = np.meshgrid(ct, ph, indexing="ij")
    st = np.sqrt(1 - CT ** 2)
    dirs = np.stack([st * np.cos(PH), st * np.sin(PH), CT], -1).reshape(-1, 3)
    w = (wt[:, None] * np.full(48, 2 * np.pi / 48)[None, :]).reshape(-1)
    B = O.sh_basis(dirs, 3)
    G = (B * w[:, None]).T @ B
    assert np.abs(G - np.eye(16)).max() < 1e-12
    zb = O.sh_basis(np.array([[0, 0, 1.0], [0, 0, -1.0]]), 3)
    m0 = [0, 2, 6, 12]
    others = [k for k in range(16) if k not in m0]
    assert np.abs(zb[:, others]).max() < 1e-15
    assert np.all(np.abs(zb[:, m0]) > 0.2)


def test_sh_basis_matches_scipy_real_harmonics():
    import brute64
    rng = np.random.default_rng(9)
    d = rng.normal(size=(200, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    assert np.abs(O.sh_basis(d, 3) - brute64.real_sh_basis(d, 3)).max() < 1e-12


# ---------------------------------------------------------------------------
# Pairs, sort, ranges
# ---------------------------------------------------------------------------
def test_pairs_sort_and_ranges_against_numpy():
    """P8: the sorted list is numpy's stable argsort of the emitted keys;
    ranges partition [0, K); sum of tiles touched is K."""
    sc = S.tiny_scene(n=5000, seed=19)
    views = [S.tiny_view(1.0), S.tiny_view(3.0).replace(width=200, height=120, cx=100.0, cy=60.0)]
    fr = O.frame(sc, views, with64=False)
    keys = np.concatenate([O.emit_pairs(v, s1, b)[0] for v, s1, b in zip(views, fr["s1"], fr["tile_base"])])
    vals = np.concatenate([O.emit_pairs(v, s1, b)[1] for v, s1, b in zip(views, fr["s1"], fr["tile_base"])])
    order = np.argsort(keys, kind="stable")
    assert np.array_equal(fr["keys"], keys[order])
    assert np.array_equal(fr["vals"], vals[order])
    K = sum(int(s1["tiles"].sum()) for s1 in fr["s1"])
    assert K == len(keys)
    hi = (fr["keys"] >> np.uint64(32)).astype(np.int64)
    r = fr["ranges"].astype(np.int64)
    t = np.arange(fr["n_tiles"])
    lo_ = np.searchsorted(hi, t, "left")
    hi_ = np.searchsorted(hi, t, "right")
    nonempty = hi_ > lo_
    assert np.array_equal(r[nonempty, 0], lo_[nonempty])
    assert np.array_equal(r[nonempty, 1], hi_[nonempty])
    assert np.all(r[~nonempty] == 0)
    assert (r[:, 1] - r[:, 0]).sum() == K


def test_tile_lists_against_fp64_brute_force():
    """Pair emission, sort and ranges together against a brute force written
    without them: for every tile of two views (the second at a non-zero tile
    base), the oracle's sorted list equals the rendered Gaussians whose FP64
    3-sigma rectangle covers the tile, nearest first (FP64 camera depth, then
    index), each tile checked against every Gaussian.  A transposed tile
    index, a wrong view offset or a depth other than camera-space z each
    break it."""
    import brute64
    sc = S.tiny_scene(n=3000, seed=23)
    views = [S.tiny_view(1.0).replace(width=96, height=80, cx=48.0, cy=40.0),
             S.look_at((2.0, -1.5, 1.0), (0, 0, 0), 72, 56, s_v=3.0)]
    fr = O.frame(sc, views, with64=False)
    vals = fr["vals"].astype(np.int64)
    r = fr["ranges"].astype(np.int64)
    assert fr["tile_base"][1] > 0
    reordered = 0
    for vi, v in enumerate(views):
        lists, P = brute64.tile_lists_brute(sc, v)
        base = fr["tile_base"][vi]
        assert sum(len(x) for x in lists) > 3000 and max(len(x) for x in lists) > 100
        for t, want in enumerate(lists):
            got = [int(i) for i in vals[r[base + t, 0]:r[base + t, 1]]]
            assert got == want, (vi, t)
            reordered += got != sorted(got)       # depth order is not index order
    assert reordered > 10


# ---------------------------------------------------------------------------
# Independent FP64 brute force and the FP64 autograd statement
# ---------------------------------------------------------------------------
def test_oracle_matches_fp64_brute_force_tiny_scene():
    """P10: 200 Gaussians, 40x40: the oracle equals a naive FP64 renderer."""
    import brute64
    sc = S.small_scene(n=200, seed=3, sh_degree=3)
    for s, flags in ((1.0, 0), (2.0, 0), (1.0, O.LOD_OFF)):
        v = S.look_at((0.4, -1.8, 1.2), (0, 0, 0), 40, 40, s_v=s, flags=flags, bg=(0.2, 0.1, 0.0))
        s1 = O.stage1(sc, v)
        out = O.render(sc, v, s1, O.stage1_f64(sc, v, s1))
        img, Tf, nc = brute64.render_brute(sc, v)
        assert s1["survive"].sum() > 20
        assert np.abs(out["img64"] - img).max() < 1e-9
        assert np.abs(out["T64"] - Tf).max() < 1e-9
        assert np.array_equal(out["ncontrib"].astype(np.int64), nc)
        assert np.abs(out["img32"] - img).max() < 2e-5


def test_torch_fp64_statement_equals_c_fp64_image():
    from oracle import grad64 as G
    sc = S.tiny_scene(n=3000, seed=20, sh_degree=0)
    v = S.tiny_view(2.0).replace(width=96, height=80, cx=48.0, cy=40.0, bg=(0.3, 0.3, 0.3))
    fr, s1, img = G.frozen_from_oracle(sc, v)
    out = G.view_forward(G.params_f64(sc, requires_grad=False), v, fr)
    assert np.abs(out["image"].numpy() - img["img64"]).max() < 1e-9
    assert np.abs(out["T"].numpy() - img["T64"]).max() < 1e-12


def test_fp32_oracle_within_tolerance_of_fp64():
    sc = S.tiny_scene()
    v = S.tiny_view(1.0)
    s1 = O.stage1(sc, v)
    out = O.render(sc, v, s1, O.stage1_f64(sc, v, s1))
    assert np.abs(out["img32"] - out["img64"]).max() < 2e-4


def test_reference_gradients_match_central_differences():
    """P11: central FP64 differences with the discrete decisions frozen."""
    import torch
    from oracle import grad64 as G
    sc = S.small_scene(n=60, seed=3, sh_degree=2)
    v = S.look_at((0.4, -1.8, 1.2), (0, 0, 0), 32, 32, s_v=2.0, bg=(0.2, 0.1, 0.0))
    fr, s1, _ = G.frozen_from_oracle(sc, v)
    rng = np.random.default_rng(1)
    gimg = rng.normal(size=(3, 32, 32))
    galpha = rng.normal(size=sc.n) * 0.1
    grads = G.reference_gradients(sc, [v], [gimg], [galpha], frozen=[fr])

    def loss(P):
        out = G.view_forward(P, v, fr)
        return float((out["image"].detach().numpy() * gimg).sum() + (out["alpha_eff"].detach().numpy() * galpha).sum())

    P0 = G.params_f64(sc, requires_grad=False)
    live = np.nonzero(s1["survive"])[0]
    for name in ("means", "scales", "quats", "opacity", "sh", "decay"):
        flat = P0[name].reshape(-1)
        per = flat.numel() // sc.n
        idxs = [int(i) * per + j for i in live[:6] for j in range(min(per, 3))]
        for k in idxs:
            x0 = float(flat[k])
            h = 1e-6 * max(1.0, abs(x0))
            flat[k] = x0 + h
            lp = loss(P0)
            flat[k] = x0 - h
            lm = loss(P0)
            flat[k] = x0
            fd = (lp - lm) / (2 * h)
            g = grads[name].reshape(-1)[k]
            assert abs(fd - g) <= 1e-5 * max(1.0, abs(g)), (name, k, fd, g)


# ---------------------------------------------------------------------------
# Training objective scalars (Sec. 3.3, Eq. 3-5)
# ---------------------------------------------------------------------------
def test_sparse_reference_gradients_equal_full():
    """The sub-scene evaluation used at full size gives the same gradients
    as the whole-scene statement when the image gradient sits on a few tiles
    and the alpha'' gradient on a few Gaussians (the others are exactly zero)."""
    from oracle import grad64 as G
    sc = S.tiny_scene(n=3000, seed=41, sh_degree=2)
    views = [S.tiny_view(1.5).replace(width=96, height=80, cx=48.0, cy=40.0),
             S.look_at((2.0, 1.5, 1.0), (0, 0, 0), 64, 64, s_v=3.0, bg=(0.5, 0.5, 0.5))]
    rng = np.random.default_rng(8)
    gimgs, galphas, frozen_t, frozen_all = [], [], [], []
    for v in views:
        tx, ty = O.tiles_of(v)
        tiles = sorted(rng.choice(tx * ty, 5, replace=False).tolist())
        sel = np.zeros((v.height, v.width), bool)
        for t in tiles:
            sel[(t // tx) * 16:(t // tx) * 16 + 16, (t % tx) * 16:(t % tx) * 16 + 16] = True
        gimgs.append(rng.normal(size=(3, v.height, v.width)) * sel[None])
        ga = np.zeros(sc.n)
        ga[rng.choice(sc.n, 50, replace=False)] = rng.normal(size=50) * 1e-2
        galphas.append(ga)
        frozen_t.append(G.frozen_on_tiles(sc, v, tiles)[0])
        frozen_all.append(G.frozen_from_oracle(sc, v)[0])
    sparse = G.reference_gradients_sparse(sc, views, frozen_t, gimgs, galphas)
    full = G.reference_gradients(sc, views, gimgs, galphas, frozen=frozen_all)
    for k in full:
        assert np.linalg.norm(full[k]) > 0, k
        assert np.abs(sparse[k] - full[k]).max() <= 1e-12 * max(1.0, np.abs(full[k]).max()), k
    assert (np.abs(full["sh"]).sum(axis=(1, 2)) > 0).sum() < sc.n // 2      # sparse indeed


def test_loss_scalars_closed_forms():
    """P7, and the golden values in tests/golden/loss_scalars.txt."""
    assert L.eta_target(1.0) == 1.0
    assert L.l_reg(1.0, 0.9) == 0.0                       # no penalty at s_v = 1
    assert L.w_s(7.0, 7.0) == 0.25                        # farthest view weighted 1/4
    assert abs(L.w_s(1e-12, 7.0) - 1.0) < 1e-12
    assert L.l_reg(4.0, 0.1) == 0.0                       # below target: ReLU
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "loss_scalars.txt")
    for line in open(path):
        line = line.split("#")[0].strip()
        if not line:
            continue
        fn, *args, expect = line.split()
        args = [float(a) for a in args]
        got = getattr(L, fn)(*args)
        assert abs(got - float(expect)) <= 1e-12 * max(1.0, abs(float(expect))), (fn, args, got, expect)


def test_oracle_regression_fixture():
    """The oracle still produces the committed digests (tests/golden/make_golden.py)."""
    import hashlib
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "tiny_scene_oracle.json")
    want = json.load(open(path))
    sc = S.tiny_scene()
    for s in (1.0, 4.0):
        fr = O.frame(sc, [S.tiny_view(s)], with64=False)
        w = want["s=%g" % s]
        s1 = fr["s1"][0]
        assert int(s1["mask"].sum()) == w["mask"]
        assert int(len(fr["keys"])) == w["pairs"]
        assert hashlib.sha256(fr["keys"].tobytes()).hexdigest() == w["keys"]
        assert hashlib.sha256(fr["img"][0]["img32"].tobytes()).hexdigest() == w["img32"]


# ---------------------------------------------------------------------------
# D-SSIM term of L_render (Sec. 3.3)
# ---------------------------------------------------------------------------
def test_ssim_window_matches_scipy_gaussian_filter():
    """The 11x11 window (sigma 1.5, zero outside) is SciPy's Gaussian filter
    truncated at radius 5 with constant padding."""
    import scipy.ndimage
    from oracle import ssim as SS
    img = np.random.default_rng(60).uniform(size=(2, 23, 31))
    ref = np.stack([scipy.ndimage.gaussian_filter(c, SS.SIGMA, mode="constant", cval=0.0,
                                                  truncate=SS.RADIUS / SS.SIGMA) for c in img])
    assert np.abs(SS.blur(img) - ref).max() < 1e-14


def test_ssim_closed_forms():
    from oracle import ssim as SS
    rng = np.random.default_rng(61)
    x = rng.uniform(size=(3, 40, 40))
    assert abs(SS.ssim(x, x) - 1.0) < 1e-12
    # constant images: zero variance, so S = (2ab + C1) / (a^2 + b^2 + C1) away from the border
    a, b = 0.3, 0.7
    S = SS.ssim_map(np.full((1, 40, 40), a), np.full((1, 40, 40), b))
    assert abs(S[0, 20, 20] - (2 * a * b + SS.C1) / (a * a + b * b + SS.C1)) < 1e-12
    # SSIM is symmetric and below 1 for different images
    y = rng.uniform(size=(3, 40, 40))
    assert abs(SS.ssim(x, y) - SS.ssim(y, x)) < 1e-12 and SS.ssim(x, y) < 0.5


def test_render_loss_gradient_central_differences():
    from oracle import ssim as SS
    rng = np.random.default_rng(62)
    x = rng.uniform(size=(2, 14, 17))
    y = rng.uniform(size=(2, 14, 17))
    v, g = SS.render_loss_grad(x, y)
    assert abs(v - SS.render_loss(x, y)) < 1e-12
    for idx in [(0, 0, 0), (1, 7, 8), (0, 13, 16), (1, 3, 12)]:
        h = 1e-6
        xp = x.copy(); xp[idx] += h
        xm = x.copy(); xm[idx] -= h
        fd = (SS.render_loss(xp, y) - SS.render_loss(xm, y)) / (2 * h)
        assert abs(fd - g[idx]) < 1e-6, (idx, fd, g[idx])


# ---------------------------------------------------------------------------
# Primitive budget (Sec. 4.2: keep the primitives of highest alpha'')
# ---------------------------------------------------------------------------
def test_budget_threshold_equivalence():
    """The threshold mask alpha'' > tau s_v keeps exactly the top-|M| set by
    alpha'' (every kept alpha'' exceeds every dropped one), so a budget equal
    to |M| reproduces Stage I bit for bit."""
    sc = S.tiny_scene(n=5000, seed=70)
    for s in (2.0, 6.0):
        thr = O.stage1(sc, S.tiny_view(s))
        B = int(thr["mask"].sum())
        assert 0 < B < sc.n
        bud = O.stage1(sc, S.tiny_view(s, budget=B))
        for k in ("alpha_eff", "mask", "survive", "rec", "rect", "tiles"):
            assert np.array_equal(thr[k], bud[k]), k


def test_budget_selects_top_alpha_by_brute_force():
    """Exactly min(B, n) Gaussians kept: the first B of (alpha'' descending,
    index ascending), checked against a NumPy lexicographic order."""
    sc = S.tiny_scene(n=3000, seed=71)
    for B in (1, 17, 1000, 2999, 3000, 5000):
        s1 = O.stage1(sc, S.tiny_view(3.0, budget=B))
        order = np.lexsort((np.arange(sc.n), -s1["alpha_eff"].astype(np.float64)))
        ref = np.zeros(sc.n, np.uint8)
        ref[order[:B]] = 1
        assert np.array_equal(s1["mask"], ref), B
        assert int(s1["mask"].sum()) == min(B, sc.n)


def test_budget_ties_go_to_lower_indices():
    """Equal alpha'' (level of detail off, one opacity for all): the budget keeps
    the lowest indices."""
    sc = S.tiny_scene(n=2000, seed=72)
    sc = S.Scene(sc.means, sc.scales, sc.quats, np.full(sc.n, 0.5, np.float32), sc.sh, sc.decay)
    s1 = O.stage1(sc, S.tiny_view(4.0, flags=O.LOD_OFF, budget=123))
    assert np.array_equal(np.flatnonzero(s1["mask"]), np.arange(123))
    # mixed: two opacity levels, ties inside each level by index
    op = np.where(np.arange(sc.n) % 3 == 0, 0.9, 0.5).astype(np.float32)
    sc2 = S.Scene(sc.means, sc.scales, sc.quats, op, sc.sh, sc.decay)
    s2 = O.stage1(sc2, S.tiny_view(4.0, flags=O.LOD_OFF, budget=800))
    hi = np.flatnonzero(op == np.float32(0.9))
    lo = np.flatnonzero(op == np.float32(0.5))
    assert np.array_equal(np.flatnonzero(s2["mask"]), np.sort(np.concatenate([hi, lo[:800 - hi.size]])))
