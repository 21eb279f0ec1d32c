"""Pins of the oracle's Stage II with FP64 decisions (CPU only).

Eq. 1 (Sec. 3.1) is stated in real arithmetic, so its three per-pixel
decisions (positive power, opacity below 1/255, transmittance below 1e-4)
are decisions on real values.  ``oracle.render_f64dec`` takes them in FP64,
flags those within a band of their thresholds and follows both outcomes.
These tests fix its main path against an independent naive FP64 renderer,
its flags against closed-form threshold crossings, and show that the check
it feeds (``branches.match_fp64_branches``) accepts the FP32 specification's
image and rejects images with plausible decision mistakes planted in a
throw-away copy of the oracle.
"""
import ctypes
import math
import os
import subprocess

import numpy as np
import pytest

from oracle import oracle as O
from paper_2510_09997_gb300 import synth as S

from branches import match_fp64_branches

SH_C0 = 1.0 / (2.0 * math.sqrt(math.pi))   # Y_0^0 of the real SH basis


def axis_view(W=64, H=64, f=200.0, **kw):
    """Camera at the origin looking along +z; principal point on a pixel
    centre, so a Gaussian on the axis projects onto pixel (W/2, H/2)."""
    vm = np.zeros((3, 4), np.float32)
    vm[:, :3] = np.eye(3)
    return S.View(width=W, height=H, viewmat=vm, fx=f, fy=f, cx=W / 2 + 0.5, cy=H / 2 + 0.5,
                  campos=np.zeros(3, np.float32), **kw)


def gaussians(k, mu=(0.0, 0.0, 2.0), scale=0.02, opacity=0.5, fdcs=None):
    fdcs = np.zeros((k, 3)) if fdcs is None else fdcs
    sh = np.zeros((k, 1, 3), np.float32)
    sh[:, 0] = fdcs
    return S.Scene(np.tile(np.array(mu, np.float32), (k, 1)), np.full((k, 3), scale, np.float32),
                   np.tile(np.array([1, 0, 0, 0], np.float32), (k, 1)), np.full(k, opacity, np.float32), sh,
                   np.ones(k, np.float32))


def passes(scene, view):
    s1 = O.stage1(scene, view)
    r64 = O.stage1_f64(scene, view, s1)
    return s1, r64, O.render(scene, view, s1, r64), O.render_f64dec(view, s1, r64)


def outcomes(dec, y, x, W):
    """All (r, g, b, T, n_contrib) outcomes of pixel (y, x): main path first."""
    out = [tuple(dec["img"][:, y, x]) + (dec["T"][y, x], int(dec["ncontrib"][y, x]))]
    for k in np.nonzero(dec["alt_pix"] == y * W + x)[0]:
        out.append(tuple(dec["alt_val"][k]) + (int(dec["alt_nc"][k]),))
    return out


def test_main_path_matches_fp64_brute_force():
    """The main path (every decision in FP64) equals a naive FP64 renderer
    written without sorting or tiles, to 1e-9, with the same contributor
    counts (P10's scenes)."""
    import brute64
    sc = S.small_scene(n=200, seed=3, sh_degree=3)
    for s, flags in ((1.0, 0), (2.0, 0), (1.0, O.LOD_OFF)):
        v = S.look_at((0.4, -1.8, 1.2), (0, 0, 0), 40, 40, s_v=s, flags=flags, bg=(0.2, 0.1, 0.0))
        s1 = O.stage1(sc, v)
        dec = O.render_f64dec(v, s1, O.stage1_f64(sc, v, s1))
        img, Tf, nc = brute64.render_brute(sc, v)
        assert s1["survive"].sum() > 20
        assert np.abs(dec["img"] - img).max() < 1e-9
        assert np.abs(dec["T"] - Tf).max() < 1e-9
        assert np.array_equal(dec["ncontrib"].astype(np.int64), nc)


@pytest.mark.parametrize("side", [1.0 + 1e-7, 1.0 - 1e-7])
def test_opacity_threshold_is_flagged_and_both_outcomes_follow(side):
    """A lone Gaussian whose opacity at four pixels (three pixels from its
    centre) is 1/255 to within 1e-7: exactly those four pixels are flagged, and
    their two outcomes are the contribution alpha rgb + (1 - alpha) bg and
    the background alone; the main path is the side of 1/255 the FP64 value
    lies on.  A value 1e-3 away from the threshold is not flagged."""
    v = axis_view(flags=O.LOD_OFF, bg=(0.25, 0.5, 0.75))
    sc = gaussians(1, fdcs=np.array([[0.4, -0.2, 0.1]]))
    s1 = O.stage1(sc, v)
    r64 = O.stage1_f64(sc, v, s1)
    A, B, C = r64[0, 3:6]
    assert abs(B) < 1e-12 and abs(A - C) < 1e-12 * A
    p = -0.5 * A * 9.0                                  # dx = 3, dy = 0
    sc.opacity[0] = np.float32(side / 255.0 / math.exp(p))
    s1, r64, _, dec = passes(sc, v)
    a = r64[0, 2] * math.exp(-0.5 * r64[0, 3] * 9.0)
    assert abs(a * 255.0 - 1.0) < 1e-6
    flagged = np.argwhere(dec["n_paths"] > 1)
    assert sorted(map(tuple, flagged)) == [(29, 32), (32, 29), (32, 35), (35, 32)]
    rgb = SH_C0 * np.float32(sc.sh[0, 0]).astype(np.float64) + 0.5
    bg = np.asarray(v.bg, np.float32).astype(np.float64)
    for y, x in flagged:
        outs = outcomes(dec, y, x, v.width)
        assert len(outs) == 2
        contrib = [o for o in outs if o[4] == 1][0]
        skipped = [o for o in outs if o[4] == 0][0]
        assert np.abs(np.array(contrib[:3]) - (rgb * a + (1 - a) * bg)).max() < 1e-12
        assert abs(contrib[3] - (1 - a)) < 1e-15
        assert np.abs(np.array(skipped[:3]) - bg).max() == 0.0 and skipped[3] == 1.0
        assert outs[0][4] == (1 if a >= 1 / 255 else 0)
    sc.opacity[0] = np.float32(1.001 / 255.0 / math.exp(p))
    _, _, _, dec = passes(sc, v)
    assert dec["n_paths"].max() == 1 and dec["alt_pix"].size == 0


def test_stop_threshold_is_flagged_and_both_outcomes_follow():
    """P2 at the stop: 14 co-located Gaussians of opacity a at a pixel
    centre with (1 - a)^10 = 1e-4 (to float rounding of a).  The tenth layer
    is flagged; one outcome stops before it (9 contributors), the other takes
    it and stops before the eleventh (10), each with the closed-form colour
    sum_k c_k a (1 - a)^k."""
    n = 14
    a = 1.0 - 1e-4 ** (1.0 / 10.0)
    rng = np.random.default_rng(7)
    fdcs = rng.uniform(-1, 1, size=(n, 3))
    sc = gaussians(n, opacity=a, fdcs=fdcs)
    v = axis_view(flags=O.LOD_OFF)
    s1, r64, ref, dec = passes(sc, v)
    y = x = 32
    a32 = float(np.float32(a))
    assert abs(r64[0, 2] - a32) == 0.0
    outs = outcomes(dec, y, x, v.width)
    assert len(outs) == 2 and sorted(o[4] for o in outs) == [9, 10]
    cols = SH_C0 * fdcs.astype(np.float32).astype(np.float64) + 0.5
    for o in outs:
        k = o[4]
        want = sum(cols[j] * a32 * (1 - a32) ** j for j in range(k))
        assert np.abs(np.array(o[:3]) - want).max() < 1e-12
        assert abs(o[3] - (1 - a32) ** k) < 1e-15
    # the FP32 specification takes one of them
    m = match_fp64_branches(ref["img32"], ref["T32"], ref["ncontrib"], dec)
    assert m["bad"] == 0 and m["nc_differs"] == 0 and m["flagged"] >= 1


@pytest.mark.parametrize("s", [1.0, 4.0])
def test_fp32_specification_is_an_accepted_branch(s):
    """The FP32 specification's image (the one the GPU reproduces bit for
    bit) lies within 2e-4 of an FP64-decision outcome at every pixel of the
    20,000-Gaussian scene, with that outcome's contributor count; few pixels
    are flagged."""
    sc = S.tiny_scene()
    v = S.tiny_view(s)
    s1, r64, ref, dec = passes(sc, v)
    m = match_fp64_branches(ref["img32"], ref["T32"], ref["ncontrib"], dec)
    print("flagged pixels", m)
    assert m["bad"] == 0 and m["nc_differs"] == 0 and m["capped"] == 0
    assert m["flagged"] < 0.01 * m["pixels"]


PLANTS = {
    # skip threshold 1/256 instead of 1/255
    "skip_256": ("const float one255 = 1.0f / 255.0f;", "const float one255 = 1.0f / 256.0f;"),
    # the stopping Gaussian is blended before the stop
    "stop_includes": ("if (tt < 1e-4f) break;\n                    float wgt = a * T;",
                      "float wgt = a * T;\n                    if (tt < 1e-4f) { C0 = fmaf(R[8], wgt, C0); "
                      "C1 = fmaf(R[9], wgt, C1); C2 = fmaf(R[10], wgt, C2); T = tt; break; }"),
    # stop threshold 1e-3 instead of 1e-4
    "stop_1e-3": ("if (tt < 1e-4f) break;", "if (tt < 1e-3f) break;"),
}


@pytest.mark.parametrize("plant", sorted(PLANTS))
def test_planted_decision_mistakes_are_rejected(plant, tmp_path, monkeypatch):
    """A decision mistake planted in the FP32 evaluation of a throw-away copy
    of the oracle -- the kind of mistake a kernel that copies that evaluation
    would share -- makes pixels fall outside every FP64-decision outcome."""
    old, new = PLANTS[plant]
    src = open(O.SRC).read()
    assert src.count(old) == 1
    path = tmp_path / "planted.c"
    path.write_text(src.replace(old, new))
    so = str(tmp_path / "planted.so")
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                           "-o", so, str(path), "-lm"])
    sc = S.tiny_scene(n=8000, seed=31)
    sc.opacity[:] = np.maximum(sc.opacity, np.float32(0.9))    # opaque enough that pixels reach the stop
    sc.scales *= np.float32(2.0)
    v = S.tiny_view(1.0).replace(width=128, height=128, cx=64.0, cy=64.0)
    s1, r64, ref, dec = passes(sc, v)
    assert (ref["T32"] < 2e-4).mean() > 0.5
    assert match_fp64_branches(ref["img32"], ref["T32"], ref["ncontrib"], dec)["bad"] == 0
    monkeypatch.setattr(O, "_lib", O.bind(ctypes.CDLL(os.path.abspath(so))))
    bad = O.render(sc, v, s1, r64)
    m = match_fp64_branches(bad["img32"], bad["T32"], bad["ncontrib"], dec)
    assert m["bad"] > 0, m
