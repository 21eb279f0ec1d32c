"""The blends skip the exponential for powers below a Gaussian's floor,
max(-5.6, -(1.001 ln(255 alpha'') + 1e-3)) (the preprocessing stores it with
the record).  The skip is exact only if every skipped power has opacity
alpha'' exp_spec(power) < 1/255 in FP32; this checks that claim against the
oracle's exp_spec on the powers just below the floor, for alpha'' spread over
[1/255, 1] (logf here is numpy's float32 log; the floor's margin is four
orders of magnitude above either log's error)."""
import numpy as np

from oracle import oracle as O

ONE255 = np.float32(1.0) / np.float32(255.0)


def _floor(a2):
    a255 = np.float32(255.0) * a2
    f = -(np.log(a255).astype(np.float32) * np.float32(1.001) + np.float32(1e-3))
    return np.maximum(np.float32(-5.6), f.astype(np.float32))


def test_powers_below_the_floor_have_opacity_below_1_over_255():
    O.build()
    rng = np.random.default_rng(0)
    a2 = np.concatenate([[np.float32(1.0 / 255.0) * np.float32(1.0000001)],
                         rng.uniform(1.0 / 255.0, 1.0, 20000),
                         np.geomspace(1.0 / 255.0, 1.0, 2000), [1.0]]).astype(np.float32)
    a2 = a2[255.0 * a2.astype(np.float64) >= 1.0]
    pf = _floor(a2)
    # the float just below the floor, and a spread of powers further below
    below = [np.nextafter(pf, np.float32(-np.inf))]
    for dlt in (1e-6, 1e-4, 1e-2, 0.3):
        below.append((pf - np.float32(dlt)).astype(np.float32))
    for p in below:
        g = O.exp_spec(p.astype(np.float32)).astype(np.float32)
        al = np.minimum(np.float32(0.99), (a2 * g).astype(np.float32))
        assert np.all(al < ONE255), (a2[al >= ONE255][:5], p[al >= ONE255][:5])


def test_floor_is_tight_enough_to_matter():
    """Not vacuous: just above the exact threshold -ln(255 alpha'') the
    opacity reaches 1/255, and the floor lies within 0.1 % + 1e-3 of it."""
    O.build()
    a2 = np.geomspace(0.01, 1.0, 200).astype(np.float32)
    thr = -np.log(255.0 * a2.astype(np.float64))
    p = (thr + 1e-3).astype(np.float32)
    g = O.exp_spec(p).astype(np.float32)
    assert np.all((a2 * g).astype(np.float32) >= ONE255)
    pf = _floor(a2).astype(np.float64)
    assert np.all(thr - pf <= 1.001e-3 * np.abs(thr) + 1.01e-3 + 1e-6)


def _reach(nA, nB, nC, a2):
    """The preprocessing's reach half-extents (float32 steps as in the kernel)."""
    f = np.float32
    A, B, C = f(-2.0) * nA, -nB, f(-2.0) * nC
    det = A * C - B * B
    a255 = f(255.0) * a2
    P = np.minimum(f(5.6), np.log(a255).astype(f))
    r2 = f(2.0) * P * f(1.001) + f(1e-3)
    ex = np.sqrt(r2 * (C / det)).astype(f) * f(1.001) + f(0.01)
    ey = np.sqrt(r2 * (A / det)).astype(f) * f(1.001) + f(0.01)
    return ex, ey


def test_pixels_outside_the_reach_box_stay_below_1_over_255():
    """A warp skips list entries whose reach box misses its patch: every pixel
    outside the box must have power out of range or opacity < 1/255."""
    O.build()
    f = np.float32
    rng = np.random.default_rng(2)
    m = 20000
    # conics of Gaussians a few pixels to ~100 pixels wide, up to 10:1 anisotropy
    sx = rng.uniform(0.7, 40.0, m)
    sy = sx * rng.uniform(0.1, 1.0, m)
    th = rng.uniform(0, np.pi, m)
    c, s = np.cos(th), np.sin(th)
    cxx = c * c * sx * sx + s * s * sy * sy + 0.3
    cyy = s * s * sx * sx + c * c * sy * sy + 0.3
    cxy = c * s * (sx * sx - sy * sy)
    det = cxx * cyy - cxy * cxy
    A, B, C = (cyy / det).astype(f), (-cxy / det).astype(f), (cxx / det).astype(f)
    nA, nB, nC = f(-0.5) * A, -B, f(-0.5) * C
    a2 = rng.uniform(1.0 / 255.0, 1.0, m).astype(f)
    ex, ey = _reach(nA, nB, nC, a2)
    # points just outside the box: on each side, at random positions along it
    for side in range(4):
        t = rng.uniform(-1.0, 1.0, m).astype(f)
        if side < 2:
            dx = (ex * f(1.0 + 1e-6) + f(1e-4)) * f(1 if side == 0 else -1)
            dy = t * ey
        else:
            dy = (ey * f(1.0 + 1e-6) + f(1e-4)) * f(1 if side == 2 else -1)
            dx = t * ex
        dx, dy = dx.astype(f), dy.astype(f)
        p = (dx * (nA * dx + nB * dy) + (nC * dy) * dy).astype(f)
        inr = (p <= 0) & (p >= f(-5.6))
        g = O.exp_spec(np.where(inr, p, f(0)).astype(f)).astype(f)
        al = np.minimum(f(0.99), (a2 * g).astype(f))
        assert np.all(~inr | (al < ONE255))
        # not vacuous: many such points are in range, some close to 1/255
        assert inr.mean() > 0.2 and al[inr].max() > f(0.9) * ONE255
