"""Direction of the point-count regularisation under its straight-through
gradient (Sec. 3.3, Eq. 3-4).

Plain gradient descent on L_reg alone: the oracle's Stage I gives the count
(eta_actual = sum M_i / N), the straight-through derivative
dL_reg/dalpha''_i = 2 (s_v - 1)^2 ReLU(eta_actual - eta_target) / N goes to
every Gaussian, and the oracle's FP64 chain rule carries it to the opacity
(through its logit) and to the decay sigma_d.  The regulariser must lower the
count toward eta_target = s_v^-1.5 and leave every parameter unchanged once
the count is at or below it (the ReLU).  A flipped sign in the
straight-through derivative, planted here in the oracle's numbers, raises
the count instead, so the checks are not vacuous.
"""
import dataclasses

import numpy as np

from oracle import grad64 as G
from oracle import losses as L
from oracle import oracle as O
from paper_2510_09997_gb300 import synth as S

S_V = 4.0
W = H = 64


def _setup():
    sc = S.tiny_scene(n=3000, seed=5, sh_degree=0)
    v = S.look_at((0.0, 0.0, 3.0), (0.0, 0.0, 0.0), W, H, up=(0.0, 1.0, 0.0), s_v=S_V)
    return sc, v


def _eta(sc, v):
    return L.eta_actual(int(O.stage1(sc, v)["mask"].sum()), sc.n)


def _step(sc, v, lr, sign=1.0):
    """One descent step on L_reg; returns the new scene and the eta_actual
    and straight-through derivative the step used."""
    eta = _eta(sc, v)
    g = sign * L.dlreg_dalpha_ste(S_V, eta, sc.n)
    gr = G.reference_gradients(sc, [v], [np.zeros((3, H, W))], [np.full(sc.n, g)])
    a = sc.opacity.astype(np.float64)
    logit = np.log(a / (1.0 - a)) - lr * gr["opacity"] * a * (1.0 - a)
    dec = sc.decay.astype(np.float64) - lr * gr["decay"]
    new = dataclasses.replace(sc, opacity=(1.0 / (1.0 + np.exp(-logit))).astype(np.float32),
                              decay=dec.astype(np.float32))
    return new, eta, g


def test_lreg_lowers_count_toward_target():
    sc, v = _setup()
    target = L.eta_target(S_V)
    etas, regs = [], []
    for _ in range(10):
        sc, eta, _ = _step(sc, v, lr=1e3)
        etas.append(eta)
        regs.append(L.l_reg(S_V, eta))
    etas.append(_eta(sc, v))
    assert etas[0] > 3 * target            # starts well above the target
    # monotone toward the target from above, and close to it after 10 steps
    assert all(b < a for a, b in zip(etas, etas[1:]) if a > target + 0.002)
    assert all(b <= a for a, b in zip(regs, regs[1:]))
    assert target <= etas[-1] <= target + 0.005


def test_lreg_stops_below_target():
    sc, v = _setup()
    target = L.eta_target(S_V)
    sc, eta0, g0 = _step(sc, v, lr=4e3)     # a step large enough to overshoot
    assert eta0 > target and g0 > 0.0
    eta1 = _eta(sc, v)
    assert eta1 < target
    # below the target the ReLU gives exactly zero: nothing moves any more
    sc2, eta, g = _step(sc, v, lr=4e3)
    assert eta == eta1 and g == 0.0
    assert np.array_equal(sc2.opacity, sc.opacity) and np.array_equal(sc2.decay, sc.decay)


def test_flipped_straight_through_sign_raises_count():
    sc, v = _setup()
    eta0 = _eta(sc, v)
    for _ in range(3):
        sc, _, g = _step(sc, v, lr=1e3, sign=-1.0)
        assert g < 0.0
    assert _eta(sc, v) > eta0 + 0.05
