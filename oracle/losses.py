"""FP64 reference for the virtual-distance training objective (Sec. 3.3).

TEST INFRASTRUCTURE ONLY (see ``clod_oracle.c``).  Plain Python floats.
"""
from __future__ import annotations

import math


def eta_target(s_v: float) -> float:
    """Target primitive ratio, Eq. 3: 1 / s_v^1.5."""
    return 1.0 / (s_v ** 1.5)


def eta_actual(n_rendered: int, n_total: int) -> float:
    """Ratio of rendered primitives, sum_i M_i / N_total (Sec. 3.3)."""
    return n_rendered / n_total


def l_reg(s_v: float, eta_act: float) -> float:
    """Point-count regularisation, Eq. 4: (s_v - 1)^2 ReLU(eta_actual - eta_target)^2."""
    return (s_v - 1.0) ** 2 * max(eta_act - eta_target(s_v), 0.0) ** 2


def w_s(s_v: float, s_max: float) -> float:
    """Scale weight of Eq. 5: (1 - 0.5 s_v / max(s_v))^2."""
    return (1.0 - 0.5 * s_v / s_max) ** 2


def l_total(s_v: float, s_max: float, l_render: float, eta_act: float, lam: float = 1.0) -> float:
    """Eq. 5: w_s (L_render + lambda_reg L_reg)."""
    return w_s(s_v, s_max) * (l_render + lam * l_reg(s_v, eta_act))


def dlreg_dalpha_ste(s_v: float, eta_act: float, n_total: int) -> float:
    """Straight-through derivative of L_reg with respect to each alpha''_i when
    dM_i/dalpha''_i is read as 1: 2 (s_v-1)^2 ReLU(eta_a - eta_t) / N_total."""
    return 2.0 * (s_v - 1.0) ** 2 * max(eta_act - eta_target(s_v), 0.0) / n_total


def l1(img, target) -> float:
    """Mean absolute error over all pixels and channels (the L1 term of L_render)."""
    n = 0
    acc = 0.0
    for a, b in zip(img.reshape(-1).tolist(), target.reshape(-1).tolist()):
        acc += abs(a - b)
        n += 1
    return acc / max(n, 1)
