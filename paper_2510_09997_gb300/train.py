"""Virtual-distance-scaling training step of CLoD-GS (Sec. 3.3).

Per view a virtual scale s_v is drawn (log-uniform on [1, s_max] by default;
the paper's example is uniform on [1, 10]), the view is rendered with that
s_v, and the objective is

    L_total = w_s (L_render + lambda_reg L_reg)                     (Eq. 5)
    w_s     = (1 - 0.5 s_v / s_max)^2
    L_reg   = (s_v - 1)^2 ReLU(eta_actual - eta_target)^2           (Eq. 4)
    eta_target = s_v^-1.5                                            (Eq. 3)
    eta_actual = sum_i M_i / N_total

L_render = (1 - w) L1 + w D-SSIM (the clod_render_loss kernel; w = 0.2 as in
the 3DGS training the paper builds on; w = 0 gives L1 alone).  eta_actual is a
count of the binary mask; its gradient is taken straight through,
dM_i/dalpha''_i := 1, so every alpha'' receives 2 w_s lambda (s_v - 1)^2
ReLU(eta_a - eta_t) / N and the rasterizer's backward carries it on to alpha,
sigma_d and the means.  Parameters are kept raw (log-scales, opacity logits)
and activated with exp / sigmoid before the rasterizer; Adam updates them,
sigma_d with learning rate 1e-2 and lambda_reg = 1 (Sec. 4.1).
"""
from __future__ import annotations

import math
from typing import List, Optional, Sequence

import numpy as np
import torch

from . import autograd as A


def eta_target(s_v: float) -> float:
    return s_v ** -1.5


def w_s(s_v: float, s_max: float) -> float:
    return (1.0 - 0.5 * s_v / s_max) ** 2


class GaussianModel(torch.nn.Module):
    def __init__(self, scene, device="cuda"):
        super().__init__()
        f = lambda a: torch.nn.Parameter(torch.tensor(np.asarray(a, np.float32), device=device))
        self.means = f(scene.means)
        self.log_scales = f(np.log(scene.scales))
        self.quats = f(scene.quats)
        op = np.clip(scene.opacity, 1e-6, 1 - 1e-6)
        self.opacity_logit = f(np.log(op / (1 - op)))
        self.sh = f(scene.sh)
        self.decay = f(scene.decay)

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    def activated(self):
        return (self.means, torch.exp(self.log_scales), self.quats, torch.sigmoid(self.opacity_logit),
                self.sh, self.decay)

    def optimizer(self, extent: float = 1.0):
        groups = [
            {"params": [self.means], "lr": 1.6e-4 * extent},
            {"params": [self.log_scales], "lr": 5e-3},
            {"params": [self.quats], "lr": 1e-3},
            {"params": [self.opacity_logit], "lr": 5e-2},
            {"params": [self.sh], "lr": 2.5e-3},
            {"params": [self.decay], "lr": 1e-2},
        ]
        return torch.optim.Adam(groups, eps=1e-15, fused=True)


class TrainStep:
    """One optimisation step over a batch of views."""

    def __init__(self, model: GaussianModel, s_max: float = 16.0, lam_reg: float = 1.0, sampler: str = "log",
                 seed: int = 0, extent: float = 1.0, dssim_weight: float = 0.2):
        self.model = model
        self.dssim = float(dssim_weight)
        self.s_max = float(s_max)
        self.lam = float(lam_reg)
        self.sampler = sampler
        self.rng = np.random.default_rng(seed)
        self.opt = model.optimizer(extent)

    def sample_scale(self) -> float:
        if self.s_max <= 1.0:
            return 1.0
        if self.sampler == "uniform":
            s = self.rng.uniform(1.0, self.s_max)
        else:
            s = math.exp(self.rng.uniform(0.0, math.log(self.s_max)))
        return float(np.float32(s))

    def loss(self, views: Sequence, targets: Sequence[torch.Tensor], scales: Optional[List[float]] = None):
        """Returns (L_total, per-view diagnostics)."""
        if scales is None:
            scales = [self.sample_scale() for _ in views]
        views = [v.replace(s_v=s) for v, s in zip(views, scales)]
        imgs, alpha, mask, counts = A.render(*self.model.activated(), views)
        self.last = dict(images=imgs, alpha=alpha, views=views)
        N = self.model.n
        total = 0.0
        info = []
        cnt = counts.detach().cpu().numpy()
        for k, (v, s) in enumerate(zip(views, scales)):
            l1 = (A.RenderLoss.apply(imgs[k], targets[k], self.dssim) if self.dssim > 0
                  else A.L1Loss.apply(imgs[k], targets[k]))
            eta_a_count = float(cnt[k, 0]) / N
            # straight-through estimator: value of the count, gradient of sum alpha'' / N
            a_sum = alpha[k].sum()
            eta_a = eta_a_count + (a_sum - a_sum.detach()) / N
            relu = torch.relu(eta_a - eta_target(s))
            l_reg = (s - 1.0) ** 2 * relu * relu
            ws = w_s(s, self.s_max)
            total = total + ws * (l1 + self.lam * l_reg)
            info.append(dict(s_v=s, l_render=float(l1.detach()), l1=float(l1.detach()), l_reg=float(l_reg.detach()), eta_actual=eta_a_count,
                             eta_target=eta_target(s), w_s=ws, rendered=int(cnt[k, 1])))
        return total / len(views), info

    def step(self, views: Sequence, targets: Sequence[torch.Tensor], scales: Optional[List[float]] = None):
        self.opt.zero_grad(set_to_none=True)
        total, info = self.loss(views, targets, scales)
        total.backward()
        self.opt.step()
        return float(total.detach()), info
