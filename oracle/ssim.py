"""FP64 reference of the D-SSIM term of the rendering loss (Sec. 3.3:
L_render is a weighted sum of L1 and D-SSIM).

TEST INFRASTRUCTURE ONLY (see ``clod_oracle.c``).

SSIM (structural similarity) per pixel and channel, with local statistics from
an 11 x 11 Gaussian window (sigma 1.5, normalised, zero outside the image):

    mu_x = w * x, mu_y = w * y,
    s_xx = w * x^2 - mu_x^2, s_yy = w * y^2 - mu_y^2, s_xy = w * (x y) - mu_x mu_y,
    S = (2 mu_x mu_y + C1)(2 s_xy + C2) / ((mu_x^2 + mu_y^2 + C1)(s_xx + s_yy + C2)),

C1 = 0.01^2, C2 = 0.03^2 (dynamic range 1); SSIM = mean of S over pixels and
channels; D-SSIM = 1 - SSIM.  The loss weight lambda = 0.2 of
L_render = (1 - lambda) L1 + lambda D-SSIM is the 3DGS setting the paper's
training builds on (its own weights are not stated).
"""
from __future__ import annotations

import math

import numpy as np
import torch

C1 = 0.01 ** 2
C2 = 0.03 ** 2
RADIUS = 5
SIGMA = 1.5
LAMBDA_DSSIM = 0.2


def window_1d() -> np.ndarray:
    x = np.arange(-RADIUS, RADIUS + 1, dtype=np.float64)
    g = np.exp(-x * x / (2.0 * SIGMA * SIGMA))
    return g / g.sum()


def blur(img: np.ndarray) -> np.ndarray:
    """Separable window, zero padding, same size.  img: (..., H, W) float64."""
    g = window_1d()
    H, W = img.shape[-2:]
    p = np.zeros(img.shape[:-2] + (H + 2 * RADIUS, W + 2 * RADIUS))
    p[..., RADIUS:RADIUS + H, RADIUS:RADIUS + W] = img
    rows = sum(g[k] * p[..., :, k:k + W] for k in range(2 * RADIUS + 1))
    return sum(g[k] * rows[..., k:k + H, :] for k in range(2 * RADIUS + 1))


def ssim_map(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    mx, my = blur(x), blur(y)
    sxx = blur(x * x) - mx * mx
    syy = blur(y * y) - my * my
    sxy = blur(x * y) - mx * my
    return ((2 * mx * my + C1) * (2 * sxy + C2)) / ((mx * mx + my * my + C1) * (sxx + syy + C2))


def ssim(x, y) -> float:
    return float(ssim_map(x, y).mean())


def render_loss(x, y, lam: float = LAMBDA_DSSIM) -> float:
    """(1 - lambda) mean |x - y| + lambda (1 - SSIM)."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    return (1.0 - lam) * float(np.abs(x - y).mean()) + lam * (1.0 - ssim(x, y))


def _blur_t(t: torch.Tensor) -> torch.Tensor:
    g = torch.tensor(window_1d(), dtype=torch.float64)
    k = (g[:, None] * g[None, :])[None, None]
    C = t.shape[0]
    return torch.nn.functional.conv2d(t[:, None], k, padding=RADIUS).reshape(C, *t.shape[1:])


def render_loss_grad(x, y, lam: float = LAMBDA_DSSIM):
    """Value and gradient with respect to x of render_loss (FP64 autograd of the
    same formulas; the L1 subgradient is sign(x - y))."""
    xt = torch.tensor(np.asarray(x, np.float64), requires_grad=True)
    yt = torch.tensor(np.asarray(y, np.float64))
    mx, my = _blur_t(xt), _blur_t(yt)
    sxx = _blur_t(xt * xt) - mx * mx
    syy = _blur_t(yt * yt) - my * my
    sxy = _blur_t(xt * yt) - mx * my
    S = ((2 * mx * my + C1) * (2 * sxy + C2)) / ((mx * mx + my * my + C1) * (sxx + syy + C2))
    loss = (1.0 - lam) * (xt - yt).abs().mean() + lam * (1.0 - S.mean())
    loss.backward()
    return float(loss), xt.grad.numpy()
