"""Seeded synthetic scenes and cameras shaped like the CLoD-GS workloads.

This module only draws random inputs and builds camera poses.  It contains none
of the rasterizer's or the level-of-detail method's arithmetic, so both the CUDA
path and the CPU oracle can take their inputs from it.

Parameters are returned *activated*, the way the C-ABI takes them: opacity in
(0, 1), scales > 0, quaternions of any norm (w, x, y, z), raw decay sigma_d.
SH coefficients are stored per Gaussian as (deg+1)^2 rows of RGB.

Scene recipes (all numpy ``default_rng(seed)``):

* ``tiny``   -- 20,000 Gaussians, means U[-1,1]^3, log-scales N(-4, 0.5),
  quaternions N(0, I4) (uniform rotations once normalised), opacity
  sigmoid(N(0,1)), SH degree 0 with the DC coefficient U[-sqrt(pi), sqrt(pi)]
  (the band-0 basis constant maps that to colour U[0,1]), decay U[0, 2].
* ``object`` -- 1M Gaussians, 90% from four isotropic blobs (centres U[-1,1]^3,
  sigma 0.25) plus 10% uniform in [-1.5,1.5]^3, SH degree 3 with bands 1-3
  N(0, 0.05); other attributes as ``tiny``.
* ``outdoor`` -- the ``object`` mixture stretched over a 10 x 10 x 4 box with
  blob sigma 1.0 (training-step scene).
* ``city``   -- 80% of the points on 64 random planes (10 x 10 patches, normal
  offset N(0, 0.02)) plus 20% uniform in a 100 x 100 x 30 box, SH degree 3.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

SQRT_PI = math.sqrt(math.pi)

# view flags (mirrors of the C-ABI flag bits; plain integers)
FLAG_LOD_OFF = 1
FLAG_NO_NORMALIZE = 2
FLAG_FAST_EXP = 4       # blends with the hardware exponential (not bit-reproducible)


@dataclasses.dataclass
class Scene:
    means: np.ndarray      # (n, 3) float32
    scales: np.ndarray     # (n, 3) float32, > 0
    quats: np.ndarray      # (n, 4) float32, (w, x, y, z), any norm
    opacity: np.ndarray    # (n,)   float32 in (0, 1)
    sh: np.ndarray         # (n, (deg+1)^2, 3) float32
    decay: np.ndarray      # (n,)   float32, raw sigma_d

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    @property
    def sh_degree(self) -> int:
        k = self.sh.shape[1]
        return int(round(math.sqrt(k))) - 1

    def subset(self, idx) -> "Scene":
        return Scene(*(np.ascontiguousarray(a[idx]) for a in
                       (self.means, self.scales, self.quats, self.opacity, self.sh, self.decay)))


@dataclasses.dataclass
class View:
    """Pinhole camera.  ``viewmat`` is the 3x4 world->camera [R|t] (camera x right,
    y down, z forward); ``campos`` the camera centre in world coordinates."""
    width: int
    height: int
    viewmat: np.ndarray    # (3, 4) float32
    fx: float
    fy: float
    cx: float
    cy: float
    campos: np.ndarray     # (3,) float32
    s_v: float = 1.0
    tau: float = 1.0 / 255.0
    eps: float = 1e-6
    near: float = 0.2
    bg: Sequence[float] = (0.0, 0.0, 0.0)
    flags: int = 0
    # window of a larger frame (full_width > 0): the camera fields describe the full frame
    region_x: int = 0
    region_y: int = 0
    full_width: int = 0
    full_height: int = 0
    budget: int = 0        # > 0: keep the `budget` Gaussians of highest alpha'' instead of the tau s_v test

    def replace(self, **kw) -> "View":
        return dataclasses.replace(self, **kw)

    @property
    def tiles(self) -> int:
        return ((self.width + 15) // 16) * ((self.height + 15) // 16)


# ----------------------------------------------------------------------------
# cameras
# ----------------------------------------------------------------------------

def look_at(eye, target, width, height, fovy_deg=60.0, up=(0.0, 0.0, 1.0), **kw) -> View:
    eye = np.asarray(eye, np.float64)
    target = np.asarray(target, np.float64)
    fwd = target - eye
    fwd /= np.linalg.norm(fwd)
    upv = np.asarray(up, np.float64)
    if abs(np.dot(fwd, upv)) > 0.999:
        upv = np.array([0.0, 1.0, 0.0])
    right = np.cross(fwd, upv)
    right /= np.linalg.norm(right)
    down = np.cross(fwd, right)
    R = np.stack([right, down, fwd])             # rows: camera axes in world
    t = -R @ eye
    vm = np.concatenate([R, t[:, None]], axis=1).astype(np.float32)
    f = (height / 2.0) / math.tan(math.radians(fovy_deg) / 2.0)
    return View(width=width, height=height, viewmat=vm, fx=float(np.float32(f)), fy=float(np.float32(f)),
                cx=width / 2.0, cy=height / 2.0, campos=eye.astype(np.float32), **kw)


def orbit_cameras(n: int, width: int, height: int, d_min=2.0, d_max=20.0, elev_deg=20.0,
                  seed: int = 1, **kw) -> List[View]:
    """``n`` cameras looking at the origin, azimuth uniform, distances geometric
    from ``d_min`` to ``d_max``."""
    rng = np.random.default_rng(seed + 1000)
    az = rng.uniform(0.0, 2 * math.pi, size=n)
    dists = np.geomspace(d_min, d_max, n) if n > 1 else np.array([d_min])
    el = math.radians(elev_deg)
    views = []
    for a, d in zip(az, dists):
        eye = d * np.array([math.cos(el) * math.cos(a), math.cos(el) * math.sin(a), math.sin(el)])
        views.append(look_at(eye, (0.0, 0.0, 0.0), width, height, **kw))
    return views


def random_cameras(n: int, widths_heights, d_range=(1.0, 50.0), s_range=(1.0, 32.0),
                   seed: int = 4, jitter: float = 0.1) -> List[View]:
    """Serving-style poses: random direction, distance U[d_range], looking at the
    origin +- jitter, resolution drawn from ``widths_heights``, s_v log-uniform."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        w, h = widths_heights[rng.integers(len(widths_heights))]
        v = rng.normal(size=3)
        v /= np.linalg.norm(v)
        d = rng.uniform(*d_range)
        tgt = rng.normal(scale=jitter, size=3)
        s = math.exp(rng.uniform(math.log(s_range[0]), math.log(s_range[1])))
        out.append(look_at(d * v, tgt, int(w), int(h), s_v=float(np.float32(s))))
    return out


# ----------------------------------------------------------------------------
# scenes
# ----------------------------------------------------------------------------

def _attributes(rng, n: int, sh_degree: int, band_std: float = 0.05):
    scales = np.exp(rng.normal(-4.0, 0.5, size=(n, 3))).astype(np.float32)
    quats = rng.normal(size=(n, 4)).astype(np.float32)
    opacity = (1.0 / (1.0 + np.exp(-rng.normal(size=n)))).astype(np.float32)
    k = (sh_degree + 1) ** 2
    sh = np.zeros((n, k, 3), np.float32)
    sh[:, 0, :] = rng.uniform(-SQRT_PI, SQRT_PI, size=(n, 3))
    if k > 1:
        sh[:, 1:, :] = rng.normal(0.0, band_std, size=(n, k - 1, 3))
    decay = rng.uniform(0.0, 2.0, size=n).astype(np.float32)
    return scales, quats, opacity, sh, decay


def tiny_scene(n: int = 20000, seed: int = 0, sh_degree: int = 0) -> Scene:
    rng = np.random.default_rng(seed)
    means = rng.uniform(-1.0, 1.0, size=(n, 3)).astype(np.float32)
    return Scene(means, *_attributes(rng, n, sh_degree))


def blob_mixture(rng, n: int, n_blobs=4, centre_range=1.0, blob_sigma=0.25, bg_range=1.5,
                 box=(1.0, 1.0, 1.0)) -> np.ndarray:
    n_bg = n // 10
    n_fg = n - n_bg
    centres = rng.uniform(-centre_range, centre_range, size=(n_blobs, 3))
    which = rng.integers(n_blobs, size=n_fg)
    fg = centres[which] + rng.normal(0.0, blob_sigma, size=(n_fg, 3))
    bg = rng.uniform(-bg_range, bg_range, size=(n_bg, 3))
    pts = np.concatenate([fg, bg]) * np.asarray(box)
    rng.shuffle(pts)
    return pts.astype(np.float32)


def object_scene(n: int = 1_000_000, seed: int = 1, sh_degree: int = 3) -> Scene:
    rng = np.random.default_rng(seed)
    means = blob_mixture(rng, n)
    return Scene(means, *_attributes(rng, n, sh_degree))


def outdoor_scene(n: int = 3_000_000, seed: int = 2, sh_degree: int = 3) -> Scene:
    rng = np.random.default_rng(seed)
    means = blob_mixture(rng, n, centre_range=1.0, blob_sigma=0.2, bg_range=1.0, box=(5.0, 5.0, 2.0))
    return Scene(means, *_attributes(rng, n, sh_degree))


def city_scene(n: int = 6_000_000, seed: int = 5, sh_degree: int = 3, n_planes: int = 64) -> Scene:
    rng = np.random.default_rng(seed)
    n_vol = n // 5
    n_pl = n - n_vol
    normals = rng.normal(size=(n_planes, 3))
    normals /= np.linalg.norm(normals, axis=1, keepdims=True)
    centres = rng.uniform([-50, -50, 0], [50, 50, 30], size=(n_planes, 3))
    a = np.cross(normals, np.array([0.0, 0.0, 1.0]))
    bad = np.linalg.norm(a, axis=1) < 1e-3
    a[bad] = np.array([1.0, 0.0, 0.0])
    a /= np.linalg.norm(a, axis=1, keepdims=True)
    b = np.cross(normals, a)
    which = rng.integers(n_planes, size=n_pl)
    uv = rng.uniform(-5.0, 5.0, size=(n_pl, 2))
    off = rng.normal(0.0, 0.02, size=n_pl)
    pl = centres[which] + uv[:, :1] * a[which] + uv[:, 1:] * b[which] + off[:, None] * normals[which]
    vol = rng.uniform([-50, -50, 0], [50, 50, 30], size=(n_vol, 3))
    pts = np.concatenate([pl, vol])
    rng.shuffle(pts)
    means = pts.astype(np.float32)
    return Scene(means, *_attributes(rng, n, sh_degree))


def city_views(width: int = 3840, height: int = 2160, scales=(1.0, 4.0, 16.0, 64.0, 1.0, 4.0, 16.0, 64.0),
               seed: int = 55) -> List[View]:
    """Cameras around the city block: azimuth uniform, distance U[40, 90],
    height U[15, 45], looking at a jittered point 10 up; one view per scale."""
    rng = np.random.default_rng(seed)
    views = []
    for s in scales:
        ang = rng.uniform(0, 2 * np.pi)
        d = rng.uniform(40.0, 90.0)
        eye = (d * np.cos(ang), d * np.sin(ang), rng.uniform(15.0, 45.0))
        views.append(look_at(eye, (rng.normal(0, 5), rng.normal(0, 5), 10.0), width, height, s_v=float(s)))
    return views


def small_scene(n: int = 200, seed: int = 3, sh_degree: int = 3, extent: float = 0.6,
                log_scale_mean: float = -3.0) -> Scene:
    """Few large Gaussians for finite-difference and brute-force checks."""
    rng = np.random.default_rng(seed)
    means = rng.uniform(-extent, extent, size=(n, 3)).astype(np.float32)
    scales, quats, opacity, sh, decay = _attributes(rng, n, sh_degree, band_std=0.2)
    scales = np.exp(rng.normal(log_scale_mean, 0.4, size=(n, 3))).astype(np.float32)
    return Scene(means, scales, quats, opacity, sh, decay)


def target_image(h: int, w: int, seed: int) -> np.ndarray:
    """Seeded smooth noise texture (3, h, w) in [0, 1] used as a training target."""
    rng = np.random.default_rng(seed)
    img = np.zeros((3, h, w), np.float32)
    yy, xx = np.mgrid[0:h, 0:w].astype(np.float32)
    for c in range(3):
        for _ in range(6):
            kx, ky = rng.uniform(0.5, 8.0, size=2) * 2 * math.pi
            ph = rng.uniform(0, 2 * math.pi)
            img[c] += np.sin(kx * xx / w + ky * yy / h + ph).astype(np.float32)
    img = 0.5 + img / 12.0
    return np.clip(img, 0.0, 1.0).astype(np.float32)


def log_uniform(rng, lo: float, hi: float, size=None):
    return np.exp(rng.uniform(math.log(lo), math.log(hi), size=size))


def tiny_view(s_v: float = 1.0, **kw) -> View:
    return look_at((0.0, 0.0, 3.0), (0.0, 0.0, 0.0), 256, 256, up=(0.0, 1.0, 0.0), s_v=s_v, **kw)
