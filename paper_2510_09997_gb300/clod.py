"""Python binding of libclod: the same entry points as include/clod.h, taking
torch tensors (device memory and streams come from PyTorch; every step of the
rasterizer runs in libclod's CUDA kernels).
"""
from __future__ import annotations

import ctypes
import dataclasses
from typing import List, Optional, Sequence

import numpy as np
import torch

from . import abi
from ._lib import load

_FIELDS = ("means", "scales", "quats", "opacity", "sh", "decay")
MAX_VIEWS = 64          # views per launch


class ClodError(RuntimeError):
    def __init__(self, fn: str, status: int, msg: str):
        super().__init__("%s -> %s: %s" % (fn, abi.STATUS_NAMES.get(status, status), msg))
        self.status = status


def lib():
    return load()


def check(fn: str, status: int) -> None:
    if status != abi.CLOD_OK:
        raise ClodError(fn, status, lib().clod_last_error().decode())


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream: Optional[torch.cuda.Stream]):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def require_cuda():
    if not torch.cuda.is_available():
        raise RuntimeError("libclod needs a CUDA device (GB300, sm_103a); none is available")


# ---------------------------------------------------------------------------
class DeviceScene:
    """A scene resident in device memory (activated parameters, float32)."""

    def __init__(self, means, scales, quats, opacity, sh, decay):
        require_cuda()
        self.t = {}
        for k, a in zip(_FIELDS, (means, scales, quats, opacity, sh, decay)):
            if not isinstance(a, torch.Tensor):
                a = torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32))
            self.t[k] = a.to(device="cuda", dtype=torch.float32).contiguous()
        self.n = int(self.t["means"].shape[0])
        k = self.t["sh"].shape[1] if self.t["sh"].dim() == 3 else self.t["sh"].shape[1] // 3
        self.sh_degree = int(round(k ** 0.5)) - 1
        self.refresh()

    def refresh(self) -> None:
        t = self.t
        self.c = abi.clod_scene(self.n, self.sh_degree, 0, *[t[k].data_ptr() for k in _FIELDS])

    @classmethod
    def from_scene(cls, scene) -> "DeviceScene":
        return cls(*(getattr(scene, k) for k in _FIELDS))

    @classmethod
    def from_tensors(cls, *tensors) -> "DeviceScene":
        """A scene over existing contiguous float32 CUDA tensors (aliased, not
        copied: later writes to them are seen by the next render)."""
        return cls(*tensors)

    def __getattr__(self, k):
        if k in _FIELDS:
            return self.t[k]
        raise AttributeError(k)


def cview(v) -> abi.clod_view:
    c = abi.clod_view()
    c.width, c.height = int(v.width), int(v.height)
    vm = np.asarray(v.viewmat, np.float32).reshape(-1)
    for i in range(12):
        c.viewmat[i] = float(vm[i])
    c.fx, c.fy, c.cx, c.cy = float(v.fx), float(v.fy), float(v.cx), float(v.cy)
    c.near_z = float(v.near)
    for i in range(3):
        c.campos[i] = float(v.campos[i])
        c.bg[i] = float(v.bg[i])
    c.s_v, c.tau, c.eps = float(v.s_v), float(v.tau), float(v.eps)
    c.flags = int(v.flags)
    c.region_x, c.region_y = int(getattr(v, "region_x", 0)), int(getattr(v, "region_y", 0))
    c.full_width, c.full_height = int(getattr(v, "full_width", 0)), int(getattr(v, "full_height", 0))
    c.budget = int(getattr(v, "budget", 0))
    return c


def band_views(view, x_bounds: Sequence[int], s_values: Sequence[float]) -> list:
    """Split a full-frame view into vertical bands [x_bounds[k], x_bounds[k+1])
    rendered at s_values[k] (regional level of detail, Sec. 4.4).  Inner bounds
    must be multiples of 16; the bands share the full frame's camera, frustum and
    d_max."""
    xb = [int(x) for x in x_bounds]
    if len(xb) != len(s_values) + 1 or xb[0] != 0 or xb[-1] != view.width or any(
            b <= a for a, b in zip(xb, xb[1:])):
        raise ValueError("x_bounds must rise from 0 to the view width, one band per s value")
    out = []
    for k, s in enumerate(s_values):
        out.append(view.replace(width=xb[k + 1] - xb[k], region_x=xb[k], region_y=0,
                                full_width=view.width, full_height=view.height, s_v=float(s)))
    return out


def view_array(views: Sequence) -> ctypes.Array:
    arr = (abi.clod_view * len(views))()
    for i, v in enumerate(views):
        arr[i] = cview(v)
    return arr


def frame_layout(n: int, views: Sequence):
    arr = view_array(views)
    nbytes = ctypes.c_size_t()
    lay = abi.clod_frame_layout()
    check("clod_frame_workspace_size",
          lib().clod_frame_workspace_size(n, arr, len(views), ctypes.byref(nbytes), ctypes.byref(lay)))
    return int(nbytes.value), lay


# ---------------------------------------------------------------------------
# Entry points with the C-ABI names
# ---------------------------------------------------------------------------
def clod_preprocess(scene: DeviceScene, views, ws: torch.Tensor, mask=None, alpha_eff=None, counts=None,
                    n_pairs=None, stream=None):
    arr = view_array(views)
    check("clod_preprocess", lib().clod_preprocess(ctypes.byref(scene.c), arr, len(views), _ptr(ws), ws.numel(),
                                                   _ptr(mask), _ptr(alpha_eff), _ptr(counts), _ptr(n_pairs),
                                                   _stream(stream)))


def clod_bin_sort(ws, cap: int, keys, vals, ranges, stream=None):
    check("clod_bin_sort", lib().clod_bin_sort(_ptr(ws), cap, _ptr(keys), _ptr(vals), _ptr(ranges),
                                               _stream(stream)))


def clod_render_fwd(ws, vals, ranges, image, T_final=None, n_contrib=None, stream=None, evaluated=None):
    if evaluated is None:
        check("clod_render_fwd", lib().clod_render_fwd(_ptr(ws), _ptr(vals), _ptr(ranges), _ptr(image),
                                                       _ptr(T_final), _ptr(n_contrib), _stream(stream)))
    else:
        check("clod_render_fwd_count",
              lib().clod_render_fwd_count(_ptr(ws), _ptr(vals), _ptr(ranges), _ptr(image), _ptr(T_final),
                                          _ptr(n_contrib), _ptr(evaluated), _stream(stream)))


def clod_frame_check(ws, cap: int, stream=None) -> int:
    k = ctypes.c_uint64()
    check("clod_frame_check", lib().clod_frame_check(_ptr(ws), cap, ctypes.byref(k), _stream(stream)))
    return int(k.value)


# ---------------------------------------------------------------------------
@dataclasses.dataclass
class Frame:
    """Buffers of one forward pass over a batch of views."""
    views: list
    ws: torch.Tensor
    layout: object
    mask: torch.Tensor          # u8 [V, n]
    alpha_eff: torch.Tensor     # f32 [V, n]
    counts: torch.Tensor        # u32 (as int32) [V, 2]: sum M, rendered
    n_pairs: int
    keys: Optional[torch.Tensor]
    vals: torch.Tensor
    ranges: torch.Tensor        # [total_tiles, 2]
    image: torch.Tensor         # packed f32
    T_final: torch.Tensor
    n_contrib: torch.Tensor
    pix_base: List[int]

    def view_image(self, v: int) -> torch.Tensor:
        w = self.views[v]
        b = self.pix_base[v]
        return self.image[3 * b: 3 * (b + w.width * w.height)].view(3, w.height, w.width)

    def view_T(self, v: int) -> torch.Tensor:
        w = self.views[v]
        b = self.pix_base[v]
        return self.T_final[b: b + w.width * w.height].view(w.height, w.width)

    def view_ncontrib(self, v: int) -> torch.Tensor:
        w = self.views[v]
        b = self.pix_base[v]
        return self.n_contrib[b: b + w.width * w.height].view(w.height, w.width)

    def ws_array(self, name: str, dtype, count: int) -> torch.Tensor:
        off = getattr(self.layout, name)
        nbytes = count * torch.empty(0, dtype=dtype).element_size()
        return self.ws[off: off + nbytes].view(dtype)


def pixel_bases(views) -> List[int]:
    out, b = [], 0
    for v in views:
        out.append(b)
        b += v.width * v.height
    return out


def render(scene: DeviceScene, views, want_keys: bool = True, stream=None, evaluated=None) -> Frame:
    """One forward pass over ``views``: preprocess, read K back (one
    synchronisation), bin/sort with exactly K slots, blend."""
    require_cuda()
    views = list(views)
    dev = torch.device("cuda")
    nbytes, lay = frame_layout(scene.n, views)
    ws = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    V = len(views)
    mask = torch.empty((V, scene.n), dtype=torch.uint8, device=dev)
    alpha = torch.empty((V, scene.n), dtype=torch.float32, device=dev)
    counts = torch.empty((V, 2), dtype=torch.int32, device=dev)
    npairs = torch.zeros(1, dtype=torch.int64, device=dev)
    clod_preprocess(scene, views, ws, mask, alpha, counts, npairs, stream)
    K = int(npairs.item())
    cap = max(K, 1)
    keys = torch.empty(cap, dtype=torch.int64, device=dev) if want_keys else None
    vals = torch.empty(cap, dtype=torch.int32, device=dev)
    ranges = torch.empty((lay.total_tiles, 2), dtype=torch.int32, device=dev)
    clod_bin_sort(ws, cap, keys, vals, ranges, stream)
    bases = pixel_bases(views)
    P = sum(v.width * v.height for v in views)
    image = torch.empty(3 * P, dtype=torch.float32, device=dev)
    T = torch.empty(P, dtype=torch.float32, device=dev)
    nc = torch.empty(P, dtype=torch.int32, device=dev)
    clod_render_fwd(ws, vals, ranges, image, T, nc, stream, evaluated=evaluated)
    return Frame(views, ws, lay, mask, alpha, counts, K, keys[:K] if keys is not None else None, vals[:K], ranges,
                 image, T, nc, bases)


class Renderer:
    """Reusable buffers for repeated forward passes without a mid-frame
    synchronisation: the pair capacity is fixed up front (grow() re-sizes),
    overflow is detected afterwards with check()."""

    def __init__(self, scene: DeviceScene, views, pair_capacity: int, want_keys: bool = False):
        self.scene = scene
        self.views = list(views)
        dev = torch.device("cuda")
        nbytes, self.layout = frame_layout(scene.n, self.views)
        self.ws = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        self.cap = int(pair_capacity)
        self.keys = torch.empty(self.cap, dtype=torch.int64, device=dev) if want_keys else None
        self.vals = torch.empty(self.cap, dtype=torch.int32, device=dev)
        self.ranges = torch.empty((self.layout.total_tiles, 2), dtype=torch.int32, device=dev)
        P = sum(v.width * v.height for v in self.views)
        self.image = torch.empty(3 * P, dtype=torch.float32, device=dev)
        self.T = torch.empty(P, dtype=torch.float32, device=dev)
        self.nc = torch.empty(P, dtype=torch.int32, device=dev)
        self.npairs = torch.zeros(1, dtype=torch.int64, device=dev)
        self.carr = view_array(self.views)

    def set_views(self, views) -> None:
        views = list(views)
        assert len(views) == len(self.views)
        assert all(a.width == b.width and a.height == b.height for a, b in zip(views, self.views))
        self.views = views
        self.carr = view_array(views)

    def run(self, stream=None) -> None:
        L = lib()
        st = _stream(stream)
        check("clod_preprocess", L.clod_preprocess(ctypes.byref(self.scene.c), self.carr, len(self.views),
                                                   _ptr(self.ws), self.ws.numel(), None, None, None,
                                                   _ptr(self.npairs), st))
        check("clod_bin_sort", L.clod_bin_sort(_ptr(self.ws), self.cap, _ptr(self.keys), _ptr(self.vals),
                                               _ptr(self.ranges), st))
        check("clod_render_fwd", L.clod_render_fwd(_ptr(self.ws), _ptr(self.vals), _ptr(self.ranges),
                                                   _ptr(self.image), _ptr(self.T), _ptr(self.nc), st))

    def check(self, stream=None) -> int:
        return clod_frame_check(self.ws, self.cap, stream)
