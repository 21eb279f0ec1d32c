"""Python front end of the CPU oracle (``clod_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
benchmark's CPU-baseline leg, never by the product path.  It shares no code
with the CUDA path; inputs come from the seeded generators as plain numpy
arrays and plain view objects (any object with the ``View`` attributes).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Dict, List, Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "clod_oracle.c")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "liboracle.so")

REC = 12      # FP32 record floats per Gaussian
REC64 = 9     # FP64 record doubles per Gaussian
TILE = 16
LOD_OFF = 1
NO_NORMALIZE = 2

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no contraction, no fast math)."""
    os.makedirs(BUILD, exist_ok=True)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + ".tmp.%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-o", tmp, SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, LIB)
    return LIB


def bind(L):
    """Declare the argument types of the oracle's C functions on a loaded
    library (the built oracle, or a test's modified copy of it)."""
    P = ctypes.c_void_p
    I64 = ctypes.c_int64
    L.oracle_exp_spec.argtypes = [ctypes.c_float]
    L.oracle_exp_spec.restype = ctypes.c_float
    L.oracle_exp_spec_batch.argtypes = [P, P, I64]
    L.oracle_exp_spec_monotone_violations.argtypes = [ctypes.c_float, ctypes.c_float, P]
    L.oracle_exp_spec_monotone_violations.restype = I64
    L.oracle_sh_basis.argtypes = [P, I64, ctypes.c_int, P]
    L.oracle_stage1.argtypes = [I64, ctypes.c_int] + [P] * 7 + [P] * 10
    L.oracle_stage1_f64.argtypes = [I64, ctypes.c_int] + [P] * 7 + [I64, P, P]
    L.oracle_emit_pairs.argtypes = [I64, P, ctypes.c_uint32, P, P, P, P, P, I64]
    L.oracle_emit_pairs.restype = I64
    L.oracle_stable_sort.argtypes = [P, P, I64]
    L.oracle_stable_sort.restype = ctypes.c_int
    L.oracle_ranges.argtypes = [P, I64, I64, P]
    L.oracle_render.argtypes = [I64, P, P, P, P, P, P, I64, P, P, P, P, P, P, P, I64, P]
    L.oracle_render.restype = I64
    L.oracle_render_f64dec.argtypes = ([I64, P, P, P, P, P, P, I64, ctypes.c_double, ctypes.c_double, ctypes.c_int]
                                       + [P] * 8 + [I64])
    L.oracle_render_f64dec.restype = I64
    return L


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = bind(ctypes.CDLL(LIB))
    return _lib


def _p(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# ----------------------------------------------------------------------------
def exp_spec(x) -> np.ndarray:
    x = _c(np.atleast_1d(x), np.float32)
    y = np.empty_like(x)
    lib().oracle_exp_spec_batch(_p(x), _p(y), x.size)
    return y


def exp_spec_monotone_violations(lo: float, hi: float):
    first = np.zeros(1, np.float32)
    n = lib().oracle_exp_spec_monotone_violations(lo, hi, _p(first))
    return int(n), float(first[0])


def sh_basis(dirs: np.ndarray, deg: int) -> np.ndarray:
    d = _c(dirs, np.float64).reshape(-1, 3)
    out = np.zeros((d.shape[0], 16), np.float64)
    lib().oracle_sh_basis(_p(d), d.shape[0], deg, _p(out))
    return out


def pack_view(v) -> np.ndarray:
    a = np.zeros(32, np.float32)
    vm = np.asarray(v.viewmat, np.float32).reshape(3, 4)
    a[0:9] = vm[:, :3].reshape(-1)
    a[9:12] = vm[:, 3]
    a[12], a[13], a[14], a[15] = v.fx, v.fy, v.cx, v.cy
    a[16] = v.near
    a[17:20] = np.asarray(v.campos, np.float32)
    a[20], a[21], a[22] = v.s_v, v.tau, v.eps
    a[23:26] = np.asarray(v.bg, np.float32)
    a[26], a[27] = v.width, v.height
    a[28] = v.flags
    a[29:30] = np.array([int(getattr(v, "budget", 0))], np.uint32).view(np.float32)
    if int(getattr(v, "full_width", 0)) > 0:
        raise ValueError("the oracle renders whole frames; compare a region with the crop of its frame")
    return a


def tiles_of(v):
    tx = (v.width + TILE - 1) // TILE
    ty = (v.height + TILE - 1) // TILE
    return tx, ty


def _scene_arrays(scene):
    return (_c(scene.means, np.float32), _c(scene.scales, np.float32), _c(scene.quats, np.float32),
            _c(scene.opacity, np.float32), _c(scene.sh, np.float32), _c(scene.decay, np.float32))


def sh_degree(scene) -> int:
    return int(round(np.sqrt(scene.sh.shape[1]))) - 1


def stage1(scene, view) -> Dict[str, np.ndarray]:
    """FP32 Stage I for one view (see ``oracle_stage1``)."""
    n = scene.means.shape[0]
    arrs = _scene_arrays(scene)
    V = pack_view(view)
    out = dict(
        dist=np.zeros(n, np.float32), in_view=np.zeros(n, np.uint8), dmax=np.zeros(1, np.float32),
        argmax=np.zeros(1, np.int64), alpha_eff=np.zeros(n, np.float32), mask=np.zeros(n, np.uint8),
        survive=np.zeros(n, np.uint8), rec=np.zeros((n, REC), np.float32), rect=np.zeros((n, 4), np.int32),
        tiles=np.zeros(n, np.uint32))
    lib().oracle_stage1(n, sh_degree(scene), *[_p(a) for a in arrs], _p(V),
                        _p(out["dist"]), _p(out["in_view"]), _p(out["dmax"]), _p(out["argmax"]),
                        _p(out["alpha_eff"]), _p(out["mask"]), _p(out["survive"]), _p(out["rec"]),
                        _p(out["rect"]), _p(out["tiles"]))
    return out


def stage1_f64(scene, view, s1) -> np.ndarray:
    n = scene.means.shape[0]
    arrs = _scene_arrays(scene)
    V = pack_view(view)
    rec64 = np.zeros((n, REC64), np.float64)
    lib().oracle_stage1_f64(n, sh_degree(scene), *[_p(a) for a in arrs], _p(V), int(s1["argmax"][0]),
                            _p(s1["survive"]), _p(rec64))
    return rec64


def emit_pairs(view, s1, tile_base: int = 0):
    n = s1["survive"].shape[0]
    V = pack_view(view)
    k = int(np.sum(s1["tiles"], dtype=np.int64))
    keys = np.zeros(max(k, 1), np.uint64)
    vals = np.zeros(max(k, 1), np.uint32)
    got = lib().oracle_emit_pairs(n, _p(V), tile_base, _p(s1["survive"]), _p(s1["rec"]), _p(s1["rect"]),
                                  _p(keys), _p(vals), k)
    assert got == k
    return keys[:k], vals[:k]


def stable_sort(keys: np.ndarray, vals: np.ndarray):
    k = keys.copy()
    v = vals.copy()
    if lib().oracle_stable_sort(_p(k), _p(v), k.size) != 0:
        raise MemoryError("oracle sort")
    return k, v


def ranges(keys: np.ndarray, n_tiles: int) -> np.ndarray:
    r = np.zeros((n_tiles, 2), np.uint32)
    lib().oracle_ranges(_p(keys), keys.size, n_tiles, _p(r))
    return r


def render(scene, view, s1, rec64=None, tiles: Optional[Sequence[int]] = None, contrib: bool = False):
    """Stage II for one view.  ``tiles`` (tile indices) limits the work; pixels
    of other tiles are left at zero.  Returns a dict with img32 (3,H,W) f32,
    img64 (3,H,W) f64 (if rec64 given), T32, T64, ncontrib, evaluated and, if
    ``contrib``, the contributing (pixel, gaussian) pairs in blending order."""
    n = s1["survive"].shape[0]
    V = pack_view(view)
    W, H = view.width, view.height
    tx, ty = tiles_of(view)
    tl = _c(np.arange(tx * ty) if tiles is None else np.asarray(tiles), np.int32)
    img32 = np.zeros((3, H, W), np.float32)
    T32 = np.zeros((H, W), np.float32)
    nc = np.zeros((H, W), np.uint32)
    img64 = np.zeros((3, H, W), np.float64) if rec64 is not None else None
    T64 = np.zeros((H, W), np.float64) if rec64 is not None else None
    ev = np.zeros(1, np.int64)
    L = lib()
    args = [n, _p(V), _p(s1["survive"]), _p(s1["rec"]), _p(s1["rect"]), _p(rec64), _p(tl), tl.size,
            _p(img32), _p(img64), _p(T32), _p(T64), _p(nc)]
    out = dict(img32=img32, img64=img64, T32=T32, T64=T64, ncontrib=nc)
    if contrib:
        total = L.oracle_render(*args, None, None, 0, _p(ev))
        pix = np.zeros(max(total, 1), np.int64)
        gid = np.zeros(max(total, 1), np.int32)
        total2 = L.oracle_render(*args, _p(pix), _p(gid), total, _p(ev))
        assert total2 == total
        out["contrib_pix"] = pix[:total]
        out["contrib_gid"] = gid[:total]
    else:
        total = L.oracle_render(*args, None, None, 0, _p(ev))
    if total < 0:
        raise MemoryError("oracle render")
    out["n_contrib_pairs"] = int(total)
    out["evaluated"] = int(ev[0])
    return out


def render_f64dec(view, s1, rec64, tiles: Optional[Sequence[int]] = None, rel: float = 1e-5,
                  max_paths: int = 16, dev: float = 1.0):
    """Stage II with every per-pixel decision taken in FP64 (see
    ``oracle_render_f64dec``).  Returns a dict with the main path's img (3,H,W)
    f64, T, ncontrib; per pixel n_paths (outcomes followed) and n_capped
    (flags beyond ``max_paths``); and the other outcomes as alt_pix (flat
    pixel index), alt_val (r, g, b, T) and alt_nc.  Pixels outside ``tiles``
    hold zeros.  ``dev`` scales the FP32 deviation bound in the bands (0: the
    relative band ``rel`` alone)."""
    n = s1["survive"].shape[0]
    V = pack_view(view)
    W, H = view.width, view.height
    tx, ty = tiles_of(view)
    tl = _c(np.arange(tx * ty) if tiles is None else np.asarray(tiles), np.int32)
    img = np.zeros((3, H, W), np.float64)
    T = np.zeros((H, W), np.float64)
    nc = np.zeros((H, W), np.uint32)
    npath = np.zeros((H, W), np.uint8)
    ncap = np.zeros((H, W), np.uint8)
    L = lib()
    cap = 1 << 16
    while True:
        pix = np.zeros(cap, np.int64)
        val = np.zeros((cap, 4), np.float64)
        anc = np.zeros(cap, np.uint32)
        got = L.oracle_render_f64dec(n, _p(V), _p(s1["survive"]), _p(s1["rec"]), _p(s1["rect"]), _p(rec64),
                                     _p(tl), tl.size, float(rel), float(dev), int(max_paths), _p(img), _p(T), _p(nc),
                                     _p(npath), _p(ncap), _p(pix), _p(val), _p(anc), cap)
        if got < 0:
            raise MemoryError("oracle render_f64dec")
        if got <= cap:
            break
        cap = int(got)
    return dict(img=img, T=T, ncontrib=nc, n_paths=npath, n_capped=ncap, alt_pix=pix[:got], alt_val=val[:got],
                alt_nc=anc[:got])


def frame(scene, views: Sequence, with64: bool = True, tiles: Optional[List[Optional[Sequence[int]]]] = None,
          pairs: bool = True, contrib: bool = False, dec64: bool = False):
    """Whole oracle pipeline over several views: Stage I per view, pairs with
    view-offset tile ids, stable sort and ranges over all views, Stage II per
    view (and, with ``dec64``, Stage II with FP64 decisions in each view's
    ``img[v]["dec64"]``).  Returns a dict of per-view lists plus the global
    keys/vals/ranges."""
    res = dict(s1=[], rec64=[], img=[], tile_base=[])
    base = 0
    all_k, all_v = [], []
    for vi, v in enumerate(views):
        s1 = stage1(scene, v)
        r64 = stage1_f64(scene, v, s1) if with64 else None
        res["s1"].append(s1)
        res["rec64"].append(r64)
        res["tile_base"].append(base)
        if pairs:
            k, val = emit_pairs(v, s1, base)
            all_k.append(k)
            all_v.append(val)
        tl = None if tiles is None else tiles[vi]
        res["img"].append(render(scene, v, s1, r64, tl, contrib=contrib))
        if dec64:
            if r64 is None:
                raise ValueError("FP64 decisions need the FP64 records (with64=True)")
            res["img"][-1]["dec64"] = render_f64dec(v, s1, r64, tl)
        tx, ty = tiles_of(v)
        base += tx * ty
    res["n_tiles"] = base
    if pairs:
        keys = np.concatenate(all_k) if all_k else np.zeros(0, np.uint64)
        vals = np.concatenate(all_v) if all_v else np.zeros(0, np.uint32)
        sk, sv = stable_sort(keys, vals)
        res["keys"], res["vals"] = sk, sv
        res["ranges"] = ranges(sk, base)
    return res
