"""clod_render_noalloc: the forward render for callers that cannot allocate
device memory (its scratch is a fixed array inside the library).  Checked
through the C ABI against the allocating path (clod_preprocess /
clod_bin_sort / clod_render_fwd), bit for bit, on several calls in a row
(including a primitive budget and a window of a frame): no call may see
anything an earlier one left in the shared array.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2510_09997_gb300 import synth as S

pytestmark = pytest.mark.gpu


def test_noalloc_matches_allocating_path_two_calls():
    from paper_2510_09997_gb300 import clod as C
    C.require_cuda()
    L = C.lib()
    sc = S.tiny_scene(n=20000, seed=0, sh_degree=1)
    ds = C.DeviceScene.from_scene(sc)
    full = S.look_at((2.0, 1.0, 1.5), (0, 0, 0), 200, 150, s_v=4.0, bg=(0.0, 0.0, 0.0))
    views = [S.tiny_view(1.0, bg=(0.1, 0.2, 0.3)), full,
             S.tiny_view(2.0, budget=3000),                                      # primitive budget
             full.replace(width=96, height=80, region_x=64, region_y=48, full_width=200, full_height=150)]
    for v in views:
        fr = C.render(ds, [v], want_keys=False)
        img = torch.full((3, v.height, v.width), -1.0, device="cuda")
        T = torch.full((v.height, v.width), -1.0, device="cuda")
        nc = torch.full((v.height, v.width), -1, dtype=torch.int32, device="cuda")
        cv = C.cview(v)
        st = L.clod_render_noalloc(ctypes.byref(ds.c), ctypes.byref(cv), C._ptr(img), C._ptr(T), C._ptr(nc),
                                   C._stream(None))
        C.check("clod_render_noalloc", st)
        torch.cuda.synchronize()
        assert torch.equal(img, fr.view_image(0))
        assert torch.equal(T, fr.view_T(0))
        assert torch.equal(nc, fr.view_ncontrib(0))


def test_noalloc_rejects_oversize():
    from paper_2510_09997_gb300 import clod as C
    C.require_cuda()
    L = C.lib()
    sc = S.tiny_scene(n=70000, seed=1)
    ds = C.DeviceScene.from_scene(sc)
    v = S.tiny_view(1.0)
    img = torch.zeros((3, v.height, v.width), device="cuda")
    cv = C.cview(v)
    assert L.clod_render_noalloc(ctypes.byref(ds.c), ctypes.byref(cv), C._ptr(img), None, None, C._stream(None)) == 1
    assert b"65536" in L.clod_last_error()
    big = C.cview(v.replace(width=2048, height=64, cx=1024.0))
    small = C.DeviceScene.from_scene(sc.subset(np.arange(100)))
    assert L.clod_render_noalloc(ctypes.byref(small.c), ctypes.byref(big), C._ptr(img), None, None,
                                 C._stream(None)) == 1


def test_noalloc_pair_overflow_writes_nothing_then_recovers():
    """A frame within the argument limits whose pairs exceed the array's 2^21
    (60,000 wide Gaussians at 1024x1024): CLOD_ERR_CAPACITY with the pair
    count in the message, and the caller's image, T and contributor buffers
    untouched; the next, normal call still equals the allocating path bit
    for bit."""
    from paper_2510_09997_gb300 import clod as C
    C.require_cuda()
    L = C.lib()
    sc = S.tiny_scene(n=60000, seed=2, sh_degree=0)
    sc.scales *= np.float32(3.0)          # about 7.7M pairs
    ds = C.DeviceScene.from_scene(sc)
    v = S.tiny_view(1.0).replace(width=1024, height=1024, cx=512.0, cy=512.0, fx=886.8, fy=886.8,
                                 flags=S.FLAG_LOD_OFF)
    K = int(C.render(ds, [v], want_keys=False).n_pairs)
    assert K > (1 << 21)
    img = torch.full((3, 1024, 1024), -1.0, device="cuda")
    T = torch.full((1024, 1024), -1.0, device="cuda")
    nc = torch.full((1024, 1024), -1, dtype=torch.int32, device="cuda")
    cv = C.cview(v)
    st = L.clod_render_noalloc(ctypes.byref(ds.c), ctypes.byref(cv), C._ptr(img), C._ptr(T), C._ptr(nc),
                               C._stream(None))
    torch.cuda.synchronize()
    assert st == 2
    assert str(K).encode() in L.clod_last_error()
    assert bool((img == -1.0).all()) and bool((T == -1.0).all()) and bool((nc == -1).all())
    small = C.DeviceScene.from_scene(S.tiny_scene(n=20000, seed=0, sh_degree=1))
    w = S.tiny_view(1.0, bg=(0.1, 0.2, 0.3))
    fr = C.render(small, [w], want_keys=False)
    img2 = torch.full((3, w.height, w.width), -1.0, device="cuda")
    cw = C.cview(w)
    C.check("clod_render_noalloc", L.clod_render_noalloc(ctypes.byref(small.c), ctypes.byref(cw), C._ptr(img2),
                                                         None, None, C._stream(None)))
    torch.cuda.synchronize()
    assert torch.equal(img2, fr.view_image(0))
