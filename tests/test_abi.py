"""The C ABI library loads without a GPU and exports every entry point that
include/clod.h declares; argument validation works without a device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "clod.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(clod_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def L():
    from paper_2510_09997_gb300 import _lib
    return _lib.load()


def test_every_declared_symbol_is_exported(L):
    names = declared()
    assert len(names) >= 12
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_header_and_binding_agree():
    from paper_2510_09997_gb300 import abi
    for n in declared():
        assert n in abi.SIGNATURES, n


def test_validation_without_gpu(L):
    from paper_2510_09997_gb300 import abi, clod, synth as S
    nbytes = ctypes.c_size_t()
    views = clod.view_array([S.tiny_view(1.0)])
    assert L.clod_frame_workspace_size(1000, views, 1, ctypes.byref(nbytes), None) == abi.CLOD_OK
    assert nbytes.value > 1000 * 60
    assert L.clod_frame_workspace_size(-1, views, 1, ctypes.byref(nbytes), None) == abi.CLOD_ERR_ARG
    assert b"outside" in L.clod_last_error()
    assert L.clod_frame_workspace_size(10, views, 0, ctypes.byref(nbytes), None) == abi.CLOD_ERR_ARG
    bad = clod.view_array([S.tiny_view(1.0).replace(width=0)])
    assert L.clod_frame_workspace_size(10, bad, 1, ctypes.byref(nbytes), None) == abi.CLOD_ERR_ARG
    assert L.clod_render_noalloc(None, None, None, None, None, None) == abi.CLOD_ERR_ARG
    assert L.clod_preprocess(None, views, 1, None, 0, None, None, None, None, None) == abi.CLOD_ERR_ARG
    assert L.clod_bin_sort(None, 0, None, None, None, None) == abi.CLOD_ERR_ARG
    assert L.clod_backward_workspace_size(5, 0, ctypes.byref(nbytes)) == abi.CLOD_ERR_ARG
    for bwd in (L.clod_render_bwd, L.clod_render_bwd_set):
        assert bwd(None, None, None, None, None, None, None, None, None, None, 0,
                   None, None, None, None, None, None, None) == abi.CLOD_ERR_ARG
    # the Adam configuration struct as the header lays it out (keep_grads last)
    assert ctypes.sizeof(abi.clod_adam_cfg) == 4 * 10 + 4
    assert abi.clod_adam_cfg.keep_grads.offset == 40


def test_region_view_validation_without_gpu(L):
    """Regional views: tile-aligned origins inside the full frame only."""
    from paper_2510_09997_gb300 import abi, clod, synth as S
    nbytes = ctypes.c_size_t()
    full = S.look_at((2.5, -1.0, 1.0), (0, 0, 0), 250, 130)
    good = clod.band_views(full, [0, 64, 128, 176, 250], [8.0, 4.0, 2.0, 1.0])
    assert [b.width for b in good] == [64, 64, 48, 74]
    assert L.clod_frame_workspace_size(100, clod.view_array(good), 4, ctypes.byref(nbytes), None) == abi.CLOD_OK
    for bad in (good[1].replace(region_x=40),                  # not a multiple of 16
                good[3].replace(width=90),                      # leaves the frame
                good[0].replace(region_y=-16),
                good[0].replace(full_height=0)):
        assert L.clod_frame_workspace_size(100, clod.view_array([bad]), 1, ctypes.byref(nbytes),
                                           None) == abi.CLOD_ERR_ARG
        assert b"view 0" in L.clod_last_error()
    with pytest.raises(ValueError):
        clod.band_views(full, [0, 64, 250], [1.0])
    assert ctypes.sizeof(abi.clod_view) == 136


def test_step_weights_closed_form(L):
    """clod_step_weights gives Eq. 5's w_s(s_v) = (1 - s_v / (2 s_max))^2 per
    view, divided by the view count (host call, no GPU)."""
    from oracle import losses as OL
    from paper_2510_09997_gb300 import abi  # noqa: F401  (declares the signatures)
    s = [1.0, 3.5, 16.0]
    sa = (ctypes.c_float * 3)(*s)
    w = (ctypes.c_float * 3)()
    assert L.clod_step_weights(sa, 3, 16.0, w) == 0
    for k in range(3):
        assert w[k] == pytest.approx(OL.w_s(float(ctypes.c_float(s[k]).value), 16.0) / 3, rel=1e-6)
    assert w[2] == pytest.approx(0.25 / 3, rel=1e-7)           # w_s(s_max) = 1/4
    assert L.clod_step_weights(sa, 3, 0.0, w) == 1
    bad = (ctypes.c_float * 1)(-1.0)
    assert L.clod_step_weights(bad, 1, 16.0, w) == 1


def test_fast_exp_flag_must_agree_across_views(L):
    """One frame blends with one exponential: views that disagree on
    CLOD_FAST_EXP are rejected before any device work."""
    from paper_2510_09997_gb300 import abi, clod, synth as S
    views = clod.view_array([S.tiny_view(1.0), S.tiny_view(2.0).replace(flags=S.FLAG_FAST_EXP)])
    nbytes = ctypes.c_size_t()
    assert L.clod_frame_workspace_size(1000, views, 2, ctypes.byref(nbytes), None) == abi.CLOD_ERR_ARG
    assert b"CLOD_FAST_EXP" in L.clod_last_error()
    same = clod.view_array([S.tiny_view(1.0).replace(flags=S.FLAG_FAST_EXP),
                            S.tiny_view(2.0).replace(flags=S.FLAG_FAST_EXP)])
    assert L.clod_frame_workspace_size(1000, same, 2, ctypes.byref(nbytes), None) == 0
