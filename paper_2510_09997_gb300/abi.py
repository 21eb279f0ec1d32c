"""ctypes mirror of include/clod.h (argument marshalling only)."""
from __future__ import annotations

import ctypes

c_status = ctypes.c_int32
P = ctypes.c_void_p

CLOD_OK = 0
CLOD_ERR_ARG = 1
CLOD_ERR_CAPACITY = 2
CLOD_ERR_CUDA = 3
CLOD_ERR_TIMEOUT = 4
CLOD_ERR_QUEUE_FULL = 5
CLOD_ERR_NOT_READY = 6
CLOD_ERR_NAN = 7

CLOD_LOD_OFF = 1
CLOD_NO_NORMALIZE = 2
CLOD_FAST_EXP = 4

STATUS_NAMES = {0: "CLOD_OK", 1: "CLOD_ERR_ARG", 2: "CLOD_ERR_CAPACITY", 3: "CLOD_ERR_CUDA",
                4: "CLOD_ERR_TIMEOUT", 5: "CLOD_ERR_QUEUE_FULL", 6: "CLOD_ERR_NOT_READY", 7: "CLOD_ERR_NAN"}


class clod_scene(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("sh_degree", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("means", P), ("scales", P), ("quats", P), ("opacity", P), ("sh", P), ("decay", P)]


class clod_view(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32), ("viewmat", ctypes.c_float * 12),
                ("fx", ctypes.c_float), ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("near_z", ctypes.c_float), ("campos", ctypes.c_float * 3), ("s_v", ctypes.c_float),
                ("tau", ctypes.c_float), ("eps", ctypes.c_float), ("bg", ctypes.c_float * 3),
                ("flags", ctypes.c_uint32), ("region_x", ctypes.c_int32), ("region_y", ctypes.c_int32),
                ("full_width", ctypes.c_int32), ("full_height", ctypes.c_int32), ("budget", ctypes.c_uint32)]


class clod_frame_layout(ctypes.Structure):
    _fields_ = [(k, ctypes.c_uint64) for k in
                ("total_bytes", "views", "dmax_key", "n_survivors", "rec0", "rec1", "rec2", "depth", "rect",
                 "tile_count", "tile_offset")] + [("total_tiles", ctypes.c_uint32), ("n_views", ctypes.c_uint32)]


class clod_server_cfg(ctypes.Structure):
    _fields_ = [("max_views_per_batch", ctypes.c_int32), ("n_slots", ctypes.c_int32),
                ("queue_capacity", ctypes.c_int32), ("use_graphs", ctypes.c_int32),
                ("max_pixels_per_batch", ctypes.c_uint64), ("pair_capacity", ctypes.c_uint64),
                ("batch_window_us", ctypes.c_int32), ("max_width", ctypes.c_int32),
                ("max_height", ctypes.c_int32), ("fast_exp", ctypes.c_int32)]


class clod_adam_cfg(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_float * 6), ("beta1", ctypes.c_float), ("beta2", ctypes.c_float),
                ("eps", ctypes.c_float), ("step", ctypes.c_int32), ("keep_grads", ctypes.c_int32)]


class clod_req_stats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("batch_size", ctypes.c_int32), ("submit_us", ctypes.c_double),
                ("launch_us", ctypes.c_double), ("done_us", ctypes.c_double), ("n_rendered", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32), ("n_pairs", ctypes.c_uint64)]


SIGNATURES = {
    "clod_last_error": ([], ctypes.c_char_p),
    "clod_version": ([], ctypes.c_char_p),
    "clod_frame_workspace_size": ([ctypes.c_int64, P, ctypes.c_int32, P, P], c_status),
    "clod_preprocess": ([P, P, ctypes.c_int32, P, ctypes.c_size_t, P, P, P, P, P], c_status),
    "clod_bin_sort": ([P, ctypes.c_uint64, P, P, P, P], c_status),
    "clod_render_fwd": ([P, P, P, P, P, P, P], c_status),
    "clod_render_fwd_count": ([P, P, P, P, P, P, P, P], c_status),
    "clod_frame_check": ([P, ctypes.c_uint64, P, P], c_status),
    # backward
    "clod_backward_workspace_size": ([ctypes.c_int64, ctypes.c_int32, P], c_status),
    "clod_render_bwd": ([P, P, P, P, P, P, P, P, P, P, ctypes.c_size_t, P, P, P, P, P, P, P], c_status),
    "clod_render_bwd_set": ([P, P, P, P, P, P, P, P, P, P, ctypes.c_size_t, P, P, P, P, P, P, P], c_status),
    "clod_l1_loss": ([P, P, ctypes.c_int64, ctypes.c_float, P, P, P], c_status),
    "clod_probe_fma": ([ctypes.c_int32, P, P, P], c_status),
    "clod_render_loss_workspace_size": ([ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, P], c_status),
    "clod_render_loss": ([P, P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_float, ctypes.c_float, P,
                          ctypes.c_size_t, P, P, P], c_status),
    "clod_step_weights": ([P, ctypes.c_int32, ctypes.c_float, P], c_status),
    "clod_lreg_grad": ([P, ctypes.c_int64, ctypes.c_int32, P, P, ctypes.c_float, P, P, P, P, P], c_status),
    "clod_adam_state_size": ([ctypes.c_int64, ctypes.c_int32, P], c_status),
    "clod_adam_step": ([P, ctypes.c_int64, ctypes.c_int32, P, P, P, P, P, P, P], c_status),
    "clod_render_noalloc": ([P, P, P, P, P, P], c_status),
    # serving
    "clod_server_create": ([P, P, P], c_status),
    "clod_serve_submit": ([P, P, P, P], c_status),
    "clod_serve_poll": ([P, ctypes.c_uint64, P, P], c_status),
    "clod_serve_wait": ([P, ctypes.c_uint64, ctypes.c_int64, P], c_status),
    "clod_server_destroy": ([P], c_status),
}


def declare(L) -> None:
    for name, (args, res) in SIGNATURES.items():
        fn = getattr(L, name, None)
        if fn is None:
            continue
        fn.argtypes = args
        fn.restype = res
