"""Python binding of the continuous-batching render server (clod_server_* in
include/clod.h).  The server, its worker thread, batching, CUDA graphs and
admission all live in libclod; this wraps the calls."""
from __future__ import annotations

import ctypes
from typing import Optional

import torch

from . import abi
from . import clod as C


class Server:
    def __init__(self, scene: "C.DeviceScene", max_views_per_batch: int = 8, n_slots: int = 2,
                 queue_capacity: int = 100000, use_graphs: bool = True, max_pixels_per_batch: Optional[int] = None,
                 pair_capacity: int = 1 << 25, batch_window_us: int = 0, max_width: int = 3840,
                 max_height: int = 2160, fast_exp: bool = False):
        C.require_cuda()
        self.scene = scene          # keeps the device arrays alive
        cfg = abi.clod_server_cfg()
        cfg.max_views_per_batch = max_views_per_batch
        cfg.n_slots = n_slots
        cfg.queue_capacity = queue_capacity
        cfg.use_graphs = 1 if use_graphs else 0
        cfg.max_pixels_per_batch = max_pixels_per_batch or max_width * max_height * 2
        cfg.pair_capacity = pair_capacity
        cfg.batch_window_us = batch_window_us
        cfg.max_width = max_width
        cfg.max_height = max_height
        cfg.fast_exp = 1 if fast_exp else 0
        self.cfg = cfg
        self.h = ctypes.c_void_p()
        C.check("clod_server_create", C.lib().clod_server_create(ctypes.byref(scene.c), ctypes.byref(cfg),
                                                                 ctypes.byref(self.h)))
        self._views = {}

    def submit(self, view, out: torch.Tensor) -> int:
        cv = C.cview(view)
        t = ctypes.c_uint64()
        C.check("clod_serve_submit", C.lib().clod_serve_submit(self.h, ctypes.byref(cv), C._ptr(out), ctypes.byref(t)))
        self._views[t.value] = out
        return int(t.value)

    def poll(self, ticket: int):
        done = ctypes.c_int32()
        st = abi.clod_req_stats()
        s = C.lib().clod_serve_poll(self.h, ticket, ctypes.byref(done), ctypes.byref(st))
        if s == abi.CLOD_ERR_NOT_READY:
            return None
        self._views.pop(ticket, None)
        C.check("clod_serve_poll", s)
        return st

    def wait(self, ticket: int, timeout_s: float = 60.0):
        st = abi.clod_req_stats()
        C.check("clod_serve_wait", C.lib().clod_serve_wait(self.h, ticket, int(timeout_s * 1e6), ctypes.byref(st)))
        self._views.pop(ticket, None)
        return st

    def close(self):
        if self.h:
            C.check("clod_server_destroy", C.lib().clod_server_destroy(self.h))
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
