"""Batched reconstruction of datasets with uneven widths and angle counts.

A thin wrapper of the tcp_batch_* calls of include/tcp.h: per dataset the
fused normalise+filter kernel, then one persistent backprojection launch over
all datasets, optionally captured once into a CUDA graph and replayed.  The
backprojector configuration is autotuned on the batch itself.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib


class Batch:
    """datasets: list of dicts with keys raw, dark, flat, vol (CUDA tensors),
    theta (angles), center, and optionally filter ('shepp') and pad ('edge').
    The tensors must outlive the batch."""

    def __init__(self, datasets, sino_dtype=torch.float16, autotune: bool = True, stream=None, config=None):
        self._keep = []
        items = (_lib.BatchItem * len(datasets))()
        for i, d in enumerate(datasets):
            th = _lib.theta_array(d["theta"])
            self._keep.append(th)
            it = items[i]
            it.raw = _lib.desc(d["raw"], _lib.U16)
            it.dark = _lib.desc(d["dark"], _lib.U16 if d["dark"].dim() == 3 else None)
            it.flat = _lib.desc(d["flat"], _lib.U16 if d["flat"].dim() == 3 else None)
            it.vol = _lib.desc(d["vol"])
            it.theta = th.ctypes.data
            it.center = float(d["center"])
            it.filter = _lib.FILTERS[d.get("filter", "shepp")]
            it.pad_mode = _lib.PADS[d.get("pad", "edge")]
        opts = _lib.BatchOpts()
        opts.sino_dtype = _lib._TORCH_DTYPE[_lib.DTYPES[sino_dtype]]
        opts.autotune = int(bool(autotune))
        h = ctypes.c_void_p()
        if config is not None:  # (k_slices, theta_stage, rows_per_thread, kernel), used without autotune
            _lib.call("tcp_set_backproject_config", ctypes.byref(_lib.BpConfig(*config)))
        try:
            _lib.call("tcp_batch_create", items, len(datasets), ctypes.byref(opts), _lib.stream_ptr(stream),
                      ctypes.byref(h))
        finally:
            if config is not None:
                _lib.call("tcp_set_backproject_config", None)
        self._h = h
        self.datasets = datasets

    def run(self, stream=None):
        _lib.call("tcp_batch_run", self._h, _lib.stream_ptr(stream))

    def capture(self, stream: torch.cuda.Stream):
        """Capture one run into a CUDA graph (on a non-default stream)."""
        _lib.call("tcp_batch_capture", self._h, _lib.stream_ptr(stream))

    def replay(self, stream=None):
        _lib.call("tcp_batch_replay", self._h, _lib.stream_ptr(stream))

    def info(self) -> dict:
        c = _lib.BpConfig()
        ms = ctypes.c_float()
        units = ctypes.c_int64()
        blocks = ctypes.c_int32()
        _lib.call("tcp_batch_info", self._h, ctypes.byref(c), ctypes.byref(ms), ctypes.byref(units),
                  ctypes.byref(blocks))
        return {"config": (c.k_slices, c.theta_stage, c.rows_per_thread), "kernel": c.kernel, "tuned_ms": ms.value,
                "work_units": units.value, "grid_blocks": blocks.value}

    def close(self):
        if getattr(self, "_h", None):
            _lib.call("tcp_batch_destroy", self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def autotune_backproject(sino: torch.Tensor, theta, center: float, vol: torch.Tensor, stream=None):
    """Time every backprojector configuration on these tensors; later calls
    with the same shapes use the fastest.  Returns (config, ms)."""
    th = _lib.theta_array(theta)
    a, b = _lib.desc(sino), _lib.desc(vol)
    c = _lib.BpConfig()
    ms = ctypes.c_float()
    _lib.call("tcp_autotune_backproject", _lib.ref(a), th.ctypes.data_as(ctypes.c_void_p), float(center),
              _lib.ref(b), _lib.stream_ptr(stream), ctypes.byref(c), ctypes.byref(ms))
    return (c.k_slices, c.theta_stage, c.rows_per_thread, c.kernel), ms.value
