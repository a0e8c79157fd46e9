"""Reconstruction plans (the tcp_plan_* calls of include/tcp.h): argument
marshalling only.

A plan is created once per geometry (angles, detector width, volume side,
slices, options) and owns every table and buffer the reconstruction needs, so
that `fbp`, `filter_`, `backproject` and `project` through it allocate
nothing and never synchronise: their first call may be captured into a CUDA
graph.
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib


class Plan:
    """ntheta angles `theta`, ndet detector pixels, nz slices (the most one
    `fbp` call reconstructs), volume side n (default ndet), rotation axis
    `center`.  host_raw / host_vol: allocate the staging rings for host raw
    input / host volume output; host_frames: how many U16 dark/flat frames may
    come from host memory.  The remaining keywords are tcp_fbp's options."""

    def __init__(self, theta, ndet: int, nz: int, center: float, n: int | None = None, dtype=torch.float32,
                 chunk_nz: int = 0, filter: str = "shepp", pad: str = "edge", sino_dtype=None, n_buffers: int = 2,
                 algorithm: str = "linerec", width: int = 0, host_raw: bool = False, host_vol: bool = False,
                 host_frames: int = 0, trace: bool = False):
        th = _lib.theta_array(theta)
        d = _lib.PlanDesc()
        d.ntheta = th.shape[0]
        d.nz = nz
        d.ndet = ndet
        d.n = ndet if n is None else n
        d.center = float(center)
        d.vol_dtype = _lib.dtype_code(dtype)
        d.io = (_lib.IO_HOST_RAW if host_raw else 0) | (_lib.IO_HOST_VOL if host_vol else 0)
        d.host_frames = host_frames
        d.trace = int(bool(trace))
        o = d.opts
        o.chunk_nz = chunk_nz
        o.sino_dtype = -1 if sino_dtype is None else _lib.dtype_code(sino_dtype)
        o.filter = _lib.FILTERS[filter]
        o.pad_mode = _lib.PADS[pad]
        o.n_buffers = n_buffers
        o.algorithm = _lib.ALGORITHMS[algorithm]
        o.width = width
        h = ctypes.c_void_p()
        _lib.call("tcp_plan_create", ctypes.byref(d), th.ctypes.data_as(ctypes.c_void_p), ctypes.byref(h))
        self._h = h
        self.ntheta, self.ndet, self.nz, self.n = d.ntheta, d.ndet, d.nz, d.n
        self.dtype = _lib.DTYPES[dtype]
        self.center = float(center)

    def info(self) -> dict:
        b = ctypes.c_int64()
        o = _lib.FbpOpts()
        _lib.call("tcp_plan_info", self._h, ctypes.byref(b), ctypes.byref(o))
        return {"device_bytes": b.value, "chunk_nz": o.chunk_nz, "sino_dtype": o.sino_dtype,
                "n_buffers": o.n_buffers, "width": o.width}

    def fbp(self, raw, dark, flat, out=None, stream=None) -> torch.Tensor:
        """tcp_fbp through the plan (raw U16 [ntheta][nz][ndet], nz <= the plan's)."""
        raw = raw.view(torch.int16) if raw.dtype != torch.int16 and raw.element_size() == 2 else raw
        nz = raw.shape[1]
        if out is None:
            out = torch.empty((nz, self.n, self.n), dtype=self.dtype, device=raw.device,
                              pin_memory=raw.device.type == "cpu")

        def dd(x):
            return _lib.desc(x, _lib.U16 if x.dim() == 3 else None)

        r, d, f, o = _lib.desc(raw, _lib.U16), dd(dark), dd(flat), _lib.desc(out)
        _lib.call("tcp_fbp_plan", self._h, _lib.ref(r), _lib.ref(d), _lib.ref(f), _lib.ref(o), _lib.stream_ptr(stream))
        return out

    def trace(self):
        """Per-chunk timeline of the last fbp call (plan made with trace=True):
        an array [chunks][6] of milliseconds from the call's start: upload
        start/end, compute start/end, download start/end (-1: no such copy)."""
        import numpy as np
        cnt = ctypes.c_int64()
        _lib.call("tcp_plan_trace", self._h, None, 0, ctypes.byref(cnt))
        out = np.zeros((max(cnt.value, 0), 6), dtype=np.float64)
        if cnt.value:
            _lib.call("tcp_plan_trace", self._h, out.ctypes.data_as(ctypes.c_void_p), cnt.value, ctypes.byref(cnt))
        return out

    def filter_(self, sino: torch.Tensor, stream=None) -> torch.Tensor:
        """In-place filter with the plan's filter, padding, centre and pi/ntheta weight."""
        d = _lib.desc(sino)
        _lib.call("tcp_filter_plan", self._h, _lib.ref(d), _lib.stream_ptr(stream))
        return sino

    def backproject(self, sino: torch.Tensor, center: float, out=None, dtype=None, scale: float = 1.0,
                    stream=None) -> torch.Tensor:
        split = _lib.is_split(sino)
        nz = sino.shape[1] if split else sino.shape[0]
        if out is None:
            out = torch.empty((nz, self.n, self.n), dtype=_lib.DTYPES[dtype or self.dtype], device=sino.device)
        s = _lib.desc(sino, _lib.F16X2 if split else None)
        o = _lib.desc(out)
        _lib.call("tcp_backproject_plan", self._h, _lib.ref(s), float(center), _lib.ref(o), float(scale),
                  _lib.stream_ptr(stream))
        return out

    def project(self, vol: torch.Tensor, center: float, out=None, stream=None) -> torch.Tensor:
        if out is None:
            out = torch.empty((vol.shape[0], self.ntheta, self.ndet), dtype=vol.dtype, device=vol.device)
        v, s = _lib.desc(vol), _lib.desc(out)
        _lib.call("tcp_project_plan", self._h, _lib.ref(v), float(center), _lib.ref(s), _lib.stream_ptr(stream))
        return out

    def close(self):
        if getattr(self, "_h", None):
            _lib.call("tcp_plan_destroy", self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
