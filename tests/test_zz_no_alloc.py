"""Allocation-free normalisation (tcp_normalize_noalloc), called through the C ABI.

For callers that may not allocate device memory while running (e.g. an
acquisition service that reserved the whole device for its own pool): the
frame means live in a fixed array inside the library.  The result must equal
the allocating tcp_normalize on the same frames, on two calls in a row (the
second call reuses the array the first one filled).  This file is collected
last so that a failure here stops a -x run only after every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

import synth
from paper_2209_08450_gb300 import _lib

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def _u16(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.uint16).view(np.int16)).to(DEV)


def _normalize(name, raw, dark, flat, out):
    lib = _lib.load()
    fn = getattr(lib, name)
    fn.argtypes = [ctypes.POINTER(_lib.TcpTensor)] * 4 + [ctypes.c_void_p]
    fn.restype = ctypes.c_int32
    r, d, f, o = _lib.desc(raw, _lib.U16), _lib.desc(dark, _lib.U16), _lib.desc(flat, _lib.U16), _lib.desc(out)
    st = fn(ctypes.byref(r), ctypes.byref(d), ctypes.byref(f), ctypes.byref(o), _lib.stream_ptr())
    assert st == 0, lib.tcp_last_error()


@pytest.mark.parametrize("dt", [torch.float32, torch.float16])
def test_noalloc_matches_allocating_normalize_twice(dt):
    tol = 1e-6 if dt == torch.float32 else 1e-3
    for seed, (nt, nz, nd) in enumerate([(64, 6, 200), (48, 9, 256)]):
        ds = synth.shepp_logan_dataset(ntheta=nt, ndet=nd, nz=nz, center=nd / 2, seed=seed)
        raw, dark, flat = _u16(ds.raw), _u16(ds.dark), _u16(ds.flat)
        ref = torch.empty((nz, nt, nd), dtype=dt, device=DEV)
        got = torch.full((nz, nt, nd), float("nan"), dtype=dt, device=DEV)
        _normalize("tcp_normalize", raw, dark, flat, ref)
        _normalize("tcp_normalize_noalloc", raw, dark, flat, got)
        torch.cuda.synchronize()
        err = (got.double() - ref.double()).norm() / ref.double().norm()
        assert float(err) <= tol


def test_noalloc_rejects_sizes_beyond_its_scratch():
    lib = _lib.load()
    fn = lib.tcp_normalize_noalloc
    fn.argtypes = [ctypes.POINTER(_lib.TcpTensor)] * 4 + [ctypes.c_void_p]
    fn.restype = ctypes.c_int32
    raw = torch.zeros((2, 513, 2048), dtype=torch.int16, device=DEV)   # 513 * 2048 > 2^20
    frames = torch.zeros((1, 513, 2048), dtype=torch.int16, device=DEV)
    out = torch.empty((513, 2, 2048), device=DEV)
    r, d, o = _lib.desc(raw, _lib.U16), _lib.desc(frames, _lib.U16), _lib.desc(out)
    st = fn(ctypes.byref(r), ctypes.byref(d), ctypes.byref(d), ctypes.byref(o), _lib.stream_ptr())
    assert st == 2 and b"exceeds the fixed scratch" in lib.tcp_last_error()
