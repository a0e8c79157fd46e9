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


@pytest.mark.parametrize("dt", [torch.float32, torch.float16, torch.bfloat16])
def test_noalloc_matches_allocating_normalize_twice(dt):
    tol = {torch.float32: 1e-6, torch.float16: 1e-3, torch.bfloat16: 8e-3}[dt]
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


def test_noalloc_accepts_exactly_its_maximum():
    # nz * ndet == 2^20 fills the fixed array exactly and is accepted
    nz, nd, nt = 512, 2048, 3
    g = torch.Generator(device=DEV)
    g.manual_seed(3)
    raw = torch.randint(3000, 30000, (nt, nz, nd), dtype=torch.int16, device=DEV, generator=g)
    dark = torch.randint(90, 110, (2, nz, nd), dtype=torch.int16, device=DEV, generator=g)
    flat = torch.randint(30000, 32000, (2, nz, nd), dtype=torch.int16, device=DEV, generator=g)
    ref = torch.empty((nz, nt, nd), device=DEV)
    got = torch.full((nz, nt, nd), float("nan"), device=DEV)
    _normalize("tcp_normalize", raw, dark, flat, ref)
    _normalize("tcp_normalize_noalloc", raw, dark, flat, got)
    torch.cuda.synchronize()
    assert float((got - ref).abs().max()) <= 1e-6 * float(ref.abs().max())


def _cudart():
    # the CUDA runtime the library was linked against (already loaded with it)
    for name in ("libcudart.so.13", "libcudart.so"):
        try:
            return ctypes.CDLL(name)
        except OSError:
            continue
    pytest.skip("CUDA runtime library not found by name")


def test_noalloc_takes_nothing_from_the_stream_ordered_pool():
    # tcp_normalize averages U16 frames in scratch from the device's default
    # memory pool; the allocation-free call must not touch that pool.  The
    # pool's high-water mark of used memory is reset before each call and read
    # after it: the allocating call raises it above the use at the reset (the
    # check sees allocations), the allocation-free one does not.
    rt = _cudart()
    pool = ctypes.c_void_p()
    assert rt.cudaDeviceGetDefaultMemPool(ctypes.byref(pool), torch.cuda.current_device()) == 0
    USED_CURRENT, USED_HIGH = 7, 8  # cudaMemPoolAttrUsedMemCurrent, cudaMemPoolAttrUsedMemHigh

    def attr(a):
        v = ctypes.c_uint64(0)
        assert rt.cudaMemPoolGetAttribute(pool, a, ctypes.byref(v)) == 0
        return v.value

    def reset_high():
        zero = ctypes.c_uint64(0)
        assert rt.cudaMemPoolSetAttribute(pool, USED_HIGH, ctypes.byref(zero)) == 0

    ds = synth.shepp_logan_dataset(ntheta=40, ndet=256, nz=8, center=128.0, seed=5)
    raw, dark, flat = _u16(ds.raw), _u16(ds.dark), _u16(ds.flat)
    ref = torch.empty((8, 40, 256), device=DEV)
    got = torch.empty((8, 40, 256), device=DEV)
    torch.cuda.synchronize()
    reset_high()
    base = attr(USED_CURRENT)
    _normalize("tcp_normalize", raw, dark, flat, ref)
    torch.cuda.synchronize()
    assert attr(USED_HIGH) >= base + 2 * 8 * 256 * 4  # two FP32 means were taken from the pool
    for _ in range(2):
        torch.cuda.synchronize()
        reset_high()
        base = attr(USED_CURRENT)
        _normalize("tcp_normalize_noalloc", raw, dark, flat, got)
        torch.cuda.synchronize()
        assert attr(USED_HIGH) <= base  # a reset mark stays at 0 until the next allocation
        assert attr(USED_CURRENT) == base
    assert torch.equal(got, ref)
