"""GB300-native chunked parallel-beam filtered backprojection.

Python face of libtcp (include/tcp.h), following Nikitin, "TomocuPy: efficient
GPU-based tomographic reconstruction with asynchronous data processing"
(arXiv 2209.08450): dark/flat normalisation with -log (Sec. 2.2), Fourier
ramp filtering of detector rows (Sec. 2.2), LineRec backprojection (Sec. 2.2
and Sec. 3), the adjoint projector, chunked asynchronous FBP (Sec. 2.3) and
16-bit storage with FP32 accumulation (Sec. 2.1).

Every function marshals arguments and calls one C-ABI entry point; the
computation is in the library's CUDA kernels.  Tensors live on the GPU
(torch); angles are radians.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import TcpError, load  # noqa: F401

__all__ = ["frame_mean", "normalize", "normalize_filter", "angle_major", "filter_", "backproject", "project", "fourierrec", "device_check",
           "set_checked", "cache_clear", "set_backproject_config", "get_backproject_config",
           "TcpError", "load", "padded_length", "tc_launch_shape"]


def _as_u16(t: torch.Tensor) -> torch.Tensor:
    if t.dtype == torch.int16 or (hasattr(torch, "uint16") and t.dtype == torch.uint16):
        return t
    raise TypeError("raw/dark/flat frames must be uint16 (or int16 holding the same bits)")


def padded_length(ndet: int, smooth: bool = False) -> int:
    """Padded row length of the filter (tcp_padded_length): the next power of
    two >= 2 ndet; with `smooth`, the smallest of that, the next 3 * 2^k
    (from 48 on) and the next 5 * 2^k (from 80 on) >= 2 ndet."""
    return int(_lib.load().tcp_padded_length(int(ndet), _lib.PADS["edge_smooth" if smooth else "edge"]))


def tc_launch_shape(nz: int, sino_dtype=torch.float16, theta_stage: int = 2, blocks_per_sm: int = 2) -> dict:
    """Launch shape of the tensor-core backprojector (tcp_tc_launch_shape) for
    nz slices: slices per block, angles per stage, blocks per SM, ring depths
    and shared memory per block.  sino_dtype: float16, bfloat16 or "f16x2"."""
    sh = _lib.TcShape()
    _lib.call("tcp_tc_launch_shape", int(nz), _lib.dtype_code(sino_dtype), int(theta_stage), int(blocks_per_sm),
              ctypes.byref(sh))
    return {f: getattr(sh, f) for f, _ in _lib.TcShape._fields_}


def frame_mean(frames: torch.Tensor, stream=None) -> torch.Tensor:
    """FP32 mean over frames of uint16 frames[f][z][j] (dark or flat)."""
    frames = _as_u16(frames)
    out = torch.empty(frames.shape[1:], dtype=torch.float32, device=frames.device)
    a, b = _lib.desc(frames, _lib.U16), _lib.desc(out)
    _lib.call("tcp_frame_mean", _lib.ref(a), _lib.ref(b), _lib.stream_ptr(stream))
    return out


def normalize(raw: torch.Tensor, dark: torch.Tensor, flat: torch.Tensor, out: torch.Tensor | None = None,
              dtype=torch.float32, stream=None) -> torch.Tensor:
    """raw uint16 [theta][z][j] -> sinogram [z][theta][j] = -ln((raw-dark)/(flat-dark)).

    dark/flat are uint16 frames [nf][z][j] or FP32 means [z][j]."""
    raw = _as_u16(raw)
    nt, nz, nd = raw.shape
    if out is None:
        out = torch.empty((nz, nt, nd), dtype=_lib.DTYPES[dtype], device=raw.device)

    def dd(x):
        return _lib.desc(x, _lib.U16 if x.dim() == 3 else None)

    r, d, f, o = _lib.desc(raw, _lib.U16), dd(dark), dd(flat), _lib.desc(out)
    _lib.call("tcp_normalize", _lib.ref(r), _lib.ref(d), _lib.ref(f), _lib.ref(o), _lib.stream_ptr(stream))
    return out


def angle_major(shape, dtype, device, planes: int | None = None) -> torch.Tensor:
    """Empty sinogram [z][theta][j] (or [planes][z][theta][j]) stored angle-major,
    [theta][z][j] in memory: the layout of the raw frames and of tcp_fbp's chunks.
    The tensor-core backprojector copies one angle's window of all slices at a
    time, which is then one contiguous block (2x faster for FP16 storage at
    2048^2 x 256 slices, 1.35x for F16X2 pairs, than the slice-major layout)."""
    nz, nt, nd = shape
    if planes is None:
        return torch.empty((nt, nz, nd), dtype=dtype, device=device).permute(1, 0, 2)
    return torch.empty((planes, nt, nz, nd), dtype=dtype, device=device).permute(0, 2, 1, 3)


def normalize_filter(raw: torch.Tensor, dark: torch.Tensor, flat: torch.Tensor, center: float,
                     filter: str = "shepp", pad: str = "edge", out: torch.Tensor | None = None,
                     dtype=torch.float32, weight: float | None = None, stream=None) -> torch.Tensor:
    """Fused normalise + filter: raw uint16 [theta][z][j] -> filtered sinogram
    [z][theta][j] in `dtype` (allocated angle-major, see `angle_major`), -log
    computed in FP32 in shared memory and the result rounded once (the
    16-bit-safe order of the two steps).  `weight`
    replaces the pi/ntheta factor (see backproject(scale=...)).  dtype="f16x2"
    returns [2][z][theta][j] float16: hi and lo planes of the FP32 result (use a
    weight such as 1024 so that values stay above 2^-3)."""
    raw = _as_u16(raw)
    nt, nz, nd = raw.shape
    if out is None:
        if dtype == _lib.SPLIT:  # FP16 hi/lo planes of the FP32 result
            out = angle_major((nz, nt, nd), torch.float16, raw.device, planes=2)
        else:
            out = angle_major((nz, nt, nd), _lib.DTYPES[dtype], raw.device)

    def dd(x):
        return _lib.desc(x, _lib.U16 if x.dim() == 3 else None)

    r, d, f = _lib.desc(raw, _lib.U16), dd(dark), dd(flat)
    o = _lib.desc(out, _lib.F16X2 if _lib.is_split(out) else None)
    _lib.call("tcp_normalize_filter_ex", _lib.ref(r), _lib.ref(d), _lib.ref(f), _lib.ref(o), _lib.FILTERS[filter],
              float(center), _lib.PADS[pad], float(weight or 0.0), _lib.stream_ptr(stream))
    return out


def filter_(sino: torch.Tensor, center: float, filter: str = "shepp", pad: str = "edge",
            ntheta: int | None = None, stream=None) -> torch.Tensor:
    """In-place FBP filter of every detector row; moves the axis from `center` to ndet/2."""
    d = _lib.desc(sino)
    _lib.call("tcp_filter_ex", _lib.ref(d), _lib.FILTERS[filter], float(center), _lib.PADS[pad],
              int(ntheta or 0), _lib.stream_ptr(stream))
    return sino


def backproject(sino: torch.Tensor, theta, center: float, n: int | None = None,
                out: torch.Tensor | None = None, dtype=None, scale: float = 1.0, stream=None) -> torch.Tensor:
    """LineRec backprojection sino[z][theta][j] -> vol[z][n][n]: scale x (sum over angles).
    A [2][z][theta][j] float16 sinogram is an F16X2 hi/lo pair (FP32-accurate,
    tensor cores; the default output dtype is then float32)."""
    th = _lib.theta_array(theta)
    split = _lib.is_split(sino)
    nz, nt, nd = sino.shape[1:] if split else sino.shape
    if out is None:
        n = nd if n is None else n
        odt = _lib.DTYPES[dtype] if dtype is not None else (torch.float32 if split else sino.dtype)
        out = torch.empty((nz, n, n), dtype=odt, device=sino.device)
    a, b = _lib.desc(sino, _lib.F16X2 if split else None), _lib.desc(out)
    _lib.call("tcp_backproject_ex", _lib.ref(a), th.ctypes.data_as(ctypes.c_void_p), float(center), _lib.ref(b),
              float(scale), _lib.stream_ptr(stream))
    return out


def project(vol: torch.Tensor, theta, center: float, ndet: int | None = None,
            out: torch.Tensor | None = None, dtype=None, stream=None) -> torch.Tensor:
    """Adjoint projector vol[z][n][n] -> sino[z][theta][ndet]."""
    th = _lib.theta_array(theta)
    nz, n, _ = vol.shape
    if out is None:
        ndet = n if ndet is None else ndet
        out = torch.empty((nz, th.shape[0], ndet), dtype=_lib.DTYPES[dtype or vol.dtype], device=vol.device)
    a, b = _lib.desc(vol), _lib.desc(out)
    _lib.call("tcp_project", _lib.ref(a), th.ctypes.data_as(ctypes.c_void_p), float(center), _lib.ref(b),
              _lib.stream_ptr(stream))
    return out


def fourierrec(sino: torch.Tensor, theta, center: float, n: int | None = None,
               out: torch.Tensor | None = None, dtype=None, scale: float = 1.0, width: int = 0,
               stream=None) -> torch.Tensor:
    """FourierRec backprojection sino[z][theta][j] -> vol[z][n][n] (n even): scale x
    (sum over angles of the trigonometric interpolant of each zero-padded row),
    evaluated on an oversampled Cartesian frequency grid with a window of
    `width` points (0: 7 for float32 output, 5 for 16-bit)."""
    th = _lib.theta_array(theta)
    nz, nt, nd = sino.shape
    if out is None:
        n = nd if n is None else n
        out = torch.empty((nz, n, n), dtype=_lib.DTYPES[dtype or sino.dtype], device=sino.device)
    a, b = _lib.desc(sino), _lib.desc(out)
    _lib.call("tcp_fourierrec", _lib.ref(a), th.ctypes.data_as(ctypes.c_void_p), float(center), _lib.ref(b),
              float(scale), int(width), _lib.stream_ptr(stream))
    return out


def lprec(sino: torch.Tensor, theta, center: float, n: int | None = None, out: torch.Tensor | None = None,
          dtype=None, scale: float = 1.0, oversampling: float = 0.0, stream=None) -> torch.Tensor:
    """LpRec backprojection sino[z][theta][j] -> vol[z][n][n]: scale x (sum over
    angles of each row's interpolating cubic B-spline), evaluated per third of
    the angles in log-polar coordinates (grid steps 1/oversampling pixel at
    the far radius; 0 picks 2).  The angles must be equally spaced over a half
    turn."""
    th = _lib.theta_array(theta)
    nz, nt, nd = sino.shape
    if out is None:
        n = nd if n is None else n
        out = torch.empty((nz, n, n), dtype=_lib.DTYPES[dtype or sino.dtype], device=sino.device)
    a, b = _lib.desc(sino), _lib.desc(out)
    _lib.call("tcp_lprec", _lib.ref(a), th.ctypes.data_as(ctypes.c_void_p), float(center), _lib.ref(b),
              float(scale), float(oversampling), _lib.stream_ptr(stream))
    return out


__all__.append("lprec")


def device_check(stream=None) -> int:
    """Read and clear the device error word (synchronises the stream); raises if set."""
    w = ctypes.c_uint32(0)
    _lib.call("tcp_device_check", _lib.stream_ptr(stream), ctypes.byref(w))
    return w.value


def set_checked(on: bool) -> None:
    _lib.call("tcp_set_checked", int(bool(on)))


def cache_clear() -> None:
    _lib.call("tcp_cache_clear")


def set_backproject_config(k_slices: int | None = None, theta_stage: int = 16, rows_per_thread: int = 4,
                           kernel: int = 0) -> None:
    """Fix the backprojector configuration (None: automatic).  kernel=1 selects
    the tensor-core backprojector for FP16/BF16 sinograms, kernel=2 the
    CUDA-core form for FP32 sinograms with slice pairs (packed FP32x2 FMAs,
    sample reuse down each voxel column), kernel=3 the tensor-core
    backprojector with its rings sized for two thread blocks per SM (FP16/BF16
    sinograms, at most 128 slices per block)."""
    if k_slices is None:
        _lib.load().tcp_set_backproject_config(None)
        return
    c = _lib.BpConfig(k_slices, theta_stage, rows_per_thread, kernel)
    _lib.call("tcp_set_backproject_config", ctypes.byref(c))


def get_backproject_config(nz, ntheta, ndet, n, sino_dtype=torch.float32, vol_dtype=torch.float32) -> tuple:
    c = _lib.BpConfig()
    _lib.call("tcp_get_backproject_config", nz, ntheta, ndet, n, _lib.dtype_code(sino_dtype),
              _lib.dtype_code(vol_dtype), ctypes.byref(c))
    return (c.k_slices, c.theta_stage, c.rows_per_thread, c.kernel)


def fbp(raw: torch.Tensor, dark: torch.Tensor, flat: torch.Tensor, theta, center: float,
        out: torch.Tensor | None = None, dtype=torch.float32, n: int | None = None, chunk_nz: int = 0,
        filter: str = "shepp", pad: str = "edge", sino_dtype=None, n_buffers: int = 2,
        algorithm: str = "linerec", width: int = 0, stream=None) -> torch.Tensor:
    """Chunked FBP (normalise -> filter -> backproject per z-slab, Sec. 2.3).

    raw uint16 [theta][z][j] and the output may be CUDA tensors or host tensors
    (page-locked host memory lets the slab copies overlap compute).  dark/flat
    are uint16 frames [nf][z][j] or FP32 means [z][j].  The volume is
    reconstructed about the filtered axis ndet/2 with the `center` shift folded
    into the filter.  algorithm: "linerec" (direct sum, linear interpolation),
    "fourierrec" (Fourier-slice evaluation, window `width`; n even) or
    "lprec" (log-polar evaluation with cubic B-splines, oversampling `width`,
    0 for 2; equally spaced angles).
    Returns `out` once the work is queued on the stream."""
    raw = _as_u16(raw)
    nt, nz, nd = raw.shape
    if out is None:
        n = nd if n is None else n
        out = torch.empty((nz, n, n), dtype=_lib.DTYPES[dtype], device=raw.device,
                          pin_memory=raw.device.type == "cpu")
    th = _lib.theta_array(theta)

    def dd(x):
        return _lib.desc(x, _lib.U16 if x.dim() == 3 else None)

    opts = _lib.FbpOpts()
    opts.chunk_nz = chunk_nz
    # None: the library's choice (F16X2 pairs for FP32 volumes when ndet % 8 == 0)
    opts.sino_dtype = -1 if sino_dtype is None else _lib.dtype_code(sino_dtype)
    opts.filter = _lib.FILTERS[filter]
    opts.pad_mode = _lib.PADS[pad]
    opts.n_buffers = n_buffers
    opts.algorithm = _lib.ALGORITHMS[algorithm]
    opts.width = width
    r, d, f, o = _lib.desc(raw, _lib.U16), dd(dark), dd(flat), _lib.desc(out)
    _lib.call("tcp_fbp", _lib.ref(r), _lib.ref(d), _lib.ref(f), th.ctypes.data_as(ctypes.c_void_p), float(center),
              _lib.ref(o), ctypes.byref(opts), _lib.stream_ptr(stream))
    return out


__all__.append("fbp")


def try_centers(raw: torch.Tensor, dark: torch.Tensor, flat: torch.Tensor, theta, centers,
                slice: int | None = None, n: int | None = None, out: torch.Tensor | None = None,
                dtype=torch.float32, filter: str = "shepp", algorithm: str = "linerec", width: int = 0,
                stream=None) -> torch.Tensor:
    """Multi-centre "try" reconstruction (Sec. 2.4): slice `slice` (default the
    middle one) reconstructed about every candidate axis in `centers`, by
    LineRec or FourierRec (`algorithm`); returns [len(centers)][n][n] on the
    CUDA device."""
    raw = _as_u16(raw)
    nt, nz, nd = raw.shape
    c = np.ascontiguousarray(centers, dtype=np.float64).reshape(-1)
    if slice is None:
        slice = nz // 2
    if out is None:
        n = nd if n is None else n
        out = torch.empty((c.shape[0], n, n), dtype=_lib.DTYPES[dtype], device="cuda")
    th = _lib.theta_array(theta)

    def dd(x):
        return _lib.desc(x, _lib.U16 if x.dim() == 3 else None)

    r, d, f, o = _lib.desc(raw, _lib.U16), dd(dark), dd(flat), _lib.desc(out)
    _lib.call("tcp_try_centers_ex", _lib.ref(r), int(slice), _lib.ref(d), _lib.ref(f),
              th.ctypes.data_as(ctypes.c_void_p), c.ctypes.data_as(ctypes.c_void_p), int(c.shape[0]), _lib.ref(o),
              _lib.FILTERS[filter], _lib.ALGORITHMS[algorithm], int(width), _lib.stream_ptr(stream))
    return out


__all__.append("try_centers")

from .plan import Plan  # noqa: E402

__all__.append("Plan")
