"""ctypes binding of libtcp (include/tcp.h): argument marshalling only.

Every compute step runs in the library's CUDA kernels; PyTorch supplies device
memory and streams.  There is no fallback: if the library is not built or a
call fails, an exception is raised.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtcp.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "tcp.h")

U16, F16, BF16, F32, F16X2 = 0, 1, 2, 3, 4
FILTERS = {"shepp": 0, "parzen": 1, "ramp": 2, "none": 3}
PADS = {"edge": 0, "zero": 1, "edge_smooth": 2, "zero_smooth": 3}  # _smooth: 3 * 2^k padded lengths allowed

_TORCH_DTYPE = {torch.int16: U16, torch.float16: F16, torch.bfloat16: BF16, torch.float32: F32}
if hasattr(torch, "uint16"):
    _TORCH_DTYPE[torch.uint16] = U16
DTYPES = {"f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16,
          torch.float32: torch.float32, torch.float16: torch.float16, torch.bfloat16: torch.bfloat16}
SPLIT = "f16x2"  # FP32 values as FP16 hi + lo planes: a [2][nz][ntheta][ndet] float16 tensor


def is_split(t: torch.Tensor) -> bool:
    """A [2][nz][ntheta][ndet] float16 tensor is an F16X2 sinogram."""
    return t.dim() == 4 and t.dtype == torch.float16 and t.shape[0] == 2


def dtype_code(dt) -> int:
    """tcp_dtype code of a torch dtype or name (including "f16x2")."""
    if dt == SPLIT:
        return F16X2
    return _TORCH_DTYPE[DTYPES[dt]]


class TcpError(RuntimeError):
    def __init__(self, status: int, fn: str, msg: str):
        super().__init__("%s failed with status %d: %s" % (fn, status, msg))
        self.status = status


class TcpTensor(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("dtype", ctypes.c_int32), ("ndim", ctypes.c_int32),
                ("shape", ctypes.c_int64 * 4), ("stride", ctypes.c_int64 * 4)]


class BpConfig(ctypes.Structure):
    _fields_ = [("k_slices", ctypes.c_int32), ("theta_stage", ctypes.c_int32),
                ("rows_per_thread", ctypes.c_int32), ("kernel", ctypes.c_int32)]


class TcShape(ctypes.Structure):
    _fields_ = [("slices_per_block", ctypes.c_int32), ("angles_per_stage", ctypes.c_int32),
                ("blocks_per_sm", ctypes.c_int32), ("weight_stages", ctypes.c_int32),
                ("sinogram_stages", ctypes.c_int32), ("smem_bytes", ctypes.c_int64)]


class FbpOpts(ctypes.Structure):
    _fields_ = [("chunk_nz", ctypes.c_int32), ("sino_dtype", ctypes.c_int32), ("filter", ctypes.c_int32),
                ("pad_mode", ctypes.c_int32), ("n_buffers", ctypes.c_int32), ("algorithm", ctypes.c_int32),
                ("width", ctypes.c_int32), ("reserved", ctypes.c_int32 * 1)]


ALGORITHMS = {"linerec": 0, "fourierrec": 1, "lprec": 2}


_lock = threading.Lock()
_lib = None

_P = ctypes.c_void_p
_T = ctypes.POINTER(TcpTensor)
_D = ctypes.c_double
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64

SIGNATURES = {
    "tcp_status_string": ([_I32], ctypes.c_char_p),
    "tcp_last_error": ([], ctypes.c_char_p),
    "tcp_version": ([], ctypes.c_int),
    "tcp_padded_length": ([_I64, _I32], _I64),
    "tcp_device_check": ([_P, ctypes.POINTER(ctypes.c_uint32)], _I32),
    "tcp_set_checked": ([_I32], _I32),
    "tcp_cache_clear": ([], _I32),
    "tcp_frame_mean": ([_T, _T, _P], _I32),
    "tcp_normalize": ([_T, _T, _T, _T, _P], _I32),
    "tcp_filter": ([_T, _I32, _D, _P], _I32),
    "tcp_normalize_filter": ([_T, _T, _T, _T, _I32, _D, _I32, _P], _I32),
    "tcp_normalize_filter_ex": ([_T, _T, _T, _T, _I32, _D, _I32, _D, _P], _I32),
    "tcp_backproject_ex": ([_T, _P, _D, _T, _D, _P], _I32),
    "tcp_filter_ex": ([_T, _I32, _D, _I32, _I64, _P], _I32),
    "tcp_backproject": ([_T, _P, _D, _T, _P], _I32),
    "tcp_project": ([_T, _P, _D, _T, _P], _I32),
    "tcp_fourierrec": ([_T, _P, _D, _T, _D, _I32, _P], _I32),
    "tcp_lprec": ([_T, _P, _D, _T, _D, _D, _P], _I32),
    "tcp_set_backproject_config": ([ctypes.POINTER(BpConfig)], _I32),
    "tcp_get_backproject_config": ([_I64, _I64, _I64, _I64, _I32, _I32, ctypes.POINTER(BpConfig)], _I32),
    "tcp_tc_launch_shape": ([_I64, _I32, _I32, _I32, ctypes.POINTER(TcShape)], _I32),
    "tcp_fbp": ([_T, _T, _T, _P, _D, _T, ctypes.POINTER(FbpOpts), _P], _I32),
    "tcp_try_centers": ([_T, _I64, _T, _T, _P, _P, _I64, _T, _I32, _P], _I32),
    "tcp_try_centers_ex": ([_T, _I64, _T, _T, _P, _P, _I64, _T, _I32, _I32, _I32, _P], _I32),
}


def header_functions() -> list[str]:
    """Names of the functions include/tcp.h declares."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tcp_[a-z0-9_]+)\s*\(", text)))


def load(path: str | None = None):
    """Load libtcp.so (built by paper_2209_08450_gb300.build); raises if missing."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise RuntimeError("libtcp.so is not built (%s); run __graft_entry__.build()" % p)
            lib = ctypes.CDLL(p)
            for name, (args, res) in SIGNATURES.items():
                if hasattr(lib, name):
                    f = getattr(lib, name)
                    f.argtypes = args
                    f.restype = res
            _lib = lib
    return _lib


def call(name: str, *args) -> None:
    lib = load()
    st = getattr(lib, name)(*args)
    if st != 0:
        msg = lib.tcp_last_error().decode(errors="replace")
        raise TcpError(st, name, msg)


def desc(t: torch.Tensor | None, dtype_code: int | None = None) -> TcpTensor:
    """Descriptor of a tensor: pointer, dtype code, shape, element strides."""
    d = TcpTensor()
    if t is None:
        return d
    if t.dim() > 4 or t.dim() < 1:
        raise ValueError("tensors must have 1 to 4 dimensions")
    code = dtype_code if dtype_code is not None else _TORCH_DTYPE.get(t.dtype)
    if code is None:
        raise TypeError("unsupported dtype %s" % t.dtype)
    d.data = t.data_ptr() if t.numel() > 0 else None
    d.dtype = code
    d.ndim = t.dim()
    for i in range(t.dim()):
        d.shape[i] = t.shape[i]
        d.stride[i] = t.stride(i)
    return d


def ref(d: TcpTensor):
    return ctypes.byref(d)


def stream_ptr(stream: torch.cuda.Stream | None = None) -> ctypes.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def theta_array(theta) -> np.ndarray:
    if isinstance(theta, torch.Tensor):
        theta = theta.detach().cpu().numpy()
    return np.ascontiguousarray(theta, dtype=np.float64)


class BatchItem(ctypes.Structure):
    _fields_ = [("raw", TcpTensor), ("dark", TcpTensor), ("flat", TcpTensor), ("vol", TcpTensor),
                ("theta", ctypes.c_void_p), ("center", ctypes.c_double), ("filter", ctypes.c_int32),
                ("pad_mode", ctypes.c_int32)]


class BatchOpts(ctypes.Structure):
    _fields_ = [("sino_dtype", ctypes.c_int32), ("autotune", ctypes.c_int32), ("reserved", ctypes.c_int32 * 2)]


class PlanDesc(ctypes.Structure):
    _fields_ = [("ntheta", ctypes.c_int64), ("nz", ctypes.c_int64), ("ndet", ctypes.c_int64), ("n", ctypes.c_int64),
                ("center", ctypes.c_double), ("vol_dtype", ctypes.c_int32), ("io", ctypes.c_int32),
                ("host_frames", ctypes.c_int32), ("trace", ctypes.c_int32), ("opts", FbpOpts)]


IO_HOST_RAW, IO_HOST_VOL = 1, 2

SIGNATURES.update({
    "tcp_plan_create": ([ctypes.POINTER(PlanDesc), _P, ctypes.POINTER(ctypes.c_void_p)], _I32),
    "tcp_plan_destroy": ([_P], _I32),
    "tcp_plan_info": ([_P, ctypes.POINTER(_I64), ctypes.POINTER(FbpOpts)], _I32),
    "tcp_fbp_plan": ([_P, _T, _T, _T, _T, _P], _I32),
    "tcp_plan_trace": ([_P, _P, _I64, ctypes.POINTER(_I64)], _I32),
    "tcp_filter_plan": ([_P, _T, _P], _I32),
    "tcp_backproject_plan": ([_P, _T, _D, _T, _D, _P], _I32),
    "tcp_project_plan": ([_P, _T, _D, _T, _P], _I32),
})

SIGNATURES.update({
    "tcp_autotune_backproject": ([_T, _P, _D, _T, _P, ctypes.POINTER(BpConfig), ctypes.POINTER(ctypes.c_float)], _I32),
    "tcp_batch_create": ([ctypes.POINTER(BatchItem), _I32, ctypes.POINTER(BatchOpts), _P,
                          ctypes.POINTER(ctypes.c_void_p)], _I32),
    "tcp_batch_run": ([_P, _P], _I32),
    "tcp_batch_capture": ([_P, _P], _I32),
    "tcp_batch_replay": ([_P, _P], _I32),
    "tcp_batch_info": ([_P, ctypes.POINTER(BpConfig), ctypes.POINTER(ctypes.c_float), ctypes.POINTER(_I64),
                        ctypes.POINTER(_I32)], _I32),
    "tcp_batch_destroy": ([_P], _I32),
})
