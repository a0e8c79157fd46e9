"""FP64 CPU oracle for chunked parallel-beam FBP (LineRec) and its adjoint.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library in ``paper_2209_08450_gb300``; neither imports the other.

What it computes (Nikitin, TomocuPy, arXiv 2209.08450):

* ``frame_mean`` / ``normalize`` -- Sec. 2.2 dark-flat field correction and
  negative logarithm: ``p = -ln(max((raw - dark)/(flat - dark), eps))``.
* ``filter_sino`` -- Sec. 2.2 one-dimensional filtering of each detector row
  in Fourier space (Shepp-Logan, Parzen or plain ramp), with padding
  (Sec. 2.2 and Sec. 3), the FBP angular weight pi/N_theta and a Fourier
  shift that moves the rotation axis to ``ndet/2``.  ``numpy.fft`` is the FFT.
* ``backproject`` -- Sec. 2.2 / Sec. 3 (LineRec): direct discretisation of the
  backprojection line integral with linear interpolation (C, FP64).
* ``project`` -- the exact transpose of ``backproject`` (not in the paper).
* ``fbp`` -- the three steps in the paper's order.
* ``oracle.fourierrec`` -- FourierRec (Sec. 1, 2.2, 3): backprojection with
  the band-limited interpolant of each zero-padded row, exact FP64 sums and
  the gridding steps (``tests/test_oracle_fourierrec.py``).
* ``oracle.lprec`` -- LpRec (Sec. 1, 3): the cubic-spline backprojection by
  direct sums and its log-polar evaluation (``tests/test_oracle_lprec.py``).

Every function is pinned by ``tests/test_oracle.py`` against closed forms,
brute force and invariants; none is pinned against itself.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tcp_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

EPS = 1e-6  # clamp for non-positive transmission (reading of Sec. 2.2)

FILTERS = ("shepp", "parzen", "ramp", "none")


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (FP64, no fast-math, no FMA contraction)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            I = ctypes.c_int64
            D = ctypes.c_double
            lib.or_frame_mean.argtypes = [P, I, I, I, P]
            lib.or_normalize.argtypes = [P, I, I, I, P, P, D, P]
            lib.or_backproject.argtypes = [P, I, I, I, P, D, I, P]
            lib.or_backproject_points.argtypes = [P, I, I, P, D, I, P, P, I, P]
            lib.or_project.argtypes = [P, I, I, P, I, D, I, P]
            for f in (lib.or_frame_mean, lib.or_normalize, lib.or_backproject,
                      lib.or_backproject_points, lib.or_project):
                f.restype = None
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def frame_mean(frames: np.ndarray) -> np.ndarray:
    """Mean over the frame axis of uint16 frames[f][z][j] -> float64 [z][j]."""
    frames = np.ascontiguousarray(frames, dtype=np.uint16)
    nf, nz, nd = frames.shape
    out = np.empty((nz, nd), np.float64)
    _load().or_frame_mean(_ptr(frames), nf, nz, nd, _ptr(out))
    return out


def normalize(raw: np.ndarray, dark_mean: np.ndarray, flat_mean: np.ndarray,
              eps: float = EPS) -> np.ndarray:
    """raw uint16 [theta][z][j] -> sinogram float64 [z][theta][j] (Sec. 2.2)."""
    raw = np.ascontiguousarray(raw, dtype=np.uint16)
    nt, nz, nd = raw.shape
    d = np.ascontiguousarray(dark_mean, dtype=np.float64).reshape(nz, nd)
    f = np.ascontiguousarray(flat_mean, dtype=np.float64).reshape(nz, nd)
    out = np.empty((nz, nt, nd), np.float64)
    _load().or_normalize(_ptr(raw), nt, nz, nd, _ptr(d), _ptr(f), float(eps), _ptr(out))
    return out


def padded_length(ndet: int, rule: str = "pow2") -> int:
    """Padded row length (reading of Sec. 2.2, which pads rows to FFT-friendly
    sizes: powers of two for FP16, products of small primes for FP32).

    pow2:   the next power of two >= 2*ndet (every precision, the default);
    smooth: the smallest of that, the next 3 * 2^k >= 2*ndet (from 48 on) and
            the next 5 * 2^k >= 2*ndet (from 80 on): 1536 -> 3072 and
            2560 -> 5120 instead of 4096 and 8192."""
    if rule not in ("pow2", "smooth"):
        raise ValueError("unknown padding rule %r" % rule)
    n = 1
    while n < 2 * ndet:
        n *= 2
    if rule == "smooth":
        for base, least in ((3, 48), (5, 80)):
            m = base
            while m < 2 * ndet or m < least:
                m *= 2
            n = min(n, m)
    return n


def ramp_response(npad: int) -> np.ndarray:
    """Band-limited ramp on the padded period, bins k = 0..npad/2.

    The spatial Ram-Lak kernel for unit sample spacing (Kak & Slaney 1988,
    Ch. 3), h[0] = 1/4, h[m] = -1/(pi^2 m^2) for odd m, 0 for even m != 0,
    truncated to -npad/2 <= m < npad/2, transformed by the DFT.  Its DC bin is
    small and positive; a ramp sampled in frequency with a zero DC bin biases
    every reconstruction by a constant (reading of Sec. 2.2, which names the
    filters but prints no formula).
    """
    m = np.arange(npad)
    m = np.where(m < npad // 2, m, m - npad)
    h = np.zeros(npad, np.float64)
    h[0] = 0.25
    odd = (m % 2) != 0
    h[odd] = -1.0 / (np.pi ** 2 * m[odd].astype(np.float64) ** 2)
    return np.fft.rfft(h).real


def filter_response(kind: str, npad: int) -> np.ndarray:
    """Filter response on bins k = 0..npad/2 (nu_k = k/npad cycles/pixel).

    ramp:   the band-limited ramp R_k of ``ramp_response``
    shepp:  R_k * sin(pi nu)/(pi nu)     (Shepp-Logan window)
    parzen: R_k * (1 - 2|nu|)^3          (Parzen-type taper)
    none:   1 (no filtering; only the weight and the shift are applied)
    """
    nu = np.arange(npad // 2 + 1, dtype=np.float64) / npad
    if kind == "none":
        return np.ones_like(nu)
    h = ramp_response(npad)
    if kind == "shepp":
        h = h * np.sinc(nu)  # numpy sinc(x) = sin(pi x)/(pi x)
    elif kind == "parzen":
        h = h * (1.0 - 2.0 * np.abs(nu)) ** 3
    elif kind != "ramp":
        raise ValueError("unknown filter %r" % kind)
    return h


def filter_sino(sino: np.ndarray, center: float, kind: str = "shepp", pad: str = "edge",
                ntheta: int | None = None, rule: str = "pow2") -> np.ndarray:
    """Ramp-filter every detector row of sino[..., theta, j] (Sec. 2.2).

    Steps, per row: pad to ``padded_length(ndet, rule)`` (``L = (npad-ndet)//2``
    samples on the left, the rest on the right; ``edge`` replicates the end
    samples, ``zero`` pads with zeros), real FFT, multiply bin k by
    ``H(nu_k) * pi/ntheta * exp(2 pi i nu_k (center - ndet/2))`` (the Nyquist
    bin takes the real part of that factor), inverse FFT, crop ``[L, L+ndet)``.
    The phase factor shifts each row so that the rotation axis moves from
    ``center`` to ``ndet/2``.
    """
    sino = np.asarray(sino, dtype=np.float64)
    nd = sino.shape[-1]
    nt = sino.shape[-2] if ntheta is None else ntheta
    npad = padded_length(nd, rule)
    left = (npad - nd) // 2
    widths = [(0, 0)] * (sino.ndim - 1) + [(left, npad - nd - left)]
    if pad == "edge":
        x = np.pad(sino, widths, mode="edge")
    elif pad == "zero":
        x = np.pad(sino, widths, mode="constant")
    else:
        raise ValueError("unknown pad mode %r" % pad)
    nu = np.arange(npad // 2 + 1, dtype=np.float64) / npad
    factor = filter_response(kind, npad) * (np.pi / nt) * np.exp(2j * np.pi * nu * (center - nd / 2.0))
    factor[-1] = factor[-1].real
    y = np.fft.irfft(np.fft.rfft(x, axis=-1) * factor, n=npad, axis=-1)
    return np.ascontiguousarray(y[..., left:left + nd])


def backproject(sino: np.ndarray, theta: np.ndarray, center: float, n: int) -> np.ndarray:
    """LineRec backprojection sino[z][theta][j] -> vol[z][n][n] (FP64)."""
    sino = np.ascontiguousarray(sino, dtype=np.float64)
    if sino.ndim == 2:
        sino = sino[None]
    nz, nt, nd = sino.shape
    th = np.ascontiguousarray(theta, dtype=np.float64)
    assert th.shape == (nt,)
    out = np.empty((nz, n, n), np.float64)
    _load().or_backproject(_ptr(sino), nz, nt, nd, _ptr(th), float(center), n, _ptr(out))
    return out


def backproject_points(sino_slice: np.ndarray, theta: np.ndarray, center: float, n: int,
                       ix: np.ndarray, iy: np.ndarray) -> np.ndarray:
    """Backprojection of one slice sino[theta][j] at voxels (ix[p], iy[p])."""
    q = np.ascontiguousarray(sino_slice, dtype=np.float64)
    nt, nd = q.shape
    th = np.ascontiguousarray(theta, dtype=np.float64)
    ix = np.ascontiguousarray(ix, dtype=np.int64)
    iy = np.ascontiguousarray(iy, dtype=np.int64)
    out = np.empty(ix.shape[0], np.float64)
    _load().or_backproject_points(_ptr(q), nt, nd, _ptr(th), float(center), n,
                                  _ptr(ix), _ptr(iy), ix.shape[0], _ptr(out))
    return out


def project(vol: np.ndarray, theta: np.ndarray, center: float, ndet: int) -> np.ndarray:
    """Radon projector vol[z][n][n] -> sino[z][theta][ndet], transpose of backproject."""
    vol = np.ascontiguousarray(vol, dtype=np.float64)
    if vol.ndim == 2:
        vol = vol[None]
    nz, n, n2 = vol.shape
    assert n == n2
    th = np.ascontiguousarray(theta, dtype=np.float64)
    out = np.empty((nz, th.shape[0], ndet), np.float64)
    _load().or_project(_ptr(vol), nz, n, _ptr(th), th.shape[0], float(center), ndet, _ptr(out))
    return out


def fbp(raw: np.ndarray, dark_frames: np.ndarray, flat_frames: np.ndarray, theta: np.ndarray,
        center: float, kind: str = "shepp", n: int | None = None, pad: str = "edge",
        rule: str = "pow2") -> np.ndarray:
    """Full FBP in the paper's order: normalise, filter (axis moved to ndet/2),
    backproject about ndet/2.  raw[theta][z][j] uint16 -> vol[z][n][n] FP64."""
    nd = raw.shape[-1]
    n = nd if n is None else n
    p = normalize(raw, frame_mean(dark_frames), frame_mean(flat_frames))
    q = filter_sino(p, center, kind, pad, rule=rule)
    return backproject(q, theta, nd / 2.0, n)
