"""FP64 oracle for FourierRec, the Fourier-based backprojector.

TEST INFRASTRUCTURE ONLY (same rules as the rest of ``oracle/``): only
``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs may use it,
and it shares no code with the CUDA library.

Sec. 1 and Sec. 2.2 of Nikitin, TomocuPy (arXiv 2209.08450), name the method:
the backprojection is evaluated through the Fourier-slice theorem with
Fourier transforms on unequally spaced grids; the frequency-domain
interpolation uses exponential functions; Sec. 3 adds that the frequencies are
oversampled by a factor of 2 and that the accuracy is controlled.  The paper
prints no formulas, so this module fixes the following readings.

What is computed (``backproject_exact``).  Each filtered row q[j], j < ndet, is
extended by zeros to the period M = the next power of two >= 2 ndet and
replaced by its trigonometric interpolant

    q~(s) = (1/M) sum_{k=-M/2}^{M/2} w_k Q[k] e^{2 pi i k s / M},
    Q[k]  = sum_j q[j] e^{-2 pi i k j / M},   w_{+-M/2} = 1/2, else w_k = 1,

which is real for real q and equals q[j] at integer s = j (and 0 at the padded
nodes).  The voxel (ix, iy) at (x, y) = (ix - n/2, iy - n/2) (n even) receives

    f(x, y) = sum_theta q~_theta(x cos(theta) + y sin(theta) + center),

the LineRec sum with linear interpolation replaced by this band-limited one.
``backproject_exact`` evaluates it by direct sums; it is pinned by closed forms
(the periodic sinc of a single-pixel row, exact node interpolation).

How it is computed fast (``backproject_gridding``, the algorithm's steps).
Substituting s gives f(x, y) = sum_{theta,k} P[theta][k] e^{2 pi i nu.(x, y)}
with P = (w_k / M) e^{2 pi i k center / M} Q[k] and polar frequencies
nu = (k / M)(cos theta, sin theta): a transform from unequally spaced
frequencies to the pixel grid.  It is evaluated by
  1. P from an FFT of each zero-padded row;
  2. spreading every P onto an L x L Cartesian frequency grid (L = the next
     power of two >= 2n, at least 16: oversampling >= 2) with a separable window phi of
     width W grid points;
  3. a 2-D inverse DFT of the grid;
  4. dividing pixel (x, y) by Phi(x / L) Phi(y / L), Phi the Fourier
     transform of phi, and keeping the centre n x n.
The window is the "exponential of semicircle" of Barnett, Magland and af
Klinteberg (SIAM J. Sci. Comput. 41, 2019),
phi(u) = exp(beta (sqrt(1 - (2u/W)^2) - 1)) for |u| < W/2, else 0, with
beta = 0.98 pi W (1 - 1/(2 sigma)) at oversampling sigma = 2; its error falls
about tenfold per extra grid point of W.  ``backproject_gridding`` is pinned
to ``backproject_exact`` within that error.
"""
from __future__ import annotations

import numpy as np


def period(ndet: int) -> int:
    """Interpolation period M: the next power of two >= 2 ndet."""
    m = 1
    while m < 2 * ndet:
        m *= 2
    return m


def grid_size(n: int) -> int:
    """Cartesian frequency grid L: the next power of two >= 2 n, at least 16
    (oversampling >= 2, and the window's W <= 16 points always fit)."""
    g = 16
    while g < 2 * n:
        g *= 2
    return g


def row_spectrum(q_row: np.ndarray, center: float) -> np.ndarray:
    """P[k] for k = -M/2 .. M/2 (M + 1 values): (w_k / M) e^{2 pi i k c / M} Q[k]."""
    q_row = np.asarray(q_row, dtype=np.float64)
    M = period(q_row.shape[-1])
    Q = np.fft.fft(q_row, n=M, axis=-1)
    k = np.arange(-M // 2, M // 2 + 1)
    w = np.ones(M + 1)
    w[0] = w[-1] = 0.5
    phase = np.exp(2j * np.pi * k * center / M)
    return Q[..., k % M] * (w * phase / M)


def interp_row(q_row: np.ndarray, s: np.ndarray) -> np.ndarray:
    """Trigonometric interpolant q~(s) of one zero-padded row at points s."""
    M = period(q_row.shape[0])
    P = row_spectrum(q_row, 0.0)
    k = np.arange(-M // 2, M // 2 + 1)
    s = np.asarray(s, dtype=np.float64)
    out = np.exp(2j * np.pi * np.multiply.outer(s, k) / M) @ P
    return out.real


def backproject_exact(sino: np.ndarray, theta: np.ndarray, center: float, n: int) -> np.ndarray:
    """FourierRec target by direct sums: sino[z][theta][j] -> vol[z][n][n] (FP64)."""
    if n % 2:
        raise ValueError("FourierRec needs an even n")
    sino = np.asarray(sino, dtype=np.float64)
    if sino.ndim == 2:
        sino = sino[None]
    nz, nt, nd = sino.shape
    x = np.arange(n) - n / 2.0
    out = np.zeros((nz, n, n))
    for t in range(nt):
        c, s = np.cos(theta[t]), np.sin(theta[t])
        sv = (x[None, :] * c + x[:, None] * s + center).reshape(-1)
        for z in range(nz):
            out[z] += interp_row(sino[z, t], sv).reshape(n, n)
    return out


def backproject_exact_points(sino_slice: np.ndarray, theta: np.ndarray, center: float, n: int,
                             ix: np.ndarray, iy: np.ndarray) -> np.ndarray:
    """``backproject_exact`` of one slice sino[theta][j] at voxels (ix[p], iy[p])."""
    q = np.asarray(sino_slice, dtype=np.float64)
    x = np.asarray(ix, dtype=np.float64) - n / 2.0
    y = np.asarray(iy, dtype=np.float64) - n / 2.0
    out = np.zeros(x.shape[0])
    for t in range(q.shape[0]):
        out += interp_row(q[t], x * np.cos(theta[t]) + y * np.sin(theta[t]) + center)
    return out


def es_beta(width: int) -> float:
    """Shape parameter of the exponential-of-semicircle window at oversampling 2."""
    return 0.98 * np.pi * width * (1.0 - 1.0 / (2.0 * 2.0))


def es_window(u: np.ndarray, width: int) -> np.ndarray:
    """phi(u) = exp(beta (sqrt(1 - (2u/W)^2) - 1)) for |u| < W/2, else 0."""
    z2 = (2.0 * np.asarray(u, dtype=np.float64) / width) ** 2
    inside = z2 < 1.0
    return np.where(inside, np.exp(es_beta(width) * (np.sqrt(np.where(inside, 1.0 - z2, 0.0)) - 1.0)), 0.0)


def es_fourier(xi: np.ndarray, width: int) -> np.ndarray:
    """Phi(xi) = integral of phi(u) e^{-2 pi i u xi} du (real, even), by adaptive quadrature."""
    from scipy.integrate import quad
    beta = es_beta(width)
    half = width / 2.0

    def one(v):
        f = lambda u: np.exp(beta * (np.sqrt(max(0.0, 1.0 - (u / half) ** 2)) - 1.0)) * np.cos(2 * np.pi * u * v)
        return 2.0 * quad(f, 0.0, half, limit=400, epsabs=1e-14, epsrel=1e-12)[0]

    return np.array([one(v) for v in np.atleast_1d(np.asarray(xi, dtype=np.float64))])


def backproject_gridding(sino: np.ndarray, theta: np.ndarray, center: float, n: int,
                         width: int = 8) -> np.ndarray:
    """FourierRec by the gridding steps (1)-(4) above, in FP64."""
    if n % 2:
        raise ValueError("FourierRec needs an even n")
    sino = np.asarray(sino, dtype=np.float64)
    if sino.ndim == 2:
        sino = sino[None]
    nz, nt, nd = sino.shape
    M, L = period(nd), grid_size(n)
    k = np.arange(-M // 2, M // 2 + 1)
    # (2) sample positions on the grid, in grid units about the zero frequency
    px = np.multiply.outer(np.cos(theta), k) * (L / M)
    py = np.multiply.outer(np.sin(theta), k) * (L / M)
    offs = np.arange(width + 1)
    gx = np.floor(px - width / 2.0)[..., None] + 1 + offs      # every node with |p - g| < W/2
    gy = np.floor(py - width / 2.0)[..., None] + 1 + offs
    wx = es_window(px[..., None] - gx, width)
    wy = es_window(py[..., None] - gy, width)
    ixg = (gx.astype(np.int64) % L)
    iyg = (gy.astype(np.int64) % L)
    # (4) deconvolution factors for x = -n/2 .. n/2 - 1
    x = np.arange(n) - n // 2
    dec = 1.0 / es_fourier(x / L, width)
    out = np.empty((nz, n, n))
    for z in range(nz):
        P = row_spectrum(sino[z], center)                       # (1) [theta][M + 1]
        G = np.zeros((L, L), dtype=np.complex128)               # G[gy][gx]
        contrib = P[..., None, None] * wy[..., :, None] * wx[..., None, :]
        np.add.at(G, (np.broadcast_to(iyg[..., :, None], contrib.shape),
                      np.broadcast_to(ixg[..., None, :], contrib.shape)), contrib)
        F = np.fft.ifft2(G) * (L * L)                           # (3) sum_g G[g] e^{+2 pi i g.x / L}
        img = F[np.ix_(x % L, x % L)]                           # rows y, columns x
        out[z] = (img * dec[:, None] * dec[None, :]).real
    return out
