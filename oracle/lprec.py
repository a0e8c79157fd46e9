"""FP64 oracle for LpRec, the log-polar backprojector.

TEST INFRASTRUCTURE ONLY (same rules as the rest of ``oracle/``).

Sec. 1 and Sec. 3 of Nikitin, TomocuPy (arXiv 2209.08450), name the method:
the backprojection is evaluated in log-polar coordinates, where it becomes a
convolution, with cubic-spline interpolation in the image domain, for equally
spaced angles.  The paper prints no formulas or grid sizes; this module fixes
the following reading.

What is approximated (``backproject_spline_exact``).  Each filtered row q[j]
is replaced by its interpolating cubic B-spline q~(s) (samples zero outside
[0, ndet)), and

    f(x, y) = sum_theta q~_theta(x cos(theta) + y sin(theta) + center),

x = ix - n/2, y = iy - n/2: LineRec with cubic instead of linear
interpolation.  It is evaluated here by direct sums.

How LpRec evaluates it (``backproject_lprec``).  The angles (equally spaced)
are split into three spans.  For a span centred on angle phi, put the
log-polar origin at O = -a (cos phi, sin phi), a = 4 R outside the object
(R: radius covering the voxel grid), and write a voxel as
x = O + e^rho (cos psi, sin psi).  Then for every angle theta of the span
x . e_theta + center = sh_theta + e^rho cos(psi - theta),
sh_theta = center - a cos(theta - phi), so with G_theta(tau) =
q~_theta(sh_theta + e^tau) the span's contribution is

    f_span(rho, psi) = sum_theta G_theta(rho + log cos(psi - theta)),

a function of the differences rho - tau and psi - theta only: a convolution on
a uniform (log-radius, angle) grid (|psi - theta| < pi/2 holds for every
voxel by the choice of a).  Steps: (1) sample every G_theta on a uniform
log-radius grid and take its cubic B-spline; (2) evaluate f_span on the
log-polar grid (log-radius step 1/(os (a + R)), angle step the angle spacing
divided by an integer, so that both steps are at most 1/os pixels at the far
radius); (3) interpolate f_span at the voxels with 2-D cubic B-splines; (4) sum
the three spans.  ``os`` is the oversampling of the log-polar grid; the error
to ``backproject_spline_exact`` falls with it (pinned in
tests/test_oracle_lprec.py).
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import solve_banded

PAD = 24  # zero samples added on each side before prefiltering (0.268^24 ~ 2e-14)


def bspline_coeffs(v: np.ndarray, axis: int = -1) -> np.ndarray:
    """Coefficients c of the interpolating cubic B-spline of samples v along
    `axis`, the samples extended by PAD zeros on each side: sum_k c[k]
    beta3(t - k) = v[t - PAD] at the integers.  Returns the padded coefficients
    (index k corresponds to sample k - PAD)."""
    v = np.moveaxis(np.asarray(v, dtype=np.float64), axis, 0)
    m = v.shape[0] + 2 * PAD
    rhs = np.zeros((m,) + v.shape[1:])
    rhs[PAD:PAD + v.shape[0]] = v
    ab = np.zeros((3, m))
    ab[0, 1:] = 1.0 / 6.0
    ab[1, :] = 4.0 / 6.0
    ab[2, :-1] = 1.0 / 6.0
    c = solve_banded((1, 1), ab, rhs.reshape(m, -1)).reshape(rhs.shape)
    return np.moveaxis(c, 0, axis)


def _beta3_taps(t: np.ndarray):
    """Integer base and the four cubic B-spline weights at offsets 0..3 from it."""
    t = np.asarray(t, dtype=np.float64)
    b = np.floor(t).astype(np.int64) - 1
    u = t - (b + 1)  # in [0, 1)
    w0 = (1 - u) ** 3 / 6
    w1 = (3 * u ** 3 - 6 * u ** 2 + 4) / 6
    w2 = (-3 * u ** 3 + 3 * u ** 2 + 3 * u + 1) / 6
    w3 = u ** 3 / 6
    return b, (w0, w1, w2, w3)


def bspline_eval(c: np.ndarray, t: np.ndarray) -> np.ndarray:
    """sum_k c[k] beta3(t - k) for coefficients c (1-D) at points t (0 outside)."""
    b, w = _beta3_taps(t)
    out = np.zeros(np.shape(t))
    for i in range(4):
        k = b + i
        ok = (k >= 0) & (k < c.shape[0])
        out += np.where(ok, c[np.clip(k, 0, c.shape[0] - 1)], 0.0) * w[i]
    return out


def bspline_eval2(c: np.ndarray, t0: np.ndarray, t1: np.ndarray) -> np.ndarray:
    """2-D tensor-product cubic B-spline sum at points (t0, t1) (0 outside)."""
    b0, w0 = _beta3_taps(t0)
    b1, w1 = _beta3_taps(t1)
    out = np.zeros(np.shape(t0))
    for i in range(4):
        k0 = b0 + i
        ok0 = (k0 >= 0) & (k0 < c.shape[0])
        for j in range(4):
            k1 = b1 + j
            ok = ok0 & (k1 >= 0) & (k1 < c.shape[1])
            out += np.where(ok, c[np.clip(k0, 0, c.shape[0] - 1), np.clip(k1, 0, c.shape[1] - 1)], 0.0) * w0[i] * w1[j]
    return out


def row_interp(q_row: np.ndarray, s: np.ndarray) -> np.ndarray:
    """Interpolating cubic B-spline of one row (zero samples outside) at s."""
    return bspline_eval(bspline_coeffs(q_row), np.asarray(s, dtype=np.float64) + PAD)


def backproject_spline_exact(sino: np.ndarray, theta: np.ndarray, center: float, n: int) -> np.ndarray:
    """Cubic-spline backprojection by direct sums: sino[z][theta][j] -> vol[z][n][n]."""
    sino = np.asarray(sino, dtype=np.float64)
    if sino.ndim == 2:
        sino = sino[None]
    nz, nt, nd = sino.shape
    x = np.arange(n) - n / 2.0
    out = np.zeros((nz, n, n))
    for z in range(nz):
        coef = bspline_coeffs(sino[z], axis=1)
        for t in range(nt):
            s = x[None, :] * np.cos(theta[t]) + x[:, None] * np.sin(theta[t]) + center
            out[z] += bspline_eval(coef[t], s + PAD)
    return out


def backproject_spline_points(sino_slice: np.ndarray, theta: np.ndarray, center: float, n: int,
                              ix: np.ndarray, iy: np.ndarray) -> np.ndarray:
    """backproject_spline_exact of one slice sino[theta][j] at the voxels
    (ix[k], iy[k]) only (the same direct sums)."""
    q = np.asarray(sino_slice, dtype=np.float64)
    coef = bspline_coeffs(q, axis=1)
    x = np.asarray(ix, dtype=np.float64) - n / 2.0
    y = np.asarray(iy, dtype=np.float64) - n / 2.0
    out = np.zeros(x.shape)
    for t in range(q.shape[0]):
        out += bspline_eval(coef[t], x * np.cos(theta[t]) + y * np.sin(theta[t]) + center + PAD)
    return out


def _check_equally_spaced(theta: np.ndarray) -> float:
    d = np.diff(theta)
    if theta.shape[0] < 3 or not np.allclose(d, d[0], rtol=0, atol=1e-9) or abs(d[0] * theta.shape[0] - np.pi) > 1e-9:
        raise ValueError("LpRec needs equally spaced angles covering [theta0, theta0 + pi)")
    return float(d[0])


def _span_by_fft(gcs: np.ndarray, p: int, r0: float, drho: float, dpsi: float, base: float, nrho: int,
                 npsi: int) -> np.ndarray:
    """Step (2) as one 2-D linear convolution, computed by FFT.

    gcs[u][l]: B-spline coefficients of G for the span's u-th angle.  With the
    angles placed every p columns, A[l][p u] = gcs[u][l], the sum
    f[i][k] = sum_u sum_l gcs[u][l] beta3(i + base + s(k - p u) - l),
    s(r) = log cos((r - r0) dpsi) / drho, is (A * K)[i][k] with
    K[d][r] = beta3(d + base + s(r))."""
    nu, nl = gcs.shape
    kp = p * (nu - 1) + 1
    A = np.zeros((nl, kp))
    A[:, ::p] = gcs.T
    r = np.arange(-(kp - 1), npsi)                      # every k - p u needed
    sr = np.log(np.cos((r - r0) * dpsi)) / drho
    # d = i - l spans [-(nl - 1), nrho - 1]; beta3 vanishes outside |.| < 2
    d = np.arange(-(nl - 1), nrho)
    arg = d[:, None] + base + sr[None, :]
    K = np.where(np.abs(arg) < 2.0,
                 np.where(np.abs(arg) < 1.0, 2.0 / 3.0 - arg ** 2 + np.abs(arg) ** 3 / 2.0,
                          (2.0 - np.abs(arg)) ** 3 / 6.0), 0.0)
    shape = (nl + K.shape[0] - 1, kp + K.shape[1] - 1)
    full = np.fft.irfft2(np.fft.rfft2(A, shape) * np.fft.rfft2(K, shape), shape)
    # output index (i, k) sits at (i + nl - 1, k + kp - 1) of the full product
    return full[nl - 1:nl - 1 + nrho, kp - 1:kp - 1 + npsi]


def backproject_lprec(sino: np.ndarray, theta: np.ndarray, center: float, n: int, os: float = 2.0,
                      a_factor: float = 4.0, margin: int = 12, conv: str = "direct") -> np.ndarray:
    """LpRec by the steps (1)-(4) above, in FP64.  conv="fft" evaluates step
    (2) as the span's 2-D convolution by FFT (the same sum)."""
    sino = np.asarray(sino, dtype=np.float64)
    if sino.ndim == 2:
        sino = sino[None]
    theta = np.asarray(theta, dtype=np.float64)
    nz, nt, nd = sino.shape
    dth = _check_equally_spaced(theta)
    R = n / np.sqrt(2.0) + 2.0
    a = a_factor * R
    drho = 1.0 / (os * (a + R))
    p = int(np.ceil(os * (a + R) * dth))  # angle substeps per angle spacing
    dpsi = dth / p
    x = np.arange(n) - n / 2.0
    X, Y = np.meshgrid(x, x)  # [iy][ix]
    out = np.zeros((nz, n, n))
    bounds = [int(round(m * nt / 3.0)) for m in range(4)]
    for m in range(3):
        js = np.arange(bounds[m], bounds[m + 1])
        if js.size == 0:
            continue
        phi = 0.5 * (theta[js[0]] + theta[js[-1]])
        ox, oy = -a * np.cos(phi), -a * np.sin(phi)
        # log-polar grid covering the voxels, with margins for the splines
        rho0 = np.log(a - R) - margin * drho
        nrho = int(np.ceil((np.log(a + R) - np.log(a - R)) / drho)) + 2 * margin + 1
        half = np.arcsin(R / a) + margin * dpsi
        kpsi = int(np.ceil(half / dpsi))
        rho = rho0 + drho * np.arange(nrho)
        psi = phi + dpsi * np.arange(-kpsi, kpsi + 1)
        # log-radius sample grid of G: the span grid extended by the largest
        # shift log cos(psi - theta)
        span = np.max(np.abs(psi[:, None] - theta[js][None, :]))
        ext = int(np.ceil(-np.log(np.cos(span)) / drho)) + margin
        tau0 = rho0 - ext * drho
        tau = tau0 + drho * np.arange(nrho + ext)
        # voxel coordinates in the span's log-polar system
        vr = np.log(np.hypot(X - ox, Y - oy))
        vpsi = np.arctan2(Y - oy, X - ox)
        vpsi = phi + np.angle(np.exp(1j * (vpsi - phi)))
        ti = (vr - rho0) / drho
        tk = (vpsi - psi[0]) / dpsi
        for z in range(nz):
            coef = bspline_coeffs(sino[z], axis=1)
            gcs = []
            for j in js:
                sh = center - a * np.cos(theta[j] - phi)
                g = bspline_eval(coef[j], sh + np.exp(tau) + PAD)          # (1) G_theta on the tau grid
                gcs.append(bspline_coeffs(g))
            if conv == "fft":                                                # (2) f_span on the grid
                r0 = kpsi - p * (js.size - 1) / 2.0
                f = _span_by_fft(np.array(gcs), p, r0, drho, dpsi, ext + PAD, nrho, psi.shape[0])
            else:
                f = np.zeros((nrho, psi.shape[0]))
                for u, j in enumerate(js):
                    shift = np.log(np.cos(psi - theta[j]))
                    tt = (rho[:, None] + shift[None, :] - tau0) / drho
                    f += bspline_eval(gcs[u], tt + PAD)
            fc = bspline_coeffs(bspline_coeffs(f, axis=0), axis=1)         # (3) back to the voxels
            out[z] += bspline_eval2(fc, ti + PAD, tk + PAD)
    return out
