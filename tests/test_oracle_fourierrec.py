"""Pins of the FourierRec oracle (CPU only).

The exact form is pinned by closed forms that do not go through its DFT sum:
the periodic sinc (Dirichlet kernel) of a single-pixel row, and exact
interpolation at the nodes.  The gridding form is pinned to the exact form
within the window's error, which must fall as the window widens.
"""
import numpy as np
import pytest

import oracle
from oracle import fourierrec as fr


def dirichlet(t, M):
    """Periodic sinc of period M (even), the Nyquist term split in halves:
    (1/M) [1 + 2 sum_{k<M/2} cos(2 pi k t / M) + cos(pi t)] = sin(pi t) cot(pi t / M) / M."""
    t = np.asarray(t, dtype=np.float64)
    den = np.tan(np.pi * t / M)
    safe = np.where(np.abs(den) < 1e-300, 1.0, den)
    return np.where(np.abs(den) < 1e-300, 1.0, np.sin(np.pi * t) / (M * safe))


def rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def test_period_and_grid():
    assert fr.period(12) == 32 and fr.period(16) == 32 and fr.period(17) == 64 and fr.period(1) == 2
    assert fr.grid_size(10) == 32 and fr.grid_size(64) == 128 and fr.grid_size(2048) == 4096
    assert fr.grid_size(1) == 16 and fr.grid_size(8) == 16 and fr.grid_size(9) == 32


@pytest.mark.parametrize("theta0,center,j0", [(0.3, 5.37, 4), (1.9, 6.0, 0), (2.71, 4.25, 11)])
def test_single_pixel_row_is_periodic_sinc(theta0, center, j0):
    nd, n = 12, 10
    M = fr.period(nd)
    q = np.zeros((1, 1, nd))
    q[0, 0, j0] = 1.0
    got = fr.backproject_exact(q, np.array([theta0]), center, n)[0]
    x = np.arange(n) - n / 2
    s = x[None, :] * np.cos(theta0) + x[:, None] * np.sin(theta0) + center
    want = dirichlet(s - j0, M)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12)


def test_two_angles_add():
    nd, n = 8, 6
    M = fr.period(nd)
    th = np.array([0.2, 2.0])
    q = np.zeros((1, 2, nd))
    q[0, 0, 3] = 2.0
    q[0, 1, 6] = -0.5
    got = fr.backproject_exact(q, th, 3.7, n)[0]
    x = np.arange(n) - n / 2
    want = np.zeros((n, n))
    for t, (j, a) in enumerate([(3, 2.0), (6, -0.5)]):
        s = x[None, :] * np.cos(th[t]) + x[:, None] * np.sin(th[t]) + 3.7
        want += a * dirichlet(s - j, M)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12)


def test_nodes_match_linear_interpolation():
    # theta = 0 and pi/2 with an integer centre put every ray on a detector
    # node, where both interpolants return the sample (0 on the padding)
    rng = np.random.default_rng(3)
    nd, n = 12, 10
    q = rng.standard_normal((2, 2, nd))
    th = np.array([0.0, np.pi / 2])
    got = fr.backproject_exact(q, th, 6.0, n)
    want = oracle.backproject(q, th, 6.0, n)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-11)


def test_real_and_points_agree():
    rng = np.random.default_rng(4)
    nd, n, nt = 16, 12, 9
    q = rng.standard_normal((1, nt, nd))
    th = np.sort(rng.uniform(0, np.pi, nt))
    full = fr.backproject_exact(q, th, 7.3, n)[0]
    ix = rng.integers(0, n, 20)
    iy = rng.integers(0, n, 20)
    pts = fr.backproject_exact_points(q[0], th, 7.3, n, ix, iy)
    np.testing.assert_allclose(pts, full[iy, ix], rtol=0, atol=1e-12)


def test_window_fourier_transform():
    # Phi(0) is the window's integral; Phi is even and decays past |xi| = 1/2
    for W in (4, 8):
        u = np.linspace(-W / 2, W / 2, 200001)
        integral = np.trapezoid(fr.es_window(u, W), u)
        assert abs(fr.es_fourier(np.array([0.0]), W)[0] - integral) < 1e-6 * integral
        a, b = fr.es_fourier(np.array([0.2, -0.2]), W)
        assert a == pytest.approx(b, rel=1e-12)
    # aliasing weight at oversampling 2 falls with the width
    r = [fr.es_fourier(np.array([0.75]), W)[0] / fr.es_fourier(np.array([0.25]), W)[0] for W in (4, 6, 8)]
    assert abs(r[0]) > abs(r[1]) > abs(r[2])


def test_gridding_converges_to_exact():
    rng = np.random.default_rng(5)
    nd, n, nt = 16, 16, 12
    q = rng.standard_normal((2, nt, nd))
    th = np.sort(rng.uniform(0, np.pi, nt))
    exact = fr.backproject_exact(q, th, 8.4, n)
    errs = {W: rel(fr.backproject_gridding(q, th, 8.4, n, W), exact) for W in (4, 6, 8, 10)}
    assert errs[4] > errs[6] > errs[8] > errs[10]
    for W, e in errs.items():
        assert e < 10.0 ** (-(W - 2)), (W, e)


def test_gridding_grid_larger_than_twice_n():
    # n = 12 gives L = 32 (oversampling 8/3); ndet = 20 gives M = 64
    rng = np.random.default_rng(6)
    q = rng.standard_normal((1, 7, 20))
    th = np.sort(rng.uniform(0, np.pi, 7))
    exact = fr.backproject_exact(q, th, 9.9, 12)
    assert rel(fr.backproject_gridding(q, th, 9.9, 12, 8), exact) < 1e-6


def test_odd_n_rejected():
    with pytest.raises(ValueError):
        fr.backproject_exact(np.zeros((1, 2, 4)), np.zeros(2), 2.0, 5)


def _bump_fbp_errors(backproject):
    import synth
    errs, lin = [], []
    for n in (32, 64, 128):
        R = 0.3 * n
        x0, y0 = 0.07 * n, -0.05 * n
        nt = 2 * n
        theta = synth.uniform_theta(nt)
        c = n / 2.0 + 0.3
        p = synth.smooth_bump_sinogram(theta, n, c, R, x0, y0)
        q = oracle.filter_sino(p[None], c, "ramp", "edge")
        f = synth.smooth_bump(n, R, x0, y0)
        xc = np.arange(n) - n / 2
        X, Y = np.meshgrid(xc, xc)
        m = X ** 2 + Y ** 2 < (n / 2 - 2.0) ** 2
        e = lambda r: np.linalg.norm((r - f)[m]) / np.linalg.norm(f[m])
        errs.append(e(backproject(q, theta, n / 2.0, n)[0]))
        lin.append(e(oracle.backproject(q, theta, n / 2.0, n)[0]))
    return errs, lin


def test_fourierrec_fbp_of_smooth_bump_converges_to_the_function():
    # FourierRec approximates the same FBP integral as LineRec: the FBP of the
    # analytic Radon transform of f = (1 - r^2/R^2)^2 converges to f, and the
    # band-limited interpolant does better than the linear one at every size
    errs, lin = _bump_fbp_errors(lambda q, th, c, n: fr.backproject_gridding(q, th, c, n, width=10))
    assert errs[0] > errs[1] > errs[2] and errs[2] < 3e-4, errs
    assert all(a < b for a, b in zip(errs, lin)), (errs, lin)
