"""Pins of the LpRec oracle (CPU only).

The cubic B-spline interpolant is pinned by textbook properties (it
interpolates, reproduces cubics away from the zero boundary, its weights
form a partition of unity); the exact cubic-spline backprojection by its
agreement with the LineRec oracle where every ray hits a detector node; the
log-polar evaluation by convergence to the exact sums as its grid is refined.
"""
import numpy as np
import pytest

import oracle
from oracle import lprec as lp


def rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def test_bspline_interpolates_and_reproduces_cubics():
    rng = np.random.default_rng(0)
    v = rng.standard_normal(40)
    np.testing.assert_allclose(lp.row_interp(v, np.arange(40.0)), v, rtol=0, atol=1e-12)
    # a cubic sampled on a long row is reproduced exactly far from the ends
    j = np.arange(200.0)
    cub = lambda s: 0.3 - 0.02 * s + 1e-3 * s ** 2 - 4e-6 * s ** 3
    s = np.linspace(90.0, 110.0, 57)
    np.testing.assert_allclose(lp.row_interp(cub(j), s), cub(s), rtol=0, atol=1e-9)
    # partition of unity of the four weights
    _, w = lp._beta3_taps(np.linspace(-3.0, 5.0, 33))
    np.testing.assert_allclose(sum(w), 1.0, rtol=0, atol=1e-15)


def test_spline_backprojection_at_nodes_equals_linerec():
    rng = np.random.default_rng(1)
    q = rng.standard_normal((2, 2, 12))
    th = np.array([0.0, np.pi / 2])
    got = lp.backproject_spline_exact(q, th, 6.0, 10)
    np.testing.assert_allclose(got, oracle.backproject(q, th, 6.0, 10), rtol=0, atol=1e-12)


def test_lprec_converges_to_spline_backprojection():
    rng = np.random.default_rng(2)
    nt, nd, n = 48, 32, 32
    theta = np.arange(nt) * np.pi / nt + 0.01
    q = rng.standard_normal((1, nt, nd))
    exact = lp.backproject_spline_exact(q, theta, 16.3, n)
    errs = [rel(lp.backproject_lprec(q, theta, 16.3, n, os=o), exact) for o in (2, 4, 8)]
    assert errs[0] > 4 * errs[1] > 16 * errs[2], errs
    assert errs[2] < 1e-4, errs


def test_lprec_needs_equally_spaced_angles():
    th = np.sort(np.random.default_rng(3).uniform(0, np.pi, 12))
    with pytest.raises(ValueError):
        lp.backproject_lprec(np.zeros((1, 12, 16)), th, 8.0, 16)


def test_lprec_span_convolution_by_fft_equals_direct_sum():
    # step (2) is a 2-D linear convolution on the log-polar grid (the kernel
    # uses the centred closed form of the cubic B-spline, independent of the
    # tap weights of the direct route)
    rng = np.random.default_rng(4)
    nt, nd, n = 36, 24, 24
    theta = np.arange(nt) * np.pi / nt
    q = rng.standard_normal((2, nt, nd))
    a = lp.backproject_lprec(q, theta, 11.7, n, os=2)
    b = lp.backproject_lprec(q, theta, 11.7, n, os=2, conv="fft")
    assert rel(b, a) < 1e-12


def test_lprec_fbp_of_smooth_bump_converges_to_the_function():
    # LpRec approximates the same FBP integral: with the analytic Radon
    # transform of the smooth bump its FBP converges to the bump (about
    # fourth order here), and its log-polar evaluation stays within 1 % of the
    # cubic-spline FBP's own error
    import synth
    errs = []
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
        a = e(lp.backproject_lprec(q, theta, n / 2.0, n, os=2)[0])
        b = e(lp.backproject_spline_exact(q, theta, n / 2.0, n)[0])
        assert abs(a - b) < 0.01 * b, (n, a, b)
        errs.append(a)
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5 and errs[2] < 1e-4, errs


def test_spline_points_equal_the_full_image():
    rng = np.random.default_rng(7)
    q = rng.standard_normal((1, 9, 20))
    th = rng.uniform(0, np.pi, 9)
    full = lp.backproject_spline_exact(q, th, 9.6, 18)[0]
    ix, iy = rng.integers(0, 18, 40), rng.integers(0, 18, 40)
    np.testing.assert_allclose(lp.backproject_spline_points(q[0], th, 9.6, 18, ix, iy), full[iy, ix],
                               rtol=0, atol=1e-12)
