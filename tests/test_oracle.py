"""Pins of the FP64 oracle against mathematics, not against itself.

Each test fixes a result that the paper's method (Sec. 2.2 / Sec. 3 LineRec)
or plain mathematics determines: closed forms, brute force on tiny inputs,
special angles, the adjoint identity and convergence to analytic phantoms.
"""
import numpy as np
import pytest

import oracle
import synth


# --------------------------------------------------------------- normalise ---

def test_frame_mean_exact():
    frames = np.stack([np.full((2, 3), 100 + k, np.uint16) for k in range(10)])
    frames[:, 1, 2] = np.arange(10) * 7
    m = oracle.frame_mean(frames)
    assert m.shape == (2, 3)
    assert np.all(m[0] == 104.5)
    assert m[1, 2] == 31.5


def test_normalize_closed_form_values():
    # dark 100, flat 10100: raw = flat -> 0; raw = 5100 -> r = 1/2 -> ln 2;
    # raw = dark -> r = 0 -> clamp eps; raw below dark -> clamp; 65535 -> finite.
    raw = np.array([10100, 5100, 100, 50, 65535, 2600], np.uint16).reshape(1, 1, 6)
    d = np.full((1, 6), 100.0)
    f = np.full((1, 6), 10100.0)
    p = oracle.normalize(raw, d, f)[0, 0]
    assert p[0] == 0.0
    assert abs(p[1] - np.log(2.0)) < 1e-15
    assert abs(p[2] - 13.815510557964274) < 1e-12  # -ln(1e-6)
    assert abs(p[3] - 13.815510557964274) < 1e-12
    assert abs(p[4] - (-np.log(65435.0 / 10000.0))) < 1e-14
    assert abs(p[5] - np.log(4.0)) < 1e-15


def test_normalize_degenerate_flat_is_clamped():
    raw = np.array([500, 100, 50], np.uint16).reshape(1, 1, 3)
    d = np.full((1, 3), 100.0)
    f = np.full((1, 3), 100.0)  # flat == dark: r is inf or nan -> eps
    p = oracle.normalize(raw, d, f)[0, 0]
    assert np.allclose(p, 13.815510557964274, atol=1e-12)


def test_normalize_transposes_projection_major_to_sinogram():
    nt, nz, nd = 3, 4, 5
    raw = (1000 + np.arange(nt * nz * nd)).astype(np.uint16).reshape(nt, nz, nd)
    d = np.zeros((nz, nd))
    f = np.full((nz, nd), 4096.0)
    p = oracle.normalize(raw, d, f)
    for t in range(nt):
        for z in range(nz):
            for j in range(nd):
                assert p[z, t, j] == -np.log(raw[t, z, j] / 4096.0)


# ------------------------------------------------------------------ filter ---

def test_ramp_response_closed_form():
    # DC bin: 1/4 - 2 sum_{odd m < N/2} 1/(pi^2 m^2); Nyquist bin: 1/4 + the
    # same sum; every bin within 1/N of the continuous ramp |nu|.
    n = 16
    r = oracle.filter_response("ramp", n)
    s = sum(1.0 / (np.pi ** 2 * m * m) for m in (1, 3, 5, 7))
    assert abs(r[0] - (0.25 - 2 * s)) < 1e-15
    assert abs(r[-1] - (0.25 + 2 * s)) < 1e-15
    for npad in (16, 256, 4096, 48, 3072, 80, 5120):  # 3 x 2^k and 5 x 2^k periods of the smooth padding too
        r = oracle.filter_response("ramp", npad)
        nu = np.arange(npad // 2 + 1) / npad
        assert np.max(np.abs(r - nu)) < 1.0 / npad
        assert r[0] > 0
    r = oracle.filter_response("ramp", 48)
    s = sum(1.0 / (np.pi ** 2 * m * m) for m in range(1, 24, 2))
    assert abs(r[0] - (0.25 - 2 * s)) < 1e-15


def test_window_special_values():
    n = 16
    r = oracle.filter_response("ramp", n)
    sl = oracle.filter_response("shepp", n)
    assert sl[0] == r[0]
    assert abs(sl[-1] - r[-1] * 2.0 / np.pi) < 1e-15  # sinc(1/2) = 2/pi
    assert abs(sl[4] - r[4] * np.sin(np.pi / 4) / (np.pi / 4)) < 1e-15
    pz = oracle.filter_response("parzen", n)
    assert pz[-1] == 0.0 and abs(pz[4] - r[4] * 0.125) < 1e-15
    assert np.all(oracle.filter_response("none", n) == 1.0)


def _brute_filter(row, center, kind, pad, ntheta, npad=None):
    """Brute-force reference: explicit padding, impulse response by a direct
    inverse DFT sum over the full Hermitian spectrum, then a direct circular
    convolution, then the crop."""
    nd = row.shape[0]
    if npad is None:
        npad = 1
        while npad < 2 * nd:
            npad *= 2
    left = (npad - nd) // 2
    right = npad - nd - left
    if pad == "edge":
        x = np.concatenate([np.full(left, row[0]), row, np.full(right, row[-1])])
    else:
        x = np.concatenate([np.zeros(left), row, np.zeros(right)])
    half = oracle.filter_response(kind, npad) * np.pi / ntheta
    F = np.zeros(npad, complex)
    for k in range(npad // 2 + 1):
        F[k] = half[k] * np.exp(2j * np.pi * (k / npad) * (center - nd / 2.0))
    F[npad // 2] = F[npad // 2].real
    for k in range(1, npad // 2):
        F[npad - k] = np.conj(F[k])
    m = np.arange(npad)
    h = np.array([np.sum(F * np.exp(2j * np.pi * np.arange(npad) * mm / npad)) / npad for mm in m])
    assert np.max(np.abs(h.imag)) < 1e-12
    h = h.real
    y = np.array([np.sum(x * h[(mm - m) % npad]) for mm in m])
    return y[left:left + nd]


@pytest.mark.parametrize("nd,center,kind,pad", [
    (13, 6.5, "shepp", "edge"), (20, 11.25, "shepp", "zero"), (16, 7.0, "parzen", "edge"),
    (9, 3.7, "ramp", "edge"), (32, 16.0, "none", "zero")])
def test_filter_equals_direct_convolution(nd, center, kind, pad):
    rng = np.random.default_rng(nd)
    row = rng.normal(size=nd)
    got = oracle.filter_sino(row[None, :], center, kind, pad, ntheta=7)[0]
    ref = _brute_filter(row, center, kind, pad, 7)
    assert np.max(np.abs(got - ref)) < 1e-12


def test_smooth_padded_lengths():
    # the smallest of the next 2^k, 3 * 2^k (>= 48) and 5 * 2^k (>= 80) at or above 2 ndet
    cases = {12: 32, 20: 48, 24: 48, 40: 80, 45: 96, 100: 256, 200: 512, 300: 640, 1024: 2048, 1536: 3072,
             2560: 5120, 2048: 4096, 4096: 8192, 30: 64, 38: 80, 76: 160}
    for nd, n in cases.items():
        assert oracle.padded_length(nd, "smooth") == n, nd
        assert oracle.padded_length(nd) == 1 << (2 * nd - 1).bit_length()


@pytest.mark.parametrize("nd,center,kind,pad", [
    (20, 11.25, "shepp", "edge"), (24, 12.0, "parzen", "zero"), (45, 17.6, "ramp", "edge"),
    (40, 19.3, "shepp", "edge"), (76, 40.1, "parzen", "zero")])
def test_filter_on_smooth_padding_equals_direct_convolution(nd, center, kind, pad):
    # padded lengths 48, 48, 96 (3 x 2^k), 80 and 160 (5 x 2^k): the same
    # definition, other period
    rng = np.random.default_rng(nd + 1)
    row = rng.normal(size=nd)
    npad = oracle.padded_length(nd, "smooth")
    assert npad % 3 == 0 or npad % 5 == 0
    got = oracle.filter_sino(row[None, :], center, kind, pad, ntheta=5, rule="smooth")[0]
    ref = _brute_filter(row, center, kind, pad, 5, npad=npad)
    assert np.max(np.abs(got - ref)) < 1e-12


def test_filter_constant_row_keeps_only_the_dc_bin():
    # Edge padding keeps a constant row constant, so only the DC bin survives:
    # out = value * R_0 * pi / ntheta.
    row = np.full((1, 3, 50), 2.5)
    out = oracle.filter_sino(row, 25.0, "shepp", "edge")
    expect = 2.5 * oracle.filter_response("ramp", 128)[0] * np.pi / 3
    assert np.max(np.abs(out - expect)) < 1e-13


def test_filter_integer_centre_shift_is_index_shift():
    rng = np.random.default_rng(1)
    row = rng.normal(size=(1, 40))
    base = oracle.filter_sino(row, 20.0, "shepp", "zero")[0]
    shifted = oracle.filter_sino(row, 23.0, "shepp", "zero")[0]
    assert np.max(np.abs(shifted[:-3] - base[3:])) < 1e-13


# ------------------------------------------------- backproject / project ---

def _hat_matrix(n, ndet, theta, center):
    """System matrix from the hat-function definition, by brute force:
    A[(t, j), (iy, ix)] = max(0, 1 - |s(ix, iy, theta_t) - j|)."""
    A = np.zeros((len(theta) * ndet, n * n))
    for t, th in enumerate(theta):
        for j in range(ndet):
            for iy in range(n):
                for ix in range(n):
                    s = (ix - n / 2) * np.cos(th) + (iy - n / 2) * np.sin(th) + center
                    A[t * ndet + j, iy * n + ix] = max(0.0, 1.0 - abs(s - j))
    return A


@pytest.mark.parametrize("ndet,ntheta,center", [(8, 3, 4.3), (9, 5, 3.9), (11, 7, 5.5), (8, 4, 4.0)])
def test_projector_and_backprojector_equal_brute_force_matrix(ndet, ntheta, center):
    n = 8
    rng = np.random.default_rng(ndet * 10 + ntheta)
    theta = np.sort(rng.uniform(0, np.pi, ntheta))
    A = _hat_matrix(n, ndet, theta, center)
    vol = rng.normal(size=(n, n))
    q = rng.normal(size=(ntheta, ndet))
    P = oracle.project(vol, theta, center, ndet)[0]
    assert np.max(np.abs(P.reshape(-1) - A @ vol.reshape(-1))) < 1e-12
    B = oracle.backproject(q, theta, center, n)[0]
    assert np.max(np.abs(B.reshape(-1) - A.T @ q.reshape(-1))) < 1e-12


def test_adjoint_identity():
    rng = np.random.default_rng(5)
    n, nd, nt, nz = 40, 47, 29, 2
    theta = rng.uniform(0, np.pi, nt)
    x = rng.normal(size=(nz, n, n))
    y = rng.normal(size=(nz, nt, nd))
    lhs = np.vdot(oracle.project(x, theta, 23.3, nd), y)
    rhs = np.vdot(x, oracle.backproject(y, theta, 23.3, n))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_theta_zero_gives_column_sums_and_replicated_rows():
    rng = np.random.default_rng(2)
    n = 12
    vol = rng.normal(size=(n, n))
    p = oracle.project(vol, np.array([0.0]), n / 2, n)[0, 0]
    assert np.max(np.abs(p - vol.sum(axis=0))) < 1e-13
    q = rng.normal(size=(1, n))
    b = oracle.backproject(q, np.array([0.0]), n / 2, n)[0]
    assert np.all(b == np.broadcast_to(q, (n, n)))


def test_theta_half_pi_gives_row_sums():
    rng = np.random.default_rng(3)
    n = 10
    vol = rng.normal(size=(n, n))
    p = oracle.project(vol, np.array([np.pi / 2]), n / 2, n)[0, 0]
    assert np.max(np.abs(p - vol.sum(axis=1))) < 1e-12
    q = rng.normal(size=(1, n))
    b = oracle.backproject(q, np.array([np.pi / 2]), n / 2, n)[0]
    assert np.max(np.abs(b - q.reshape(n, 1))) < 1e-12


def test_constant_sinogram_backprojects_to_ntheta_inside_circle():
    n, nd, nt = 32, 32, 17
    theta = synth.uniform_theta(nt)
    b = oracle.backproject(np.full((nt, nd), 1.5), theta, nd / 2, n)[0]
    c = np.arange(n) - n / 2
    X, Y = np.meshgrid(c, c)
    inside = X ** 2 + Y ** 2 < (nd / 2 - 1.5) ** 2
    assert np.max(np.abs(b[inside] - 1.5 * nt)) < 1e-12
    assert np.all(b <= 1.5 * nt + 1e-12)


def test_backproject_points_equal_full_slice():
    rng = np.random.default_rng(4)
    n, nd, nt = 20, 23, 11
    theta = rng.uniform(0, np.pi, nt)
    q = rng.normal(size=(nt, nd))
    full = oracle.backproject(q, theta, 10.7, n)[0]
    ix = rng.integers(0, n, 50)
    iy = rng.integers(0, n, 50)
    pts = oracle.backproject_points(q, theta, 10.7, n, ix, iy)
    assert np.max(np.abs(pts - full[iy, ix])) < 1e-12


def test_projector_axis_angles_converge_to_closed_form_at_second_order():
    # At theta = 0 and pi/2 the projector is the midpoint rule along columns
    # (rows), so for the smooth bump it converges to the exact Radon
    # transform (16/15) R (1 - t^2/R^2)^(5/2) at second order in 1/n.
    errs = []
    for n in (32, 64, 128, 256):
        R, x0, y0, c = 0.3 * n, 0.1 * n, -0.07 * n, n / 2 + 0.37
        th = np.array([0.0, np.pi / 2])
        p = oracle.project(synth.smooth_bump(n, R, x0, y0), th, c, n)[0]
        ref = synth.smooth_bump_sinogram(th, n, c, R, x0, y0)
        errs.append(np.linalg.norm(p - ref) / np.linalg.norm(ref))
    ratios = [errs[i] / errs[i + 1] for i in range(3)]
    assert min(ratios) > 3.5, (errs, ratios)
    assert errs[-1] < 2e-4


def test_projector_conserves_mass_at_every_angle():
    # Each voxel's two weights sum to one, so every projection carries the
    # total mass of an object that projects inside the detector.
    n = 64
    rng = np.random.default_rng(9)
    theta = rng.uniform(0, np.pi, 37)
    img = synth.smooth_bump(n, 0.3 * n, 3.0, -2.0)
    p = oracle.project(img, theta, n / 2 - 0.4, n)[0]
    assert np.max(np.abs(p.sum(axis=1) - img.sum())) < 1e-12 * img.sum()


def test_projector_of_shepp_logan_approaches_closed_form():
    # Sharp edges and the pixel-driven weights leave an O(1) aliasing pattern
    # at oblique angles; the error still shrinks with n and stays small.
    errs = []
    for n in (64, 128, 256):
        ells = synth.ellipses_at(synth.shepp_logan_3d(n), 0.0)
        theta = synth.uniform_theta(24)
        img = synth.rasterize_ellipses(ells, n, supersample=8)
        p = oracle.project(img, theta, n / 2.0, n)[0]
        ref = synth.ellipse_sinogram(ells, theta, n, n / 2.0)
        errs.append(np.linalg.norm(p - ref) / np.linalg.norm(ref))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 0.03


# ------------------------------------------------------------- end to end ---

def _fov_mask(n, margin=2.0):
    c = np.arange(n) - n / 2
    X, Y = np.meshgrid(c, c)
    return X ** 2 + Y ** 2 < (n / 2 - margin) ** 2


def test_fbp_of_smooth_bump_converges_to_the_function():
    # Filtered backprojection of the exact Radon transform of
    # f = (1 - r^2/R^2)^2 converges to f inside the field of view at second
    # order: this fixes the ramp's scale and DC term, the pi/N_theta weight,
    # the sign of the centre shift and the interpolation.
    errs = []
    for n in (64, 128, 256):
        R = 0.3 * n
        x0, y0 = 0.07 * n, -0.05 * n
        nt = 2 * n
        theta = synth.uniform_theta(nt)
        c = n / 2.0 + 0.3
        p = synth.smooth_bump_sinogram(theta, n, c, R, x0, y0)
        q = oracle.filter_sino(p[None], c, "ramp", "edge")
        rec = oracle.backproject(q, theta, n / 2.0, n)[0]
        f = synth.smooth_bump(n, R, x0, y0)
        m = _fov_mask(n)
        errs.append(np.linalg.norm((rec - f)[m]) / np.linalg.norm(f[m]))
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5, errs
    assert errs[2] < 3e-4


def test_filter_centre_route_equals_backprojection_route():
    # Shifting the axis in the filter, or backprojecting about the true axis,
    # both reconstruct f to interpolation accuracy.
    n = 128
    nt = 256
    R, c = 0.3 * n, n / 2.0 + 2.25
    theta = synth.uniform_theta(nt)
    p = synth.smooth_bump_sinogram(theta, n, c, R)
    f = synth.smooth_bump(n, R)
    m = _fov_mask(n, 4.0)
    a = oracle.backproject(oracle.filter_sino(p[None], c, "ramp"), theta, n / 2.0, n)[0]
    b = oracle.backproject(oracle.filter_sino(p[None], n / 2.0, "ramp"), theta, c, n)[0]
    for r in (a, b):
        assert np.linalg.norm((r - f)[m]) / np.linalg.norm(f[m]) < 1.5e-3


def test_fbp_from_raw_frames_recovers_attenuation():
    ds = synth.shepp_logan_dataset(ntheta=128, ndet=128, nz=2, center=64.0, seed=0)
    rec = oracle.fbp(ds.raw, ds.dark, ds.flat, ds.theta, ds.center, "shepp")
    ells = synth.shepp_logan_3d(128)
    zs = synth.slice_heights(2, 128)
    truth = np.stack([synth.rasterize_ellipses(synth.ellipses_at(ells, z), 128) for z in zs]) * ds.mu
    err = np.linalg.norm(rec - truth) / np.linalg.norm(truth)
    assert err < 0.3
