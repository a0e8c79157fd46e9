"""Seeded synthetic inputs shaped like the paper's workloads.

This module is shared by the tests and the benchmark.  It holds no step of the
reconstruction method (no normalisation, filter or backprojection): it only
builds phantoms, their exact parallel-beam line integrals and noisy uint16
detector frames from them, all in FP64 NumPy with ``numpy.random.default_rng``.

Geometry (pixel units): voxel (ix, iy) of an n x n slice has centre
(x, y) = (ix - n/2, iy - n/2); detector pixel j sits at coordinate j; a point
(x, y) projects at angle theta to s = x cos(theta) + y sin(theta) + center.

Noise model for uint16 frames (photon counting with a dark offset):
    raw  = min(65535, Poisson(I0 * exp(-mu * p)) + Poisson(dark_level))
    dark = Poisson(dark_level)
    flat = Poisson(I0) + Poisson(dark_level)
with mu chosen so that the largest line integral attenuates to exp(-2).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


def uniform_theta(ntheta: int) -> np.ndarray:
    """ntheta angles uniform on [0, pi)."""
    return np.pi * np.arange(ntheta, dtype=np.float64) / ntheta


@dataclass
class Ellipsoid:
    """Ellipsoid with semi-axes (a, b, c), rotated by phi about z, density rho.
    Centre (x0, y0, z0) in pixel units; z0 is measured on the slice-height axis."""
    x0: float
    y0: float
    z0: float
    a: float
    b: float
    c: float
    phi: float
    rho: float


# Ellipsoids after the 3-D Shepp-Logan head phantom (Shepp & Logan 1974;
# 3-D form in Kak & Slaney 1988, with the higher-contrast densities of Toft
# 1996), restricted to rotations about the z axis.  Columns: rho, a, b, c,
# x0, y0, z0, phi (degrees), all in units of the phantom radius.  The exact
# numbers are not load-bearing: every test compares against the closed-form
# line integrals of whatever table is used here.
_SHEPP_LOGAN_3D = [
    (1.0, 0.6900, 0.920, 0.810, 0.00, 0.0000, 0.00, 0.0),
    (-0.8, 0.6624, 0.874, 0.780, 0.00, -0.0184, 0.00, 0.0),
    (-0.2, 0.1100, 0.310, 0.220, 0.22, 0.0000, 0.00, -18.0),
    (-0.2, 0.1600, 0.410, 0.280, -0.22, 0.0000, 0.00, 18.0),
    (0.1, 0.2100, 0.250, 0.410, 0.00, 0.3500, -0.15, 0.0),
    (0.1, 0.0460, 0.046, 0.050, 0.00, 0.1000, 0.25, 0.0),
    (0.1, 0.0460, 0.046, 0.050, 0.00, -0.1000, 0.25, 0.0),
    (0.1, 0.0460, 0.023, 0.050, -0.08, -0.6050, 0.00, 0.0),
    (0.1, 0.0230, 0.023, 0.020, 0.00, -0.6060, 0.00, 0.0),
    (0.1, 0.0230, 0.046, 0.020, 0.06, -0.6050, 0.00, 0.0),
]


def shepp_logan_3d(n: int, radius_frac: float = 0.45) -> list[Ellipsoid]:
    """3-D Shepp-Logan-type phantom scaled to an n-pixel grid (radius 0.45 n)."""
    r = radius_frac * n
    return [Ellipsoid(x0 * r, y0 * r, z0 * r, a * r, b * r, c * r, np.deg2rad(phi), rho)
            for rho, a, b, c, x0, y0, z0, phi in _SHEPP_LOGAN_3D]


def slice_heights(nz: int, n: int, span: float = 0.5, radius_frac: float = 0.45) -> np.ndarray:
    """nz slice heights spread over [-span/2, span/2] of the phantom radius."""
    r = radius_frac * n
    return r * span * ((np.arange(nz) + 0.5) / nz - 0.5)


def random_ellipsoids(rng: np.random.Generator, count: int, n: int, nz_extent: float,
                      axis_range=(0.02, 0.25), fov_frac: float = 0.48) -> list[Ellipsoid]:
    """count ellipsoids with axes U(axis_range)*n, density U(0, 1), rotation
    U(0, pi) about z, centres drawn so that each stays inside the field-of-view
    cylinder of radius fov_frac*n; z centres uniform over [-nz_extent/2, nz_extent/2]."""
    out = []
    rmax = fov_frac * n
    while len(out) < count:
        a, b, c = rng.uniform(axis_range[0], axis_range[1], size=3) * n
        reach = max(a, b)
        if reach >= rmax:
            continue
        rad = (rmax - reach) * np.sqrt(rng.uniform())
        ang = rng.uniform(0, 2 * np.pi)
        z0 = rng.uniform(-nz_extent / 2, nz_extent / 2)
        phi = rng.uniform(0, np.pi)
        rho = rng.uniform(0, 1)
        out.append(Ellipsoid(rad * np.cos(ang), rad * np.sin(ang), z0, a, b, c, phi, rho))
    return out


def porous_spheres(rng: np.random.Generator, n: int, nz: int, r_range=(3.0, 40.0),
                   rho_range=(0.2, 1.0), solid_fraction: float = 0.4,
                   cyl_frac: float = 0.45) -> np.ndarray:
    """Porous medium: spheres with radius U(r_range) px and density U(rho_range)
    (additive where they overlap), centres uniform inside a cylinder of radius
    cyl_frac*n (each sphere kept inside it) and over the nz slice heights, added
    until their summed volume reaches solid_fraction of the cylinder.
    Returns an array [count, 5] of (x0, y0, z0, r, rho)."""
    rcyl = cyl_frac * n
    target = solid_fraction * np.pi * rcyl * rcyl * nz
    mean_vol = 4.0 / 3.0 * np.pi * (r_range[1] ** 4 - r_range[0] ** 4) / (4 * (r_range[1] - r_range[0]))
    est = int(target / mean_vol * 1.3) + 16
    out = []
    vol = 0.0
    while vol < target:
        r = rng.uniform(r_range[0], r_range[1], size=est)
        rho = rng.uniform(rho_range[0], rho_range[1], size=est)
        rad = (rcyl - r) * np.sqrt(rng.uniform(size=est))
        ang = rng.uniform(0, 2 * np.pi, size=est)
        z0 = rng.uniform(-nz / 2, nz / 2, size=est)
        v = 4.0 / 3.0 * np.pi * r ** 3
        cum = vol + np.cumsum(v)
        k = int(np.searchsorted(cum, target)) + 1
        k = min(k, est)
        out.append(np.stack([rad[:k] * np.cos(ang[:k]), rad[:k] * np.sin(ang[:k]), z0[:k], r[:k], rho[:k]], 1))
        vol = cum[k - 1]
    return np.concatenate(out, 0)


def ellipses_at(ellipsoids: list[Ellipsoid], z: float):
    """2-D cross-sections at height z: list of (x0, y0, A, B, phi, rho)."""
    out = []
    for e in ellipsoids:
        u = (z - e.z0) / e.c
        if abs(u) < 1.0:
            k = np.sqrt(1.0 - u * u)
            out.append((e.x0, e.y0, e.a * k, e.b * k, e.phi, e.rho))
    return out


def ellipse_sinogram(ellipses, theta: np.ndarray, ndet: int, center: float) -> np.ndarray:
    """Exact line integrals of a sum of uniform ellipses at detector centres.

    For an ellipse with semi-axes A, B rotated by phi, centre (x0, y0) and
    density rho, the integral along the line at signed distance t from the
    origin is (Kak & Slaney 1988, Ch. 3)
        p = 2 rho A B sqrt(a^2 - t'^2) / a^2  for |t'| <= a, else 0,
        a^2 = A^2 cos^2(theta - phi) + B^2 sin^2(theta - phi),
        t'  = t - (x0 cos(theta) + y0 sin(theta)),  t = j - center.
    Returns p[theta][j] in FP64.
    """
    th = np.asarray(theta, dtype=np.float64)[:, None]
    t = (np.arange(ndet, dtype=np.float64) - center)[None, :]
    out = np.zeros((th.shape[0], ndet), np.float64)
    for x0, y0, A, B, phi, rho in ellipses:
        a2 = (A * np.cos(th - phi)) ** 2 + (B * np.sin(th - phi)) ** 2
        tp = t - (x0 * np.cos(th) + y0 * np.sin(th))
        inside = a2 - tp * tp
        out += np.where(inside > 0, 2.0 * rho * A * B * np.sqrt(np.maximum(inside, 0.0)) / a2, 0.0)
    return out


def sphere_sinogram(spheres: np.ndarray, z: float, theta: np.ndarray, ndet: int,
                    center: float) -> np.ndarray:
    """Exact line integrals p[theta][j] through the slice at height z of a set
    of uniform spheres (x0, y0, z0, r, rho): each cuts the slice in a disk of
    radius rs = sqrt(r^2 - (z - z0)^2), whose chord integral is
    2 rho sqrt(rs^2 - t'^2)."""
    dz = z - spheres[:, 2]
    cut = np.abs(dz) < spheres[:, 3]
    s = spheres[cut]
    rs = np.sqrt(s[:, 3] ** 2 - dz[cut] ** 2)
    ell = [(x0, y0, r, r, 0.0, rho) for (x0, y0, _, _, rho), r in zip(s, rs)]
    return ellipse_sinogram(ell, theta, ndet, center)


def rasterize_ellipses(ellipses, n: int, supersample: int = 4) -> np.ndarray:
    """Pixel-average image [iy][ix] of a sum of uniform ellipses (supersampled)."""
    off = (np.arange(supersample) + 0.5) / supersample - 0.5
    c = np.arange(n, dtype=np.float64) - n / 2.0
    xs = (c[:, None] + off[None, :]).reshape(-1)
    X, Y = np.meshgrid(xs, xs)  # Y varies along rows (iy), X along columns (ix)
    img = np.zeros_like(X)
    for x0, y0, A, B, phi, rho in ellipses:
        dx, dy = X - x0, Y - y0
        u = dx * np.cos(phi) + dy * np.sin(phi)
        v = -dx * np.sin(phi) + dy * np.cos(phi)
        img += np.where((u / A) ** 2 + (v / B) ** 2 <= 1.0, rho, 0.0)
    return img.reshape(n, supersample, n, supersample).mean(axis=(1, 3))


def smooth_bump(n: int, R: float, x0: float = 0.0, y0: float = 0.0) -> np.ndarray:
    """f = (1 - r^2/R^2)^2 inside radius R, sampled at voxel centres [iy][ix]."""
    c = np.arange(n, dtype=np.float64) - n / 2.0
    X, Y = np.meshgrid(c, c)
    r2 = ((X - x0) ** 2 + (Y - y0) ** 2) / (R * R)
    return np.where(r2 < 1.0, (1.0 - r2) ** 2, 0.0)


def smooth_bump_sinogram(theta: np.ndarray, ndet: int, center: float, R: float,
                         x0: float = 0.0, y0: float = 0.0) -> np.ndarray:
    """Radon transform of smooth_bump: p(t') = (16/15) R (1 - t'^2/R^2)^(5/2)."""
    th = np.asarray(theta, dtype=np.float64)[:, None]
    t = (np.arange(ndet, dtype=np.float64) - center)[None, :] - (x0 * np.cos(th) + y0 * np.sin(th))
    u = 1.0 - (t / R) ** 2
    return np.where(u > 0, 16.0 / 15.0 * R * np.maximum(u, 0.0) ** 2.5, 0.0)


def frames_from_line_integrals(p: np.ndarray, rng: np.random.Generator, I0: float,
                               n_dark: int, n_flat: int, dark_level: float = 100.0,
                               max_attenuation: float = 2.0):
    """uint16 detector frames from line integrals p[theta][z][j].

    Returns (raw [theta][z][j], dark [n_dark][z][j], flat [n_flat][z][j], mu).
    Draw order: raw photons, raw dark offset, dark frames, flat photons, flat
    dark offset.
    """
    pmax = float(p.max())
    mu = max_attenuation / pmax if pmax > 0 else 1.0
    lam = I0 * np.exp(-mu * p)
    raw = rng.poisson(lam) + rng.poisson(dark_level, size=p.shape)
    raw = np.minimum(raw, 65535).astype(np.uint16)
    shp = p.shape[1:]
    dark = rng.poisson(dark_level, size=(n_dark,) + shp).astype(np.uint16)
    flat = rng.poisson(I0, size=(n_flat,) + shp) + rng.poisson(dark_level, size=(n_flat,) + shp)
    flat = np.minimum(flat, 65535).astype(np.uint16)
    return raw, dark, flat, mu


@dataclass
class Dataset:
    raw: np.ndarray      # uint16 [theta][z][j]
    dark: np.ndarray     # uint16 [n_dark][z][j]
    flat: np.ndarray     # uint16 [n_flat][z][j]
    theta: np.ndarray    # float64 [theta]
    center: float
    mu: float
    line_integrals: np.ndarray  # float64 [theta][z][j], noise-free


def shepp_logan_dataset(ntheta=256, ndet=256, nz=16, center=128.0, I0=4e4, n_dark=10,
                        n_flat=10, seed=0) -> Dataset:
    """Plain FBP workload: 3-D Shepp-Logan, analytic projections, uint16 frames
    (defaults: 256 angles, 256 pixels x 16 slices, centre 128, I0 = 4e4)."""
    rng = np.random.default_rng(seed)
    theta = uniform_theta(ntheta)
    ells = shepp_logan_3d(ndet)
    zs = slice_heights(nz, ndet)
    p = np.stack([ellipse_sinogram(ellipses_at(ells, z), theta, ndet, center) for z in zs], 1)
    raw, dark, flat, mu = frames_from_line_integrals(p, rng, I0, n_dark, n_flat)
    return Dataset(raw, dark, flat, theta, center, mu, p)


def ellipsoid_dataset(ntheta=1500, ndet=1024, nz=16, count=64, I0=2e4, n_dark=20, n_flat=20,
                      seed=0, z_extent=None, center=None) -> Dataset:
    """Random-ellipsoid workload: 64 seeded ellipsoids, centre ndet/2 - 0.5 + U(-2, 2),
    uint16 frames with I0 = 2e4 and 20 dark/flat frames (sizes are arguments so
    the same recipe serves small test cases)."""
    rng = np.random.default_rng(seed)
    if center is None:
        center = ndet / 2.0 - 0.5 + rng.uniform(-2, 2)
    z_extent = float(ndet) if z_extent is None else z_extent
    ells = random_ellipsoids(rng, count, ndet, z_extent)
    theta = uniform_theta(ntheta)
    zs = (np.arange(nz) + 0.5 - nz / 2.0) * (z_extent / max(nz, 1))
    p = np.stack([ellipse_sinogram(ellipses_at(ells, z), theta, ndet, center) for z in zs], 1)
    raw, dark, flat, mu = frames_from_line_integrals(p, rng, I0, n_dark, n_flat)
    return Dataset(raw, dark, flat, theta, center, mu, p)


def porous_dataset(ntheta=2048, ndet=2048, nz=8, n_total=None, z_first=0, I0=3e4, n_dark=20,
                   n_flat=20, seed=0, center=None) -> Dataset:
    """Porous-medium workload on the host: seeded spheres (r = 3-40 px,
    density 0.2-1.0) filling 40 % of a 0.45 n cylinder through n_total slices;
    returns slices [z_first, z_first + nz) only."""
    rng = np.random.default_rng(seed)
    n_total = ndet if n_total is None else n_total
    center = ndet / 2.0 if center is None else center
    spheres = porous_spheres(rng, ndet, n_total)
    theta = uniform_theta(ntheta)
    zs = np.arange(z_first, z_first + nz) + 0.5 - n_total / 2.0
    p = np.stack([sphere_sinogram(spheres, z, theta, ndet, center) for z in zs], 1)
    raw, dark, flat, mu = frames_from_line_integrals(p, rng, I0, n_dark, n_flat)
    return Dataset(raw, dark, flat, theta, center, mu, p)
