"""Torch generator of the porous-medium workload at full size (on any device).

Same recipe as ``synth.porous_dataset`` (seeded spheres r = 3-40 px, density
0.2-1.0, 40 % solid fraction of a 0.45 n cylinder, exact chord integrals,
Poisson counts), written with plain torch tensor ops so that a 2048^3 stack
(17 GB of uint16) can be synthesised on the GPU in seconds.  It holds no step
of the reconstruction method.  The phantom geometry comes from the same
``numpy.random.default_rng(seed)`` draw as the host generator; the photon
noise comes from a seeded torch generator on the target device.
"""
from __future__ import annotations

import numpy as np
import torch

from . import porous_spheres, uniform_theta

# Window half-widths (px) of the chord profiles, by disk radius.
_BUCKETS = (6, 12, 24, 41)


def sphere_line_integrals(spheres: np.ndarray, zs: np.ndarray, theta: np.ndarray, ndet: int,
                          center: float, device, theta_block: int = 128) -> torch.Tensor:
    """Exact line integrals p[theta][k][j] (FP32) of uniform spheres through the
    slices at heights zs: each sphere cuts slice k in a disk of radius
    rs = sqrt(r^2 - (z_k - z0)^2) whose chord integral at signed distance t is
    2 rho sqrt(rs^2 - t^2)."""
    nt, nz = len(theta), len(zs)
    out = torch.zeros((nt, nz, ndet), dtype=torch.float32, device=device)
    sp = torch.as_tensor(spheres, dtype=torch.float64, device=device)
    zt = torch.as_tensor(np.asarray(zs, np.float64), device=device)
    dz = zt[None, :] - sp[:, 2:3]                      # [S, nz]
    r2 = (sp[:, 3:4] ** 2 - dz ** 2)
    sidx, kidx = torch.nonzero(r2 > 0, as_tuple=True)
    if sidx.numel() == 0:
        return out
    rs = torch.sqrt(r2[sidx, kidx])
    x0, y0, rho = sp[sidx, 0], sp[sidx, 1], sp[sidx, 4]
    th = torch.as_tensor(np.asarray(theta, np.float64), device=device)
    flat = out.view(-1)
    lo = 0.0
    for hw in _BUCKETS:
        sel = (rs > lo) & (rs <= hw)
        lo = hw
        if not bool(sel.any()):
            continue
        bx, by, bk = x0[sel], y0[sel], kidx[sel]
        br2 = (rs[sel] ** 2).float()[:, None, None]
        bq2 = (2.0 * rho[sel]).float()[:, None, None]
        offs = torch.arange(-hw - 1, hw + 2, device=device, dtype=torch.int64)
        for t0 in range(0, nt, theta_block):
            tb = th[t0:t0 + theta_block]
            c = bx[:, None] * torch.cos(tb)[None, :] + by[:, None] * torch.sin(tb)[None, :] + center  # [P, tb]
            fl = torch.floor(c)
            frac = (c - fl).float()[..., None]                                  # [P, tb, 1] in [0, 1)
            d = offs.float() - frac                                              # [P, tb, W]: j - c
            d2 = br2 - d * d
            j = fl.long()[..., None] + offs
            ok = (d2 > 0) & (j >= 0) & (j < ndet)
            tt = torch.arange(t0, t0 + tb.numel(), device=device)
            idx = (tt[None, :, None] * nz + bk[:, None, None]) * ndet + j
            flat.index_add_(0, idx[ok], (bq2 * torch.sqrt(torch.clamp(d2, min=0.0)))[ok])
    return out


def porous_frames(n: int = 2048, ntheta: int = 2048, nz: int | None = None, seed: int = 0, device="cuda",
                  I0: float = 3e4, n_dark: int = 20, n_flat: int = 20, dark_level: float = 100.0,
                  z_chunk: int = 32, slices: np.ndarray | None = None):
    """uint16 frames (as int16 tensors holding the same bits) of the porous
    workload: raw [ntheta][nz][n], dark [n_dark][nz][n], flat [n_flat][nz][n].
    ``slices`` selects a subset of the nz slice heights (default: all).
    Returns (raw, dark, flat, theta, center, mu)."""
    nz = n if nz is None else nz
    rng = np.random.default_rng(seed)
    spheres = porous_spheres(rng, n, nz)
    theta = uniform_theta(ntheta)
    center = n / 2.0
    sel = np.arange(nz) if slices is None else np.asarray(slices)
    heights = sel + 0.5 - nz / 2.0
    m = len(sel)
    raw = torch.empty((ntheta, m, n), dtype=torch.int16, device=device)
    half = raw.view(torch.float16)  # line integrals stored as FP16 until converted
    pmax = 0.0
    for k0 in range(0, m, z_chunk):
        p = sphere_line_integrals(spheres, heights[k0:k0 + z_chunk], theta, n, center, device)
        pmax = max(pmax, float(p.max()))
        half[:, k0:k0 + z_chunk] = p.to(torch.float16)
        del p
    mu = 2.0 / pmax if pmax > 0 else 1.0
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    for k0 in range(0, m, z_chunk):
        p = half[:, k0:k0 + z_chunk].float()
        counts = torch.poisson(I0 * torch.exp(-mu * p), generator=g) + \
            torch.poisson(torch.full_like(p, dark_level), generator=g)
        raw[:, k0:k0 + z_chunk] = _to_u16_bits(counts)
        del p, counts
    dark = _to_u16_bits(torch.poisson(torch.full((n_dark, m, n), dark_level, device=device), generator=g))
    flat = torch.poisson(torch.full((n_flat, m, n), I0, device=device), generator=g) + \
        torch.poisson(torch.full((n_flat, m, n), dark_level, device=device), generator=g)
    flat = _to_u16_bits(flat)
    return raw, dark, flat, theta, center, mu


def _to_u16_bits(counts: torch.Tensor) -> torch.Tensor:
    """Clamp to [0, 65535] and return int16 tensors holding the uint16 bits."""
    c = torch.clamp(counts, 0, 65535).to(torch.int32)
    return torch.where(c >= 32768, c - 65536, c).to(torch.int16)


def rasterize_ellipsoids(ellipsoids, n: int, zs, device="cuda") -> torch.Tensor:
    """Voxel-centre samples vol[k][iy][ix] (FP32) of a sum of uniform
    ellipsoids (rotated about z) at slice heights zs."""
    c = torch.arange(n, dtype=torch.float32, device=device) - n / 2.0
    Y, X = torch.meshgrid(c, c, indexing="ij")
    out = torch.zeros((len(zs), n, n), dtype=torch.float32, device=device)
    for k, z in enumerate(zs):
        for e in ellipsoids:
            u = (z - e.z0) / e.c
            if abs(u) >= 1.0:
                continue
            s = float(np.sqrt(1.0 - u * u))
            A, B = e.a * s, e.b * s
            dx, dy = X - e.x0, Y - e.y0
            cu, su = float(np.cos(e.phi)), float(np.sin(e.phi))
            pu = dx * cu + dy * su
            pv = -dx * su + dy * cu
            out[k] += torch.where((pu / A) ** 2 + (pv / B) ** 2 <= 1.0, float(e.rho), 0.0)
    return out


def frames_from_line_integrals(p: torch.Tensor, seed: int, I0: float, n_dark: int, n_flat: int,
                               dark_level: float = 100.0, max_attenuation: float = 2.0):
    """Torch version of synth.frames_from_line_integrals (same model, noise
    from a seeded torch generator on p's device).  p: [theta][z][j] FP32.
    Returns (raw, dark, flat, mu) as int16 tensors holding uint16 bits."""
    g = torch.Generator(device=p.device)
    g.manual_seed(seed)
    pmax = float(p.max())
    mu = max_attenuation / pmax if pmax > 0 else 1.0
    raw = _to_u16_bits(torch.poisson(I0 * torch.exp(-mu * p), generator=g) +
                       torch.poisson(torch.full_like(p, dark_level), generator=g))
    shp = tuple(p.shape[1:])
    dark = _to_u16_bits(torch.poisson(torch.full((n_dark,) + shp, dark_level, device=p.device), generator=g))
    flat = _to_u16_bits(torch.poisson(torch.full((n_flat,) + shp, I0, device=p.device), generator=g) +
                        torch.poisson(torch.full((n_flat,) + shp, dark_level, device=p.device), generator=g))
    return raw, dark, flat, mu


def ellipsoid_frames(n: int, ntheta: int, nz: int, seed: int = 0, device="cuda", count: int = 64,
                     I0: float = 2e4, n_dark: int = 20, n_flat: int = 20, center: float | None = None):
    """Random-ellipsoid workload (as synth.ellipsoid_dataset) on a torch device:
    count seeded ellipsoids, centre ndet/2 - 0.5 + U(-2, 2) unless given, exact
    ellipse line integrals per slice, Poisson frames.
    Returns (raw, dark, flat, theta, center, mu)."""
    from . import ellipses_at, random_ellipsoids
    rng = np.random.default_rng(seed)
    if center is None:
        center = n / 2.0 - 0.5 + rng.uniform(-2, 2)
    z_extent = float(n)
    ells = random_ellipsoids(rng, count, n, z_extent)
    theta = uniform_theta(ntheta)
    zs = (np.arange(nz) + 0.5 - nz / 2.0) * (z_extent / max(nz, 1))
    th = torch.as_tensor(theta, dtype=torch.float64, device=device)
    t = torch.arange(n, dtype=torch.float32, device=device) - float(center)
    p = torch.zeros((ntheta, nz, n), dtype=torch.float32, device=device)
    for k, z in enumerate(zs):
        acc = torch.zeros((ntheta, n), dtype=torch.float32, device=device)
        for x0, y0, A, B, phi, rho in ellipses_at(ells, z):
            a2 = ((A * torch.cos(th - phi)) ** 2 + (B * torch.sin(th - phi)) ** 2).float()
            sh = (x0 * torch.cos(th) + y0 * torch.sin(th)).float()
            tp = t[None, :] - sh[:, None]
            inside = a2[:, None] - tp * tp
            acc += torch.where(inside > 0, (2.0 * rho * A * B) * torch.sqrt(torch.clamp(inside, min=0.0)) / a2[:, None],
                               0.0)
        p[:, k, :] = acc
    raw, dark, flat, mu = frames_from_line_integrals(p, seed, I0, n_dark, n_flat)
    return raw, dark, flat, theta, center, mu
