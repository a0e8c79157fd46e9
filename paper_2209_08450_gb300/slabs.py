"""z-slab split of one dataset across ranks (Sec. 2.4 of the TomocuPy paper:
one process per GPU reconstructs the slices between its start and end rows).

Parallel-beam slices are independent, so rank r of `world` reconstructs the
contiguous slab [z0, z1) = slab(nz, r, world) of the SAME projection stack:
it passes views raw[:, z0:z1], dark[:, z0:z1], flat[:, z0:z1] (no copy) and
writes vol[z0:z1] (or its own slab buffer).  No collective is on the data
path; ranks meet only in the timing barrier of the caller.
"""
from __future__ import annotations


def slab(nz: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous z-slab [z0, z1) of rank among world: the first nz % world
    ranks take one slice more, so the slabs differ by at most one slice."""
    if world < 1 or not 0 <= rank < world or nz < 0:
        raise ValueError("slab: need 0 <= rank < world and nz >= 0")
    base, extra = divmod(nz, world)
    z0 = rank * base + min(rank, extra)
    return z0, z0 + base + (1 if rank < extra else 0)


def rank_views(raw, dark, flat, vol, rank: int, world: int):
    """The views rank `rank` works on: raw/dark/flat [.., z0:z1, ..] of the
    projection stack (frames [nf][nz][ndet] or means [nz][ndet]) and its
    output slab (vol[z0:z1] when vol holds the whole volume, else vol itself,
    which must then hold exactly z1 - z0 slices)."""
    nz = raw.shape[1]
    z0, z1 = slab(nz, rank, world)

    def zsl(t):
        return t[:, z0:z1] if t.dim() == 3 else t[z0:z1]

    if vol.shape[0] == nz:
        out = vol[z0:z1]
    elif vol.shape[0] == z1 - z0:
        out = vol
    else:
        raise ValueError("slab: vol must hold all %d slices or the rank's %d" % (nz, z1 - z0))
    return (z0, z1), raw[:, z0:z1], zsl(dark), zsl(flat), out


def reconstruct_slab(raw, dark, flat, theta, center, vol, rank: int, world: int, fbp=None, **opts):
    """Reconstruct rank's slab of one dataset with `fbp` (default the
    library's chunked FBP) into its output slab; returns (z0, z1)."""
    if fbp is None:
        from . import fbp as fbp_call
        fbp = fbp_call
    (z0, z1), r, d, f, out = rank_views(raw, dark, flat, vol, rank, world)
    if z1 > z0:
        fbp(r, d, f, theta, center, out=out, **opts)
    return z0, z1
