"""Multi-rank pieces of bench.py on CPU with gloo (world size 2): the
max-over-ranks timing, the barrier, and the z-slab split (the paper's
--start-row/--end-row partition, Sec. 2.4)."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.barrier(world)
        m = bench.reduce_max(10.0 + 5.0 * rank, world)
        z0, z1 = bench.slab(2048, rank, world)
        out[rank] = (m, z0, z1, bench.dist_env())
    finally:
        dist.destroy_process_group()


def test_gloo_two_ranks_max_and_slabs():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0][0] == out[1][0] == 15.0
    assert (out[0][1], out[0][2], out[1][1], out[1][2]) == (0, 1024, 1024, 2048)
    assert out[0][3] == (0, 2, 0) and out[1][3][0] == 1


@pytest.mark.parametrize("nz,world", [(2048, 1), (2048, 3), (7, 4), (5, 8)])
def test_slabs_partition_every_slice_once(nz, world):
    seen = []
    for r in range(world):
        z0, z1 = bench.slab(nz, r, world)
        assert 0 <= z0 <= z1 <= nz
        seen.extend(range(z0, z1))
    assert seen == list(range(nz))
    sizes = [bench.slab(nz, r, world)[1] - bench.slab(nz, r, world)[0] for r in range(world)]
    assert max(sizes) - min(sizes) <= 1


def test_reduce_max_single_rank_is_identity():
    assert bench.reduce_max(3.5, 1) == 3.5


def _slab_worker(rank, world, port, out):
    # one seeded dataset per process (the shared stack every rank sees); the
    # reconstruction call is stubbed: it records the views it was given and
    # marks the output slab with the rank's id
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_2209_08450_gb300 import slabs
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        nt, nz, nd, n = 6, 11, 8, 8
        g = torch.Generator().manual_seed(0)
        raw = torch.randint(0, 30000, (nt, nz, nd), dtype=torch.int16, generator=g)
        dark = torch.randint(90, 110, (3, nz, nd), dtype=torch.int16, generator=g)
        flat = torch.rand((nz, nd), generator=g)  # F32 means form
        vol = torch.full((nz, n, n), -1.0)
        calls = []

        def fbp_stub(r, d, f, theta, center, out=None, **kw):
            calls.append({"raw": (r.data_ptr() - raw.data_ptr()) // 2, "raw_shape": tuple(r.shape),
                          "raw_stride": r.stride(), "dark": (d.data_ptr() - dark.data_ptr()) // 2,
                          "dark_shape": tuple(d.shape), "flat": (f.data_ptr() - flat.data_ptr()) // 4,
                          "flat_shape": tuple(f.shape), "out": (out.data_ptr() - vol.data_ptr()) // 4,
                          "out_shape": tuple(out.shape), "same_raw": bool(torch.equal(r, raw[:, out_z0[0]:out_z1[0]])),
                          "kw": kw})
            out.fill_(float(rank))

        out_z0, out_z1 = [0], [0]
        out_z0[0], out_z1[0] = slabs.slab(nz, rank, world)
        z0, z1 = slabs.reconstruct_slab(raw, dark, flat, np.zeros(nt), 4.0, vol, rank, world, fbp=fbp_stub,
                                        chunk_nz=4)
        mine = (vol[:, 0, 0] == rank).nonzero().flatten().tolist()
        out[rank] = (z0, z1, calls, mine)
    finally:
        dist.destroy_process_group()


def test_gloo_two_ranks_reconstruct_their_own_slab_of_one_dataset():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_slab_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    nt, nz, nd, n = 6, 11, 8, 8
    covered = []
    for rank in range(2):
        z0, z1, calls, mine = out[rank]
        assert (z0, z1) == bench.slab(nz, rank, 2) == ((0, 6), (6, 11))[rank]
        assert len(calls) == 1
        c = calls[0]
        # exactly the rank's [z0, z1) view of the shared stack, no copy
        assert c["raw"] == z0 * nd and c["raw_shape"] == (nt, z1 - z0, nd) and c["raw_stride"] == (nz * nd, nd, 1)
        assert c["same_raw"]
        assert c["dark"] == z0 * nd and c["dark_shape"] == (3, z1 - z0, nd)
        assert c["flat"] == z0 * nd and c["flat_shape"] == (z1 - z0, nd)
        assert c["out"] == z0 * n * n and c["out_shape"] == (z1 - z0, n, n)
        assert c["kw"] == {"chunk_nz": 4}
        assert mine == list(range(z0, z1))  # wrote its own slab and nothing else
        covered += mine
    assert sorted(covered) == list(range(nz))  # the two slabs cover the volume once
