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
