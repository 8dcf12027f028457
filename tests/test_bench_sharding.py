"""The multi-rank path of bench.py on CPU: two gloo ranks deal chunks of consecutive Bloch vectors
round-robin (every point of the path once per sweep, no point on two ranks in the same sweep) and
reduce the timing with max and the k-point counts with sum, as the GPU launch under torchrun does."""

import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, nk, steps, kb, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = [bench.kpoint_chunk(s, world, rank, nk, kb) for s in range(steps)]
        local_time = 1.0 + rank  # rank-dependent "time"
        t_max = bench.max_over_ranks(world, local_time, device="cpu")
        total = bench.sum_over_ranks(world, float(steps * kb), device="cpu")
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        if rank == 0:
            out.put((gathered, t_max, total))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,steps,kb", [(2, 16, 1), (2, 3, 1), (2, 2, 8), (2, 3, 8)])
def test_two_rank_sharding_and_reductions(world, steps, kb):
    nk = 31
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, nk, steps, kb, q)) for r in range(world)]
    for p in procs:
        p.start()
    gathered, t_max, total = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert t_max == 1.0 + (world - 1)
    assert total == world * steps * kb
    # step s on rank r takes the kb points of chunk s * world + r (mod nk): the first sweep covers
    # each point once
    order = [i for s in range(steps) for r in range(world) for i in gathered[r][s]]
    first = order[:nk]
    assert len(set(first)) == len(first)
    if len(order) >= nk:
        assert sorted(first) == list(range(nk))
