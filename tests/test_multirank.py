"""The multi-rank path of bench.py on CPU ranks (gloo, world size 2): every
rank runs its own whole chains (distinct random streams, no collective on the
data path), the job's time is the slowest rank's, the job's work is the sum of
the ranks', and only rank 0 reports."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist          # noqa: E402
import torch.multiprocessing as mp         # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, chains, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms, total = bench.combine_ranks(dist, 10.0 * (rank + 1), 100 * (rank + 1), "cpu")
        layout = bench.rank_chains(rank, chains)
        layouts = [None] * world
        dist.all_gather_object(layouts, layout)
        q.put((rank, ms, total, layouts, bench.reports(rank)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    world, chains = 2, 3
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    mp.start_processes(_rank_main, args=(world, _free_port(), chains, q), nprocs=world, join=True,
                       start_method="spawn")
    got = sorted(q.get() for _ in range(world))
    for rank, ms, total, layouts, rep in got:
        assert ms == 20.0                       # slowest rank
        assert total == 300.0                   # all ranks' proposals
        assert rep == (rank == 0)
        seeds = [s for s, _ in layouts]
        idx = [i for _, c in layouts for i in c]
        assert len(set(seeds)) == world         # distinct seeds per rank
        assert sorted(idx) == list(range(world * chains))   # every (rank, chain) its own stream


def test_single_rank_needs_no_collective():
    import bench
    assert bench.combine_ranks(None, 12.5, 7, "cpu") == (12.5, 7.0)
    assert bench.rank_chains(0, 2) == (1000, [0, 1])
