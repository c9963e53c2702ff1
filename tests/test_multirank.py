"""The multi-rank path of bench.py on CPU: two gloo ranks (one process each, 127.0.0.1).

Under torchrun every rank drives its own GPU with its own context and its own frequencies (the
(omega, p) systems of eq. xplin are independent: weak scaling, no collective on the data path);
the only collective reduces the timings after the timed region.  These tests run that host logic
with world_size 2 on the gloo backend: the frequency shards are disjoint and cover the grid, and
the reduction takes the slowest rank's time and the sum of the ranks' columns.
"""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, steps, per, nw, sweep, out):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", world_size=world, rank=rank)
    try:
        mine = [bench.step_frequency_indices(k, world, rank, per, nw, sweep) for k in range(steps)]
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        seconds, cols = bench.reduce_over_ranks(dist, 1.5 + rank, 10 + 3 * rank, "cpu")
        if rank == 0:
            out.put((gathered, seconds, cols))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def _run(world, steps, per, nw, sweep):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, steps, per, nw, sweep, out)) for r in range(world)]
    for p in procs:
        p.start()
    try:
        res = out.get(timeout=120)
    finally:
        for p in procs:
            p.join(timeout=60)
    assert all(p.exitcode == 0 for p in procs)
    return res


@pytest.mark.parametrize("per,sweep", [(1, False), (4, False), (8, True)])
def test_two_ranks_shard_frequencies_and_reduce_timings(per, sweep):
    nw, world = 64, 2
    steps = nw // (world * per)          # exactly one pass over the grid
    gathered, seconds, cols = _run(world, steps, per, nw, sweep)
    flat = [i for rank_steps in gathered for step in rank_steps for i in step]
    assert len(flat) == nw and sorted(flat) == list(range(nw))   # disjoint shards that cover the grid
    assert seconds == 2.5                                         # slowest rank (1.5 + rank)
    assert cols == 10 + 13                                        # columns of both ranks


def test_single_rank_indices_match_the_stride_rule():
    # world 1: step k takes grid frequency (k per + j) * FREQ_STRIDE mod nw; warm-up steps the top end
    nw = 64
    assert bench.step_frequency_indices(0, 1, 0, 1, nw) == [0]
    assert bench.step_frequency_indices(1, 1, 0, 1, nw) == [bench.FREQ_STRIDE % nw]
    assert bench.step_frequency_indices(-1, 1, 0, 2, nw) == [nw - 2, nw - 1]
    seconds, cols = bench.reduce_over_ranks(None, 3.0, 7, "cpu")
    assert (seconds, cols) == (3.0, 7)
