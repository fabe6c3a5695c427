"""Object placement on ranks and the benchmark's cross-rank reductions, on CPU with the gloo backend."""
import itertools
import os
import socket

import numpy as np
import pytest

from paper_2304_05735_gb300.sharding import lpt_partition, makespan, max_over_ranks, sum_over_ranks


def _brute_force_makespan(costs, world):
    best = float("inf")
    for assign in itertools.product(range(world), repeat=len(costs)):
        load = [0.0] * world
        for i, r in enumerate(assign):
            load[r] += costs[i]
        best = min(best, max(load))
    return best


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("world", [2, 3])
def test_lpt_covers_every_object_once_within_graham_bound(seed, world):
    rng = np.random.default_rng(seed)
    costs = list(np.exp(rng.uniform(np.log(256), np.log(16384), 7)))
    parts = lpt_partition(costs, world)
    assert sorted(i for p in parts for i in p) == list(range(len(costs)))
    opt = _brute_force_makespan(costs, world)
    assert makespan(costs, parts) <= (4 / 3 - 1 / (3 * world)) * opt + 1e-9


def test_lpt_single_rank_and_more_ranks_than_objects():
    assert lpt_partition([3, 1, 2], 1) == [[0, 1, 2]]
    parts = lpt_partition([5, 7], 4)
    assert parts == [[1], [0], [], []]
    with pytest.raises(ValueError):
        lpt_partition([1], 0)


def test_reductions_without_process_group():
    assert max_over_ranks(2.5) == 2.5
    assert sum_over_ranks(7) == 7.0


def _worker(rank, world, port, costs, q):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        parts = lpt_partition(costs, world)
        mine = parts[rank]
        # every rank derives the same placement; gather it to check the ranks agree and cover all objects
        got = [None] * world
        dist.all_gather_object(got, mine)
        step_ms = 10.0 + rank  # rank-dependent "step time"
        samples = sum(costs[i] for i in mine)
        q.put((rank, got, max_over_ranks(step_ms, dist), sum_over_ranks(samples, dist)))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_rank_placement_and_reductions_gloo():
    import torch.multiprocessing as mp

    world = 2
    costs = [4096.0 * 64] * 5 + [300.0 * 64, 9000.0 * 64, 16000.0 * 64]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, costs, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    expect = lpt_partition(costs, world)
    for rank, got, mx, sm in res:
        assert got == expect
        assert mx == 10.0 + world - 1
        assert sm == pytest.approx(sum(costs))
    assert sorted(i for p in expect for i in p) == list(range(len(costs)))
