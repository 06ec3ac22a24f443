"""Pair sharding of a batch across ranks (host logic, CPU): the LPT partition
covers every pair exactly once, keeps the largest rank load within Graham's
4/3 - 1/(3N) of the optimum's lower bound, is the same on every rank, and the
all-gather of per-pair records over two gloo ranks (127.0.0.1) returns every
pair's record on every rank."""
import multiprocessing as mp
import os
import socket
import sys

import numpy as np
import pytest

from paper_2410_04385_gb300 import sharding
from paper_2410_04385_gb300 import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def batch_costs(count=64, seed=7):
    pairs = wl.workload_batch_uneven(count=count, seed=seed)
    return [sharding.predicted_flops(Y, Z, o) for Y, Z, o in pairs]


@pytest.mark.parametrize("world", [1, 2, 3, 4, 8])
def test_lpt_partition_covers_and_balances(world):
    costs = batch_costs()
    parts = sharding.lpt_partition(costs, world)
    flat = sorted(i for p in parts for i in p)
    assert flat == list(range(len(costs)))
    loads = [sum(costs[i] for i in p) for p in parts]
    lower = max(sum(costs) / world, max(costs))
    assert max(loads) <= (4.0 / 3.0 - 1.0 / (3 * world)) * lower * (1 + 1e-12) + 1e-9
    assert sharding.lpt_partition(costs, world) == parts


def test_lpt_degenerate_cases():
    assert sharding.lpt_partition([], 3) == [[], [], []]
    assert sharding.lpt_partition([5.0], 2) == [[0], []]
    assert sharding.lpt_partition([1.0, 1.0, 1.0, 1.0], 2) == [[0, 2], [1, 3]]
    with pytest.raises(ValueError):
        sharding.lpt_partition([1.0], 0)


def test_predicted_flops_follow_the_section4_model():
    from paper_2410_04385_gb300 import costmodel
    Y, Z, opts = wl.workload_random_d20()
    n, r, s, ell = sharding.pair_ranks(Y, Z, opts)
    assert ell == [1, 32] + [50] * 17 + [32, 1]
    hp, sw = costmodel.hatt1_flops(n, r, s, ell)
    assert sharding.predicted_flops(Y, Z, opts) == pytest.approx(hp + sw)


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    from paper_2410_04385_gb300 import sharding as sh
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        costs = batch_costs(count=40, seed=5)
        mine = sh.lpt_partition(costs, world)[rank]
        records = [[j, 0, len(mine), rank] for j in mine]
        merged = sh.gather_records(records, world)
        out.put((rank, mine, merged))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_gather_over_two_gloo_ranks_returns_every_pair():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = {}
    for _ in procs:
        rank, mine, merged = q.get(timeout=180)
        got[rank] = (mine, merged)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert sorted(got[0][0] + got[1][0]) == list(range(40))
    assert not set(got[0][0]) & set(got[1][0])
    for rank in (0, 1):
        merged = got[rank][1]
        assert sorted(rec[0] for rec in merged) == list(range(40))
        assert all(rec[3] == (0 if rec[0] in got[0][0] else 1) for rec in merged)
    assert got[0][1] == got[1][1]
