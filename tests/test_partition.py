"""Instance-to-rank assignment of the batched workload (greedy longest-processing-time):
coverage, determinism, Graham's 4/3 - 1/(3m) bound against the brute-force optimum on small
cases, its tight textbook case, and two gloo ranks agreeing on the same shards."""
import itertools
import os
import socket

import numpy as np
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2603_19647_gb300 import inputs
from paper_2603_19647_gb300.partition import (instance_cost, lpt_partition, shard,
                                              workload_directions)


def _makespan(costs, parts):
    return max(sum(costs[i] for i in p) for p in parts)


def test_every_instance_once_and_deterministic():
    rng = np.random.default_rng(0)
    costs = list(rng.uniform(1, 100, 37))
    for m in (1, 2, 3, 8, 40):
        parts = lpt_partition(costs, m)
        assert len(parts) == m
        assert sorted(i for p in parts for i in p) == list(range(37))
        assert parts == lpt_partition(costs, m)


def test_graham_bound_against_brute_force():
    rng = np.random.default_rng(1)
    for trial in range(30):
        n = int(rng.integers(3, 9))
        m = int(rng.integers(2, 4))
        costs = list(rng.integers(1, 20, n).astype(float))
        best = min(max(sum(c for c, a in zip(costs, assign) if a == r) for r in range(m))
                   for assign in itertools.product(range(m), repeat=n))
        got = _makespan(costs, lpt_partition(costs, m))
        assert best <= got <= (4 / 3 - 1 / (3 * m)) * best + 1e-12, (costs, m, got, best)


def test_tight_textbook_case():
    # two ranks, costs 3,3,2,2,2: LPT gives {3,2,2} and {3,2} (7), the optimum {3,3}, {2,2,2} (6)
    costs = [3.0, 3.0, 2.0, 2.0, 2.0]
    assert _makespan(costs, lpt_partition(costs, 2)) == 7.0


def test_cost_model_and_batched_directions():
    assert instance_cost(100, 64, 3.0) == 100 * 64 * 5
    wls = inputs.batched(count=12, scale=0.05)
    assert {workload_directions(w) for w in wls} <= {64, 128}
    shards = [shard(wls, r, 3)[0] for r in range(3)]
    assert sorted(i for s in shards for i in s) == list(range(12))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    wls = inputs.batched(count=64, scale=0.05)
    idx, mine = shard(wls, rank, world)
    gathered = [None] * world
    dist.all_gather_object(gathered, idx)
    out.put((rank, gathered, [w.name for w in mine]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_disjoint_shards():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=120) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, g0, names0), (_, g1, names1) = res
    assert g0 == g1
    assert sorted(g0[0] + g0[1]) == list(range(64)) and not set(g0[0]) & set(g0[1])
    assert names0 == [f"batched[{i}]" for i in g0[0]]
    assert names1 == [f"batched[{i}]" for i in g0[1]]
