"""Host logic of the multi-process bench (independent replicas, no data-path collective):
the whole-job time is the slowest rank's, the work is the sum over ranks.  Two gloo ranks on
the CPU."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, upd = bench.reduce_over_ranks(dist, 10.0 + 5.0 * rank, 1000 * (rank + 1), "cpu")
    out.put((rank, ms, upd))
    dist.barrier()
    dist.destroy_process_group()


def test_reduce_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == [(0, 15.0, 3000.0), (1, 15.0, 3000.0)]


def test_single_process_passthrough():
    import bench
    assert bench.reduce_over_ranks(None, 12.5, 7, "cpu") == (12.5, 7.0)
