"""Host logic of the multi-process bench (independent replicas, no data-path collective):
the whole-job time is the slowest rank's, the work is the sum over ranks (two gloo ranks on
the CPU); and the oracle arm's JSON line, run alone and as two torchrun ranks."""
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


def _bench_lines(cmd):
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    res = subprocess.run([sys.executable] + cmd, cwd=root, capture_output=True, text=True,
                         timeout=300)
    assert res.returncode == 0, res.stderr[-2000:]
    return [json.loads(l) for l in res.stdout.splitlines() if l.startswith("{")]


def _check_reference_line(line, gpus):
    assert line["impl"] == "reference" and line["n_gpus"] == gpus
    for k in ("metric", "unit", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config"):
        assert k in line, k
    assert line["value"] > 0 and line["higher_is_better"] is True
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"]
    assert cb["unit"] == line["unit"] and cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_json_line():
    """The oracle arm on the host cores prints one line of the bench's contract."""
    lines = _bench_lines(["bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0",
                          "--grid", "16"])
    assert len(lines) == 1
    _check_reference_line(lines[0], 1)


def test_reference_arm_under_torchrun_prints_once():
    """Launched as two ranks, rank 0 alone runs the oracle and prints; rank 1 exits 0."""
    lines = _bench_lines(["-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
                          "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
                          "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1",
                          "--warmup", "0", "--grid", "16"])
    assert len(lines) == 1
    _check_reference_line(lines[0], 2)
