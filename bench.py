#!/usr/bin/env python
"""Benchmark of the ROM-accelerated SI-DSA time march on GB300.

Metric: cell-direction updates/s, and time per implicit step at a 1e-8 relative residual,
ROM vs SI-DSA.  One bench step is one whole march of the 2D checkerboard workload
(256 x 256 cells, CL(32,8) hemisphere = 128 directions, c dt = 0.005, 200 implicit steps,
FP64, ROM-accelerated SI-DSA with Algorithm 2's three phases): every hot-path step
(sweeps, moments, DSA CG, DMD initial guess, ROM preconditioner, incremental SVD) runs in it.
One cell-direction update is one upwind cell solve; a step counts 1 + iterations + 1 sweeps
(Sec. 4), each of N_x N_v updates.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torchrun: independent replicas (the single-problem march has no exchange
step), value = all ranks' updates / max-over-ranks time.  --impl reference times the CPU
oracle (the plain FP64 implementation the tests check against) on bounded samples of the
same workload.  Prints one JSON line on rank 0.
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
# Hardware work queues of this process's CUDA context (read when the context is created, so set
# before torch initialises CUDA): with the default 8, the streams of the 64 batched instances
# (three per instance) share queues and their kernels serialise behind one another; 32 queues
# measured 66 -> 39 ms per batched step.
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

METRIC = "cell-direction updates/s; time per implicit step at 1e-8 residual, ROM vs SI-DSA"
UNIT = "cell-direction updates/s"
# FP64 ALU peak: 152 SMs x 2 FP64 FMA (4 flop) per clock x 2.07 GHz = 1.2586 TFLOP/s.
FP64_PEAK_TFLOPS = 152 * 4 * 2.07e9 / 1e12
FLOP_PER_UPDATE = 7          # two multiply-adds, one multiply by 1/d, one multiply-add (moment)
# Q1 SI sweep: the closed-form bilinear cell solve (106 FP64 flops, multiply-add = 2) and the
# weighted moment of its four modes (8)
Q1_FLOPS_PER_UPDATE = 114
PROFILE = os.path.join(ROOT, "profiles", "sweep_si_fp64_checkerboard.md")
SWEEP_SRC = [os.path.join(ROOT, "paper_2603_19647_gb300", "csrc", f)
             for f in ("sweep.cu", "sweep_common.cuh")]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-baseline", action="store_true", help="skip the cpu_baseline leg")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the reduced-precision and batched workloads measured beside the line")
    # not "--n": under torchrun that abbreviates several of the launcher's own options
    ap.add_argument("--grid", dest="n", type=int, default=256,
                    help="grid side (256 = the benchmark workload)")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), \
        int(os.environ.get("WORLD_SIZE", 1))


class Clocks:
    """Samples SM clock and throttle reasons with nvidia-smi during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        import statistics
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(self.rows)}


def profiled_traffic():
    """DRAM bytes per SI-sweep launch from the committed ncu summary, or None when the sweep
    source changed since the capture."""
    try:
        txt = open(PROFILE).read()
        src_hash = hashlib.sha256(b"".join(open(f, "rb").read() for f in SWEEP_SRC)).hexdigest()[:16]
        vals = dict(line.split(":", 1) for line in txt.splitlines() if ":" in line and line[:1] != "#")
        vals = {k.strip("-* `"): v.strip(" `") for k, v in vals.items()}
        if vals.get("sweep_src_sha256_16") != src_hash:
            return None
        return float(vals["dram_bytes_per_launch_full_size"])
    except (OSError, KeyError, ValueError):
        return None


def reduce_over_ranks(dist, total_ms, updates, device):
    """Whole-job figures of independent replicas: the slowest rank's time and the sum of all
    ranks' updates (dist None: one process)."""
    if dist is None:
        return float(total_ms), float(updates)
    import torch
    t = torch.tensor([float(total_ms)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([float(updates)], device=device, dtype=torch.float64)
    dist.all_reduce(u)
    return float(t.item()), float(u.item())


def oracle_sample(wl, budget_s, min_steps=2):
    """Time the CPU oracle's march on the workload for about budget_s seconds."""
    from oracle import build as obuild, quadrature, stepper, transport
    obuild.build()
    mu, eta, w = quadrature.cl_hemisphere(*wl.quadrature[1:])
    p = transport.Problem(wl.nx, wl.ny, *wl.domain, mu, eta, w, wl.sigma_t, wl.sigma_s, wl.source,
                          wl.c_dt)
    o = stepper.OracleRTE(p)
    o.set_initial(wl.rho0)
    t0 = time.perf_counter()
    k = 0
    while k < wl.steps and (k < min_steps or time.perf_counter() - t0 < budget_s):
        o.step(1)
        k += 1
    dt = time.perf_counter() - t0
    updates = sum(s.sweeps for s in o.log) * wl.ncell * p.nv
    return updates / dt, k, dt, transport.num_threads(), o


def extra_workloads(rte, inputs, torch, out):
    """The other rows of the method on this GPU, each a separately timed run beside the
    headline line: the 1024^2 log-normal workload and the 2048^2 diffusive disc for their full
    lengths (500 and 300 steps) in FP64 (ROM-accelerated and plain SI-DSA) and in the reduced
    precisions (FP32 sweeps; BF16-stored f at 2048^2), each reduced-precision march compared
    with the FP64 ROM march of the same GPU every few steps (final and worst relative L2 of the
    scalar flux); and the 64 batched instances (20 of 100 steps), with the kernels launched one
    by one and with the SI iterations in captured CUDA graphs (a while node around them).
    Time per step counts the
    steps alone (the comparisons' reads of rho are outside it).  The rows go into `out` as they
    are measured, so that rows measured before a failure stay in the line."""
    import numpy as np

    def march(wl, steps, sample_every, **o):
        h = rte.create_from_workload(wl, options=rte.default_options(**o))
        h.rte_step(2)
        h.rte_restart()
        torch.cuda.synchronize()
        dt, samples, n = 0.0, {}, 0
        while n < steps:
            k = min(sample_every, steps - n)
            t0 = time.perf_counter()
            h.rte_step(k)
            dt += time.perf_counter() - t0
            n += k
            samples[n] = h.rte_get_scalar_flux()
        st = h.rte_get_stats()
        h.destroy()
        return {"steps": steps, "ms_per_step": 1e3 * dt / steps,
                "updates_per_s": st["cell_direction_updates"] / dt,
                "iterations_per_step": st["total_iterations"] / steps,
                "sweeps_per_step": st["total_sweeps"] / steps,
                "si_sweep_ms": st["si_sweep_kernel_ms"] / max(1, st["si_sweep_launches"]),
                "f_sweep_ms": st["f_sweep_kernel_ms"] / max(1, st["f_sweep_launches"]),
                "phase_end": st["phase"]}, samples

    def compare(row, samples, ref):
        errs = [float(np.linalg.norm(samples[n] - ref[n]) / np.linalg.norm(ref[n])) for n in ref]
        row["rel_l2_vs_fp64_rom_gpu"] = {"final": errs[-1], "worst": max(errs),
                                         "sampled_steps": len(errs)}

    ln = inputs.lognormal()
    r64, s64 = march(ln, ln.steps, 25, rom=rte.RTE_ROM_AUTO)
    p64, _ = march(ln, ln.steps, ln.steps, rom=rte.RTE_ROM_OFF)
    r32, s32 = march(ln, ln.steps, 25, rom=rte.RTE_ROM_AUTO, precision=rte.RTE_FP32)
    compare(r32, s32, s64)
    for r in (r64, r32):
        r["speedup_vs_sidsa_fp64"] = p64["ms_per_step"] / r["ms_per_step"]
    out[f"lognormal_1024sq_128dirs_{ln.steps}steps"] = {"rom_fp64": r64, "rom_fp32": r32,
                                                         "sidsa_fp64": p64}
    disc = inputs.diffusive_disc()
    d64, t64 = march(disc, disc.steps, 30, rom=rte.RTE_ROM_AUTO, r_max=60)
    q64, _ = march(disc, disc.steps, disc.steps, rom=rte.RTE_ROM_OFF)
    d32, t32 = march(disc, disc.steps, 30, precision=rte.RTE_FP32, r_max=60)
    dbf, tbf = march(disc, disc.steps, 30, precision=rte.RTE_FP32_BF16F, r_max=60)
    compare(d32, t32, t64)
    compare(dbf, tbf, t64)
    for r in (d64, d32, dbf):
        r["speedup_vs_sidsa_fp64"] = q64["ms_per_step"] / r["ms_per_step"]
    out[f"diffusive_disc_2048sq_256dirs_{disc.steps}steps"] = {
        "rom_fp64": d64, "rom_fp32": d32, "rom_bf16_f": dbf, "sidsa_fp64": q64}
    # the paper's own discretisation: Q1 upwind DG (options.degree = 1) on the headline
    # checkerboard, ROM-accelerated and plain SI-DSA, full length
    cb = inputs.checkerboard()
    k64, s64 = march(cb, cb.steps, 25, rom=rte.RTE_ROM_AUTO, degree=1)
    k0, _ = march(cb, cb.steps, cb.steps, rom=rte.RTE_ROM_OFF, degree=1)
    k32, s32 = march(cb, cb.steps, 25, rom=rte.RTE_ROM_AUTO, degree=1, precision=rte.RTE_FP32)
    compare(k32, s32, s64)
    for r in (k64, k32):
        r["speedup_vs_sidsa_fp64"] = k0["ms_per_step"] / r["ms_per_step"]
    # roofline of the Q1 SI sweep: FP64 flops per cell-direction of its closed-form cell solve
    # (106, FMA = 2) and the weighted moment (8), against the nominal FP64 peak
    flops = Q1_FLOPS_PER_UPDATE * cb.ncell * 128
    for r in (k64, k0):   # FP64 arms (the FP32 arm's sweeps run on the FP32 pipe)
        r["si_sweep_roofline"] = {"bound": "fp64", "achieved": flops / (r["si_sweep_ms"] * 1e-3) / 1e12,
                                  "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                                  "frac": flops / (r["si_sweep_ms"] * 1e-3) / 1e12 / FP64_PEAK_TFLOPS}
    out[f"checkerboard_256sq_128dirs_q1_{cb.steps}steps"] = {"rom_fp64": k64, "rom_fp32": k32,
                                                            "sidsa_fp64": k0}
    wls = inputs.batched()
    arms = {}
    for graph in (0, 2):   # kernels launched one by one; SI iterations in CUDA graphs (while node)
        b = rte.rte_batch_create(wls, rte.default_options(precision=rte.RTE_FP32, graph=graph))
        try:
            b.rte_batch_step(2)
            b.rte_batch_restart()
            t0 = time.perf_counter()
            b.rte_batch_step(20)
            dt = time.perf_counter() - t0
        except rte.RteError as e:   # reported in the line instead of ending the run
            arms[graph] = {"error": str(e)}
            b.destroy()
            continue
        upd = sum(b.instance(i).rte_get_stats()["cell_direction_updates"] for i in range(len(b)))
        b.destroy()
        arms[graph] = {"ms_per_step": 1e3 * dt / 20, "updates_per_s": upd / dt}
    out["batched_64_instances_20steps_fp32_rom"] = dict(arms[0], graph=arms[2])
    return out


def batched_sharded(rte, inputs, torch, dist, rank, world, steps=20):
    """The 64 batched instances sharded over the ranks by greedy longest-processing-time on
    the per-step cost model (no collective in the data path): each rank creates and steps its
    own instances; the whole-job figures are the slowest rank's time and all ranks' updates."""
    from paper_2603_19647_gb300.partition import shard
    idx, mine = shard(inputs.batched(), rank, world)
    b = rte.rte_batch_create(mine, rte.default_options(precision=rte.RTE_FP32)) if mine else None
    if b:
        b.rte_batch_step(2)
        b.rte_batch_restart()
    torch.cuda.synchronize()
    dist.barrier()
    t0 = time.perf_counter()
    if b:
        b.rte_batch_step(steps)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    upd = sum(b.instance(i).rte_get_stats()["cell_direction_updates"] for i in range(len(b))) if b else 0
    if b:
        b.destroy()
    ms, upd_all = reduce_over_ranks(dist, 1e3 * dt, upd, "cuda")
    return {"ms_per_step": ms / steps, "updates_per_s": upd_all / (ms / 1e3),
            "instances_on_rank0": len(idx), "partition": "greedy LPT on N_x N_v (k + 2)"}


def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return
    from paper_2603_19647_gb300 import inputs
    wl = inputs.checkerboard(n=args.n)
    per_step_budget = 6.0
    for _ in range(args.warmup):
        oracle_sample(wl, 0.0, min_steps=1)
    vals = []
    t_all = time.perf_counter()
    for _ in range(args.steps):
        v, k, dt, cores, _o = oracle_sample(wl, per_step_budget)
        vals.append((v, k, dt))
    wall = time.perf_counter() - t_all
    value = sum(v for v, _, _ in vals) / len(vals)
    sample = (f"each step: the first {vals[0][1]} implicit steps of the {args.n}x{args.n} x 128-direction "
              f"checkerboard march (of {wl.steps}), FP64 oracle, SI-DSA + ROM")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"checkerboard {args.n}^2 CL(32,8)=128 dirs, c*dt=0.005, 200 steps",
                   "parallelism": "host cores (OpenMP over directions)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": vals and cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def run_ours(args):
    import numpy as np
    import torch
    rank, local_rank, world = dist_env()
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2603_19647_gb300 import inputs, rte

    wl = inputs.checkerboard(n=args.n)
    nsteps = wl.steps
    # a high-priority stream: the library's ROM-update side streams run at the lowest priority
    stream = torch.cuda.Stream(priority=-1)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")

    def make(rom, precision=rte.RTE_FP64):
        h = rte.create_from_workload(wl, options=rte.default_options(
            rom=rte.RTE_ROM_AUTO if rom else rte.RTE_ROM_OFF, precision=precision))
        h.rte_set_stream(stream.cuda_stream)
        return h

    def timed_marches(h, k):
        """k marches, each timed with CUDA events on the library's stream, L2 flushed between."""
        ms, st0 = [], h.rte_get_stats()
        agg = dict(updates=0, sweeps=0, launches=0, k1_ms=0.0, k1_n=0, k2_ms=0.0, k2_n=0, its=0)
        for _ in range(k):
            h.rte_restart()
            with torch.cuda.stream(stream):
                flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            h.rte_step(nsteps)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            st = h.rte_get_stats()
            agg["updates"] += st["cell_direction_updates"]
            agg["sweeps"] += st["total_sweeps"]
            agg["its"] += st["total_iterations"]
            agg["launches"] += st["kernel_launches"]
            agg["k1_ms"] += st["si_sweep_kernel_ms"]
            agg["k1_n"] += st["si_sweep_launches"]
            agg["k2_ms"] += st["f_sweep_kernel_ms"]
            agg["k2_n"] += st["f_sweep_launches"]
            agg["phase_end"] = st["phase"]
            agg["ig_rank"], agg["pc_rank"] = st["ig_rank"], st["pc_rank"]
        return ms, agg

    h_rom = make(True)
    h_plain = make(False)
    for _ in range(args.warmup):
        h_rom.rte_restart()
        h_rom.rte_step(nsteps)
        h_plain.rte_restart()
        h_plain.rte_step(nsteps)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    with Clocks(local_rank) as clk:
        ms_rom, agg_rom = timed_marches(h_rom, args.steps)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    wall_rom = time.perf_counter() - wall0
    ms_plain, agg_plain = timed_marches(h_plain, args.steps)
    # the reduced-precision arms of the method on the same workload and GPU (FP32 sweeps and
    # BF16-stored f with the FP64 residual), against the FP64 ROM march's final scalar flux
    rho64 = h_rom.rte_get_scalar_flux()
    reduced = {}
    for name, prec in (("rom_sidsa_fp32", rte.RTE_FP32), ("rom_sidsa_bf16f", rte.RTE_FP32_BF16F)):
        hr = make(True, prec)
        hr.rte_restart()
        hr.rte_step(nsteps)
        ms_r, _ = timed_marches(hr, args.steps)
        rho_r = hr.rte_get_scalar_flux()
        reduced[name] = {"ms": sum(ms_r) / args.steps / nsteps,
                         "rel_l2_vs_fp64": float(np.linalg.norm(rho_r - rho64) / np.linalg.norm(rho64))}
        hr.destroy()

    total_ms, updates_all = reduce_over_ranks(dist, sum(ms_rom), agg_rom["updates"], "cuda")
    value = updates_all / (total_ms / 1e3)

    # e2e: the user's call sequence with host buffers (pinned): create, set_initial, march,
    # read rho back, destroy.
    n = wl.ncell
    pin = {k: torch.from_numpy(np.ascontiguousarray(getattr(wl, k))).pin_memory()
           for k in ("sigma_t", "sigma_s", "source", "rho0")}
    out = torch.empty(n, dtype=torch.float64).pin_memory()
    e2e_t = []
    e2e_updates = 0
    for _ in range(args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h = rte.rte_create(rte.mesh_from(wl), rte.quadrature_from(wl.quadrature),
                           pin["sigma_t"].numpy(), pin["sigma_s"].numpy(), pin["source"].numpy(),
                           wl.c_dt, rte.default_options())
        h.rte_set_initial(pin["rho0"].numpy())
        h.rte_step(nsteps)
        status = rte.load().rte_get_scalar_flux(h.ptr, out.numpy().ctypes.data_as(rte._dp))
        h._check(status)
        e2e_updates += h.rte_get_stats()["cell_direction_updates"]
        h.destroy()
        torch.cuda.synchronize()
        e2e_t.append(time.perf_counter() - t0)
    e2e_value = e2e_updates / sum(e2e_t)
    if dist:
        t = torch.tensor([e2e_value], device="cuda", dtype=torch.float64)
        dist.all_reduce(t)
        e2e_value = float(t.item())

    sharded = None
    if world > 1 and not args.no_extras:
        sharded = batched_sharded(rte, inputs, torch, dist, rank, world)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    k1_avg_ms = agg_rom["k1_ms"] / max(1, agg_rom["k1_n"])
    units = wl.ncell * wl.nv
    achieved = FLOP_PER_UPDATE * units / (k1_avg_ms / 1e3) / 1e12
    traffic = profiled_traffic()
    cpu = None
    if not args.no_baseline and world == 1:
        v, k, dt, cores, _o = oracle_sample(wl, 15.0)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"first {k} implicit steps of the same {args.n}^2 march (of {nsteps}), "
                         f"{dt:.1f} s, FP64 oracle, ROM on"}
    per_step_rom = total_ms / args.steps / nsteps if world == 1 else sum(ms_rom) / args.steps / nsteps
    per_step_plain = sum(ms_plain) / args.steps / nsteps
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": sum(ms_rom) / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"checkerboard {args.n}x{args.n}, CL(32,8) hemisphere = 128 directions, "
                               f"c*dt=0.005, {nsteps} implicit steps per bench step, ROM-accelerated "
                               "SI-DSA at 1e-8 relative residual",
                   "parallelism": f"replicas x{world}", "l2": "flushed (256 MiB write) between steps"},
        "time_per_implicit_step_ms": {"rom_sidsa_fp64": per_step_rom, "sidsa_fp64": per_step_plain},
        "speedup_rom_vs_sidsa": per_step_plain / per_step_rom,
        "reduced_precision_rom": {k: {"ms_per_implicit_step": v["ms"],
                                      "speedup_vs_sidsa_fp64": per_step_plain / v["ms"],
                                      "final_rel_l2_vs_fp64_rom": v["rel_l2_vs_fp64"]}
                                  for k, v in reduced.items()},
        "sweeps_per_step": {"rom": agg_rom["sweeps"] / (args.steps * nsteps),
                            "sidsa": agg_plain["sweeps"] / (args.steps * nsteps)},
        "rom_ranks_end": {"ig": agg_rom["ig_rank"], "pc": agg_rom["pc_rank"]},
        "roofline": {"kernel": "SI sweep (FP64 strip-chain)", "bound": "alu",
                     "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved / FP64_PEAK_TFLOPS, "traffic": traffic,
                     "peak_note": "FP64 nominal: 152 SMs x 4 flop/clk x 2.07 GHz",
                     "avg_launch_ms": k1_avg_ms, "flop_per_launch": FLOP_PER_UPDATE * units},
        "gpu_launches": agg_rom["launches"],
        "e2e": {"value": e2e_value, "unit": UNIT,
                "h2d_bytes_per_step": 4 * n * 8, "d2h_bytes_per_step": n * 8},
        "clocks": clk.summary(),
        "wall_s_timed_region": wall_rom,
    }
    if cpu:
        line["cpu_baseline"] = cpu
    if not args.no_extras and world == 1:
        extras = {}
        try:
            extra_workloads(rte, inputs, torch, extras)
        except rte.RteError as e:   # the headline figures stand; the line says what failed
            extras["error"] = str(e)
        line["other_workloads"] = extras
    elif sharded is not None:
        line["other_workloads"] = {"batched_64_instances_20steps_fp32_rom_sharded": sharded}
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
