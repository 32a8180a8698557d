"""Command-line march of one synthetic workload through the C ABI, printing its statistics.

    python -m paper_2603_19647_gb300.march lognormal --precision fp32 --steps 80

Workloads are the seeded generators of ``paper_2603_19647_gb300.inputs`` (checkerboard,
lognormal, diffusive_disc, slab_1d); the options map onto ``rte_options``.  It creates the
handle (with the sweep-tile tuning), sets the workload's initial state, takes the steps and
prints one JSON line with the wall time per step and ``rte_get_stats``.  Useful for profiling
one march under ncu and for trying options from the shell.
"""
import argparse
import json
import time

from . import inputs, rte

PRECISIONS = {"fp64": rte.RTE_FP64, "fp32": rte.RTE_FP32, "bf16": rte.RTE_FP32_BF16F}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("workload", choices=sorted(inputs.BY_NAME))
    ap.add_argument("--steps", type=int, default=None, help="default: the workload's own")
    ap.add_argument("--precision", choices=sorted(PRECISIONS), default="fp64")
    ap.add_argument("--rom", choices=["on", "off"], default="on")
    ap.add_argument("--pc-levels", type=int, default=1)
    ap.add_argument("--sa", choices=["dsa", "dmd"], default="dsa")
    ap.add_argument("--scheme", choices=["be", "bdf2"], default="be")
    ap.add_argument("--r-max", type=int, default=40)
    ap.add_argument("--degree", type=int, choices=[0, 1], default=0,
                    help="DG degree: 0 (one value per cell) or 1 (bilinear, 2D FP64)")
    ap.add_argument("--lanes", type=int, default=0, help="sweep_lanes (0: the library's choice)")
    ap.add_argument("--rows", type=int, default=0, help="sweep_rows (0: the library's choice)")
    ap.add_argument("--graph", type=int, choices=[0, 1, 2], default=0,
                    help="1: each SI iteration as a captured CUDA graph; 2: also the remaining "
                         "DSA iterations in one graph with a while node")
    a = ap.parse_args(argv)
    wl = inputs.BY_NAME[a.workload]()
    steps = a.steps if a.steps is not None else wl.steps
    opts = rte.default_options(
        precision=PRECISIONS[a.precision],
        rom=rte.RTE_ROM_AUTO if a.rom == "on" else rte.RTE_ROM_OFF,
        pc_levels=a.pc_levels, r_max=a.r_max,
        sa_kind=rte.RTE_SA_DMD_ITER if a.sa == "dmd" else rte.RTE_SA_DSA,
        time_scheme=rte.RTE_BDF2 if a.scheme == "bdf2" else rte.RTE_BE,
        degree=a.degree, sweep_lanes=a.lanes, sweep_rows=a.rows, graph=a.graph)
    h = rte.create_from_workload(wl, options=opts)
    t0 = time.perf_counter()
    h.rte_step(steps)
    dt = time.perf_counter() - t0
    st = h.rte_get_stats()
    h.destroy()
    print(json.dumps({"workload": a.workload, "steps": steps, "ms_per_step": 1e3 * dt / max(1, steps),
                      "stats": st}))


if __name__ == "__main__":
    main()
