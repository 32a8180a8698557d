"""options.graph: each DSA-preconditioned SI iteration (the DSA solve of l, the sweep and the
residual of l + 1; Algorithm 1) runs as one CUDA graph captured from the handle's stream the
first time l is reached and replayed in later steps (graph = 1); with graph = 2 the remaining
DSA iterations run inside one graph whose while node the residual kernel's stopping test ends.

A replay launches the kernels of the one-by-one loop with the same arguments, so the march
must be the one-by-one march bit for bit: scalar flux, iteration counts, CG counts, ROM ranks,
phases, sweeps and kernel launches.  Through Phase 3 it is also held to the oracle at 1e-10,
as the one-by-one march is."""
import numpy as np
import pytest
import torch

from conftest import cell_modes
from gpu_util import make_pair
from paper_2603_19647_gb300 import inputs, rte
from test_gpu_march import WELL_CONDITIONED_PC, _march

pytestmark = pytest.mark.gpu


def _run(wl, steps, restart_at=None, stream=None, **opts):
    h, _ = make_pair(wl, rom=rte.RTE_ROM_AUTO, **opts)
    if stream is not None:
        h.rte_set_stream(stream.cuda_stream)
    h.rte_set_initial(rho0=cell_modes(wl.rho0, opts.get("degree", 0)))
    log = []
    for n in range(1, steps + 1):
        if restart_at == n:
            h.rte_restart()
        h.rte_step(1)
        st = h.rte_get_stats()
        log.append((st["last_iterations"], st["last_cg_iterations"], st["ig_rank"],
                    st["pc_rank"], st["phase"], st["total_sweeps"], st["kernel_launches"]))
    rho = h.rte_get_scalar_flux()
    h.destroy()
    return rho, log


def _same(wl, steps, graph, **opts):
    rho0, log0 = _run(wl, steps, graph=0, **opts)
    rho1, log1 = _run(wl, steps, graph=graph, **opts)
    assert log0 == log1
    assert np.array_equal(rho0, rho1)
    return log1


GRAPH = pytest.mark.parametrize("graph", [1, 2], ids=["per_iteration", "while_loop"])


@pytest.mark.parametrize("case", [
    dict(precision=rte.RTE_FP64),
    dict(precision=rte.RTE_FP32),
    dict(precision=rte.RTE_FP32_BF16F),
    dict(precision=rte.RTE_FP64, pc_levels=2),
    dict(precision=rte.RTE_FP64, lookahead=1),
    dict(precision=rte.RTE_FP64, sweep_kernel=2),
    dict(precision=rte.RTE_FP64, degree=1),
    dict(precision=rte.RTE_FP32, degree=1),
    dict(precision=rte.RTE_FP32, dsa_cluster=1, dsa_fp64=1),
], ids=["fp64", "fp32", "bf16f", "two_pc_levels", "lookahead", "tile_kernel", "q1_fp64",
        "q1_fp32", "dsa_cluster"])
@GRAPH
def test_graph_march_is_the_launch_by_launch_march(case, graph):
    log = _same(inputs.checkerboard(n=48), 80, graph, **case)
    assert max(t[4] for t in log) == 3   # the ROM-preconditioned iteration was reached too


@GRAPH
def test_graph_march_slab(graph):
    _same(inputs.slab_1d(steps=60), 60, graph)


@GRAPH
def test_graph_bdf2_and_restart(graph):
    """BDF2 changes the time step constant after its first (backward-Euler) step, and a
    restart changes it back: the captured iterations are dropped and captured again."""
    _same(inputs.checkerboard(n=48), 40, graph, restart_at=21, time_scheme=rte.RTE_BDF2)


@GRAPH
def test_graph_on_a_caller_stream(graph):
    wl = inputs.checkerboard(n=48)
    s = torch.cuda.Stream()
    rho0, log0 = _run(wl, 30, graph=0)
    rho1, log1 = _run(wl, 30, graph=graph, stream=s)
    assert log0 == log1
    assert np.array_equal(rho0, rho1)


@GRAPH
def test_graph_march_against_the_oracle_through_phase3(graph):
    orc = _march(inputs.checkerboard(n=48), 80, 5, rom_on=True, decisions_p3=True, graph=graph,
                 **WELL_CONDITIONED_PC)
    assert sum(s.phase == 3 for s in orc.log) >= 60


def test_graph_loop_stops_at_the_iteration_cap():
    """A cap of max_iter SI iterations ends the device-side loop too: every step stops at the
    cap (RTE_ENOCONV from rte_step, the iterate still usable), as the launch-by-launch loop
    does."""
    wl = inputs.checkerboard(n=48)
    out = []
    for graph in (0, 2):
        h, _ = make_pair(wl, rom=rte.RTE_ROM_OFF, max_iter=3, eps_sisa=1e-14, graph=graph)
        h.rte_set_initial(rho0=wl.rho0)
        with pytest.raises(rte.RteError) as err:
            h.rte_step(1)
        assert err.value.status == rte.RTE_ENOCONV
        st = h.rte_get_stats()
        out.append((h.rte_get_scalar_flux(), st["last_iterations"], st["last_cg_iterations"],
                    st["kernel_launches"]))
        h.destroy()
    assert out[0][1] == out[1][1] == 3
    assert out[0][2:] == out[1][2:]
    assert np.array_equal(out[0][0], out[1][0])
