"""Batched instances (rte_batch_*): independent problems of different grids, quadratures and
cross sections, stepped side by side on their own streams and host threads.  Each instance
must give what the same problem gives on its own: the single-instance path bit for bit in
the same tile configuration, the oracle's march to the usual bounds."""
import numpy as np
import pytest

from conftest import oracle_problem
from gpu_util import rel_l2
from oracle import stepper
from paper_2603_19647_gb300 import inputs, rte

pytestmark = pytest.mark.gpu


def _small_batch(count=6, steps=24, seed=4):
    return inputs.batched(count=count, seed=seed, n_range=(128, 512), steps=steps, scale=0.1)


def _alone_options(inst, precision):
    """Options that give a handle stepped alone the same sweep tiles and DSA solve as batch
    instance `inst` (every batch solves its DSA system in FP64 in one thread-block cluster;
    FP32 batches take a fixed tile; FP64 instances tune exactly as a handle alone does)."""
    if precision == rte.RTE_FP64:
        return rte.default_options(precision=precision, dsa_cluster=1)
    st = inst.rte_get_stats()
    return rte.default_options(precision=precision, sweep_kernel=st["sweep_si_kernel"],
                               sweep_lanes=st["sweep_lanes"], sweep_rows=st["sweep_si_rows"],
                               sweep_warps=st["sweep_si_warps"], dsa_fp64=1, dsa_cluster=1)


@pytest.mark.parametrize("precision", [rte.RTE_FP64, rte.RTE_FP32])
def test_batch_matches_single_instances(precision):
    wls = _small_batch()
    opts = rte.default_options(precision=precision)
    b = rte.rte_batch_create(wls, opts)
    b.rte_batch_step(12)
    b.rte_batch_step(12)
    for i, wl in enumerate(wls):
        h = rte.create_from_workload(wl, options=_alone_options(b.instance(i), precision))
        h.rte_step(24)
        a, s = b.instance(i).rte_get_scalar_flux(), h.rte_get_scalar_flux()
        st_b, st_h = b.instance(i).rte_get_stats(), h.rte_get_stats()
        assert st_b["total_iterations"] == st_h["total_iterations"], i
        assert rel_l2(a, s) < 1e-13, (i, rel_l2(a, s))
        h.destroy()
    b.destroy()


def test_batch_rom_off_against_oracle():
    wls = _small_batch(count=4, steps=15, seed=11)
    b = rte.rte_batch_create(wls, rte.default_options(rom=rte.RTE_ROM_OFF))
    b.rte_batch_step(15)
    for i, wl in enumerate(wls):
        orc = stepper.OracleRTE(oracle_problem(wl), rom=False)
        orc.set_initial(wl.rho0)
        orc.step(15)
        assert rel_l2(b.instance(i).rte_get_scalar_flux(), orc.rho) < 1e-10, i
    b.destroy()


def test_batch_fp32_rom_against_fp64_oracle():
    wls = _small_batch(count=3, steps=40, seed=23)
    b = rte.rte_batch_create(wls, rte.default_options(precision=rte.RTE_FP32))
    b.rte_batch_step(40)
    for i, wl in enumerate(wls):
        orc = stepper.OracleRTE(oracle_problem(wl), rom=True)
        orc.set_initial(wl.rho0)
        orc.step(40)
        assert rel_l2(b.instance(i).rte_get_scalar_flux(), orc.rho) < 1e-6, i
    b.destroy()


def test_batch_restart_and_status():
    wls = _small_batch(count=3, steps=10, seed=5)
    b = rte.rte_batch_create(wls)
    b.rte_batch_step(10)
    first = [b.instance(i).rte_get_scalar_flux() for i in range(3)]
    b.rte_batch_restart()
    b.rte_batch_step(10)
    for i in range(3):
        assert np.array_equal(first[i], b.instance(i).rte_get_scalar_flux())
        assert rte.load().rte_batch_status(b.ptr, i) == rte.RTE_OK
    assert rte.load().rte_batch_status(b.ptr, 3) == rte.RTE_EINVAL
    b.destroy()


def test_batch_full_size_sampled():
    """The 64-instance log-normal batch at full size (sides 128-512, 64 or 128 directions,
    FP32, ROM on), three steps: sampled instances bit for bit against the same problems
    stepped alone, and the smallest against the FP64 oracle's march."""
    wls = inputs.batched(steps=3)
    opts = rte.default_options(precision=rte.RTE_FP32)
    b = rte.rte_batch_create(wls, opts)
    b.rte_batch_step(3)
    sides = [wl.nx for wl in wls]
    small = int(np.argmin(sides))
    for i in sorted({0, len(wls) // 2, len(wls) - 1, small, int(np.argmax(sides))}):
        h = rte.create_from_workload(wls[i], options=_alone_options(b.instance(i), rte.RTE_FP32))
        h.rte_step(3)
        a, s = b.instance(i).rte_get_scalar_flux(), h.rte_get_scalar_flux()
        assert b.instance(i).rte_get_stats()["total_iterations"] == h.rte_get_stats()["total_iterations"], i
        assert rel_l2(a, s) < 1e-13, (i, rel_l2(a, s))
        h.destroy()
    orc = stepper.OracleRTE(oracle_problem(wls[small]), rom=True)
    orc.set_initial(wls[small].rho0)
    orc.step(3)
    assert rel_l2(b.instance(small).rte_get_scalar_flux(), orc.rho) < 1e-6
    b.destroy()


def test_batch_fp32_takes_the_concurrent_tile():
    """FP32 batches whose options leave the sweep to the library take the tile sequence with
    32 directions per lane group, 4-row tiles and 8 warps per CTA (fewer if shared memory is
    short); FP64 batches and explicit choices are left alone."""
    wls = _small_batch(count=2, steps=2)
    b = rte.rte_batch_create(wls, rte.default_options(precision=rte.RTE_FP32))
    for i in range(2):
        st = b.instance(i).rte_get_stats()
        assert (st["sweep_si_kernel"], st["sweep_lanes"], st["sweep_si_rows"]) == (2, 32, 4)
        assert st["sweep_tuned"] == 0
    b.destroy()
    b = rte.rte_batch_create(wls, rte.default_options(precision=rte.RTE_FP32, sweep_rows=8,
                                                      sweep_kernel=2))
    assert b.instance(0).rte_get_stats()["sweep_si_rows"] == 8
    b.destroy()
