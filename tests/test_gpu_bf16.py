"""BF16 storage of the angular flux (RTE_FP32_BF16F) against the FP64 oracle.

f is stored as a per-cell FP32 reference (the scalar flux the step converged to) plus a BF16
remainder per cell-direction, written with unbiased stochastic rounding; sweeps, moments and
accumulation are FP32 as in RTE_FP32, and the SI residual, DSA and ROMs FP64.  A stored
remainder is within one BF16 ulp (2^-7 relative) of the exact one; the target for a march is
1e-5 relative L2 in the scalar flux against the FP64 oracle, measured here on the
diffusive-disc workload at a reduced grid."""
import numpy as np
import pytest

from conftest import oracle_problem
from gpu_util import make_pair, match_directions, rel_l2
from oracle import stepper
from oracle import transport as tr
from paper_2603_19647_gb300 import inputs, rte

pytestmark = pytest.mark.gpu

BF16 = dict(precision=rte.RTE_FP32_BF16F)


def _disc(n, quad=(16, 8), steps=40):
    return inputs.diffusive_disc(n=n, quad=quad, steps=steps)


def test_bf16_initial_state_roundtrip():
    wl = _disc(24)
    h, p = make_pair(wl, **BF16)
    perm, _, w = match_directions(h, wl.quadrature)
    rng = np.random.default_rng(3)
    f0 = rng.uniform(0.5, 1.5, (p.nv, wl.ncell))
    h.rte_set_initial(f0=f0[perm])
    ref = np.float32(p.w @ f0).astype(np.float64)          # the FP32 reference per cell
    got = h.rte_get_angular_flux()
    assert np.all(np.abs(got - f0[perm]) <= 2.0 ** -8 * np.abs(f0[perm] - ref) + 1e-6), "RN bound"
    h.destroy()


def test_bf16_fused_sweep_within_one_ulp_of_the_remainder():
    wl = _disc(40)
    h, p = make_pair(wl, **BF16)
    perm, _, _ = match_directions(h, wl.quadrature)
    rng = np.random.default_rng(1)
    f0 = rng.uniform(0.5, 1.5, (p.nv, wl.ncell))
    h.rte_set_initial(f0=f0[perm])
    f0_stored = h.rte_get_angular_flux()[np.argsort(perm)]   # what the sweep reads
    rho = rng.uniform(0.5, 1.5, wl.ncell)
    bt = h.rte_op_fsweep(rho)
    f_exact, _ = tr.final_f(p, rho, f0_stored)
    ref = np.float32(rho).astype(np.float64)
    got = h.rte_get_angular_flux()[np.argsort(perm)]
    tol = 2.0 ** -7 * np.abs(f_exact - ref) + 2e-6 * np.abs(f_exact)
    assert np.all(np.abs(got - f_exact) <= tol)
    # b~ is swept from the stored f^n, so it matches the exact b~ of that stored f
    assert rel_l2(bt, tr.b_tilde(p, got)) < 2e-6
    h.destroy()


def test_bf16_disc_march_against_fp64_oracle():
    """Diffusive disc (sigma_s = 1000 inside r < 0.3, 1 outside, sigma_a = 0.01, c dt = 0.001)
    on a 64^2 grid with the workload's 256 directions, ROM on (rank <= 60), 120 steps."""
    wl = _disc(64, quad=(32, 16), steps=120)
    h, p = make_pair(wl, r_max=60, **BF16)
    orc = stepper.OracleRTE(p, rom=True, r_max=60)
    orc.set_initial(wl.rho0)
    worst = 0.0
    for n in range(1, 121):
        h.rte_step(1)
        orc.step(1)
        if n % 20 == 0:
            worst = max(worst, rel_l2(h.rte_get_scalar_flux(), orc.rho))
    assert worst < 1e-5, worst
    h.destroy()


def test_bf16_restart_reproduces():
    wl = _disc(32)
    h, _ = make_pair(wl, **BF16)
    h.rte_step(10)
    a = h.rte_get_scalar_flux()
    h.rte_restart()
    h.rte_step(10)
    assert np.array_equal(a, h.rte_get_scalar_flux())
    h.destroy()


@pytest.mark.parametrize("kernel", [1, 2])
def test_bf16_both_kernels_fused_sweep(kernel):
    wl = _disc(37)
    h, p = make_pair(wl, sweep_kernel=kernel, **BF16)
    perm, _, _ = match_directions(h, wl.quadrature)
    rng = np.random.default_rng(kernel)
    f0 = rng.uniform(0.5, 1.5, (p.nv, wl.ncell))
    h.rte_set_initial(f0=f0[perm])
    f0_stored = h.rte_get_angular_flux()[np.argsort(perm)]
    rho = rng.uniform(0.5, 1.5, wl.ncell)
    bt = h.rte_op_fsweep(rho)
    f_exact, _ = tr.final_f(p, rho, f0_stored)
    ref = np.float32(rho).astype(np.float64)
    got = h.rte_get_angular_flux()[np.argsort(perm)]
    assert np.all(np.abs(got - f_exact) <= 2.0 ** -7 * np.abs(f_exact - ref) + 2e-6 * np.abs(f_exact))
    assert rel_l2(bt, tr.b_tilde(p, got)) < 2e-6
    h.destroy()
