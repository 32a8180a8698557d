"""Mixed-precision mode (RTE_FP32) against the FP64 oracle, through the C ABI.

In RTE_FP32 the sweeps run in FP32 on FP32 copies of sigma_t, G and the angular flux f, and
their moments are summed into FP64; the SI residual, the DSA solve and the ROMs stay FP64.
Each SI iteration sweeps only the increment rho^{l-1} - rho_ref and adds its image to the
FP64 accumulator y_ir = T Sigma_s rho_ref (iterative refinement), so the FP32 rounding enters
rho^n in proportion to the size of the increments, not of rho.  The paper is FP64 throughout;
the bounds below are the reduced-precision targets of the method's FP32 variant: a single
FP32 sweep within 2e-6 relative L2 of the FP64 operator, and a whole march within 1e-6
relative L2 of the FP64 oracle's march of the same algorithm."""
import numpy as np
import pytest

from gpu_util import make_pair, match_directions, max_rel, rel_l2
from oracle import stepper
from oracle import transport as tr
from paper_2603_19647_gb300 import inputs, rte

pytestmark = pytest.mark.gpu

SWEEP_TOL = 2e-6
MARCH_TOL = 1e-6
# element-wise: every output value within 2e-5 of the FP64 value (relative, floored at 1e-3 of
# the field's maximum): ten times the L2 bound, far below the O(1) error of a wrong value
ELEM_TOL = 2e-5
FP32 = dict(precision=rte.RTE_FP32)


def _close(got, ref):
    assert rel_l2(got, ref) < SWEEP_TOL
    assert max_rel(got, ref) < ELEM_TOL


def _hetero_2d(nx, ny, quad, seed):
    rng = np.random.default_rng(seed)
    wl = inputs.checkerboard(n=8, quad=quad)
    wl.nx, wl.ny = nx, ny
    n = nx * ny
    ss = rng.uniform(0, 50, n)
    wl.sigma_s, wl.sigma_t = ss, ss + rng.uniform(0.05, 2, n)
    wl.source = rng.uniform(0, 1, n)
    wl.rho0 = rng.uniform(0, 1, n)
    return wl, rng


@pytest.mark.parametrize("shape,quad", [((37, 29), (32, 8)), ((129, 70), (16, 8)),
                                        ((1, 1), (8, 4)), ((64, 3), (32, 16))])
def test_fp32_sweep_2d(shape, quad):
    wl, rng = _hetero_2d(*shape, quad, seed=shape[0] + quad[1])
    h, p = make_pair(wl, **FP32)
    for _ in range(2):
        rho = rng.uniform(0, 1, wl.ncell)
        _close(h.rte_op_sweep(rho), tr.apply_T_sigma_s(p, rho))
    h.destroy()


@pytest.mark.parametrize("lanes,rows,warps", [(32, 1, 1), (8, 1, 8), (16, 4, 3), (8, 8, 2), (4, 1, 8),
                                               (4, 4, 3)])
def test_fp32_tilings_fused_f(lanes, rows, warps):
    wl, rng = _hetero_2d(45, 53, (32, 8), seed=lanes * rows + warps)
    h, p = make_pair(wl, sweep_lanes=lanes, sweep_rows=rows, sweep_warps=warps, **FP32)
    rho = rng.uniform(0, 1, wl.ncell)
    _close(h.rte_op_sweep(rho), tr.apply_T_sigma_s(p, rho))
    perm, _, _ = match_directions(h, wl.quadrature)
    f0 = rng.uniform(0, 1, (p.nv, wl.ncell))
    h.rte_set_initial(f0=f0[perm])
    g = np.array([0.3, 0.6, 0.2, 0.9])
    h.rte_set_inflow(g)
    p.inflow = g
    bt = h.rte_op_fsweep(rho)
    f_ref, _ = tr.final_f(p, rho, f0)
    _close(h.rte_get_angular_flux(), f_ref[perm])
    _close(bt, tr.b_tilde(p, f_ref))
    h.destroy()


@pytest.mark.parametrize("lanes,th,warps", [(8, 4, 1), (8, 8, 2), (16, 4, 3), (32, 4, 8), (32, 8, 2),
                                             (8, 4, 8), (16, 8, 5), (8, 2, 3), (32, 2, 4),
                                             (16, 2, 8)])
@pytest.mark.parametrize("shape", [(45, 53), (8, 9), (3, 130)])
def test_fp32_tile_kernel(lanes, th, warps, shape):
    """The tile-sequence kernel (each lane solves whole TW x TH tiles): SI sweep, fused f sweep
    with inflow and b~, on ragged grids (partial tiles in both directions), every tile shape."""
    wl, rng = _hetero_2d(*shape, (32, 8), seed=lanes * th + warps + shape[0])
    h, p = make_pair(wl, sweep_kernel=2, sweep_lanes=lanes, sweep_rows=th, sweep_warps=warps,
                     **FP32)
    st = h.rte_get_stats()
    assert st["sweep_si_kernel"] == 2 and st["sweep_f_kernel"] == 2
    for _ in range(2):
        rho = rng.uniform(0, 1, wl.ncell)
        _close(h.rte_op_sweep(rho), tr.apply_T_sigma_s(p, rho))
    perm, _, _ = match_directions(h, wl.quadrature)
    f0 = rng.uniform(0, 1, (p.nv, wl.ncell))
    h.rte_set_initial(f0=f0[perm])
    g = np.array([0.3, 0.6, 0.2, 0.9])
    h.rte_set_inflow(g)
    p.inflow = g
    rho = rng.uniform(0, 1, wl.ncell)
    bt = h.rte_op_fsweep(rho)
    f_ref, _ = tr.final_f(p, rho, f0)
    _close(h.rte_get_angular_flux(), f_ref[perm])
    _close(bt, tr.b_tilde(p, f_ref))
    h.destroy()


def test_fp32_tile_kernel_march():
    wl = inputs.lognormal(n=64, steps=60)
    worst, st, orc = _march_fp32(wl, 60, 10, rom_on=True, sweep_kernel=2)
    assert st["sweep_si_kernel"] == 2


@pytest.mark.parametrize("n,nd", [(7, 4), (256, 16), (4097, 16)])
def test_fp32_sweep_1d(n, nd):
    rng = np.random.default_rng(n)
    wl = inputs.slab_1d(n=n, n_dirs=nd)
    ss = rng.uniform(0, 20, n)
    wl.sigma_s, wl.sigma_t = ss, ss + rng.uniform(0.01, 1, n)
    h, p = make_pair(wl, **FP32)
    rho = rng.uniform(0, 1, n)
    _close(h.rte_op_sweep(rho), tr.apply_T_sigma_s(p, rho))
    h.destroy()


def _march_fp32(wl, steps, check_every, rom_on, **opts):
    o = dict(rom=rte.RTE_ROM_AUTO if rom_on else rte.RTE_ROM_OFF, **FP32)
    o.update(opts)
    h, p = make_pair(wl, **o)
    orc = stepper.OracleRTE(p, rom=rom_on, **{k: v for k, v in opts.items()
                                              if k in stepper.DEFAULTS})
    orc.set_initial(wl.rho0)
    worst = 0.0
    for n in range(1, steps + 1):
        h.rte_step(1)
        orc.step(1)
        if n % check_every == 0 or n == steps:
            err = rel_l2(h.rte_get_scalar_flux(), orc.rho)
            worst = max(worst, err)
            assert err < MARCH_TOL, (n, err)
    st = h.rte_get_stats()
    h.destroy()
    return worst, st, orc


def test_fp32_slab_full_workload():
    """1D slab, 256 cells, S16, c dt = 0.01, 100 steps at 1e-8."""
    wl = inputs.slab_1d()
    _march_fp32(wl, wl.steps, 10, rom_on=False)


def test_fp32_lognormal_downscaled_rom():
    """The log-normal workload's statistics (std 2, correlation length 0.1, sigma_a 0.05,
    c dt = 0.002, 128 directions) on a 64^2 grid, ROM on."""
    wl = inputs.lognormal(n=64, steps=120)
    worst, st, orc = _march_fp32(wl, wl.steps, 10, rom_on=True)
    assert max(s.phase for s in orc.log) >= 2


def test_fp32_checkerboard_rom_with_inflow():
    wl = inputs.checkerboard(n=48)
    wl.inflow = np.array([0.5, 0.0, 0.25, 0.0])
    _march_fp32(wl, 80, 10, rom_on=True)


def test_fp32_restart_reproduces():
    """rte_restart puts the FP32 state (f, the refinement accumulator) back exactly."""
    wl = inputs.checkerboard(n=32)
    h, _ = make_pair(wl, **FP32)
    h.rte_set_initial(rho0=wl.rho0)
    h.rte_step(15)
    a = h.rte_get_scalar_flux()
    h.rte_restart()
    h.rte_step(15)
    b = h.rte_get_scalar_flux()
    h.destroy()
    assert np.array_equal(a, b)
