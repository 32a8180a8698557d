"""GPU parity of the Q1 upwind DG path (Sec. 2.1 Eq. (DG) with K = 1, options.degree = 1)
against the oracle's Q1 scheme, through the C ABI, in FP64 (and the FP32 mode at the end).

Bounds as for the Q0 path: relative L2 <= 1e-12 (and element-wise 1e-11 against the field's
scale) for single sweeps, 1e-10 where an iterative solve sits in between; whole marches with
equal iteration counts and ROM ranks."""
import numpy as np
import pytest

from conftest import cell_modes, oracle_problem
from gpu_util import make_pair, match_directions, max_rel, rel_l2
from oracle import dsa as ods
from oracle import stepper
from oracle import transport as tr
from paper_2603_19647_gb300 import inputs, rte

pytestmark = pytest.mark.gpu

Q1 = dict(degree=1)


def _hetero(nx, ny, quad, seed):
    rng = np.random.default_rng(seed)
    wl = inputs.checkerboard(n=8, quad=quad)
    wl.nx, wl.ny = nx, ny
    n = nx * ny
    ss = rng.uniform(0, 50, n)
    wl.sigma_s, wl.sigma_t = ss, ss + rng.uniform(0.05, 2, n)
    wl.source = rng.uniform(0, 1, n)
    wl.rho0 = rng.uniform(0, 1, n)
    wl.domain = (0.0, 1.3, 0.0, 0.7)
    return wl, rng


@pytest.mark.parametrize("quad", [(32, 8), (8, 4), (16, 8)])
@pytest.mark.parametrize("shape", [(37, 29), (1, 1), (5, 40), (40, 3), (70, 66)])
def test_q1_si_sweep(quad, shape):
    wl, rng = _hetero(*shape, quad, seed=shape[0] * 5 + quad[1])
    h, p = make_pair(wl, **Q1)
    for _ in range(2):   # twice: the control block resets itself between launches
        rho = rng.uniform(-1, 1, 4 * wl.ncell)
        got = h.rte_op_sweep(rho)
        ref = tr.apply_T_sigma_s(p, rho)
        assert rel_l2(got, ref) < 1e-12
        assert max_rel(got, ref) < 1e-11
    h.destroy()


@pytest.mark.parametrize("lanes,rows", [(2, 1), (2, 4), (4, 1), (4, 2), (8, 1), (8, 2), (8, 4),
                                        (16, 1), (16, 4), (32, 1), (32, 2), (32, 4)])
@pytest.mark.parametrize("mode", ["si", "f"])
def test_q1_sweep_tilings(lanes, rows, mode):
    """Every tile (directions per lane group, rows per lane group) gives the same SI sweep and
    fused f sweep on a ragged grid, with inflow on every side for the fused sweep."""
    wl, rng = _hetero(45, 53, (32, 8), seed=lanes + rows)
    h, p = make_pair(wl, sweep_lanes=lanes, sweep_rows=rows, **Q1)
    if mode == "si":
        rho = rng.uniform(-1, 1, 4 * wl.ncell)
        got, ref = h.rte_op_sweep(rho), tr.apply_T_sigma_s(p, rho)
        assert rel_l2(got, ref) < 1e-12 and max_rel(got, ref) < 1e-11
    else:
        perm, _, _ = match_directions(h, wl.quadrature)
        f0 = rng.uniform(0, 1, (p.nv, 4 * wl.ncell))
        h.rte_set_initial(f0=f0[perm])
        g = np.array([0.3, 0.6, 0.2, 0.9])
        h.rte_set_inflow(g)
        p.inflow = g
        rho = rng.uniform(0, 1, 4 * wl.ncell)
        bt = h.rte_op_fsweep(rho)
        f_ref, _ = tr.final_f(p, rho, f0)
        f_got = h.rte_get_angular_flux()
        assert rel_l2(f_got, f_ref[perm]) < 1e-12 and max_rel(f_got, f_ref[perm]) < 1e-11
        bt_ref = tr.b_tilde(p, f_ref)
        assert rel_l2(bt, bt_ref) < 1e-12 and max_rel(bt, bt_ref) < 1e-11
    st = h.rte_get_stats()
    assert st["sweep_si_kernel"] == 3 and st["sweep_lanes"] == lanes
    h.destroy()


def test_q1_initial_state_round_trip():
    wl, rng = _hetero(19, 23, (16, 8), seed=3)
    h, p = make_pair(wl, **Q1)
    f0 = rng.normal(size=(p.nv, 4 * wl.ncell))
    h.rte_set_initial(f0=f0)
    assert np.array_equal(h.rte_get_angular_flux(), f0)
    _, (mu, eta, w), _ = match_directions(h, wl.quadrature)
    assert np.allclose(h.rte_get_scalar_flux(), w @ f0, rtol=0, atol=1e-14)
    rho0 = rng.normal(size=4 * wl.ncell)
    h.rte_set_initial(rho0)
    assert np.array_equal(h.rte_get_angular_flux(), np.tile(rho0, (p.nv, 1)))
    h.destroy()


@pytest.mark.parametrize("shape", [(24, 20), (7, 1), (96, 80)])
def test_q1_dsa(shape):
    wl, rng = _hetero(*shape, (16, 8), seed=11)
    h, p = make_pair(wl, cg_rtol=1e-10, cg_max_iter=2000, **Q1)
    A = ods.dsa_matrix(p)
    for _ in range(2):
        res = rng.normal(size=4 * wl.ncell)
        got, its = h.rte_op_dsa(res)
        ref, its_ref = ods.dsa_correction(p, A, res, 1e-10, 2000)
        assert rel_l2(got, ref) < 1e-9
        assert abs(its - its_ref) <= 1, (its, its_ref)
    h.destroy()


def test_q1_dsa_large_grid():
    """The Jacobi-preconditioned CG on 260^2 cells (270 400 unknowns, two blocks per SM)."""
    wl, rng = _hetero(260, 260, (8, 4), seed=5)
    h, p = make_pair(wl, cg_rtol=1e-8, cg_max_iter=3000, **Q1)
    res = rng.normal(size=4 * wl.ncell)
    got, its = h.rte_op_dsa(res)
    ref, its_ref = ods.dsa_correction(p, ods.dsa_matrix(p), res, 1e-8, 3000)
    assert rel_l2(got, ref) < 1e-7 and abs(its - its_ref) <= 2
    h.destroy()


def _q1_workload(n=24, steps=40, seed=0):
    wl = inputs.checkerboard(n=n, steps=steps)
    return wl


def test_q1_march_plain_sidsa():
    from test_gpu_march import _march
    _march(_q1_workload(), 30, 5, rom_on=False, **Q1)


def test_q1_march_rom_through_phase3():
    """Algorithm 2 on the Q1 scheme: the same N0, N1, iteration counts and ROM ranks, and
    rho^n at 1e-10, through Phase 3 (preconditioner ROM truncated at 1e-3, where the reduced
    operator stays well conditioned)."""
    from test_gpu_march import _march
    orc = _march(_q1_workload(steps=60), 60, 5, rom_on=True, eps_pc=1e-3, decisions_p3=True, **Q1)
    assert max(s.phase for s in orc.log) == 3


def test_q1_march_rom_working_tolerance():
    from test_gpu_march import _march
    orc = _march(_q1_workload(steps=60), 60, 10, rom_on=True, exact=False, **Q1)
    assert max(s.phase for s in orc.log) >= 2


def test_q1_march_inflow_and_bdf2():
    from test_gpu_march import _march
    wl = _q1_workload(n=20, steps=30)
    _march(wl, 30, 5, rom_on=True, eps_pc=1e-3, decisions_p3=True,
           inflow_at={1: [0.5, 0.0, 0.25, 0.0], 12: [0.0, 0.3, 0.0, 0.1]},
           time_scheme=rte.RTE_BDF2, **Q1)


def test_q1_checkpoint_resume_is_bit_exact():
    wl = _q1_workload(n=20, steps=30)
    opts = dict(sweep_lanes=8, sweep_rows=2, **Q1)
    a = rte.create_from_workload(wl, options=rte.default_options(**opts))
    a.rte_step(12)
    blob = a.rte_save()
    a.rte_step(10)
    b = rte.create_from_workload(wl, options=rte.default_options(**opts))
    b.rte_load(blob)
    b.rte_step(10)
    assert np.array_equal(a.rte_get_scalar_flux(), b.rte_get_scalar_flux())
    assert np.array_equal(a.rte_get_angular_flux(), b.rte_get_angular_flux())
    # a Q0 handle of the same mesh refuses the blob
    c = rte.create_from_workload(wl, options=rte.default_options(sweep_lanes=8))
    with pytest.raises(rte.RteError):
        c.rte_load(blob)
    for x in (a, b, c):
        x.destroy()


@pytest.mark.slow
def test_q1_full_size_sweeps():
    """The 256^2 checkerboard with CL(32, 8) (128 directions) in the tile the library picks:
    the SI sweep and the fused sweep against the oracle, element by element."""
    wl = inputs.checkerboard()
    h, p = make_pair(wl, **Q1)
    rng = np.random.default_rng(9)
    rho = rng.uniform(0, 1, 4 * wl.ncell)
    got, ref = h.rte_op_sweep(rho), tr.apply_T_sigma_s(p, rho)
    assert rel_l2(got, ref) < 1e-12 and max_rel(got, ref) < 1e-11
    perm, _, _ = match_directions(h, wl.quadrature)
    h.rte_set_initial(cell_modes(wl.rho0, 1))
    bt = h.rte_op_fsweep(rho)
    f_ref, _ = tr.final_f(p, rho, np.tile(cell_modes(wl.rho0, 1), (p.nv, 1)))
    assert rel_l2(h.rte_get_angular_flux(), f_ref[perm]) < 1e-12
    assert rel_l2(bt, tr.b_tilde(p, f_ref)) < 1e-12
    h.destroy()


# ---- FP32 sweeps with the FP64 residual (options.precision = RTE_FP32) ---------------------

FP32 = dict(degree=1, precision=rte.RTE_FP32)


@pytest.mark.parametrize("lanes,rows", [(2, 1), (4, 1), (8, 1), (8, 4), (16, 2), (32, 1)])
def test_q1_fp32_sweeps(lanes, rows):
    """FP32 cell solves: the SI sweep and the fused sweep within 2e-6 (relative L2) of the FP64
    oracle, and element by element within 2e-5 relative for every value above 1 % of the field's
    largest (the linear modes of f run down to zero, where FP32's error relative to the field,
    about 1e-7, is what remains)."""
    wl, rng = _hetero(45, 53, (32, 8), seed=7 * lanes + rows)
    h, p = make_pair(wl, sweep_lanes=lanes, sweep_rows=rows, **FP32)
    rho = rng.uniform(0, 1, 4 * wl.ncell)
    got, ref = h.rte_op_sweep(rho), tr.apply_T_sigma_s(p, rho)
    assert rel_l2(got, ref) < 2e-6 and max_rel(got, ref) < 2e-5, (rel_l2(got, ref), max_rel(got, ref))
    perm, _, _ = match_directions(h, wl.quadrature)
    f0 = rng.uniform(0, 1, (p.nv, 4 * wl.ncell))
    h.rte_set_initial(f0=f0[perm])
    g = np.array([0.3, 0.6, 0.2, 0.9])
    h.rte_set_inflow(g)
    p.inflow = g
    bt = h.rte_op_fsweep(rho)
    f_ref, _ = tr.final_f(p, rho, f0)
    f_got = h.rte_get_angular_flux()
    assert rel_l2(f_got, f_ref[perm]) < 2e-6 and max_rel(f_got, f_ref[perm], floor=1e-2) < 2e-5
    bt_ref = tr.b_tilde(p, f_ref)
    assert rel_l2(bt, bt_ref) < 2e-6 and max_rel(bt, bt_ref, floor=1e-2) < 2e-5
    h.destroy()


@pytest.mark.parametrize("rom_on", [False, True])
def test_q1_fp32_march_within_1e6_of_fp64_oracle(rom_on):
    """The FP32 march (FP32 sweeps and f, FP64 residual, DSA and ROMs) stays within 1e-6 of the
    FP64 oracle's march at every step, through Phase 3 with the ROMs on."""
    wl = _q1_workload(n=32, steps=60)
    o = dict(rom=rte.RTE_ROM_AUTO if rom_on else rte.RTE_ROM_OFF, **FP32)
    h, p = make_pair(wl, **o)
    orc = stepper.OracleRTE(p, rom=rom_on)
    orc.set_initial(cell_modes(wl.rho0, 1))
    worst = 0.0
    for n in range(1, 61):
        h.rte_step(1)
        orc.step(1)
        worst = max(worst, rel_l2(h.rte_get_scalar_flux(), orc.rho))
    assert worst < 1e-6, worst
    if rom_on:
        assert h.rte_get_stats()["phase"] == 3
    h.destroy()


@pytest.mark.slow
def test_q1_full_size_march_against_oracle():
    """The 256^2 x 128 benchmark grid in the Q1 scheme with the ROMs on, against the oracle's
    march of the same algorithm for 24 steps: relative L2 <= 1e-10 with equal iteration counts,
    ROM ranks and phase changes at every step."""
    from test_gpu_march import _march
    wl = inputs.checkerboard(steps=24)
    _march(wl, 24, 1, rom_on=True, **Q1)


def test_q1_two_preconditioner_roms_strict():
    """Two preconditioner ROMs (iterations 1 and 2) on the Q1 scheme: the same decisions, ranks
    of both ROMs and 1e-10 while the second ROM is built from steps that applied the first."""
    from test_gpu_march import _march
    orc = _march(_q1_workload(n=24, steps=100), 100, 5, rom_on=True, decisions_p3=True,
                 pc_levels=2, eps_pc=1e-3, **Q1)
    assert orc.pcs[1].rank > 0


def test_q1_dmd_across_iterations_strict():
    """The DMD-across-iterations SA steps in place of DSA on the Q1 scheme, with the ROMs: the
    same decisions, the same number of jumps and 1e-10 throughout, and no CG at all."""
    from test_gpu_march import _march
    orc = _march(_q1_workload(n=24, steps=50), 50, 5, rom_on=True, decisions_p3=True,
                 sa_kind=rte.RTE_SA_DMD_ITER, eps_pc=1e-3, **Q1)
    assert sum(s.cg_iterations for s in orc.log) == 0


@pytest.mark.parametrize("precision", [rte.RTE_FP64, rte.RTE_FP32])
def test_q1_batch_matches_single_instances(precision):
    """Batched Q1 instances of different sizes step exactly as the same problems alone."""
    wls = [inputs.checkerboard(n=n, steps=20) for n in (24, 40, 16)]
    b = rte.rte_batch_create(wls, rte.default_options(degree=1, precision=precision))
    b.rte_batch_step(15)
    for i, wl in enumerate(wls):
        st = b.instance(i).rte_get_stats()
        o = rte.default_options(degree=1, precision=precision, sweep_lanes=st["sweep_lanes"],
                                sweep_rows=st["sweep_si_rows"], dsa_fp64=1)
        h = rte.create_from_workload(wl, options=o)
        h.rte_step(15)
        assert h.rte_get_stats()["total_iterations"] == st["total_iterations"], i
        assert rel_l2(b.instance(i).rte_get_scalar_flux(), h.rte_get_scalar_flux()) < 1e-13, i
        h.destroy()
    b.destroy()
