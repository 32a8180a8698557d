"""GPU time marches (Algorithms 1 and 2) against the oracle's march of the same algorithm,
through the C ABI, in FP64.

Parity of rho^n at a relative L2 error <= 1e-10, with equal iteration counts and ROM ranks,
holds whenever the march does not amplify rounding: ROM-off marches, ROM-on marches through
Phases 1 and 2, tight tolerances (eps_SISA = 1e-12), and Phase 3 at the working tolerance
eps_SISA = 1e-8 when the preconditioner ROM is truncated at eps_PC = 1e-3.

At the working tolerance with the default eps_PC = 1e-6 the preconditioner ROM keeps singular
values down to 1e-6 of their sum, and its reduced operator reaches condition numbers of 1e5
and more (measured on the oracle for the 48^2 checkerboard): the method itself then amplifies
a rounding difference by that much per step.  The oracle against itself, with its source
perturbed by 2e-16 relative, drifts to a few 1e-9 in Phase 3 (and flips iteration counts); a
1e-10 bound is not a property of the method there.  Those marches are held to the method's
own sensitivity instead: the oracle is run three more times with such perturbations, and the
library's distance to the unperturbed oracle must stay within 50 times the largest distance
seen so far among the oracle runs (never below 1e-10).  A real defect (a wrong pairing, a
wrong gate, a wrong kernel) moves the march by orders of magnitude more."""
import numpy as np
import pytest

from conftest import cell_modes, oracle_problem
from gpu_util import make_pair, rel_l2
from oracle import stepper
from paper_2603_19647_gb300 import inputs, rte

pytestmark = pytest.mark.gpu

TOL = 1e-10


ENVELOPE_FACTOR = 50.0
PERTURBATION = 2e-16
# A phase change one step apart is accepted only where the oracle's own decision value stood
# within this relative distance of its threshold.  The construction phases end on the ratio
# s_last / sum s of Eq. (ig_stop) / Eq. (pc_stop).  The PC-ROM's snapshots are differences of
# SI iterates converged to eps_SISA, so at eps_PC = 1e-6 its smallest singular values carry
# the solves' tolerance relative to themselves: measured on the 48^2 checkerboard at
# eps_SISA = 1e-12, library and oracle singular values agree to 2e-7 .. 1.5e-6 of the largest,
# and the ratio at the Phase-2 end differs by 5 % (0.985e-6 against 1.040e-6 with one sweep
# tile, 1.090e-6 against 1.040e-6 with another).  A decision 10 % or more from its threshold
# must agree.
DECISION_MARGIN = 0.1


class _LoggedOracle(stepper.OracleRTE):
    """The oracle's march with every decision recorded: (step, kind, value, threshold)."""

    def __init__(self, *a, **k):
        super().__init__(*a, **k)
        self.decisions = []

    def decide(self, kind, own, value, threshold):
        self.decisions.append((self.n + 1, kind, float(value), float(threshold)))
        return own

    def margin(self, kind, first, last):
        """Smallest relative distance to the threshold of the decisions `kind` taken at the ends
        of steps first .. last (0-based step indices; step k's decision sets step k+1's phase)."""
        m = [abs(v - t) / abs(t) for n, k, v, t in self.decisions
             if k == kind and first <= n <= last + 1 and t != 0]
        return min(m) if m else float("inf")


def _perturbed_oracles(wl, rom_on, oopts, k=3, degree=0):
    """k oracle marches whose source (or, without one, sigma_t) is perturbed by a relative
    2e-16 (seeded normal numbers): rounding-sized changes of the input."""
    out = []
    for seed in range(1, k + 1):
        p = oracle_problem(wl, degree=degree)
        rng = np.random.default_rng(seed)
        if np.any(p.source):
            p.source = p.source * (1 + PERTURBATION * rng.standard_normal(p.ndof))
        else:
            p.sigma_t = p.sigma_t * (1 + PERTURBATION * rng.standard_normal(p.ncell))
        o = stepper.OracleRTE(p, rom=rom_on, **oopts)
        o.set_initial(cell_modes(wl.rho0, degree))
        out.append(o)
    return out


def _march(wl, steps, check_every, rom_on, exact=True, inflow_at=None, decisions_p3=False,
           **opts):
    """exact=False: exact parity until the first Phase 3 step, then within the envelope of the
    oracle's own rounding sensitivity (module docstring).  decisions_p3: iteration counts and
    ROM ranks must also agree in Phase 3.
    inflow_at: {step: g} sets the isotropic inflow of both sides before that step."""
    o = dict(rom=rte.RTE_ROM_AUTO if rom_on else rte.RTE_ROM_OFF)
    o.update(opts)
    h, p = make_pair(wl, **o)
    oopts = {k: v for k, v in opts.items() if k in stepper.DEFAULTS}
    if "residual_norm" in oopts:   # the library's enum -> the oracle's names
        oopts["residual_norm"] = "abs" if oopts["residual_norm"] == rte.RTE_ABS_INF else "rel"
    if "up_rel" in oopts:
        oopts["up_rel"] = bool(oopts["up_rel"])
    if "sa_kind" in opts:
        oopts["sa"] = "mh" if opts["sa_kind"] == rte.RTE_SA_DMD_ITER else "dsa"
    if "time_scheme" in opts:
        oopts["scheme"] = "bdf2" if opts["time_scheme"] == rte.RTE_BDF2 else "be"
    deg = opts.get("degree", 0)
    orc = _LoggedOracle(p, rom=rom_on, **oopts)
    orc.set_initial(cell_modes(wl.rho0, deg))
    pert = [] if exact else _perturbed_oracles(wl, rom_on, oopts, degree=deg)
    envelope = 0.0
    in_p3 = False
    phases_lib, phases_orc = [], []
    for n in range(1, steps + 1):
        if inflow_at and n in inflow_at:
            h.rte_set_inflow(inflow_at[n])
            for o in [orc] + pert:
                o.set_inflow(inflow_at[n])
        h.rte_step(1)
        orc.step(1)
        for o in pert:
            o.step(1)
            envelope = max(envelope, rel_l2(o.rho, orc.rho))
        st = h.rte_get_stats()
        lg = orc.log[-1]
        phases_lib.append(st["phase"])
        phases_orc.append(lg.phase)
        in_p3 = in_p3 or lg.phase == 3 or st["phase"] == 3
        same_decisions = decisions_p3 or not in_p3
        strict = exact or not in_p3
        if same_decisions:
            assert st["last_iterations"] == lg.iterations, n
            if "sa_kind" in opts:
                assert st["total_mh_jumps"] == sum(s.mh_jumps for s in orc.log), n
        if n % check_every == 0 or n == steps or not in_p3:
            err = rel_l2(h.rte_get_scalar_flux(), orc.rho)
            bound = TOL if strict else max(TOL, ENVELOPE_FACTOR * envelope)
            assert err < bound, (n, err, envelope)
            if rom_on and same_decisions:
                assert st["ig_rank"] == orc.ig.rank and st["pc_rank"] == orc.pc.rank, n
                assert st["pc_level_rank"][:len(orc.pcs)] == [v.rank for v in orc.pcs], n
    if rom_on:   # the same N0 and N1, up to a decision within rounding of its threshold
        for ph in (2, 3):
            a = phases_lib.index(ph) if ph in phases_lib else -1
            b = phases_orc.index(ph) if ph in phases_orc else -1
            if a != b:
                kind = "ig_built" if ph == 2 else "pc_built"
                assert min(a, b) >= 0 and abs(a - b) == 1, (ph, a, b)
                margin = orc.margin(kind, min(a, b), max(a, b))
                assert margin < DECISION_MARGIN, (ph, a, b, margin)
    h.destroy()
    return orc


def test_slab_full_workload_plain_sidsa():
    """1D slab, 256 cells, S16, c dt = 0.01, 100 steps, plain SI-DSA in FP64 at 1e-8."""
    wl = inputs.slab_1d()
    _march(wl, wl.steps, 10, rom_on=False)


TIGHT = dict(eps_sisa=1e-12, eps_ig=1e-9, eps_pc=1e-6, eps_up=1e-9, cg_rtol=1e-8)


def test_slab_rom():
    wl = inputs.slab_1d(steps=60)
    _march(wl, 60, 10, rom_on=True, exact=False)


def test_slab_rom_tight():
    wl = inputs.slab_1d(steps=60)
    _march(wl, 60, 10, rom_on=True, **TIGHT)


def test_checkerboard_downscaled_plain():
    _march(inputs.checkerboard(n=48), 80, 10, rom_on=False)


def test_checkerboard_downscaled_rom():
    orc = _march(inputs.checkerboard(n=48), 80, 10, rom_on=True, exact=False)
    assert max(s.phase for s in orc.log) == 3


def test_checkerboard_downscaled_rom_tight():
    orc = _march(inputs.checkerboard(n=48), 80, 10, rom_on=True, **TIGHT)
    assert max(s.phase for s in orc.log) >= 2


def test_checkerboard_tile_kernel_rom_tight():
    """The same march with the tile-sequence sweep kernel for both sweep modes."""
    orc = _march(inputs.checkerboard(n=48), 80, 10, rom_on=True, sweep_kernel=2, **TIGHT)
    assert max(s.phase for s in orc.log) >= 2


# Phase 3 at the working tolerance with a well-conditioned preconditioner ROM: the oracle's
# decisions stand at least 6e-4 (relative) from their thresholds on these marches, so both
# sides take the same ones and stay within 1e-10 for the whole march.
WELL_CONDITIONED_PC = dict(eps_pc=1e-3)


def test_checkerboard_phase3_working_tolerance_strict():
    orc = _march(inputs.checkerboard(n=48), 80, 5, rom_on=True, decisions_p3=True,
                 **WELL_CONDITIONED_PC)
    assert sum(s.phase == 3 for s in orc.log) >= 60


@pytest.mark.parametrize("precision", [rte.RTE_FP64, rte.RTE_FP32])
def test_checkerboard_dsa_in_one_cluster_strict(precision):
    """options.dsa_cluster (the DSA solve batched instances take): the FP64 march through
    Phase 3 with the same decisions and 1e-10 throughout; the FP32 march (FP32 sweeps, FP64
    residual and DSA) within 1e-6."""
    if precision == rte.RTE_FP64:
        orc = _march(inputs.checkerboard(n=48), 80, 5, rom_on=True, decisions_p3=True,
                     dsa_cluster=1, **WELL_CONDITIONED_PC)
        assert sum(s.phase == 3 for s in orc.log) >= 60
        return
    wl = inputs.checkerboard(n=48)
    h, p = make_pair(wl, precision=precision, dsa_cluster=1, dsa_fp64=1, **WELL_CONDITIONED_PC)
    orc = stepper.OracleRTE(p, rom=True, **WELL_CONDITIONED_PC)
    orc.set_initial(wl.rho0)
    h.rte_step(80)
    orc.step(80)
    assert rel_l2(h.rte_get_scalar_flux(), orc.rho) < 1e-6
    h.destroy()


def test_slab_phase3_working_tolerance_strict():
    orc = _march(inputs.slab_1d(steps=60), 60, 5, rom_on=True, decisions_p3=True,
                 **WELL_CONDITIONED_PC)
    assert sum(s.phase == 3 for s in orc.log) >= 40


@pytest.mark.parametrize("eps_sisa", [1e-8, 1e-10])
def test_two_preconditioner_roms_strict(eps_sisa):
    """A preconditioner ROM for the first and for the second SI iteration (the second built
    only from steps that applied the first): the same decisions, ranks of both ROMs and 1e-10
    for the whole march, with updates of the second ROM in Phase 3 (the oracle's decisions
    stand at least 7e-4 relative from their thresholds)."""
    orc = _march(inputs.checkerboard(n=48), 80, 5, rom_on=True, decisions_p3=True,
                 pc_levels=2, eps_sisa=eps_sisa, **WELL_CONDITIONED_PC)
    assert sum(s.phase == 3 for s in orc.log) >= 60
    assert sum(s.pc_ups[1] for s in orc.log if s.phase == 3) >= 5


@pytest.mark.parametrize("case", ["rom_working_tolerance", "rom_off", "slab", "two_levels_fp32"])
def test_dmd_across_iterations_in_place_of_dsa(case):
    """The DMD-across-iterations SA steps (options.sa_kind) against the oracle's, in the
    ROM-accelerated march (Phases 1-3, the hybrid of the paper's Sec. 4) and in plain SI with
    them alone: the same decisions, the same number of jumps and 1e-10 throughout (FP32 sweeps:
    within 1e-6 of the FP64 oracle)."""
    wl = inputs.slab_1d(steps=60) if case == "slab" else inputs.checkerboard(n=48)
    steps = 60 if case == "slab" else 80
    extra = dict(pc_levels=2, precision=rte.RTE_FP32) if case == "two_levels_fp32" else {}
    rom_on = case != "rom_off"
    if case == "two_levels_fp32":
        h, p = make_pair(wl, rom=rte.RTE_ROM_AUTO, sa_kind=rte.RTE_SA_DMD_ITER, eps_pc=1e-3,
                         **extra)
        orc = stepper.OracleRTE(p, sa="mh", eps_pc=1e-3, pc_levels=2)
        orc.set_initial(wl.rho0)
        for n in range(1, steps + 1):
            h.rte_step(1)
            orc.step(1)
            if n % 10 == 0:
                assert rel_l2(h.rte_get_scalar_flux(), orc.rho) < 1e-6, n
        h.destroy()
        return
    orc = _march(wl, steps, 5, rom_on=rom_on, decisions_p3=True, sa_kind=rte.RTE_SA_DMD_ITER,
                 **WELL_CONDITIONED_PC)
    assert sum(s.cg_iterations for s in orc.log) == 0
    if rom_on:
        assert sum(s.phase == 3 for s in orc.log) >= 40


def test_two_preconditioner_roms_exact_on_an_invariant_span():
    """The oracle pin of the sequentially built second preconditioner ROM, run by the library:
    a five-mode slab march (f0 from eigenvectors of the step's dense system matrix) with every
    ROM capped at rank 2, where the second ROM is exact and every Phase 3 step ends at l = 3."""
    from oracle import dense
    from gpu_util import match_directions
    wl = inputs.slab_1d(n=16, n_dirs=8, steps=16, c_dt=0.05)
    rng = np.random.default_rng(5)
    wl.sigma_s = 0.9 * (0.5 + rng.uniform(0, 1, 16))
    wl.sigma_t = wl.sigma_s + rng.uniform(0.2, 1.0, 16)
    p = oracle_problem(wl)
    lam, V = np.linalg.eig(dense.assemble(p))
    order = [i for i in np.argsort(np.abs(lam)) if abs(lam[i].imag) < 1e-12]
    f0 = sum(c * V[:, i].real / np.abs(V[:, i].real).max()
             for c, i in zip([1.0, 0.7, 0.5, 0.4, 0.3], order)).reshape(p.nv, p.ncell)
    o = dict(eps_sisa=1e-12, cg_rtol=1e-12, eps_ig=1e-6, eps_pc=1e-6, eps_up=0.5, r_max=2,
             pc_levels=2)
    h, _ = make_pair(wl, rom=rte.RTE_ROM_AUTO, **o)
    perm, _, _ = match_directions(h, wl.quadrature)
    h.rte_set_initial(f0=f0[perm])
    orc = stepper.OracleRTE(p, **o)
    orc.set_initial(np.zeros(p.ncell), f0=f0)
    for n in range(1, 17):
        h.rte_step(1)
        orc.step(1)
        st, lg = h.rte_get_stats(), orc.log[-1]
        assert st["phase"] == lg.phase and st["last_iterations"] == lg.iterations, n
        assert st["pc_level_rank"][:2] == list(lg.pc_ranks), n
        assert rel_l2(h.rte_get_scalar_flux(), orc.rho) < TOL, n
        if lg.phase == 3:
            assert st["last_iterations"] == 3, n
    h.destroy()
    assert sum(s.phase == 3 for s in orc.log) >= 8


@pytest.mark.parametrize("precision,levels", [(rte.RTE_FP64, 1), (rte.RTE_FP32, 1),
                                              (rte.RTE_FP64, 2)])
def test_lookahead_gives_the_same_march(precision, levels):
    """options.lookahead queues SI iteration l+1 before the host reads the stopping test of l;
    the work queued past convergence skips itself on the device, so the march, its iteration
    counts and its ROM ranks are those of the waiting loop, bit for bit."""
    wl = inputs.checkerboard(n=48)
    out = []
    for la in (0, 1):
        h, _ = make_pair(wl, rom=rte.RTE_ROM_AUTO, precision=precision, lookahead=la,
                         pc_levels=levels)
        h.rte_set_initial(rho0=wl.rho0)
        its = []
        for _ in range(80):
            h.rte_step(1)
            st = h.rte_get_stats()
            its.append((st["last_iterations"], st["last_cg_iterations"], st["ig_rank"],
                        st["pc_rank"], st["phase"]))
        out.append((h.rte_get_scalar_flux(), its, h.rte_get_stats()["total_sweeps"]))
        h.destroy()
    (rho0, its0, sw0), (rho1, its1, sw1) = out
    assert its0 == its1 and sw0 == sw1
    assert max(t[4] for t in its0) == 3
    assert np.array_equal(rho0, rho1)


def test_paper_absolute_rules():
    """The paper's own rules: the absolute stopping test ||rho^{l-1/2} - rho^{l-1}||_inf < eps
    (RTE_ABS_INF) and the absolute ROM-update threshold (up_rel = 0), against the oracle's
    march under the same rules."""
    orc = _march(inputs.checkerboard(n=48), 80, 10, rom_on=True, residual_norm=rte.RTE_ABS_INF,
                 up_rel=0, **TIGHT)
    assert max(s.phase for s in orc.log) >= 2


def test_checkerboard_ragged_small_rule():
    wl = inputs.checkerboard(n=8, quad=(8, 4))
    wl.nx, wl.ny = 27, 19
    n = wl.ncell
    rng = np.random.default_rng(2)
    ss = np.where(rng.random(n) < 0.5, 100.0, 0.01)
    wl.sigma_s, wl.sigma_t, wl.source = ss, ss + 0.1, rng.uniform(0, 1, n)
    wl.rho0 = np.zeros(n)
    wl.inflow = np.array([0.5, 0.0, 0.25, 0.0])
    _march(wl, 40, 5, rom_on=True, **TIGHT)
    _march(wl, 40, 5, rom_on=True, exact=False)


def test_degenerate_zero_state_then_inflow():
    """Nothing to transport for five steps: every iterate, snapshot and stopping test is
    exactly zero (the relative test accepts 0 <= eps * 0 at l = 1; a zero snapshot does not
    grow the IG-ROM, whose stop ratio is then 0, so Phase 2 starts with a rank-0 ROM that
    gives the initial guess 0 = rho^{n-1}); then an inflow switches on and the march follows
    the oracle's through all three phases."""
    wl = inputs.checkerboard(n=16, quad=(8, 4))
    n = wl.ncell
    wl.source, wl.rho0, wl.inflow = np.zeros(n), np.zeros(n), np.zeros(4)
    orc = _march(wl, 40, 5, rom_on=True, inflow_at={6: [0.5, 0.0, 0.25, 0.0]}, **TIGHT)
    assert all(s.iterations == 1 and s.residual == 0.0 for s in orc.log[:5])
    assert max(s.phase for s in orc.log) == 3


def test_degenerate_pure_absorber():
    """sigma_s = 0: the DSA right side sigma_s (rho^{l-1/2} - rho^{l-1}) vanishes, so CG takes
    no iteration and every step converges at l = 2; the preconditioner snapshot
    rho^n - rho^{n,1/2} is exactly zero, so the PC-ROM stays at rank 0 (Phase 3 with a zero
    correction, the same iterate as the zero DSA correction)."""
    wl = inputs.checkerboard(n=16, quad=(8, 4))
    n = wl.ncell
    wl.sigma_s = np.zeros(n)
    wl.sigma_t = np.where(np.arange(n) % 3 == 0, 5.0, 0.5)
    wl.inflow = np.array([0.3, 0.0, 0.6, 0.1])
    h, _ = make_pair(wl, rom=rte.RTE_ROM_AUTO, **TIGHT)
    for _ in range(12):
        h.rte_step(1)
        st = h.rte_get_stats()
        assert st["last_cg_iterations"] == 0 and st["last_iterations"] <= 2
    assert st["phase"] == 3 and st["pc_rank"] == 0
    h.destroy()
    orc = _march(wl, 40, 5, rom_on=True, **TIGHT)
    assert all(s.cg_iterations == 0 for s in orc.log)


@pytest.mark.parametrize("shape", [(1, 1), (1, 23), (23, 1)])
def test_degenerate_single_cell_and_strips(shape):
    """One cell (the ROMs reach their full rank 1 at once) and one-cell-wide strips along
    either axis, ROM on."""
    wl = inputs.checkerboard(n=8, quad=(8, 4))
    wl.nx, wl.ny = shape
    n = wl.ncell
    rng = np.random.default_rng(3)
    ss = rng.uniform(0, 50, n)
    wl.sigma_s, wl.sigma_t, wl.source = ss, ss + 0.2, rng.uniform(0, 1, n)
    wl.rho0 = np.zeros(n)
    wl.inflow = np.array([0.5, 0.0, 0.25, 0.0])
    _march(wl, 30, 5, rom_on=True, **TIGHT)


def test_degenerate_single_cell_slab():
    wl = inputs.slab_1d(n=1, steps=20)
    _march(wl, 20, 5, rom_on=True, **TIGHT)


@pytest.mark.slow
def test_checkerboard_full_workload_rom():
    """The benchmark workload (256^2, 128 directions, c dt = 0.005, 200 steps, ROM on)."""
    wl = inputs.checkerboard()
    _march(wl, wl.steps, 25, rom_on=True, exact=False)


@pytest.mark.slow
def test_checkerboard_full_workload_phase3_strict():
    """The benchmark workload at the working tolerance with the preconditioner ROM truncated at
    eps_PC = 1e-3: 1e-10 and the same decisions for all 200 steps, 189 of them in Phase 3
    (the oracle's decisions stand at least 6e-4 relative from their thresholds)."""
    wl = inputs.checkerboard()
    orc = _march(wl, wl.steps, 25, rom_on=True, decisions_p3=True, **WELL_CONDITIONED_PC)
    assert sum(s.phase == 3 for s in orc.log) >= 180


@pytest.mark.parametrize("case", ["checkerboard_rom", "slab_rom", "checkerboard_plain"])
def test_bdf2_march(case):
    """BDF2 (options.time_scheme): a backward-Euler first step, then the BDF2 step's system with
    its history; against the oracle's BDF2 march with the same decisions and 1e-10 (ROM on:
    the preconditioner ROM truncated at eps_PC = 1e-3, §2 item 13 of the design notes)."""
    wl = inputs.slab_1d(steps=60) if case == "slab_rom" else inputs.checkerboard(n=48)
    steps = 60 if case == "slab_rom" else 80
    rom_on = case != "checkerboard_plain"
    o = dict(time_scheme=rte.RTE_BDF2, **WELL_CONDITIONED_PC)
    h, p = make_pair(wl, rom=rte.RTE_ROM_AUTO if rom_on else rte.RTE_ROM_OFF, **o)
    orc = stepper.OracleRTE(p, rom=rom_on, scheme="bdf2", **WELL_CONDITIONED_PC)
    h.rte_set_initial(rho0=wl.rho0)
    orc.set_initial(wl.rho0)
    for n in range(1, steps + 1):
        h.rte_step(1)
        orc.step(1)
        st, lg = h.rte_get_stats(), orc.log[-1]
        assert st["last_iterations"] == lg.iterations, n
        assert st["phase"] == (lg.phase if rom_on else 0), n
        assert rel_l2(h.rte_get_scalar_flux(), orc.rho) < TOL, n
    if rom_on:
        assert max(s.phase for s in orc.log) == 3
    h.destroy()


@pytest.mark.parametrize("precision", [rte.RTE_FP64, rte.RTE_FP32])
def test_bdf2_angular_flux_restart_and_checkpoint(precision):
    """The angular flux of a BDF2 march is f^n (not the stored history) and matches the
    oracle's; rte_restart begins again with a backward-Euler step (the march repeats bit for
    bit); a checkpoint taken mid-march resumes bit for bit."""
    from gpu_util import match_directions
    wl = inputs.checkerboard(n=32)
    wl.inflow = np.array([0.3, 0.0, 0.1, 0.0])
    opts = dict(time_scheme=rte.RTE_BDF2, precision=precision)
    h, p = make_pair(wl, **opts)
    orc = stepper.OracleRTE(p, scheme="bdf2")
    h.rte_set_initial(rho0=wl.rho0)
    orc.set_initial(wl.rho0)
    h.rte_step(12)
    orc.step(12)
    perm, _, _ = match_directions(h, wl.quadrature)
    tol = TOL if precision == rte.RTE_FP64 else 1e-6
    assert rel_l2(h.rte_get_angular_flux(), orc.f[perm]) < tol
    rho12 = h.rte_get_scalar_flux()
    blob = h.rte_save()
    h.rte_step(6)
    rho18 = h.rte_get_scalar_flux()
    h.rte_restart()
    h.rte_step(12)
    assert np.array_equal(h.rte_get_scalar_flux(), rho12)
    for pre_steps in (3, 0):   # a handle past its first step, and a fresh one
        b, _ = make_pair(wl, **opts)
        b.rte_set_initial(rho0=wl.rho0)
        b.rte_step(pre_steps)
        b.rte_load(blob)
        b.rte_step(6)
        assert np.array_equal(b.rte_get_scalar_flux(), rho18), pre_steps
        b.destroy()
    h.destroy()
