"""Pins of the oracle's Algorithm 2 bookkeeping (Sec. 3.2): the snapshot pairs of both ROMs,
the ends of both construction phases, the two update gates of Phase 3 and the rule that a step
without a correction gives the preconditioner ROM no snapshot.

Each pin is a consequence of the mathematics, checked on marches whose answer is known:

* Exact span.  The implicit step is linear, f^n = tau A^{-1} f^{n-1} with A the dense system
  matrix of the step (G = 0, vacuum), so an f^0 made of k real eigenvectors of A keeps every
  f^n, and so every rho^n, in a k-dimensional space.  Since A~ rho^n = b~^{n-1}, the IG-ROM
  built from the pairs (rho^n, b~^{n-1}) has A_r = U^T A~ U, and once rho^n lies in span U the
  DMD initial guess is rho^n itself: SI stops at l = 1 (Eq. (dmd-ig)).
* Exact correction.  With a fixed, inexact IG, e = rho^n - rho^{n,(0)} stays in the span of
  the march, the first correction rho^n - rho^{n,1/2} = T Sigma_s e and its residual
  rho^{n,1/2} - rho^{n,(0)} = A~ e are fixed linear images of e, so once the PC-ROM holds the
  span of those corrections the l = 1 correction (Eq. (dmd-sa)) is exact and every Phase 3
  step ends at l = 2.
* Construction ends.  Phases 1 and 2 append without truncation, so the IG-ROM and PC-ROM
  singular values are those of the stacked snapshots, here taken from LAPACK's SVD; each phase
  ends at the first snapshot count m with s_m / sum s <= eps (Eq. (ig_stop), Eq. (pc_stop)).

Every pin is also run with one plausible mistake planted in the oracle (a subclass that
replaces one piece of Algorithm 2), and must fail for it."""
import numpy as np
import pytest

from oracle import dense, stepper
from oracle import quadrature as q
from oracle import transport as tr


def _slab(ss=0.9, c_dt=0.05, seed=5, nx=16, nd=8):
    mu, eta, w = q.gl_slab(nd)
    rng = np.random.default_rng(seed)
    sig_s = ss * (0.5 + rng.uniform(0, 1, nx))
    sig_t = sig_s + rng.uniform(0.2, 1.0, nx)
    return tr.Problem(nx, 1, 0.0, 1.0, 0.0, 1.0, mu, eta, w, sig_t, sig_s, np.zeros(nx), c_dt,
                      np.zeros(4))


def _span_start(p, coeffs):
    """f^0 = sum_i c_i v_i over the real eigenvectors v_i of the step's dense system matrix
    with the slowest decay (each scaled to max |v_i| = 1)."""
    lam, V = np.linalg.eig(dense.assemble(p))
    order = [i for i in np.argsort(np.abs(lam)) if abs(lam[i].imag) < 1e-12]
    f0 = np.zeros(p.nv * p.ncell)
    for c, i in zip(coeffs, order):
        v = V[:, i].real
        f0 += c * v / np.abs(v).max()
    return f0.reshape(p.nv, p.ncell)


def _run(p, f0, steps, cls=stepper.OracleRTE, inflow_at=None, **opts):
    r = cls(p, record=True, **opts)
    r.set_initial(np.zeros(p.ncell), f0=f0)
    for n in range(1, steps + 1):
        if inflow_at and n in inflow_at:
            r.set_inflow(inflow_at[n])
        r.step()
    return r


# ---- planted mistakes (each replaces one piece of Algorithm 2) ----
class PairRhoWithNextBtilde(stepper.OracleRTE):
    """The IG pair (rho^n, b~^n), as the printed text of Phase 3 reads literally."""

    def ig_pair(self, rho_n, btilde_prev, f_new):
        return rho_n, tr.b_tilde(self.p, f_new)


class CorrectionEveryStep(stepper.OracleRTE):
    """A PC snapshot from every step, also from those that converged at l = 1."""

    def has_correction(self, info):
        return True


class IGGateAlwaysOpen(stepper.OracleRTE):
    def decide(self, kind, own, value, threshold):
        return True if kind == "ig_update" else own


class IGGateNeverOpens(stepper.OracleRTE):
    def decide(self, kind, own, value, threshold):
        return False if kind == "ig_update" else own


class ResidualAgainstPreviousRho(stepper.OracleRTE):
    """The PC residual snapshot rho^{n,1/2} - rho^{n-1} instead of rho^{n,1/2} - rho^{n,(0)}."""

    def pc_pair(self, rho_n, info, level):
        return rho_n - info.rho_half[level - 1], info.rho_half[level - 1] - self.rho


class PCGateAlwaysOpen(stepper.OracleRTE):
    def decide(self, kind, own, value, threshold):
        return True if kind == "pc_update" else own


class PCGateNeverOpens(stepper.OracleRTE):
    def decide(self, kind, own, value, threshold):
        return False if kind == "pc_update" else own


class PCIgnoresIGUpdate(stepper.OracleRTE):
    """The PC update gate without the 'IG updated in the same step' clause."""

    def pc_update_due(self, ig_up, err, threshold):
        return self.decide("pc_update", err > threshold, err, threshold)


# ---- exact span: the IG-ROM reproduces rho^n, and nothing else moves ----
EXACT = dict(eps_sisa=1e-12, cg_rtol=1e-12, eps_ig=1e-6, eps_pc=1e-6, eps_up=1e-8)


def _ig_exact_violations(cls):
    p = _slab()
    f0 = _span_start(p, [1.0, 0.7, 0.5])
    try:
        r = _run(p, f0, 14, cls=cls, **EXACT)
    except Exception as e:   # a planted mistake may break the march outright
        return [f"raised {e!r}"]
    bad = []
    ph = [s.phase for s in r.log]
    # three independent modes: Phase 1 takes the three growing snapshots and the fourth, which
    # lies in their span, ends it
    if ph[:4] != [1] * 4 or ph[4:] != [2] * 10:
        bad.append(f"phases {ph}")
    for s in r.log[4:]:
        if s.iterations != 1:
            bad.append(f"step {s.n}: {s.iterations} iterations with an exact initial guess")
        if np.linalg.norm(s.rho_init - s.rho) > 1e-11 * np.linalg.norm(s.rho):
            bad.append(f"step {s.n}: initial guess off the solution")
        if s.ig_updated or s.pc_updated or s.pc_rank != 0:
            bad.append(f"step {s.n}: ROM changed without a reason")
    if r.log[-1].ig_rank != 3:
        bad.append(f"IG rank {r.log[-1].ig_rank}")
    return bad


def test_ig_rom_is_exact_on_an_invariant_span():
    assert _ig_exact_violations(stepper.OracleRTE) == []


@pytest.mark.parametrize("planted", [PairRhoWithNextBtilde, CorrectionEveryStep, IGGateAlwaysOpen])
def test_ig_exactness_pin_catches(planted):
    assert _ig_exact_violations(planted)


def _ig_gate_violations(cls):
    """A march in the exact span until an inflow switches on at step 9: from then on rho^n
    leaves span U, the IG indicator jumps far above eps_UP ||rho^n|| and the IG-ROM must be
    updated in that very step (and not before)."""
    p = _slab()
    f0 = _span_start(p, [1.0, 0.7, 0.5])
    r = _run(p, f0, 12, cls=cls, inflow_at={9: [0.3, 0.1, 0.0, 0.0]}, **EXACT)
    bad = []
    for s in r.log[4:8]:
        if s.ig_updated:
            bad.append(f"step {s.n}: IG update inside the span")
    s9 = r.log[8]
    if not s9.ig_error > 1e3 * EXACT["eps_up"] * np.linalg.norm(s9.rho):
        bad.append("the perturbation did not move the IG indicator")   # the setup itself
    if not (s9.ig_updated and s9.ig_rank == 4):
        bad.append(f"step 9: ig_updated {s9.ig_updated}, rank {s9.ig_rank}")
    return bad


def test_ig_update_gate_opens_when_the_state_leaves_the_span():
    assert _ig_gate_violations(stepper.OracleRTE) == []


@pytest.mark.parametrize("planted", [IGGateNeverOpens, IGGateAlwaysOpen])
def test_ig_gate_pin_catches(planted):
    assert _ig_gate_violations(planted)


# ---- exact correction: the PC-ROM makes every Phase 3 step end at l = 2 ----
# eps_IG = 0.9 ends Phase 1 after two snapshots (an inexact IG of rank 2 for a four-mode
# march); eps_UP = 0.5 ||rho^n|| keeps that IG fixed.
PCX = dict(eps_sisa=1e-12, cg_rtol=1e-12, eps_ig=0.9, eps_pc=1e-6, eps_up=0.5)


def _pc_exact_violations(cls):
    p = _slab()
    f0 = _span_start(p, [1.0, 0.7, 0.5, 0.4])
    r = _run(p, f0, 16, cls=cls, inflow_at={13: [20.0, 5.0, 0.0, 0.0]}, **PCX)
    bad = []
    p3 = [s for s in r.log if s.phase == 3]
    if not p3 or p3[0].n > 8:
        return [f"Phase 3 never reached (phases {[s.phase for s in r.log]})"]
    for s in p3:
        if s.n >= 13:
            break
        if s.iterations != 2:
            bad.append(f"step {s.n}: {s.iterations} iterations with an exact correction")
        if s.ig_updated or s.pc_updated:
            bad.append(f"step {s.n}: ROM changed without a reason")
    # step 13: a strong inflow moves the IG indicator above eps_UP ||rho^n||; the IG-ROM is
    # updated, and the PC-ROM must be updated with it whatever its own indicator says
    s13 = r.log[12]
    thr = PCX["eps_up"] * np.linalg.norm(s13.rho)
    if not (s13.ig_error > thr and s13.pc_error < thr):
        bad.append("setup: the inflow did not separate the two indicators")
    if not (s13.ig_updated and s13.pc_updated):
        bad.append(f"step 13: ig_updated {s13.ig_updated}, pc_updated {s13.pc_updated}")
    return bad


def test_pc_rom_correction_is_exact_on_an_invariant_span():
    assert _pc_exact_violations(stepper.OracleRTE) == []


@pytest.mark.parametrize("planted", [ResidualAgainstPreviousRho, PCGateAlwaysOpen,
                                     PCIgnoresIGUpdate])
def test_pc_exactness_pin_catches(planted):
    assert _pc_exact_violations(planted)


def _pc_gate_violations(cls):
    """Phase 3 with an exact correction until a weak inflow at step 10: the IG indicator
    stays below eps_UP ||rho^n|| (no IG update), but the stale PC-ROM, applied to a residual
    with a new component, returns a correction far off the true one (its reduced operator
    amplifies the slow modes), so the PC indicator exceeds the threshold and the PC-ROM must
    be updated on its own."""
    p = _slab(ss=0.9, c_dt=1.0, seed=2)
    f0 = _span_start(p, [1.0, 0.7, 0.5, 0.4])
    r = _run(p, f0, 11, cls=cls, inflow_at={10: [1e-3, 3e-4, 0.0, 0.0]}, **PCX)
    bad = []
    for s in r.log[5:9]:
        if s.phase != 3 or s.pc_updated:
            bad.append(f"step {s.n}: phase {s.phase}, pc_updated {s.pc_updated}")
    s10 = r.log[9]
    thr = PCX["eps_up"] * np.linalg.norm(s10.rho)
    if not (s10.ig_error < 0.8 * thr and s10.pc_error > 2 * thr):
        bad.append("setup: the indicators are not well apart from the threshold")
    if s10.ig_updated or not s10.pc_updated:
        bad.append(f"step 10: ig_updated {s10.ig_updated}, pc_updated {s10.pc_updated}")
    return bad


def test_pc_update_gate_opens_on_its_own_indicator():
    assert _pc_gate_violations(stepper.OracleRTE) == []


@pytest.mark.parametrize("planted", [PCGateNeverOpens, PCGateAlwaysOpen])
def test_pc_gate_pin_catches(planted):
    assert _pc_gate_violations(planted)


# ---- construction ends against LAPACK's SVD of the stacked snapshots ----
class StopOnFirstRatio(stepper.OracleRTE):
    """A construction test on s_1 / sum s (the largest value) instead of the newest."""

    def _built(self, kind, svd, grew, eps):
        ratio = float(svd.S[0] / np.sum(svd.S)) if svd.rank else 0.0
        return ratio <= eps or svd.rank >= self.o["r_max"]


class BuildGateNeverCloses(stepper.OracleRTE):
    def decide(self, kind, own, value, threshold):
        return False if kind in ("ig_built", "pc_built") else own


def _first_below(snapshots, eps):
    """First m with s_m / sum_{k<=m} s_k <= eps for the SVD of the first m snapshots."""
    for m in range(1, len(snapshots) + 1):
        s = np.linalg.svd(np.column_stack(snapshots[:m]), compute_uv=False)
        ratio = s[m - 1] / s.sum()
        assert abs(ratio - eps) > 0.1 * eps, "pin setup: a ratio within 10 % of eps"
        if ratio <= eps:
            return m
    return None


CONSTRUCT = dict(eps_sisa=1e-12, cg_rtol=1e-12, eps_ig=2e-3, eps_pc=2e-2, eps_up=1e-6)


def _construction_violations(cls):
    p = _slab(seed=7, c_dt=0.2)
    rng = np.random.default_rng(3)
    f0 = rng.uniform(0.0, 1.0, (p.nv, p.ncell))
    try:
        r = _run(p, f0, 30, cls=cls, **CONSTRUCT)
    except Exception as e:
        return [f"raised {e!r}"]
    ph = [s.phase for s in r.log]
    bad = []
    m_ig = _first_below([s.rho for s in r.log], CONSTRUCT["eps_ig"])
    n0 = ph.index(2) if 2 in ph else None   # steps in Phase 1
    if m_ig is None or n0 != m_ig:
        bad.append(f"Phase 1 ended after {n0} steps, LAPACK says {m_ig}")
        return bad
    corr = [s.rho - s.rho_half_1 for s in r.log[n0:] if s.iterations > 1]
    m_pc = _first_below(corr, CONSTRUCT["eps_pc"])
    n1 = (ph.index(3) - n0) if 3 in ph else None   # steps in Phase 2
    steps_pc = [s for s in r.log[n0:] if s.iterations > 1]
    if m_pc is None or n1 is None or steps_pc[m_pc - 1].n != n0 + n1:
        bad.append(f"Phase 2 ended after {n1} steps, LAPACK says snapshot {m_pc}")
        return bad
    # the ROMs of the construction phases are the SVDs of the stacked snapshots
    s_ig = np.linalg.svd(np.column_stack([s.rho for s in r.log[:n0]]), compute_uv=False)
    s_pc = np.linalg.svd(np.column_stack(corr[:m_pc]), compute_uv=False)
    got_ig, got_pc = r.log[n0 - 1].ig_s, steps_pc[m_pc - 1].pc_s
    if got_ig.size != s_ig.size or np.max(np.abs(got_ig - s_ig)) > 1e-10 * s_ig[0]:
        bad.append(f"IG singular values {got_ig} vs LAPACK {s_ig}")
    if got_pc.size != s_pc.size or np.max(np.abs(got_pc - s_pc)) > 1e-10 * s_pc[0]:
        bad.append(f"PC singular values {got_pc} vs LAPACK {s_pc}")
    return bad


def test_construction_phases_end_where_lapack_says():
    assert _construction_violations(stepper.OracleRTE) == []


@pytest.mark.parametrize("planted", [StopOnFirstRatio, BuildGateNeverCloses])
def test_construction_pin_catches(planted):
    assert _construction_violations(planted)


# ---- a second preconditioner ROM (iteration l = 2; Sec. 3.2, key feature 1) ----
# A five-mode march with every ROM capped at rank 2 (r_max = 2) and the IG frozen
# (eps_UP = 0.5 ||rho^n||): the ROM of iteration 1 is exact on a two-dimensional part of the
# first corrections only, so Phase 3 with it alone takes four iterations.  The map from the
# first-iteration error to the second-iteration error, e -> (T Sigma_s - P_1 A~) e with P_1 the
# first ROM's correction, vanishes on that part, so the second-iteration errors span at most
# the rest (two dimensions here): built sequentially, from steps that already applied the
# first ROM, the second ROM is exact and every Phase 3 step ends at l = 3.
LEVELS = dict(eps_sisa=1e-12, cg_rtol=1e-12, eps_ig=1e-6, eps_pc=1e-6, eps_up=0.5, r_max=2)


class LevelsConcurrent(stepper.OracleRTE):
    """The ROM of iteration 2 built at the same time as that of iteration 1, from steps whose
    first iteration still used DSA."""

    def sequential_ready(self, level, built_before):
        return True


class LevelTwoResidualFromInitialGuess(stepper.OracleRTE):
    """The second-iteration residual snapshot measured from rho^{n,(0)} instead of rho^{n,(1)}."""

    def pc_pair(self, rho_n, info, level):
        return rho_n - info.rho_half[level - 1], info.rho_half[level - 1] - info.rho_prev[0]


def _levels_violations(cls, levels=2):
    p = _slab()
    f0 = _span_start(p, [1.0, 0.7, 0.5, 0.4, 0.3])
    r = _run(p, f0, 16, cls=cls, pc_levels=levels, **LEVELS)
    bad = []
    p3 = [s for s in r.log if s.phase == 3]
    if len(p3) < 8:
        return [f"Phase 3 for {len(p3)} steps (phases {[s.phase for s in r.log]})"]
    want = 3 if levels == 2 else 4
    for s in p3:
        if s.iterations != want:
            bad.append(f"step {s.n}: {s.iterations} iterations, {want} expected")
        if any(s.pc_ups):
            bad.append(f"step {s.n}: a preconditioner ROM changed without a reason")
    if levels == 2:
        # the second ROM started only once the first was built: its first snapshot comes from
        # a step after the first ROM's last construction step
        first_built = next(s.n for s in r.log if s.pc_ranks[0] == 2)
        first_l2 = next((s.n for s in r.log if s.pc_ranks[1] > 0), None)
        if first_l2 is None or first_l2 <= first_built:
            bad.append(f"level 2 began at step {first_l2}, level 1 was built at {first_built}")
    return bad


def test_one_preconditioner_rom_leaves_four_iterations():
    assert _levels_violations(stepper.OracleRTE, levels=1) == []


def test_second_preconditioner_rom_is_exact_when_built_sequentially():
    assert _levels_violations(stepper.OracleRTE) == []


@pytest.mark.parametrize("planted", [LevelsConcurrent, LevelTwoResidualFromInitialGuess])
def test_second_level_pin_catches(planted):
    assert _levels_violations(planted)
