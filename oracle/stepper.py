"""Algorithm 2: on-the-fly DMD-enhanced SI-SA for implicit time marching (test infrastructure).

Per time step n (Sec. 3.2, Algorithm 2):
  1. b_tilde^{n-1} by a transport sweep (Eq. (implicit_linear_system_rho)).
  2. rho^{n,(0)} = U_IG c (Eq. (dmd-ig)) when Flag_IG, else rho^{n-1}.
  3. Algorithm 1; at l = 1 the ROM preconditioner (Eq. (dmd-sa)) when Flag_PC, DSA otherwise.
  4. f^n by one more sweep (Eq. (sweep_to_obtain_f)).
  5. ROM construction / adaptive update (Phases 1-3).

Readings where the paper is silent or loose (each listed in the design notes):
* Snapshot pair of the IG ROM is (rho^n, b_tilde^{n-1}), since A~ rho^n = b_tilde^{n-1}
  (Eq. (implicit_linear_system_rho), Eq. (snapshots)); the "b_tilde^n" of the Phase 3 text
  is read as this pair.
* Phases 1 and 2 append without truncation (capped at r_max; reaching the cap ends the phase).
* Phase 3 updates truncate with eps_IG (IG ROM) and eps_PC (PC ROM).
* The update indicators compare with eps_UP * ||rho^n||_2 (up_rel=True, default) or with
  eps_UP itself (up_rel=False, the paper's absolute form).
* The PC ROM's adaptive update applies only once Flag_PC held at the start of the step
  (in Phase 2 its snapshots are appended by the construction branch already).
* A step whose first sweep already converged has no first correction, so no PC snapshot
  is taken from it.
* Step 1's initial guess is rho^0 (the isotropic initial state).
* scheme = "bdf2" marches with the second-order backward difference formula the paper names as
  an alternative to backward Euler (Sec. 2.1): (3 f^n - 4 f^{n-1} + f^{n-2}) / (2 c dt) replaces
  (f^n - f^{n-1}) / (c dt), i.e. the step's system is that of backward Euler with
  tau' = 3 / (2 c dt) and the history h^n = (4 f^{n-1} - f^{n-2}) / 3 in place of f^{n-1}.
  The first step is a backward-Euler step of dt (its local error O(dt^2) keeps the march
  second order), and it gives the ROMs no snapshot: they learn the BDF2 step's system
  A~ rho^n = b~^{n-1} (b~ built from h), on which Algorithm 2 runs unchanged from step 2.

Each decision of the algorithm (the SI stopping test, the end of each construction phase, the
two update gates) goes through ``decide``, which returns the algorithm's own decision; a
test may override it to follow another implementation's log where both sides stand within
rounding of a threshold.  The snapshot pairs and the correction rule are methods of their own
so that a test can plant a mistake in exactly one of them.
"""
import dataclasses
from dataclasses import dataclass, field

import numpy as np

from . import dsa as _dsa
from . import rom as _rom
from . import sisa as _sisa
from . import transport as _tr

DEFAULTS = dict(eps_sisa=1e-8, eps_ig=1e-6, eps_pc=1e-6, eps_up=1e-6, max_iter=500, r_max=40,
                rom=True, residual_norm="rel", cg_rtol=1e-6, cg_max_iter=500, up_rel=True,
                pc_levels=1, sa="dsa", mh_window=4, scheme="be")


@dataclass
class StepLog:
    n: int
    phase: int
    iterations: int
    sweeps: int
    cg_iterations: int
    ig_rank: int
    pc_rank: int
    ig_updated: bool
    pc_updated: bool
    residual: float
    ig_error: float = float("nan")
    pc_error: float = float("nan")
    # record=True: rho^n, rho^{n,1/2} and the initial guess rho^{n,(0)} of the step, and the
    # singular values of both ROMs after its update
    rho: np.ndarray = None
    rho_half_1: np.ndarray = None
    rho_init: np.ndarray = None
    ig_s: np.ndarray = None
    pc_s: np.ndarray = None
    # every preconditioner ROM (iterations l = 1 .. pc_levels): ranks and updates
    pc_ranks: tuple = ()
    pc_ups: tuple = ()
    mh_jumps: int = 0   # DMD-across-iterations jumps of the step (sa = "mh")


class OracleRTE:
    """The time march of Algorithm 2 on an oracle.transport.Problem."""

    def __init__(self, problem, record=False, **opts):
        self.p = problem
        self.record = record
        self.o = dict(DEFAULTS)
        self.o.update(opts)
        if self.o["scheme"] not in ("be", "bdf2"):
            raise ValueError("scheme must be 'be' or 'bdf2'")
        # the step's system: backward Euler's with tau' = 3 / (2 c dt) for BDF2
        self.q = (problem if self.o["scheme"] == "be"
                  else dataclasses.replace(problem, c_dt=problem.c_dt * 2.0 / 3.0))
        self.A = _dsa.dsa_matrix(self.q)
        self.A_start = self.A if self.o["scheme"] == "be" else _dsa.dsa_matrix(problem)
        self.rho = np.zeros(problem.ndof)
        self.f = np.zeros((problem.nv, problem.ndof))
        self.f_prev = self.f.copy()
        self.n = 0
        self.flag_ig = False
        self.ig = _rom.IncrementalSVD(problem.ndof, self.o["r_max"])
        # one preconditioner ROM per SI iteration l = 1 .. pc_levels, each with its Flag_PC
        L = int(self.o["pc_levels"])
        self.pcs = [_rom.IncrementalSVD(problem.ndof, self.o["r_max"]) for _ in range(L)]
        self.flags_pc = [False] * L
        self.log = []

    @property
    def pc(self):
        """The preconditioner ROM of the first iteration."""
        return self.pcs[0]

    @property
    def flag_pc(self):
        """Every preconditioner ROM is built (Phase 3)."""
        return all(self.flags_pc)

    def set_initial(self, rho0, f0=None):
        """f^0 = rho0 in every direction (isotropic) unless f0 [nv, ndof] is given."""
        self.rho = np.array(rho0, dtype=np.float64).ravel().copy()
        if f0 is None:
            self.f = np.tile(self.rho, (self.p.nv, 1))
        else:
            self.f = np.array(f0, dtype=np.float64).reshape(self.p.nv, self.p.ndof).copy()
            self.rho = self.p.w @ self.f
        self.f_prev = self.f.copy()   # BDF2: f^{-1} = f^0

    def set_inflow(self, g):
        self.p.inflow = np.asarray(g, dtype=np.float64).ravel().copy()
        self.q.inflow = self.p.inflow

    def starting_step(self):
        """BDF2's first step, a backward-Euler step."""
        return self.o["scheme"] == "bdf2" and self.n == 0

    def history(self):
        """What the step's sweeps scale by tau: f^{n-1} (backward Euler and BDF2's first step)
        or h^n = (4 f^{n-1} - f^{n-2}) / 3 (BDF2)."""
        if self.o["scheme"] == "be" or self.starting_step():
            return self.f
        return (4.0 * self.f - self.f_prev) / 3.0

    def phase(self):
        return 1 if not self.flag_ig else (2 if not self.flag_pc else 3)

    def step(self, nsteps=1):
        for _ in range(nsteps):
            self._step()

    # ---- the pieces of Algorithm 2 a test may replace one at a time ----
    def decide(self, kind, own, value, threshold):
        """A decision of the algorithm: kind is "si_stop", "ig_built", "pc_built", "ig_update"
        or "pc_update"; own is the algorithm's answer for value against threshold."""
        return own

    def ig_pair(self, rho_n, btilde_prev, f_new):
        """IG-ROM snapshot pair: (rho^n, b~^{n-1}), since A~ rho^n = b~^{n-1}."""
        return rho_n, btilde_prev

    def pc_pair(self, rho_n, info, level):
        """PC-ROM snapshot pair of iteration l = level: the ideal correction
        rho^n - rho^{n,(l-1/2)} and its residual rho^{n,(l-1/2)} - rho^{n,(l-1)} (Sec. 3.2,
        Phase 2; for l = 1 the residual is measured from the initial guess rho^{n,(0)})."""
        rho_half, rho_prev = info.rho_half[level - 1], info.rho_prev[level - 1]
        return rho_n - rho_half, rho_half - rho_prev

    def sequential_ready(self, level, built_before):
        """The ROM of iteration `level` takes snapshots only from steps that applied the ROMs of
        all earlier iterations (Sec. 3.2, key feature 1)."""
        return all(built_before[:level - 1])

    def has_correction(self, info, level=1):
        """A step that met the stopping test at iteration l <= level took no correction at
        iteration `level`."""
        return info.iterations > level

    def pc_update_due(self, ig_up, err, threshold):
        """Phase 3 PC-ROM update: when the IG-ROM (or, for the ROM of iteration l > 1, any ROM
        of an earlier iteration) was updated in the same step, or when the PC indicator
        exceeds the threshold (Sec. 3.2, Phase 3 and key feature 1)."""
        return ig_up or self.decide("pc_update", err > threshold, err, threshold)

    def _built(self, kind, svd, grew, eps):
        """End of a construction phase: s_m / sum s <= eps (Eq. (ig_stop), Eq. (pc_stop)) or
        the rank cap reached."""
        ratio = svd.stop_ratio(grew)
        own = ratio <= eps or svd.rank >= self.o["r_max"]
        return self.decide(kind, own, ratio, eps)

    def _step(self):
        start = self.starting_step()
        p, o = (self.p if start else self.q), self.o
        A = self.A_start if start else self.A
        L = len(self.pcs)
        phase = self.phase()
        hist = self.history()
        btilde = _tr.b_tilde(p, hist)
        use_rom = o["rom"] and not start
        rho_ig = None
        if use_rom and self.flag_ig:
            rho_ig = self.ig.solve_apply(btilde)
            rho0 = rho_ig
        else:
            rho0 = self.rho
        # the ROM of iteration l applies once it and the ROMs of iterations 1 .. l-1 are built
        pcs = [self.pcs[k].solve_apply if use_rom and all(self.flags_pc[:k + 1]) else None
               for k in range(L)]
        rho_n, info = _sisa.si_sa(p, rho0, btilde, o, A, pc=pcs, decide=self.decide)
        f_new, _ = _tr.final_f(p, rho_n, hist)
        ig_up = False
        pc_ups, pc_errs = [False] * L, [float("nan")] * L
        ig_err = float("nan")
        if use_rom:
            scale = float(np.linalg.norm(rho_n)) if o["up_rel"] else 1.0
            thr = o["eps_up"] * scale
            x_ig, b_ig = self.ig_pair(rho_n, btilde, f_new)
            if not self.flag_ig:
                grew = self.ig.append(x_ig, b_ig)
                ig_up = True
                if self._built("ig_built", self.ig, grew, o["eps_ig"]):
                    self.flag_ig = True
            else:
                ig_err = float(np.linalg.norm(rho_ig - rho_n))
                if self.decide("ig_update", ig_err > thr, ig_err, thr):
                    self.ig.append(x_ig, b_ig, trunc_eps=o["eps_ig"])
                    ig_up = True
                earlier_up = ig_up
                built_before = list(self.flags_pc)   # as this step found them
                for k in range(L):
                    if not self.sequential_ready(k + 1, built_before):
                        break
                    if not self.has_correction(info, k + 1):
                        break
                    svd = self.pcs[k]
                    d_rho, d_b = self.pc_pair(rho_n, info, k + 1)
                    if not self.flags_pc[k]:
                        grew = svd.append(d_rho, d_b)
                        pc_ups[k] = True
                        if self._built("pc_built", svd, grew, o["eps_pc"]):
                            self.flags_pc[k] = True
                    else:
                        pc_errs[k] = float(np.linalg.norm(info.delta_pc[k] - d_rho))
                        if self.pc_update_due(earlier_up, pc_errs[k], thr):
                            svd.append(d_rho, d_b, trunc_eps=o["eps_pc"])
                            pc_ups[k] = True
                    earlier_up = earlier_up or pc_ups[k]
        self.rho = rho_n
        self.f_prev = self.f
        self.f = f_new
        self.n += 1
        sweeps = info.iterations + 2
        lg = StepLog(self.n, phase, info.iterations, sweeps, info.cg_iterations, self.ig.rank,
                     self.pcs[0].rank, ig_up, pc_ups[0], info.residual, ig_err, pc_errs[0],
                     pc_ranks=tuple(v.rank for v in self.pcs), pc_ups=tuple(pc_ups),
                     mh_jumps=info.mh_corrections)
        if self.record:
            lg.rho, lg.rho_half_1, lg.rho_init = rho_n.copy(), info.rho_half_1.copy(), rho0.copy()
            lg.ig_s, lg.pc_s = self.ig.S.copy(), self.pcs[0].S.copy()
        self.log.append(lg)
