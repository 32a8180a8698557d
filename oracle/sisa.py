"""Memory-efficient source iteration with synthetic acceleration, Algorithm 1 (test infrastructure).

Sec. 2.3: iterate on rho only,
    rho^{l-1/2} = T Sigma_s rho^{l-1} + b_tilde                      (Eq. (SI_rho))
    stop when ||rho^{l-1/2} - rho^{l-1}||_inf < eps  and return rho^{l-1/2}
    else rho^l = rho^{l-1/2} + delta_rho^l, delta_rho from the SA step.

Readings where the paper leaves a choice:
* The stopping test is relative by default, ||.||_inf <= eps ||rho^{l-1/2}||_inf
  (mode "rel"); mode "abs" is the paper's absolute test.  "<=" instead of "<" so
  that an all-zero state counts as converged.
* The SA step at l = 1 uses the ROM preconditioner when one is given (Sec. 3.2
  Phase 3, Eq. (dmd-sa)); every other SA step is DSA (Eq. (rho_residual)).  With a sequence
  of preconditioner ROMs (Sec. 3.2, key feature 1: ROMs for the first l - 1 iterations before
  the one for iteration l), the SA step of iteration l uses the l-th ROM when there is one.
* opts["sa"] = "mh" replaces DSA by the DMD-across-iterations acceleration the paper combines
  with its ROMs in Sec. 4 ("hybrid with McClarren-Haut method", compared in Sec. 3.3), which it
  gives by citation only.  Reading: the SA steps that would be DSA are plain SI steps
  (delta = 0) collecting this cycle's residuals r_l = rho^{l-1/2} - rho^{l-1}; for plain SI,
  r_{l+1} = T Sigma_s r_l, so the pairs (r_l, r_l - r_{l+1}) sample I - T Sigma_s.  After
  K = opts["mh_window"] residuals a DMD reduced model of I - T Sigma_s is built from the K - 1
  pairs (the incremental SVD and reduced operator of Sec. 3.1) and the iterate jumps to
  rho^l = rho^{l-1} + C_r^{-1} r_l, the fixed point rho = T Sigma_s rho + b~ restricted to
  the span of the residuals; the cycle then starts again.
"""
from dataclasses import dataclass

import numpy as np

from . import dsa as _dsa
from . import rom as _rom
from . import transport as _tr


class NoConvergence(RuntimeError):
    pass


@dataclass
class SolveInfo:
    iterations: int = 0          # SI sweeps done (l at return)
    cg_iterations: int = 0       # total CG iterations over the DSA solves
    rho_half_1: np.ndarray = None   # rho^{n,(1/2)}, kept for the PC snapshot (Sec. 3.2 Phase 2)
    delta_pc_1: np.ndarray = None   # delta_rho_DMD^{n,(1)} when the ROM PC was applied at l = 1
    residual: float = 0.0
    # per iteration l = 1, 2, ... (index l - 1): rho^{n,(l-1/2)}, rho^{n,(l-1)} and the ROM
    # correction delta_rho_DMD^{n,(l)} (None where DSA was used)
    rho_half: list = None
    rho_prev: list = None
    delta_pc: list = None
    mh_corrections: int = 0      # DMD-across-iterations jumps (opts["sa"] = "mh")


def converged(diff, rho_half, eps, mode):
    dn = float(np.max(np.abs(diff))) if diff.size else 0.0
    if mode == "abs":
        return dn <= eps, dn
    rn = float(np.max(np.abs(rho_half))) if rho_half.size else 0.0
    return dn <= eps * rn, (dn / rn if rn > 0 else dn)


def mh_step(cycle, r, window, rho_prev, rho_half):
    """One SA step of the DMD-across-iterations acceleration (reading in the module docstring):
    append the residual r to the cycle; a plain SI step (delta = 0) until the cycle holds
    `window` residuals, then the jump rho^l = rho^{l-1} + C_r^{-1} r of the DMD model of
    I - T Sigma_s built from the pairs (r_i, r_i - r_{i+1}), returned as delta = rho^l -
    rho^{l-1/2}, and the cycle is emptied."""
    cycle.append(r.copy())
    if len(cycle) < window:
        return np.zeros_like(r)
    svd = _rom.IncrementalSVD(r.size, window)
    for a, b in zip(cycle[:-1], cycle[1:]):
        svd.append(a, a - b)
    cycle.clear()
    if svd.rank == 0:
        return np.zeros_like(r)
    return rho_prev + svd.solve_apply(r) - rho_half


def si_sa(p, rho_init, btilde, opts, A_dsa, pc=None, decide=None):
    """Algorithm 1.  pc: callable(rhs) -> delta for the l = 1 SA step, or a list of such
    callables for the SA steps l = 1, 2, ..., or None for DSA only.  The ROM correction of
    iteration l maps the residual rho^{n,(l-1/2)} - rho^{n,(l-1)} to delta (Eq. (dmd-sa)).
    decide: optional callable(kind, own, value, threshold) -> bool that may replace the
    stopping decision ("si_stop"; value = the residual in the test's own units).

    Returns (rho^n, SolveInfo).  Raises NoConvergence after opts['max_iter'] sweeps.
    """
    pcs = [] if pc is None else (list(pc) if isinstance(pc, (list, tuple)) else [pc])
    info = SolveInfo(rho_half=[], rho_prev=[], delta_pc=[])
    rho_prev = np.array(rho_init, dtype=np.float64, copy=True)
    mh = opts.get("sa", "dsa") == "mh"
    window = int(opts.get("mh_window", 4))
    cycle = []   # residuals of the current DMD-across-iterations cycle
    for l in range(1, opts["max_iter"] + 1):
        rho_half = _tr.apply_T_sigma_s(p, rho_prev) + btilde
        diff = rho_half - rho_prev
        if l == 1:
            info.rho_half_1 = rho_half.copy()
        if l <= len(pcs) + 1:   # what the ROM snapshots of iteration l need
            info.rho_half.append(rho_half.copy())
            info.rho_prev.append(rho_prev.copy())
        ok, res = converged(diff, rho_half, opts["eps_sisa"], opts["residual_norm"])
        if decide is not None:
            ok = decide("si_stop", ok, res, opts["eps_sisa"])
        info.iterations = l
        info.residual = res
        if ok:
            return rho_half, info
        if l <= len(pcs) and pcs[l - 1] is not None:
            delta = pcs[l - 1](rho_half - rho_prev)
            info.delta_pc.append(delta.copy())
            if l == 1:
                info.delta_pc_1 = delta.copy()
        else:
            if l <= len(pcs):
                info.delta_pc.append(None)
            if mh:
                delta = mh_step(cycle, diff, window, rho_prev, rho_half)
                info.mh_corrections += 0 if cycle else 1
            else:
                delta, its = _dsa.dsa_correction(p, A_dsa, diff, opts["cg_rtol"],
                                                 opts["cg_max_iter"])
                info.cg_iterations += its
        rho_prev = rho_half + delta
    raise NoConvergence(f"SI-SA did not converge in {opts['max_iter']} iterations")
