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
  Phase 3, Eq. (dmd-sa)); every other SA step is DSA (Eq. (rho_residual)).
"""
from dataclasses import dataclass

import numpy as np

from . import dsa as _dsa
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


def converged(diff, rho_half, eps, mode):
    dn = float(np.max(np.abs(diff))) if diff.size else 0.0
    if mode == "abs":
        return dn <= eps, dn
    rn = float(np.max(np.abs(rho_half))) if rho_half.size else 0.0
    return dn <= eps * rn, (dn / rn if rn > 0 else dn)


def si_sa(p, rho_init, btilde, opts, A_dsa, pc=None, decide=None):
    """Algorithm 1.  pc: callable(rhs) -> delta for the l = 1 SA step, or None for DSA only.
    decide: optional callable(kind, own, value, threshold) -> bool that may replace the
    stopping decision ("si_stop"; value = the residual in the test's own units).

    Returns (rho^n, SolveInfo).  Raises NoConvergence after opts['max_iter'] sweeps.
    """
    info = SolveInfo()
    rho_prev = np.array(rho_init, dtype=np.float64, copy=True)
    for l in range(1, opts["max_iter"] + 1):
        rho_half = _tr.apply_T_sigma_s(p, rho_prev) + btilde
        diff = rho_half - rho_prev
        if l == 1:
            info.rho_half_1 = rho_half.copy()
        ok, res = converged(diff, rho_half, opts["eps_sisa"], opts["residual_norm"])
        if decide is not None:
            ok = decide("si_stop", ok, res, opts["eps_sisa"])
        info.iterations = l
        info.residual = res
        if ok:
            return rho_half, info
        if l == 1 and pc is not None:
            delta = pc(rho_half - rho_init)
            info.delta_pc_1 = delta.copy()
        else:
            delta, its = _dsa.dsa_correction(p, A_dsa, diff, opts["cg_rtol"], opts["cg_max_iter"])
            info.cg_iterations += its
        rho_prev = rho_half + delta
    raise NoConvergence(f"SI-SA did not converge in {opts['max_iter']} iterations")
