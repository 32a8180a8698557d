"""Pins of the oracle's DMD-across-iterations acceleration, the alternative to DSA that the
paper combines with its ROMs in Sec. 4 ("hybrid with McClarren-Haut method", set against its
own method in Sec. 3.3) and gives by citation only.  Reading (oracle/sisa.py): plain SI steps
collect a cycle of K residuals r_l = rho^{l-1/2} - rho^{l-1}; since r_{l+1} = T Sigma_s r_l for
plain SI, the K - 1 pairs (r_l, r_l - r_{l+1}) sample I - T Sigma_s, and the jump
rho^l = rho^{l-1} + C_r^{-1} r_l with their DMD model C_r is the fixed point restricted to the
span of the residuals.

Pins from the mathematics:
* when the initial error lies in a k-dimensional invariant subspace of T Sigma_s (real
  eigenvectors of the dense T Sigma_s, assembled column by column from oracle sweeps), the
  residuals span exactly that subspace, so with K = k + 1 the jump lands on the fixed point of
  a dense solve of (I - T Sigma_s) rho = b~ and SI stops at l = K + 1; a model of the wrong
  operator (the pairs (r_l, r_{l+1}), i.e. T Sigma_s) fails this;
* the acceleration changes only the path: a ROM-accelerated march with it ends where the
  one with DSA ends."""
import numpy as np
import pytest

from oracle import dsa, rom, sisa, stepper
from oracle import transport as tr
from conftest import oracle_problem
from paper_2603_19647_gb300 import inputs
from test_oracle_alg2 import _slab


def _setup():
    p = _slab(ss=5.0, c_dt=1.0)
    n = p.ncell
    TS = np.column_stack([tr.apply_T_sigma_s(p, np.eye(n)[:, j]) for j in range(n)])
    lam, V = np.linalg.eig(TS)
    real = [i for i in np.argsort(-np.abs(lam)) if abs(lam[i].imag) < 1e-12]
    bt = tr.b_tilde(p, np.random.default_rng(1).uniform(0, 1, (p.nv, n)))
    rho_star = np.linalg.solve(np.eye(n) - TS, bt)
    modes = [V[:, i].real / np.abs(V[:, i].real).max() for i in real]
    return p, bt, rho_star, modes


def _jump(p, bt, rho0, window):
    o = dict(stepper.DEFAULTS, eps_sisa=1e-12, cg_rtol=1e-12, sa="mh", mh_window=window)
    return sisa.si_sa(p, rho0, bt, o, dsa.dsa_matrix(p))


@pytest.mark.parametrize("k", [1, 2, 3])
def test_jump_lands_on_the_fixed_point_of_an_invariant_span(k):
    p, bt, rho_star, modes = _setup()
    rho0 = rho_star + sum(0.7 ** i * modes[i] for i in range(k))
    rho, info = _jump(p, bt, rho0, window=k + 1)
    assert info.mh_corrections == 1 and info.iterations == k + 2
    assert np.linalg.norm(rho - rho_star) < 1e-12 * np.linalg.norm(rho_star)


def test_model_of_the_wrong_operator_is_caught(monkeypatch):
    """Planted: the DMD model built from (r_l, r_{l+1}) (the operator T Sigma_s itself)."""
    def wrong_step(cycle, r, window, rho_prev, rho_half):
        cycle.append(r.copy())
        if len(cycle) < window:
            return np.zeros_like(r)
        svd = rom.IncrementalSVD(r.size, window)
        for a, b in zip(cycle[:-1], cycle[1:]):
            svd.append(a, b)
        cycle.clear()
        return rho_prev + svd.solve_apply(r) - rho_half
    p, bt, rho_star, modes = _setup()
    rho0 = rho_star + modes[0] + 0.7 * modes[1]
    monkeypatch.setattr(sisa, "mh_step", wrong_step)
    rho, info = _jump(p, bt, rho0, window=3)
    assert info.iterations > 4


def test_hybrid_march_ends_where_the_dsa_march_ends():
    """The ROM-accelerated march with the DMD-across-iterations steps in place of DSA (both
    phases of construction and Phase 3) against the same march with DSA, at a tight tolerance:
    the fixed point of every step is the same."""
    wl = inputs.checkerboard(n=16, quad=(8, 4))
    out = {}
    for sa in ("dsa", "mh"):
        r = stepper.OracleRTE(oracle_problem(wl), eps_sisa=1e-12, cg_rtol=1e-10, eps_ig=1e-9,
                              eps_up=1e-9, sa=sa)
        r.set_initial(wl.rho0)
        r.step(30)
        out[sa] = r
    assert max(s.phase for s in out["mh"].log) == 3
    assert sum(s.cg_iterations for s in out["mh"].log) == 0
    a, b = out["dsa"].rho, out["mh"].rho
    assert np.linalg.norm(a - b) < 1e-10 * np.linalg.norm(a)
