"""Pins of the oracle's BDF2 time marching (the second-order backward difference formula the
paper names beside backward Euler in Sec. 2.1):

* the march equals, step by step, dense LU solves assembled without any sweep
  (oracle/dense.py): a backward-Euler first step, then the BDF2 system with
  tau' = 3 / (2 c dt) and the history (4 f^{n-1} - f^{n-2}) / 3 on the right side, with and
  without the ROMs;
* in a uniform absorbing medium whose inflow follows the exact solution rho0 exp(-c sigma_a t),
  the error at a fixed time falls by about 4 when the time step halves (second order), where
  backward Euler's falls by about 2."""
import numpy as np
import pytest

from oracle import dense, stepper
from oracle import quadrature as q
from oracle import transport as tr
from test_oracle_step import _small_1d, _small_2d


@pytest.mark.parametrize("dim", [1, 2])
@pytest.mark.parametrize("rom", [False, True])
def test_bdf2_march_matches_direct_solve(dim, rom, rng):
    p = _small_2d(rng) if dim == 2 else _small_1d(rng)
    r = stepper.OracleRTE(p, scheme="bdf2", eps_sisa=1e-13, rom=rom, cg_rtol=1e-10, eps_ig=1e-8,
                          eps_pc=1e-8, eps_up=1e-10)
    rho0 = rng.uniform(0, 1, p.ncell)
    r.set_initial(rho0)
    q2 = tr.Problem(p.nx, p.ny, p.x0, p.x1, p.y0, p.y1, p.mu, p.eta, p.w, p.sigma_t, p.sigma_s,
                    p.source, p.c_dt * 2.0 / 3.0, p.inflow)
    A = dense.assemble(q2)
    f0 = np.tile(rho0, (p.nv, 1))
    f_prev, f = f0, dense.step(p, f0)[0]      # the backward-Euler first step
    r.step()
    assert np.max(np.abs(r.f - f)) <= 1e-10 * np.max(np.abs(f))
    for n in range(11):
        r.step()
        h = (4.0 * f - f_prev) / 3.0
        f_prev, f = f, np.linalg.solve(A, dense.rhs(q2, h)).reshape(p.nv, p.ncell)
        rho = p.w @ f
        assert np.linalg.norm(r.rho - rho) <= 1e-11 * np.linalg.norm(rho)
        assert np.max(np.abs(r.f - f)) <= 1e-10 * np.max(np.abs(f))


def _decay_error(scheme, steps, T=0.4):
    mu, eta, w = q.cl_hemisphere(8, 4)
    nx = ny = 4
    n = nx * ny
    st, ss, rho0 = 3.0, 1.0, 1.0
    c_dt = T / steps
    p = tr.Problem(nx, ny, 0, 1, 0, 1, mu, eta, w, np.full(n, st), np.full(n, ss), np.zeros(n),
                   c_dt, np.zeros(4))
    r = stepper.OracleRTE(p, scheme=scheme, eps_sisa=1e-14, cg_rtol=1e-12, rom=False)
    r.set_initial(np.full(n, rho0))
    for k in range(1, steps + 1):
        r.set_inflow([rho0 * np.exp(-(st - ss) * k * c_dt)] * 4)
        r.step()
    exact = rho0 * np.exp(-(st - ss) * T)
    return float(np.max(np.abs(r.rho - exact)))


def test_bdf2_is_second_order_in_time():
    e = [_decay_error("bdf2", s) for s in (8, 16, 32)]
    b = [_decay_error("be", s) for s in (8, 16, 32)]
    for k in range(2):
        assert 3.3 < e[k] / e[k + 1] < 4.7, e
        assert 1.7 < b[k] / b[k + 1] < 2.3, b
    assert e[-1] < b[-1] / 10
