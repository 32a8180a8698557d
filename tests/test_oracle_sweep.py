"""Pins of the oracle's Q0 upwind sweep and transport operator T (Sec. 2.1-2.3).

Each pin is fixed by the mathematics, not by re-running the oracle's own formula:
closed-form lattice-path solutions of the pure-absorber recurrence, a dense inverse of
independently assembled L_j, and exact particle balance.
"""
import math

import numpy as np
import pytest

from oracle import quadrature as q
from oracle import transport as tr
from conftest import oracle_problem
from paper_2603_19647_gb300 import inputs


def _problem(nx, ny, mu, eta, w, sig_t, sig_s=None, G=None, c_dt=0.1, lx=1.0, ly=1.0, g=None):
    n = nx * ny
    sig_t = np.broadcast_to(np.asarray(sig_t, float), (n,)).copy()
    sig_s = np.zeros(n) if sig_s is None else np.broadcast_to(np.asarray(sig_s, float), (n,)).copy()
    G = np.zeros(n) if G is None else np.broadcast_to(np.asarray(G, float), (n,)).copy()
    return tr.Problem(nx, ny, 0.0, lx, 0.0, ly, np.atleast_1d(mu), np.atleast_1d(eta),
                      np.atleast_1d(w), sig_t, sig_s, G, c_dt,
                      np.zeros(4) if g is None else np.asarray(g, float))


@pytest.mark.parametrize("mu", [0.3, -0.7])
def test_1d_pure_absorber_closed_form(mu):
    n, g, sig, c_dt = 40, 2.5, 3.0, 0.2
    p = _problem(n, 1, [mu], [0.0], [1.0], sig, c_dt=c_dt, lx=2.0, g=[g, g, 0, 0])
    _, psi = tr.sweep(p, inflow=p.inflow, want_psi=True)
    a = abs(mu) / p.hx
    alpha = a / (p.tau + sig + a)
    k = np.arange(1, n + 1)               # cells counted from the inflow side
    expect = g * alpha ** k
    got = psi[0] if mu > 0 else psi[0][::-1]
    assert np.max(np.abs(got - expect) / expect) < 1e-13


def test_1d_pure_absorber_continuum_limit():
    """With tau -> 0 (a very long step) the upwind cell values of a pure absorber approach the
    steady solution g exp(-sigma x / |mu|) of the transport equation at the cell's outflow face
    (the upwind cell value is the flux it passes on), with an error of first order in h: the
    error must halve as h halves (a centred or downwind scheme, or a wrong face, would not)."""
    mu, g, sig, L = 0.4, 1.3, 2.0, 1.0
    errs = []
    for n in (50, 100, 200, 400):
        p = _problem(n, 1, [mu], [0.0], [1.0], sig, c_dt=1e12, lx=L, g=[g, 0, 0, 0])
        _, psi = tr.sweep(p, inflow=p.inflow, want_psi=True)
        x_out = (np.arange(n) + 1.0) * p.hx
        errs.append(np.max(np.abs(psi[0] - g * np.exp(-sig * x_out / mu))))
    ratios = [errs[i] / errs[i + 1] for i in range(len(errs) - 1)]
    assert all(1.9 < r < 2.1 for r in ratios), ratios
    assert errs[-1] < 5e-3 * g


@pytest.mark.parametrize("sx,sy", [(1, 1), (-1, 1), (1, -1), (-1, -1)])
def test_2d_pure_absorber_lattice_paths(sx, sy):
    # Inflow g on the x-inflow face only: psi_ij = g sum_{k=1}^{j} C(i-1+j-k, i-1) a^i b^{j-k}
    nx, ny, g = 9, 7, 1.7
    mu, eta = 0.45 * sx, 0.62 * sy
    side_x = 0 if sx > 0 else 1
    inflow = np.zeros(4)
    inflow[side_x] = g
    p = _problem(nx, ny, [mu], [eta], [1.0], 0.8, c_dt=0.5, lx=1.3, ly=0.9, g=inflow)
    _, psi = tr.sweep(p, inflow=inflow, want_psi=True)
    psi = psi[0].reshape(ny, nx)
    a, b = abs(mu) / p.hx, abs(eta) / p.hy
    d = p.tau + 0.8 + a + b
    al, be = a / d, b / d
    for jy in range(ny):
        for ix in range(nx):
            i = (ix + 1) if sx > 0 else (nx - ix)
            j = (jy + 1) if sy > 0 else (ny - jy)
            expect = g * sum(math.comb(i - 1 + j - k, i - 1) * al ** i * be ** (j - k)
                             for k in range(1, j + 1))
            assert abs(psi[jy, ix] - expect) <= 1e-13 * expect


def _dense_T(p):
    """sum_j w_j L_j^{-1} with L_j assembled as a matrix (never swept)."""
    nx, ny, nc = p.nx, p.ny, p.ncell
    T = np.zeros((nc, nc))
    for j in range(p.nv):
        a = abs(p.mu[j]) / p.hx
        b = abs(p.eta[j]) / p.hy if p.dim == 2 else 0.0
        L = np.diag(p.tau + p.sigma_t + a + b)
        for jy in range(ny):
            for ix in range(nx):
                c = ix + nx * jy
                iu = ix - (1 if p.mu[j] > 0 else -1)
                ju = jy - (1 if p.eta[j] >= 0 else -1)
                if 0 <= iu < nx:
                    L[c, iu + nx * jy] = -a
                if b and 0 <= ju < ny:
                    L[c, ix + nx * ju] = -b
        T += p.w[j] * np.linalg.inv(L)
    return T


@pytest.mark.parametrize("dim", [1, 2])
def test_T_matches_dense_inverse(dim, rng):
    if dim == 2:
        mu, eta, w = q.cl_hemisphere(8, 4)
        nx, ny = 6, 5
    else:
        mu, eta, w = q.gl_slab(8)
        nx, ny = 11, 1
    n = nx * ny
    sig_s = rng.uniform(0.0, 3.0, n)
    p = _problem(nx, ny, mu, eta, w, sig_s + rng.uniform(0.1, 1.0, n), sig_s, c_dt=0.3,
                 lx=1.2, ly=0.8)
    T = _dense_T(p)
    cols = np.stack([tr.sweep(p, s_iso=np.eye(n)[c])[0] for c in range(n)], axis=1)
    assert np.max(np.abs(cols - T)) < 1e-14 * np.max(np.abs(T)) * 10
    rho = rng.uniform(0, 1, n)
    assert np.allclose(tr.apply_T_sigma_s(p, rho), T @ (p.sigma_s * rho), rtol=1e-13, atol=0)


@pytest.mark.parametrize("name", ["checkerboard", "slab"])
def test_particle_balance_exact(name, rng):
    """Summing the upwind cell equations over cells and directions telescopes the streaming
    terms into leakage minus inflow:
      sum_c A [tau (rho^ - rho^_old) + sigma_a rho^ - G] + leak - inflow = sum_c A sigma_s (rho - rho^)
    with rho^ the moment of the swept f and rho the scattering density fed to the sweep."""
    if name == "slab":
        wl = inputs.slab_1d(n=64)
    else:
        wl = inputs.checkerboard(n=24, quad=(16, 4))
    p = oracle_problem(wl)
    p.inflow = np.array([0.3, 0.1, 0.7, 0.2]) if p.dim == 2 else np.array([0.4, 0.9, 0, 0])
    n = p.ncell
    f_old = rng.uniform(0, 1, (p.nv, n))
    rho = rng.uniform(0, 2, n)
    f_new, mom = tr.final_f(p, rho, f_old)
    A = p.hx * (p.hy if p.dim == 2 else 1.0)
    rho_hat_old = p.w @ f_old
    sa = p.sigma_t - p.sigma_s
    lhs = np.sum(A * (p.tau * (mom - rho_hat_old) + sa * mom - p.source))
    F = f_new.reshape(p.nv, p.ny, p.nx)
    leak = inflow = 0.0
    for j in range(p.nv):
        ex = abs(p.mu[j]) * (p.hy if p.dim == 2 else 1.0)
        out_col = -1 if p.mu[j] > 0 else 0
        gx = p.inflow[0] if p.mu[j] > 0 else p.inflow[1]
        leak += p.w[j] * ex * np.sum(F[j][:, out_col])
        inflow += p.w[j] * ex * gx * p.ny
        if p.dim == 2:
            ey = abs(p.eta[j]) * p.hx
            out_row = -1 if p.eta[j] > 0 else 0
            gy = p.inflow[2] if p.eta[j] > 0 else p.inflow[3]
            leak += p.w[j] * ey * np.sum(F[j][out_row, :])
            inflow += p.w[j] * ey * gy * p.nx
    rhs = np.sum(A * p.sigma_s * (rho - mom))
    scale = np.sum(A * p.tau * (np.abs(mom) + np.abs(rho_hat_old))) + leak + inflow
    assert abs(lhs + leak - inflow - rhs) < 1e-13 * scale


def test_planted_wrong_upwind_side_is_caught():
    """A sweep that takes the downwind neighbour (a flipped direction) must fail the
    lattice-path pin: plant the mistake in the oracle's inputs and check the pin bites."""
    nx, ny, g = 6, 5, 1.0
    p = _problem(nx, ny, [-0.45], [0.62], [1.0], 0.8, c_dt=0.5, g=[g, 0, 0, 0])
    _, psi = tr.sweep(p, inflow=p.inflow, want_psi=True)   # sweeps east->west, west inflow unused
    a, b = 0.45 / p.hx, 0.62 / p.hy
    al = a / (p.tau + 0.8 + a + b)
    assert abs(psi[0].reshape(ny, nx)[0, 0] - g * al) > 1e-3
