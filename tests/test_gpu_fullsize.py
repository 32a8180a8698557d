"""Parity at the full sizes of the 1024^2 log-normal (1.34e8 cell-directions) and 2048^2
diffusive-disc (1.07e9) workloads.

One SI sweep T Sigma_s rho (the hot path's dominant kernel, in the tile the autotuner picks for
that size) against the oracle's sweep of the same rho, every output: the oracle sweeps these
sizes in seconds.  A whole march at these sizes it cannot follow; there the check is a
property that holds at any size:

Particle balance of the fused f sweep.  f^n solves the discrete transport equation of the step,
(tau + sigma_t + a_k + b_k) f^n_k = sigma_s rho^n + G + tau f^{n-1}_k + a_k f_up,x + b_k f_up,y,
so weighting by w_k and summing over directions and cells telescopes the streaming terms to the
outflow through the boundary (vacuum inflow) and leaves, exactly up to rounding,

    sum_c [tau (F^n - F^{n-1}) + sigma_t F^n - sigma_s rho^n - G]
        + sum_k w_k (|mu_k| / h_x  sum_rows f^n_k(x-outflow cell)
                     + |eta_k| / h_y sum_cols f^n_k(y-outflow cell)) = 0,

with F = sum_k w_k f_k.  The check covers the sweep's whole data path at this size (families,
row blocks, CTA hand-offs, the stored f and its layout) for both precisions."""
import numpy as np
import pytest

from conftest import oracle_problem
from gpu_util import match_directions, max_rel, rel_l2
from oracle import dsa, rom
from oracle import transport as tr
from paper_2603_19647_gb300 import inputs, rte

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name,precision,tol", [("lognormal", rte.RTE_FP64, 1e-12),
                                                ("lognormal", rte.RTE_FP32, 2e-6),
                                                ("diffusive_disc", rte.RTE_FP32, 2e-6),
                                                ("diffusive_disc", rte.RTE_FP32_BF16F, 2e-6)])
def test_si_sweep_full_size(name, precision, tol):
    wl = inputs.BY_NAME[name]()
    h = rte.create_from_workload(wl, options=rte.default_options(precision=precision))
    rho = np.random.default_rng(7).uniform(0.0, 1.0, wl.ncell)
    got = h.rte_op_sweep(rho)
    h.destroy()
    ref = tr.apply_T_sigma_s(oracle_problem(wl), rho)
    assert rel_l2(got, ref) < tol
    assert max_rel(got, ref) < 10 * tol   # every cell, not only the norm


@pytest.mark.parametrize("precision,tol", [(rte.RTE_FP64, 1e-12), (rte.RTE_FP32, 2e-6)])
def test_fused_sweep_full_size(precision, tol):
    """The fused f sweep (f^n in place, then b~ from f^n) at 1024^2 x 128 against the oracle's,
    from a random f^{n-1}, with isotropic inflow on every side."""
    wl = inputs.lognormal()
    rng = np.random.default_rng(11)
    h = rte.create_from_workload(wl, options=rte.default_options(precision=precision))
    p = oracle_problem(wl)
    perm, _, _ = match_directions(h, wl.quadrature)
    f0 = rng.uniform(0.0, 1.0, (p.nv, wl.ncell))
    h.rte_set_initial(f0=f0[perm])
    g = np.array([0.7, 0.2, 0.4, 1.1])
    h.rte_set_inflow(g)
    p.inflow = g
    rho = rng.uniform(0.0, 1.0, wl.ncell)
    bt = h.rte_op_fsweep(rho)
    f_lib = h.rte_get_angular_flux()
    h.destroy()
    f_ref, _ = tr.final_f(p, rho, f0)
    assert rel_l2(f_lib, f_ref[perm]) < tol
    assert rel_l2(bt, tr.b_tilde(p, f_ref)) < tol
    assert max_rel(f_lib, f_ref[perm]) < 10 * tol   # every cell-direction
    assert max_rel(bt, tr.b_tilde(p, f_ref)) < 10 * tol


def test_dsa_full_size():
    """The DSA solve at 1024^2 (the two-phase CG above 2^18 cells) against the oracle's CG:
    the same iteration count and the correction within 1e-10."""
    wl = inputs.lognormal()
    h = rte.create_from_workload(wl, options=rte.default_options(cg_rtol=1e-8))
    p = oracle_problem(wl)
    res = np.random.default_rng(5).uniform(-1.0, 1.0, wl.ncell)
    got, its = h.rte_op_dsa(res)
    h.destroy()
    ref, its_ref = dsa.dsa_correction(p, dsa.dsa_matrix(p), res, 1e-8, 500)
    assert its == its_ref
    assert rel_l2(got, ref) < 1e-10


def test_rom_full_size():
    """Incremental SVD appends and the ROM apply on 1024^2-cell snapshots (the tall-skinny
    products at full length) against the oracle's iSVD."""
    wl = inputs.lognormal()
    n = wl.ncell
    h = rte.create_from_workload(wl, options=rte.default_options(r_max=12))
    rng = np.random.default_rng(13)
    X, Y = np.meshgrid(np.linspace(0, 1, wl.nx), np.linspace(0, 1, wl.ny))
    o = rom.IncrementalSVD(n, 12)
    for k in range(8):
        x = (np.exp(-((X - 0.2 - 0.05 * k) ** 2 + (Y - 0.5) ** 2) / 0.02) * (1 + 0.05 * k)).ravel()
        x = x + 1e-4 * rng.standard_normal(n)
        b = x + 0.1 * np.roll(x, 3) + 1e-3 * rng.standard_normal(n)
        assert h.rte_op_rom_append(rte.RTE_ROM_IG, x, b, -1.0) == o.append(x, b, trunc_eps=None)
    S, _, _ = h.rte_op_rom_get(rte.RTE_ROM_IG)
    assert np.max(np.abs(S - o.S) / o.S) < 1e-10
    rhs = b + 0.01 * rng.standard_normal(n)
    assert rel_l2(h.rte_op_rom_apply(rte.RTE_ROM_IG, rhs), o.solve_apply(rhs)) < 1e-9
    h.destroy()


def _balance(wl, quad, f_prev, f_now, rho_now):
    mu, eta, w = quad
    nx, ny = wl.nx, wl.ny
    x0, x1, y0, y1 = wl.domain
    hx, hy = (x1 - x0) / nx, (y1 - y0) / ny
    tau = 1.0 / wl.c_dt
    F_prev, F_now = w @ f_prev, w @ f_now
    body = tau * (F_now - F_prev) + wl.sigma_t * F_now - wl.sigma_s * rho_now - wl.source
    fn = f_now.reshape(len(w), ny, nx)
    leak = 0.0
    for k in range(len(w)):
        col = fn[k, :, -1] if mu[k] > 0 else fn[k, :, 0]
        row = fn[k, -1, :] if eta[k] > 0 else fn[k, 0, :]
        leak += w[k] * (abs(mu[k]) / hx * col.sum() + abs(eta[k]) / hy * row.sum())
    scale = np.sum((tau + wl.sigma_t) * np.abs(F_now))
    return (body.sum() + leak) / scale


@pytest.mark.parametrize("precision,tol", [(rte.RTE_FP64, 1e-12), (rte.RTE_FP32, 2e-6)])
def test_lognormal_full_size_particle_balance(precision, tol):
    wl = inputs.lognormal()
    h = rte.create_from_workload(wl, options=rte.default_options(precision=precision))
    h.rte_set_initial(rho0=wl.rho0)
    h.rte_step(2)
    f_prev = h.rte_get_angular_flux()
    h.rte_step(1)
    f_now = h.rte_get_angular_flux()
    rho_now = h.rte_get_scalar_flux()
    quad = h.rte_get_quadrature()
    h.destroy()
    assert np.all(np.isfinite(f_now))
    assert abs(_balance(wl, quad, f_prev, f_now, rho_now)) < tol
