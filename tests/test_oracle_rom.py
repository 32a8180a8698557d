"""Pins of the oracle's incremental SVD (App. B), DMD operators (Sec. 3.1) and the ROM
phases of Algorithm 2 against full SVDs, exact data and ROM-off runs."""
import numpy as np
import pytest

from oracle import quadrature as q
from oracle import dsa, rom, sisa, stepper
from oracle import transport as tr


def _snapshots(rng, n=400, m=14):
    x = np.linspace(0, 1, n)
    cols = [np.exp(-(x - 0.2 - 0.04 * k) ** 2 / 0.01) * (1 + 0.1 * k) + 1e-3 * rng.standard_normal(n)
            for k in range(m)]
    return np.stack(cols, axis=1)


def test_isvd_matches_full_svd(rng):
    R = _snapshots(rng)
    B = rng.standard_normal(R.shape)
    s = rom.IncrementalSVD(R.shape[0], r_max=40)
    for k in range(R.shape[1]):
        assert s.append(R[:, k], B[:, k])
    U, S, Vt = np.linalg.svd(R, full_matrices=False)
    assert np.max(np.abs(s.S - S) / S) < 1e-10
    assert np.max(np.abs(s.U.T @ s.U - np.eye(s.rank))) < 1e-12
    # principal angles between the subspaces
    cosines = np.linalg.svd(U.T @ s.U, compute_uv=False)
    assert np.min(cosines) > 1 - 1e-10
    # W = B V, hence A_r = U^T B V S^{-1}
    sg = np.sign(np.sum(U * s.U, axis=0))[None, :]
    Ui, Vi = U * sg, Vt.T * sg
    assert np.max(np.abs(s.U - Ui)) < 1e-10
    assert np.allclose(s.W, B @ Vi, rtol=0, atol=1e-8 * np.max(np.abs(B)))
    Ar = Ui.T @ B @ Vi / S[None, :]
    assert np.max(np.abs(s.operator() - Ar)) < 1e-9 * np.max(np.abs(Ar))


def test_dmd_operator_is_galerkin_projection_for_exact_data(rng):
    """With B = A~ R exactly and R of full column rank, U^T B V S^{-1} = U^T A~ U."""
    mu, eta, w = q.cl_hemisphere(8, 4)
    n = 30
    ss = rng.uniform(0, 5, n)
    p = tr.Problem(6, 5, 0, 1, 0, 1, mu, eta, w, ss + 0.5, ss, np.zeros(n), 0.2, np.zeros(4))
    T = np.stack([tr.apply_T_sigma_s(p, e) for e in np.eye(n)], axis=1)
    At = np.eye(n) - T
    R = rng.standard_normal((n, 9))
    s = rom.IncrementalSVD(n, 40)
    for k in range(9):
        s.append(R[:, k], At @ R[:, k])
    assert np.allclose(s.operator(), s.U.T @ At @ s.U, atol=1e-12)
    rho = R @ rng.standard_normal(9)              # a state inside span U
    assert np.allclose(s.solve_apply(At @ rho), rho, rtol=0, atol=1e-11 * np.linalg.norm(rho))


def test_rank_guard_and_stop_ratio(rng):
    R = rng.standard_normal((200, 3))
    s = rom.IncrementalSVD(200, 40)
    for k in range(3):
        assert s.append(R[:, k], R[:, k])
        assert s.stop_ratio(True) > 0
    grew = s.append(R @ np.array([0.3, -1.0, 2.0]), np.zeros(200))
    assert not grew and s.rank == 3 and s.stop_ratio(grew) == 0.0
    U, S, _ = np.linalg.svd(np.hstack([R, (R @ np.array([0.3, -1.0, 2.0]))[:, None]]),
                            full_matrices=False)
    assert np.allclose(s.S, S[:3], rtol=1e-12)


def test_truncation_and_cap(rng):
    R = _snapshots(rng, m=20)
    s = rom.IncrementalSVD(R.shape[0], r_max=6)
    for k in range(20):
        s.append(R[:, k], R[:, k], trunc_eps=1e-3)
    assert s.rank <= 6
    assert np.all(s.S / s.S.sum() > 1e-3)
    assert np.all(np.diff(s.S) <= 0)


@pytest.mark.parametrize("dim", [2])
def test_rom_march_invariance_and_phases(dim):
    """ROM on and off reach the same states within the solver tolerance (Sec. 4 reports
    1e-9 to 1e-16 differences) and the ROM phases advance to Phase 3."""
    mu, eta, w = q.cl_hemisphere(16, 4)
    n = 16
    X, Y = np.meshgrid((np.arange(n) + .5) / n, (np.arange(n) + .5) / n)
    ss = np.where(X < 0.5, 40.0, 2.0).ravel()
    G = np.exp(-((X - .5) ** 2 + (Y - .5) ** 2) / 0.02).ravel()
    mk = lambda: tr.Problem(n, n, 0, 1, 0, 1, mu, eta, w, ss + 0.1, ss, G, 0.02, np.zeros(4))
    runs = {}
    for rom_on in (False, True):
        r = stepper.OracleRTE(mk(), eps_sisa=1e-12, rom=rom_on, cg_rtol=1e-8, eps_ig=1e-8,
                              eps_pc=1e-6, eps_up=1e-9)
        r.set_initial(np.zeros(n * n))
        r.step(40)
        runs[rom_on] = r
    a, b = runs[False].rho, runs[True].rho
    assert np.linalg.norm(a - b) <= 1e-9 * np.linalg.norm(a)
    log = runs[True].log
    assert {s.phase for s in log} >= {1, 2}
    it_rom = np.mean([s.iterations for s in log[-10:]])
    it_plain = np.mean([s.iterations for s in runs[False].log[-10:]])
    assert it_rom < it_plain


def test_rom_pc_exact_when_correction_in_span(rng):
    """Eq. (dmd-sa) with exact data.  With K = T Sigma_s, rho^{1/2} = K rho^{(0)} + b~ and the
    fixed point rho^n = K rho^n + b~, the step's error e = rho^n - rho^{(0)} gives the ideal
    first correction delta = rho^n - rho^{1/2} = K e and the right side of the correction
    equation rho^{1/2} - rho^{(0)} = e - K e.  A PC-ROM built from the pairs (K e_k, e_k - K e_k)
    represents the correction operator exactly on span{K e_k}; when e lies in span{e_k} the
    l = 1 correction lands on rho^n and the second sweep meets a 1e-12 test.  DSA from the same
    guess takes more sweeps, and a planted sign error in the correction is caught."""
    mu, eta, w = q.cl_hemisphere(8, 4)
    nx, ny = 6, 5
    n = nx * ny
    ss = rng.uniform(0.0, 20.0, n)
    p = tr.Problem(nx, ny, 0, 1, 0, 0.8, mu, eta, w, ss + rng.uniform(0.05, 1.0, n), ss,
                   rng.uniform(0, 1, n), 0.05, np.array([0.3, 0.0, 0.5, 0.1]))
    K = lambda v: tr.apply_T_sigma_s(p, v)
    bt = tr.b_tilde(p, rng.uniform(0, 1, (p.nv, n)))
    Kmat = np.stack([K(e) for e in np.eye(n)], axis=1)
    rho_n = np.linalg.solve(np.eye(n) - Kmat, bt)
    E = rng.standard_normal((n, 6))
    pc = rom.IncrementalSVD(n, 40)
    for k in range(E.shape[1]):
        assert pc.append(K(E[:, k]), E[:, k] - K(E[:, k]))
    e = E @ rng.standard_normal(E.shape[1])
    rho0 = rho_n - e
    opts = dict(stepper.DEFAULTS, eps_sisa=1e-12, cg_rtol=1e-10)
    A = dsa.dsa_matrix(p)
    got, info = sisa.si_sa(p, rho0, bt, opts, A, pc=pc.solve_apply)
    assert info.iterations == 2
    assert np.linalg.norm(info.delta_pc_1 - K(e)) <= 1e-10 * np.linalg.norm(K(e))
    assert np.linalg.norm(got - rho_n) <= 1e-11 * np.linalg.norm(rho_n)
    _, info_dsa = sisa.si_sa(p, rho0, bt, opts, A)
    assert info_dsa.iterations > 2
    _, info_bad = sisa.si_sa(p, rho0, bt, opts, A, pc=lambda r: -pc.solve_apply(r))
    assert info_bad.iterations > 2
