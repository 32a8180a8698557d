"""Pins of the oracle's Q1 upwind DG scheme (Sec. 2.1 Eq. (DG) with K = 1 in Eq. (dg_space))
and its interior-penalty DSA operator.

None of these re-types the oracle's closed-form 2 x 2 building blocks.  The independent side
evaluates the weak forms directly: basis functions and their gradients at Gauss points of
every cell and face, upwind values taken from whichever side the direction says, the
boundary data as a function on the face.  Pins:

* the sweep equals a dense solve of the weak form assembled by quadrature (random data);
* the scheme reproduces a bilinear exact solution (DG consistency: a continuous solution in
  the space satisfies the discrete equations, so the unique discrete solution is it);
* the pure-absorber solution converges to exp(-sigma s / |mu|) at second order;
* one SI-DSA time step equals a dense direct solve of the scattering problem;
* the DSA matrix equals the quadrature assembly of its bilinear form, is SPD on rough
  coefficient fields, and its solution converges at second order to a manufactured solution
  of the diffusion equation with the Marshak condition;
* SI-DSA contracts fast on an optically thick, highly scattering grid (the acceleration acts).
"""
import numpy as np
import pytest
from scipy.optimize import brentq

from oracle import dsa as ods
from oracle import quadrature as oq
from oracle import sisa as osisa
from oracle import stepper as ost
from oracle import transport as tr

R3 = np.sqrt(3.0)
GX, GWT = np.polynomial.legendre.leggauss(3)


def phi(k, xi, ze):
    """Basis k = a + 2 b at local coordinates (xi, zeta) of a cell: orthonormal under the cell
    average, p_0 = 1, p_1 = sqrt(3) t."""
    a, b = k & 1, k >> 1
    return (R3 * xi if a else 1.0) * (R3 * ze if b else 1.0)


def dphi(k, xi, ze, hx, hy):
    a, b = k & 1, k >> 1
    px, pxd = (R3 * xi, R3) if a else (1.0, 0.0)
    py, pyd = (R3 * ze, R3) if b else (1.0, 0.0)
    return (2.0 / hx) * pxd * py, (2.0 / hy) * px * pyd


def _problem(nx, ny, mu, eta, w, sig_t, sig_s=None, G=None, c_dt=0.1, lx=1.0, ly=1.0):
    n = nx * ny
    sig_t = np.broadcast_to(np.asarray(sig_t, float), (n,)).copy()
    sig_s = np.zeros(n) if sig_s is None else np.broadcast_to(np.asarray(sig_s, float), (n,)).copy()
    G = np.zeros(4 * n) if G is None else np.asarray(G, float)
    return tr.Problem(nx, ny, 0.0, lx, 0.0, ly, np.atleast_1d(mu), np.atleast_1d(eta),
                      np.atleast_1d(w), sig_t, sig_s, G, c_dt, np.zeros(4), degree=1)


# faces of a cell: (outward normal, the local coordinate that is fixed and its value)
FACES = (((-1.0, 0.0), "xi", -1.0), ((1.0, 0.0), "xi", 1.0),
         ((0.0, -1.0), "ze", -1.0), ((0.0, 1.0), "ze", 1.0))


def dense_transport(p, mu, eta, gfun=None):
    """Weak form of Eq. (DG) for one direction, tested with every basis function and divided
    by the cell area, assembled by Gauss quadrature.  Unknowns k ncell + c.  gfun(side, t):
    the inflow value at the face point t (the face's own coordinate in [-1, 1]) of boundary
    side 0 west / 1 east (t along y), 2 south / 3 north (t along x), row or column index
    passed as the side's third argument; None = vacuum.  Returns (A, boundary right side)."""
    nx, ny, nc = p.nx, p.ny, p.ncell
    A = np.zeros((4 * nc, 4 * nc))
    rb = np.zeros(4 * nc)
    for j in range(ny):
        for i in range(nx):
            c = i + nx * j
            for k in range(4):
                row = k * nc + c
                for qx, wx in zip(GX, GWT):
                    for qy, wy in zip(GX, GWT):
                        wq = wx * wy / 4.0
                        gxk, gyk = dphi(k, qx, qy, p.hx, p.hy)
                        for m in range(4):
                            fm = phi(m, qx, qy)
                            A[row, m * nc + c] += wq * ((p.tau + p.sigma_t[c]) * fm * phi(k, qx, qy)
                                                        - fm * (mu * gxk + eta * gyk))
                for (nxn, nyn), which, val in FACES:
                    on = mu * nxn + eta * nyn
                    h = p.hx if which == "xi" else p.hy
                    di, dj = int(nxn), int(nyn)
                    ni, nj = i + di, j + dj
                    inside = 0 <= ni < nx and 0 <= nj < ny
                    for t, wt in zip(GX, GWT):
                        xi, ze = (val, t) if which == "xi" else (t, val)
                        wf = wt / (2.0 * h)
                        pk = phi(k, xi, ze)
                        if on > 0:
                            for m in range(4):
                                A[row, m * nc + c] += on * wf * phi(m, xi, ze) * pk
                        elif inside:
                            nb = ni + nx * nj
                            # the same point in the neighbour's coordinates
                            xn, zn = (-xi, ze) if which == "xi" else (xi, -ze)
                            for m in range(4):
                                A[row, m * nc + nb] += on * wf * phi(m, xn, zn) * pk
                        elif on < 0 and gfun is not None:
                            side = (0 if nxn < 0 else 1) if which == "xi" else (2 if nyn < 0 else 3)
                            idx = j if which == "xi" else i
                            rb[row] -= on * wf * gfun(side, idx, t) * pk
    return A, rb


def _traces_from(gfun, nx, ny):
    """Face modes (average of g p_0 and g p_1 over the face) of a boundary function."""
    gx, gy = np.zeros((2, ny, 2)), np.zeros((2, nx, 2))
    for side in range(4):
        n = ny if side < 2 else nx
        for idx in range(n):
            m0 = sum(wt * gfun(side, idx, t) for t, wt in zip(GX, GWT)) / 2.0
            m1 = sum(wt * gfun(side, idx, t) * R3 * t for t, wt in zip(GX, GWT)) / 2.0
            (gx[side] if side < 2 else gy[side - 2])[idx] = (m0, m1)
    return gx, gy


def _linear_g(rng):
    coef = rng.uniform(0.2, 1.5, size=(4, 64, 2))
    return lambda side, idx, t: coef[side, idx, 0] + coef[side, idx, 1] * t


@pytest.mark.parametrize("seed", [0, 1])
def test_q1_sweep_equals_dense_weak_form(seed):
    rng = np.random.default_rng(seed)
    nx, ny = 5, 4
    mu = np.array([0.6, -0.35, 0.2, -0.8, 0.45, 0.0])
    eta = np.array([0.3, 0.7, -0.5, -0.15, 0.0, -0.9])
    w = rng.uniform(0.5, 1.5, mu.size)
    w /= w.sum()
    p = _problem(nx, ny, mu, eta, w, rng.uniform(0.2, 6.0, nx * ny), c_dt=0.3, lx=1.3, ly=0.9)
    s_iso = rng.normal(size=4 * p.ncell)
    s_dir = rng.normal(size=(mu.size, 4 * p.ncell))
    gfun = _linear_g(rng)
    mom, psi = tr.sweep(p, s_iso=s_iso, s_dir=s_dir, s_dir_scale=0.7, want_psi=True,
                        traces=_traces_from(gfun, nx, ny))
    want_mom = np.zeros(4 * p.ncell)
    for j in range(mu.size):
        A, rb = dense_transport(p, mu[j], eta[j], gfun)
        want = np.linalg.solve(A, s_iso + 0.7 * s_dir[j] + rb)
        assert np.max(np.abs(psi[j] - want)) <= 1e-12 * np.max(np.abs(want)), j
        want_mom += w[j] * want
    assert np.max(np.abs(mom - want_mom)) <= 1e-12 * np.max(np.abs(want_mom))


def _cell_projection(fun, p):
    """Degrees of freedom of fun(x, y) on every cell (cell average of fun phi_k, Gauss)."""
    out = np.zeros(4 * p.ncell)
    for j in range(p.ny):
        for i in range(p.nx):
            c = i + p.nx * j
            for k in range(4):
                s = 0.0
                for qx, wx in zip(GX, GWT):
                    for qy, wy in zip(GX, GWT):
                        x = p.x0 + (i + 0.5 + 0.5 * qx) * p.hx
                        y = p.y0 + (j + 0.5 + 0.5 * qy) * p.hy
                        s += wx * wy / 4.0 * fun(x, y) * phi(k, qx, qy)
                out[k * p.ncell + c] = s
    return out


def test_q1_reproduces_bilinear_solution():
    rng = np.random.default_rng(3)
    nx, ny = 6, 5
    mu = np.array([0.5, -0.6, 0.25, -0.3])
    eta = np.array([0.4, 0.2, -0.7, -0.55])
    w = np.full(4, 0.25)
    sig = rng.uniform(0.5, 4.0, nx * ny)
    p = _problem(nx, ny, mu, eta, w, sig, c_dt=0.5, lx=1.2, ly=0.8)
    coef = rng.uniform(-1.0, 2.0, size=(mu.size, 4))
    s_dir = np.zeros((mu.size, 4 * p.ncell))
    exact = np.zeros((mu.size, 4 * p.ncell))
    for j in range(mu.size):
        al, be, ga, de = coef[j]
        f = lambda x, y: al + be * x + ga * y + de * x * y
        exact[j] = _cell_projection(f, p)
        # source (tau + sigma_t) f + Omega . grad f, cell by cell (sigma_t constant per cell)
        tf = _cell_projection(lambda x, y: mu[j] * (be + de * y) + eta[j] * (ga + de * x), p)
        s_dir[j] = np.tile(p.tau + sig, 4) * exact[j] + tf
    for j in range(mu.size):
        al, be, ga, de = coef[j]
        f = lambda x, y: al + be * x + ga * y + de * x * y

        def gfun(side, idx, t):
            if side < 2:
                x = p.x0 if side == 0 else p.x1
                y = p.y0 + (idx + 0.5 + 0.5 * t) * p.hy
            else:
                y = p.y0 if side == 2 else p.y1
                x = p.x0 + (idx + 0.5 + 0.5 * t) * p.hx
            return f(x, y)

        q = _problem(nx, ny, [mu[j]], [eta[j]], [1.0], sig, c_dt=0.5, lx=1.2, ly=0.8)
        _, psi = tr.sweep(q, s_dir=s_dir[j:j + 1], want_psi=True, traces=_traces_from(gfun, nx, ny))
        assert np.max(np.abs(psi[0] - exact[j])) < 1e-12 * np.max(np.abs(exact[j])), j


def test_q1_pure_absorber_converges_at_second_order():
    """Steady pure absorber (tau -> 0) with unit inflow on the west face: the exact solution is
    exp(-sigma x / mu); the Q1 cell averages approach its cell averages at second order (a
    first-order scheme, a wrong face trace or a sign error would not)."""
    mu, sig = 0.5, 2.0
    errs = []
    for n in (8, 16, 32, 64):
        p = _problem(n, 2, [mu], [0.0], [1.0], sig, c_dt=1e14, ly=1.0)
        gx = np.zeros((2, 2, 2))
        gx[0, :, 0] = 1.0
        _, psi = tr.sweep(p, want_psi=True, traces=(gx, np.zeros((2, n, 2))))
        exact = _cell_projection(lambda x, y: np.exp(-sig * x / mu), p)
        errs.append(np.sqrt(np.mean((psi[0][:n] - exact[:n]) ** 2)))
    ratios = [errs[i] / errs[i + 1] for i in range(len(errs) - 1)]
    assert all(r > 3.5 for r in ratios), ratios


def dense_step(p, f_old):
    """One backward-Euler step of the Q1 scheme with scattering, as one dense system in all
    directions' unknowns: the quadrature-assembled transport blocks, minus Sigma_s times the
    quadrature moment on the diagonal blocks' mass term (cell average of sigma_s rho phi_k)."""
    nv, nd = p.nv, p.ndof
    A = np.zeros((nv * nd, nv * nd))
    b = np.zeros(nv * nd)
    gx, gy = tr.q1_traces(p, p.inflow)

    def gfun(side, idx, t):
        return (gx[side, idx, 0] if side < 2 else gy[side - 2, idx, 0])

    S = np.diag(p.sig_s_dof)
    for j in range(nv):
        Aj, rb = dense_transport(p, p.mu[j], p.eta[j], gfun)
        A[j * nd:(j + 1) * nd, j * nd:(j + 1) * nd] += Aj
        for k in range(nv):
            A[j * nd:(j + 1) * nd, k * nd:(k + 1) * nd] -= p.w[k] * S
        b[j * nd:(j + 1) * nd] = p.tau * f_old[j] + p.source + rb
    f = np.linalg.solve(A, b).reshape(nv, nd)
    return f, p.w @ f


def _scattering_problem(nx=4, ny=3, seed=5, inflow=(0.4, 0.0, 0.2, 0.1)):
    rng = np.random.default_rng(seed)
    mu, eta, w = oq.cl_hemisphere(4, 2)
    sig_t = rng.uniform(1.0, 8.0, nx * ny)
    sig_s = sig_t * rng.uniform(0.3, 0.95, nx * ny)
    G = np.zeros(4 * nx * ny)
    G[:nx * ny] = rng.uniform(0.0, 2.0, nx * ny)
    G[nx * ny:] = rng.normal(scale=0.2, size=3 * nx * ny)
    p = tr.Problem(nx, ny, 0.0, 1.0, 0.0, 0.8, mu, eta, w, sig_t, sig_s, G, 0.05,
                   np.asarray(inflow, float), degree=1)
    return p, rng


def test_q1_si_dsa_step_equals_dense_solve():
    p, rng = _scattering_problem()
    rho0 = rng.uniform(0.5, 1.5, p.ndof)
    f_old = np.tile(rho0, (p.nv, 1)) + rng.normal(scale=0.1, size=(p.nv, p.ndof))
    m = ost.OracleRTE(p, rom=False, eps_sisa=1e-13, cg_rtol=1e-12)
    m.set_initial(rho0, f_old)
    f_ref, rho_ref = dense_step(p, f_old)
    m.step(1)
    assert np.max(np.abs(m.rho - rho_ref)) < 1e-10 * np.max(np.abs(rho_ref))
    assert np.max(np.abs(m.f - f_ref)) < 1e-10 * np.max(np.abs(f_ref))


def test_q1_rom_march_keeps_the_dense_fixed_point():
    """Algorithm 2 with the ROMs on: every step still lands on the implicit step's solution."""
    p, rng = _scattering_problem(seed=7)
    rho0 = rng.uniform(0.5, 1.5, p.ndof)
    m = ost.OracleRTE(p, rom=True, eps_sisa=1e-12, cg_rtol=1e-12, eps_ig=1e-4, eps_pc=1e-3)
    m.set_initial(rho0)
    f = m.f.copy()
    for _ in range(12):
        f, rho = dense_step(p, f)
        m.step(1)
        assert np.max(np.abs(m.rho - rho)) < 1e-9 * np.max(np.abs(rho))
    assert m.phase() >= 2


# ---- DSA operator ---------------------------------------------------------------------------

def dense_dsa(p):
    """The interior-penalty bilinear form of oracle.dsa (Q1) assembled by Gauss quadrature from
    basis values and gradients: volume D grad u . grad v + sigma_a~ u v; interior faces
    kappa [u][v] - {D du/dn}[v] - [u]{D dv/dn}; boundary faces u v / 2; divided by the cell
    area."""
    nx, ny, nc = p.nx, p.ny, p.ncell
    D = 1.0 / (3.0 * (p.sigma_t + p.tau))
    sa = p.sigma_t - p.sigma_s + p.tau
    A = np.zeros((4 * nc, 4 * nc))
    for j in range(ny):
        for i in range(nx):
            c = i + nx * j
            for qx, wx in zip(GX, GWT):
                for qy, wy in zip(GX, GWT):
                    wq = wx * wy / 4.0
                    for k in range(4):
                        gk = dphi(k, qx, qy, p.hx, p.hy)
                        for m in range(4):
                            gm = dphi(m, qx, qy, p.hx, p.hy)
                            A[k * nc + c, m * nc + c] += wq * (
                                D[c] * (gk[0] * gm[0] + gk[1] * gm[1])
                                + sa[c] * phi(k, qx, qy) * phi(m, qx, qy))
            # faces on the high x / high y side of the cell (each interior face once)
            for axis in ("x", "y"):
                h = p.hx if axis == "x" else p.hy
                hi_in = (i + 1 < nx) if axis == "x" else (j + 1 < ny)
                lo_bd = (i == 0) if axis == "x" else (j == 0)
                for t, wt in zip(GX, GWT):
                    wf = wt / (2.0 * h)
                    if axis == "x":
                        pl, pr = (1.0, t), (-1.0, t)
                    else:
                        pl, pr = (t, 1.0), (t, -1.0)
                    n_idx = 0 if axis == "x" else 1
                    if lo_bd:
                        plo = (-1.0, t) if axis == "x" else (t, -1.0)
                        for k in range(4):
                            for m in range(4):
                                A[k * nc + c, m * nc + c] += wf * 0.5 * phi(k, *plo) * phi(m, *plo)
                    if not hi_in:
                        for k in range(4):
                            for m in range(4):
                                A[k * nc + c, m * nc + c] += wf * 0.5 * phi(k, *pl) * phi(m, *pl)
                        continue
                    r = c + 1 if axis == "x" else c + nx
                    kap = max(2.0 * (D[c] + D[r]) / h, 0.25)
                    cells = ((c, pl, +1.0), (r, pr, -1.0))   # (cell, face point, jump sign)
                    for ct, ptt, st in cells:          # test function side
                        for cu, ptu, su in cells:      # trial function side
                            for k in range(4):
                                vk = phi(k, *ptt)
                                dvk = D[ct] * dphi(k, *ptt, p.hx, p.hy)[n_idx]
                                for m in range(4):
                                    um = phi(m, *ptu)
                                    dum = D[cu] * dphi(m, *ptu, p.hx, p.hy)[n_idx]
                                    v = kap * (su * um) * (st * vk)
                                    v -= 0.5 * dum * (st * vk)
                                    v -= (su * um) * 0.5 * dvk
                                    A[k * nc + ct, m * nc + cu] += wf * v
    return A


def test_q1_dsa_matrix_equals_quadrature_assembly():
    rng = np.random.default_rng(11)
    nx, ny = 4, 3
    sig_t = np.exp(rng.normal(1.0, 1.2, nx * ny))
    sig_s = sig_t * rng.uniform(0.2, 0.99, nx * ny)
    p = _problem(nx, ny, [0.5], [0.5], [1.0], sig_t, sig_s, c_dt=0.07, lx=1.1, ly=0.7)
    C = ods.dsa_matrix(p).toarray()
    want = dense_dsa(p)
    assert np.max(np.abs(C - want)) <= 1e-12 * np.max(np.abs(want))


@pytest.mark.parametrize("seed,scale", [(0, 0.1), (1, 1.0), (2, 30.0), (3, 400.0)])
def test_q1_dsa_matrix_is_spd(seed, scale):
    rng = np.random.default_rng(seed)
    nx, ny = 7, 6
    sig_t = scale * np.exp(rng.normal(0.0, 1.5, nx * ny))
    sig_s = sig_t * rng.uniform(0.0, 0.9999, nx * ny)
    p = _problem(nx, ny, [0.5], [0.5], [1.0], sig_t, sig_s, c_dt=1e3)
    C = ods.dsa_matrix(p).toarray()
    assert np.max(np.abs(C - C.T)) <= 1e-13 * np.max(np.abs(C))
    assert np.linalg.eigvalsh(C).min() > 0.0


def test_q1_dsa_converges_to_marshak_diffusion_solution():
    """-D Lap u + sigma_a u = R on the unit square with -D du/dn = u / 2 on every side:
    u = X(x) X(y), X = cos(k (t - 1/2)) with k tan(k / 2) = 1 / (2 D).  The DG solution's error
    against the cell projection of u falls at (at least) second order."""
    sig_t, sig_s = 2.0, 1.5
    D = 1.0 / (3.0 * sig_t)
    kk = brentq(lambda k: k * np.tan(k / 2.0) - 1.0 / (2.0 * D), 1e-6, np.pi - 1e-9)
    u = lambda x, y: np.cos(kk * (x - 0.5)) * np.cos(kk * (y - 0.5))
    sa = sig_t - sig_s
    errs = []
    for n in (4, 8, 16, 32):
        p = _problem(n, n, [0.5], [0.5], [1.0], sig_t, sig_s, c_dt=1e15)
        C = ods.dsa_matrix(p)
        R = _cell_projection(lambda x, y: (2.0 * D * kk ** 2 + sa) * u(x, y), p)
        from scipy.sparse.linalg import spsolve
        uh = spsolve(C.tocsc(), R)
        e = uh - _cell_projection(u, p)
        errs.append(np.sqrt(np.sum(e ** 2) / p.ncell))
    ratios = [errs[i] / errs[i + 1] for i in range(len(errs) - 1)]
    assert all(r > 3.5 for r in ratios), ratios


def test_q1_si_dsa_contracts_on_thick_scattering_grid():
    """sigma_t h = 5, scattering ratio 0.999: unaccelerated source iteration would contract by
    about 0.999 per sweep; with the DSA step a few iterations reach 1e-10."""
    n = 12
    mu = np.array([0.5, -0.5, 0.5, -0.5, 0.2, -0.2, 0.2, -0.2, 0.85, -0.85, 0.85, -0.85])
    eta = np.array([0.5, 0.5, -0.5, -0.5, 0.8, 0.8, -0.8, -0.8, 0.3, 0.3, -0.3, -0.3])
    w = np.full(mu.size, 1.0 / mu.size)
    sig_t = np.full(n * n, 60.0)
    p = _problem(n, n, mu, eta, w, sig_t, 0.999 * sig_t, c_dt=1e3)
    rng = np.random.default_rng(2)
    bt = rng.uniform(0.0, 1.0, p.ndof)
    opts = dict(ost.DEFAULTS)
    opts.update(eps_sisa=1e-10, cg_rtol=1e-12)
    _, info = osisa.si_sa(p, np.zeros(p.ndof), bt, opts, ods.dsa_matrix(p))
    assert info.iterations <= 25, info.iterations


def test_q1_dsa_preconditioned_cg():
    """The Q1 DSA solve is CG preconditioned by the diagonal of C: it reaches the direct solve's
    answer, in fewer iterations than plain CG on a rough field, and with M = I it is plain CG
    iterate for iterate."""
    from scipy.sparse.linalg import spsolve
    rng = np.random.default_rng(21)
    nx, ny = 20, 18
    sig_t = np.exp(rng.normal(1.5, 1.5, nx * ny))
    p = _problem(nx, ny, [0.5], [0.5], [1.0], sig_t, sig_t * rng.uniform(0.5, 0.999, nx * ny),
                 c_dt=0.5)
    A = ods.dsa_matrix(p)
    b = rng.normal(size=p.ndof)
    x_direct = spsolve(A.tocsc(), b)
    m_inv = ods.preconditioner(p, A)
    assert np.array_equal(m_inv, 1.0 / A.diagonal())
    x, its = ods.cg(A, b, 1e-12, 5000, m_inv)
    assert np.linalg.norm(x - x_direct) <= 1e-9 * np.linalg.norm(x_direct)
    x0, its0 = ods.cg(A, b, 1e-12, 5000)
    assert its < its0, (its, its0)
    x1, its1 = ods.cg(A, b, 1e-12, 5000, np.ones(p.ndof))
    assert its1 == its0 and np.array_equal(x1, x0)
