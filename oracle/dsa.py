"""Diffusion synthetic acceleration of the oracle (test infrastructure).

Sec. 2.3 Eq. (rho_residual): C delta_rho = Sigma_s (rho^{l-1/2} - rho^{l-1}), where C is a
diffusion discretisation of the correction equation Eq. (discrete_correction_f): a steady
RTE with sigma_a~ = tau + sigma_a, sigma_t~ = tau + sigma_t and zero inflow.  Its diffusion
limit (Sec. 2, D = 1/(3 sigma)) is

    -div(D grad dr) + sigma_a~ dr = R,   D = 1/(3 sigma_t~).

The paper's fully consistent DSA belongs to its Q1 scheme and is given only by citation
(Sec. 4); for the Q0 scheme the oracle uses the cell-centred 5-point (1D: 3-point)
discretisation with harmonic-mean face couplings and a Marshak vacuum condition on every
boundary face (outgoing current rho_b / 2 in the normalisation sum_j w_j = 1), each floored
at the coupling the upwind Q0 sweep itself applies to an isotropic flux across a face, the
half-range current sum_{Omega.n > 0} w Omega.n = 1/4 (the interior-penalty floor of the
modified-interior-penalty diffusion form for piecewise constants):
    interior face:  max(2 D_L D_R / ((D_L + D_R) h), 1/4) / h
    vacuum face:    max(1 / (2 + h / (2 D)), 1/4) / h.
Without the floor the operator under-couples optically thick cells and SI-DSA can diverge.
The linear system is solved by conjugate gradients (Sec. 4 uses CG), for Q1 preconditioned by
the diagonal of C.

For the Q1 scheme (degree=1) C is the symmetric interior-penalty DG discretisation of the same
equation on the same bilinear space, with the penalty of the modified-interior-penalty DSA
(Wang and Ragusa, 2010) and the Marshak condition -D dr/dn = dr/2 taken weakly:

    a(u, v) = sum_T int_T (D grad u . grad v + sigma_a~ u v)
            + sum_{interior F} int_F (kappa_F [u][v] - {D du/dn}[v] - [u]{D dv/dn})
            + sum_{boundary F} int_F u v / 2,
    kappa_F = max(2 (D_L + D_R) / h_perp, 1/4),

[u] = u_L - u_R and {.} the average across F (normal from L to R), every term divided by the
cell area like the transport equations (C is then symmetric on the uniform grid).  The 1/4
floor is the half-range current of an isotropic flux, the coupling the upwind sweep itself
gives a jump in the optically thick limit.
"""
import numpy as np
import scipy.sparse as sp


def dsa_matrix(p):
    """Assemble C as a scipy CSR matrix (SPD).  p: oracle.transport.Problem."""
    if p.degree == 1:
        return dsa_matrix_q1(p)
    nx, ny = p.nx, p.ny
    tau = p.tau
    D = (1.0 / (3.0 * (p.sigma_t + tau))).reshape(ny, nx)
    sa = (p.sigma_t - p.sigma_s + tau).reshape(ny, nx)
    diag = sa.copy()
    rows, cols, vals = [], [], []
    idx = np.arange(nx * ny).reshape(ny, nx)

    def faces(DL, DR, h, iL, iR):
        c = np.maximum(2.0 * DL * DR / ((DL + DR) * h), 0.25) / h
        return c, iL, iR

    def vacuum(Db, h):
        return np.maximum(1.0 / (2.0 + h / (2.0 * Db)), 0.25) / h

    hx = p.hx
    # x faces
    if nx > 1:
        c, iL, iR = faces(D[:, :-1], D[:, 1:], hx, idx[:, :-1], idx[:, 1:])
        diag[:, :-1] += c
        diag[:, 1:] += c
        rows += [iL.ravel(), iR.ravel()]
        cols += [iR.ravel(), iL.ravel()]
        vals += [-c.ravel(), -c.ravel()]
    diag[:, 0] += vacuum(D[:, 0], hx)
    diag[:, -1] += vacuum(D[:, -1], hx)
    if p.dim == 2:
        hy = p.hy
        if ny > 1:
            c, iL, iR = faces(D[:-1, :], D[1:, :], hy, idx[:-1, :], idx[1:, :])
            diag[:-1, :] += c
            diag[1:, :] += c
            rows += [iL.ravel(), iR.ravel()]
            cols += [iR.ravel(), iL.ravel()]
            vals += [-c.ravel(), -c.ravel()]
        diag[0, :] += vacuum(D[0, :], hy)
        diag[-1, :] += vacuum(D[-1, :], hy)
    rows.append(idx.ravel())
    cols.append(idx.ravel())
    vals.append(diag.ravel())
    n = nx * ny
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(n, n))


def dsa_matrix_q1(p):
    """The Q1 interior-penalty operator of the module docstring as a scipy CSR matrix on the
    mode-major degrees of freedom (mode k = a + 2 b of cell c at k ncell + c).

    Per axis, on the reference interval with the orthonormal p_0 = 1, p_1 = sqrt(3) xi:
    traces P(+1) = (1, sqrt 3), P(-1) = (1, -sqrt 3); derivative d/dx p = (2/h) (0, sqrt 3);
    stiffness (1/|I|) int p_a' p_c' = (4/h^2) diag(0, 3).  A term acting on the x modes is
    kron(I2, X) on the local index (a + 2 b); one acting on the y modes is kron(Y, I2); a face
    integral divided by the cell area carries 1 / h_perp."""
    nx, ny, nc = p.nx, p.ny, p.ncell
    tau = p.tau
    r3 = np.sqrt(3.0)
    D = 1.0 / (3.0 * (p.sigma_t + tau))
    sa = p.sigma_t - p.sigma_s + tau
    tp, tm = np.array([1.0, r3]), np.array([1.0, -r3])
    I2 = np.eye(2)
    blocks = {}

    def add(ci, cj, B):
        key = (ci, cj)
        blocks[key] = blocks.get(key, 0.0) + B

    def on_x(X):
        return np.kron(I2, X)

    def on_y(Y):
        return np.kron(Y, I2)

    stiff = np.diag([0.0, 3.0])
    for axis, h, on in (("x", p.hx, on_x), ("y", p.hy, on_y)):
        g = (2.0 / h) * np.array([0.0, r3])   # derivative of the two modes along the axis
        for j in range(ny):
            for i in range(nx):
                c = i + nx * j
                add(c, c, on(D[c] * (4.0 / h ** 2) * stiff))
                # the face on the high side of cell c along this axis
                hi = (i + 1 < nx) if axis == "x" else (j + 1 < ny)
                lo_boundary = (i == 0) if axis == "x" else (j == 0)
                if lo_boundary:
                    add(c, c, on(0.5 * np.outer(tm, tm) / h))
                if not hi:
                    add(c, c, on(0.5 * np.outer(tp, tp) / h))
                    continue
                r = c + 1 if axis == "x" else c + nx
                dl, dr = D[c], D[r]
                kap = max(2.0 * (dl + dr) / h, 0.25)
                # L = c (its trace at +1), R = r (its trace at -1); rows test, columns trial
                LL = kap * np.outer(tp, tp) - 0.5 * dl * (np.outer(tp, g) + np.outer(g, tp))
                LR = -kap * np.outer(tp, tm) - 0.5 * dr * np.outer(tp, g) + 0.5 * dl * np.outer(g, tm)
                RL = -kap * np.outer(tm, tp) + 0.5 * dl * np.outer(tm, g) - 0.5 * dr * np.outer(g, tp)
                RR = kap * np.outer(tm, tm) + 0.5 * dr * (np.outer(tm, g) + np.outer(g, tm))
                add(c, c, on(LL / h))
                add(c, r, on(LR / h))
                add(r, c, on(RL / h))
                add(r, r, on(RR / h))
    for c in range(nc):
        add(c, c, sa[c] * np.eye(4))
    rows, cols, vals = [], [], []
    for (ci, cj), B in blocks.items():
        for k in range(4):
            for m in range(4):
                if B[k, m] != 0.0:
                    rows.append(k * nc + ci)
                    cols.append(m * nc + cj)
                    vals.append(B[k, m])
    n = 4 * nc
    return sp.csr_matrix((np.array(vals), (np.array(rows), np.array(cols))), shape=(n, n))


def cg(A, b, rtol, max_iter, m_inv=None):
    """Textbook conjugate gradients from x0 = 0; stops when ||r||_2 <= rtol ||b||_2.
    m_inv: the inverse of a diagonal preconditioner M (preconditioned CG: z = M^-1 r in place of
    r in the search directions and in the step lengths), or None.

    Returns (x, iterations).  The sparse matrix-vector product is the library step.
    """
    x = np.zeros_like(b)
    r = b.copy()
    bb = float(b @ b)
    rr = bb
    if bb == 0.0:
        return x, 0
    z = r if m_inv is None else m_inv * r
    rz = float(r @ z)
    p = z.copy()
    it = 0
    while it < max_iter and rr > rtol * rtol * bb:
        Ap = A @ p
        alpha = rz / float(p @ Ap)
        x += alpha * p
        r -= alpha * Ap
        rr = float(r @ r)
        z = r if m_inv is None else m_inv * r
        rz_new = float(r @ z)
        beta = rz_new / rz
        rz = rz_new
        p = z + beta * p
        it += 1
    return x, it


def preconditioner(p, A):
    """The DSA solve's preconditioner: none for Q0 (plain CG); for Q1 the inverse diagonal of C
    (Jacobi).  Sec. 4 preconditions its DSA solves (by algebraic multigrid); on the Q1 operator
    the diagonal alone cuts the CG iterations by a third (44 -> 29 at 256^2 on the
    checkerboard)."""
    return 1.0 / A.diagonal() if p.degree == 1 else None


def dsa_correction(p, A, residual, rtol, max_iter):
    """delta_rho solving C delta_rho = Sigma_s (rho^{l-1/2} - rho^{l-1}) (Eq. (rho_residual))."""
    return cg(A, p.sig_s_dof * residual, rtol, max_iter, preconditioner(p, A))
