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
The linear system is solved by conjugate gradients (Sec. 4 uses CG).
"""
import numpy as np
import scipy.sparse as sp


def dsa_matrix(p):
    """Assemble C as a scipy CSR matrix (SPD).  p: oracle.transport.Problem."""
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


def cg(A, b, rtol, max_iter):
    """Textbook conjugate gradients from x0 = 0; stops when ||r||_2 <= rtol ||b||_2.

    Returns (x, iterations).  The sparse matrix-vector product is the library step.
    """
    x = np.zeros_like(b)
    r = b.copy()
    bb = float(b @ b)
    rr = bb
    if bb == 0.0:
        return x, 0
    p = r.copy()
    it = 0
    while it < max_iter and rr > rtol * rtol * bb:
        Ap = A @ p
        alpha = rr / float(p @ Ap)
        x += alpha * p
        r -= alpha * Ap
        rr_new = float(r @ r)
        beta = rr_new / rr
        rr = rr_new
        p = r + beta * p
        it += 1
    return x, it


def dsa_correction(p, A, residual, rtol, max_iter):
    """delta_rho solving C delta_rho = Sigma_s (rho^{l-1/2} - rho^{l-1}) (Eq. (rho_residual))."""
    return cg(A, p.sigma_s * residual, rtol, max_iter)
