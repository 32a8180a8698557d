"""Direct solve of one implicit step on tiny grids (test infrastructure).

Assembles Eq. (kinetic_dg_discrete) for the Q0 scheme as one dense linear system in all
unknowns f_j (j = 1..N_v) and solves it with LU (numpy.linalg.solve):

    (tau + sigma_t + a_j + b_j) f_j[c] - a_j f_j[upx(c)] - b_j f_j[upy(c)]
        - sigma_s[c] sum_k w_k f_k[c] = tau f_j^{n-1}[c] + G[c] + g_j^bc[c],

where upx / upy are the upwind neighbours for Omega_j and g_j^bc[c] = a_j g_x + b_j g_y on
inflow-boundary cells (Sec. 2.1 Eq. (DG), upwind flux; K = 0).  This never sweeps, so it
pins the sweep-based solvers from outside.
"""
import numpy as np


def assemble(p):
    nx, ny, nv = p.nx, p.ny, p.nv
    nc = nx * ny
    N = nv * nc
    A = np.zeros((N, N))
    for j in range(nv):
        a = abs(p.mu[j]) / p.hx
        b = abs(p.eta[j]) / p.hy if p.dim == 2 else 0.0
        sx = 1 if p.mu[j] > 0 else -1
        sy = 1 if p.eta[j] >= 0 else -1
        for jy in range(ny):
            for ix in range(nx):
                c = ix + nx * jy
                r = j * nc + c
                A[r, r] += p.tau + p.sigma_t[c] + a + b
                iu = ix - sx
                if 0 <= iu < nx:
                    A[r, j * nc + iu + nx * jy] -= a
                ju = jy - sy
                if 0 <= ju < ny and b != 0.0:
                    A[r, j * nc + ix + nx * ju] -= b
                for k in range(nv):
                    A[r, k * nc + c] -= p.sigma_s[c] * p.w[k]
    return A


def rhs(p, f_old, inflow=None):
    g = p.inflow if inflow is None else np.asarray(inflow, dtype=np.float64)
    nx, ny, nv = p.nx, p.ny, p.nv
    nc = nx * ny
    out = np.zeros(nv * nc)
    f_old = np.asarray(f_old, dtype=np.float64).reshape(nv, nc)
    for j in range(nv):
        a = abs(p.mu[j]) / p.hx
        b = abs(p.eta[j]) / p.hy if p.dim == 2 else 0.0
        gx = g[0] if p.mu[j] > 0 else g[1]
        gy = g[2] if p.eta[j] >= 0 else g[3]
        for jy in range(ny):
            for ix in range(nx):
                c = ix + nx * jy
                v = p.tau * f_old[j, c] + p.source[c]
                if (p.mu[j] > 0 and ix == 0) or (p.mu[j] < 0 and ix == nx - 1):
                    v += a * gx
                if b != 0.0 and ((p.eta[j] >= 0 and jy == 0) or (p.eta[j] < 0 and jy == ny - 1)):
                    v += b * gy
                out[j * nc + c] = v
    return out


def step(p, f_old, inflow=None):
    """One backward-Euler step solved directly.  Returns (f^n [nv, ncell], rho^n)."""
    f = np.linalg.solve(assemble(p), rhs(p, f_old, inflow)).reshape(p.nv, p.ncell)
    return f, p.w @ f
