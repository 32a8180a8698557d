"""Angular quadratures of the oracle (test infrastructure).

Sec. 2.1: S_N directions {Omega_j} with weights summing to one, so that
rho = sum_j w_j f(Omega_j) approximates (1/4pi) * integral of f over S^2.
"""
import numpy as np


def gauss_legendre(n: int):
    """n-point Gauss-Legendre nodes and weights on [-1, 1] (weights sum to 2).

    The library routine numpy.polynomial.legendre.leggauss serves as the step.
    """
    x, w = np.polynomial.legendre.leggauss(n)
    return np.asarray(x, dtype=np.float64), np.asarray(w, dtype=np.float64)


def gl_slab(n: int):
    """1D slab S_N rule (Sec. 2.1: Gauss-Legendre in 1D): mu = GL nodes, w = GL weights / 2.

    Returns (mu, eta, w) with eta = 0 so the 1D rule plugs into the 2D sweep.
    """
    mu, w = gauss_legendre(n)
    return mu, np.zeros_like(mu), w / 2.0


def chebyshev_legendre(n_phi: int, n_vz: int):
    """Full-sphere CL(n_phi, n_vz) rule of App. A.

    phi_j = (2j-1) pi / n_phi with weight 1/n_phi; v_z from the normalised
    n_vz-point GL rule (weights / 2); direction
    (cos(phi) sqrt(1-vz^2), sin(phi) sqrt(1-vz^2), vz), weight product,
    index j = (j2-1) n_phi + j1.
    Returns (ox, oy, oz, w).
    """
    vz, wz = gauss_legendre(n_vz)
    wz = wz / 2.0
    j1 = np.arange(1, n_phi + 1)
    phi = (2 * j1 - 1) * np.pi / n_phi
    ox, oy, oz, w = [], [], [], []
    for j2 in range(n_vz):
        s = np.sqrt(1.0 - vz[j2] ** 2)
        ox.append(np.cos(phi) * s)
        oy.append(np.sin(phi) * s)
        oz.append(np.full(n_phi, vz[j2]))
        w.append(np.full(n_phi, wz[j2] / n_phi))
    return (np.concatenate(ox), np.concatenate(oy), np.concatenate(oz), np.concatenate(w))


def cl_hemisphere(n_phi: int, n_vz: int):
    """CL(n_phi, n_vz) restricted to v_z > 0 with doubled weights, for X-Y geometry.

    In X-Y geometry f does not depend on z and is even in v_z, so the two
    directions (ox, oy, +vz) and (ox, oy, -vz) carry equal f and are merged.
    Returns (mu, eta, w) with mu = Omega_x, eta = Omega_y.
    """
    if n_vz % 2:
        raise ValueError("n_vz must be even for the hemisphere rule")
    ox, oy, oz, w = chebyshev_legendre(n_phi, n_vz)
    keep = oz > 0
    return ox[keep].copy(), oy[keep].copy(), 2.0 * w[keep]
