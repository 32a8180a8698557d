"""Problem description and the upwind sweeps of the oracle (test infrastructure).

The sweeps themselves are the plain C loop nests in ``csrc/oracle_sweep.c`` (Q0: one value
per cell; Q1: four bilinear modes per cell, ``degree=1``); this module marshals NumPy arrays
into them and writes out the operators of Sec. 2.3:

* T q       = sum_j w_j L_j^{-1} q           (Eq. (implicit_linear_system_rho), zero inflow)
* b_tilde   = sum_j w_j L_j^{-1}(tau f_j + G + g_j^bc)   (same equation)
* f_j       = L_j^{-1}(Sigma_s rho + tau f_j^old + G + g_j^bc)   (Eq. (sweep_to_obtain_f),
              with the tau f^{n-1} term of Eq. (dg_discrete1))

with L_j = tau M + D_j + Sigma_t, tau = 1/(c dt), M = I for the orthonormal bases.

Vectors over the degrees of freedom (rho, the source G, each direction's f) hold ncell values
for Q0 and 4 ncell values for Q1, mode-major: mode k of cell c at k ncell + c, with the modes
1, sqrt(3) xi, sqrt(3) zeta, 3 xi zeta of the cell's local coordinates (orthonormal under the
cell average).  Sigma_t and Sigma_s are constant per cell.
"""
import ctypes
from dataclasses import dataclass, field

import numpy as np

from . import build as _build

_lib = None


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(_build.build())
        d = ctypes.POINTER(ctypes.c_double)
        _lib.oracle_sweep.restype = ctypes.c_int
        _lib.oracle_sweep.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_int, d, d, d, ctypes.c_double, d, d, d,
                                      ctypes.c_double, d, d, d]
        _lib.oracle_sweep_q1.restype = ctypes.c_int
        _lib.oracle_sweep_q1.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_int, d, d, d, ctypes.c_double,
                                         d, d, d, ctypes.c_double, d, d, d, d]
        _lib.oracle_num_threads.restype = ctypes.c_int
    return _lib


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def _ptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


@dataclass
class Problem:
    """One-group linear RTE problem, Sec. 2 Eq. (rte), on a uniform Cartesian grid.

    nx, ny: cells (1D slab: ny = 1).  [x0,x1] x [y0,y1]: domain.
    mu, eta, w: S_N directions and weights (sum w = 1).  sigma_t >= sigma_s >= 0, source G: per cell.
    c_dt: c * dt, so tau = 1/(c dt) takes the place of 1/dt in Eq. (time_discrete).
    inflow: isotropic inflow value per side (west, east, south, north), Eq. (boundary).
    degree: K of the DG space Eq. (dg_space), 0 (one constant per cell) or 1 (bilinear, 2D);
    the source G then holds ndof = nb ncell values (mode-major, see the module docstring).
    """
    nx: int
    ny: int
    x0: float
    x1: float
    y0: float
    y1: float
    mu: np.ndarray
    eta: np.ndarray
    w: np.ndarray
    sigma_t: np.ndarray
    sigma_s: np.ndarray
    source: np.ndarray
    c_dt: float
    inflow: np.ndarray = field(default_factory=lambda: np.zeros(4))
    degree: int = 0

    def __post_init__(self):
        for k in ("mu", "eta", "w", "sigma_t", "sigma_s", "source", "inflow"):
            setattr(self, k, _f64(getattr(self, k)).ravel())
        if self.degree not in (0, 1):
            raise ValueError("degree must be 0 or 1")
        if self.degree == 1 and self.dim != 2:
            raise ValueError("the Q1 scheme is built for 2D grids")
        if self.source.size != self.ndof:
            raise ValueError(f"source must hold {self.ndof} values")

    @property
    def ncell(self):
        return self.nx * self.ny

    @property
    def nb(self):
        """Basis functions per cell: 1 (Q0) or 4 (Q1)."""
        return 1 if self.degree == 0 else 4

    @property
    def ndof(self):
        return self.nb * self.ncell

    @property
    def sig_s_dof(self):
        """Sigma_s on every degree of freedom (piecewise constant: the same for each mode)."""
        return np.tile(self.sigma_s, self.nb)

    @property
    def nv(self):
        return self.mu.size

    @property
    def hx(self):
        return (self.x1 - self.x0) / self.nx

    @property
    def hy(self):
        return (self.y1 - self.y0) / self.ny

    @property
    def tau(self):
        return 1.0 / self.c_dt

    @property
    def dim(self):
        return 1 if self.ny == 1 and not np.any(self.eta) else 2


def q1_traces(p: Problem, inflow):
    """Face modes of an isotropic inflow value per side (west, east, south, north) for the Q1
    sweep: the constant g has face modes (g, 0) on every boundary face."""
    g = _f64(inflow).ravel()
    gx = np.zeros((2, p.ny, 2))
    gy = np.zeros((2, p.nx, 2))
    gx[0, :, 0], gx[1, :, 0] = g[0], g[1]
    gy[0, :, 0], gy[1, :, 0] = g[2], g[3]
    return gx, gy


def sweep(p: Problem, s_iso=None, s_dir=None, s_dir_scale=1.0, inflow=None, want_psi=False,
          traces=None):
    """Apply L_j^{-1} to (s_iso + s_dir_scale * s_dir[j] + g_j^bc) for every direction j.

    Returns (moment, psi) where moment = sum_j w_j psi_j and psi is [nv, ndof]
    (None unless want_psi).  inflow=None means vacuum (the SI and DSA sweeps of
    Sec. 2.3 run with zero inflow).  Q1 only: traces = (gx [2, ny, 2], gy [2, nx, 2]) gives
    the face modes of a non-constant inflow instead (west / east rows, south / north columns).
    """
    if p.degree == 1:
        return _sweep_q1(p, s_iso, s_dir, s_dir_scale, inflow, want_psi, traces)
    lib = _load()
    s_iso = _f64(s_iso)
    s_dir = _f64(s_dir)
    if s_dir is not None:
        s_dir = s_dir.reshape(p.nv, p.ncell)
    g = _f64(inflow)
    mom = np.empty(p.ncell)
    psi = np.empty((p.nv, p.ncell)) if want_psi else None
    rc = lib.oracle_sweep(p.nx, p.ny, p.hx, p.hy, p.nv, _ptr(p.mu), _ptr(p.eta), _ptr(p.w), p.tau,
                          _ptr(p.sigma_t), _ptr(s_iso), _ptr(s_dir), float(s_dir_scale), _ptr(g),
                          _ptr(psi), _ptr(mom))
    if rc != 0:
        raise MemoryError("oracle sweep: allocation failed")
    return mom, psi


def _sweep_q1(p, s_iso, s_dir, s_dir_scale, inflow, want_psi, traces):
    lib = _load()
    s_iso = _f64(s_iso)
    s_dir = _f64(s_dir)
    if s_dir is not None:
        s_dir = s_dir.reshape(p.nv, p.ndof)
    if traces is not None:
        gx, gy = (_f64(t) for t in traces)
    elif inflow is not None:
        gx, gy = q1_traces(p, inflow)
    else:
        gx = gy = None
    mom = np.empty(p.ndof)
    psi = np.empty((p.nv, p.ndof)) if want_psi else None
    rc = lib.oracle_sweep_q1(p.nx, p.ny, p.hx, p.hy, p.nv, _ptr(p.mu), _ptr(p.eta), _ptr(p.w),
                             p.tau, _ptr(p.sigma_t), _ptr(s_iso), _ptr(s_dir),
                             float(s_dir_scale), _ptr(gx), _ptr(gy), _ptr(psi), _ptr(mom))
    if rc != 0:
        raise MemoryError("oracle sweep: allocation failed")
    return mom, psi


def apply_T_sigma_s(p: Problem, rho):
    """T Sigma_s rho with zero inflow: the SI map of Eq. (SI_rho) without b_tilde."""
    return sweep(p, s_iso=p.sig_s_dof * rho)[0]


def b_tilde(p: Problem, f_old, inflow=None):
    """b_tilde^{n-1} = sum_j w_j L_j^{-1}(tau f_j^{n-1} + G + g_j^bc), Eq. (implicit_linear_system_rho)."""
    return sweep(p, s_iso=p.source, s_dir=f_old, s_dir_scale=p.tau,
                 inflow=p.inflow if inflow is None else inflow)[0]


def final_f(p: Problem, rho, f_old, inflow=None):
    """f_j^n = L_j^{-1}(Sigma_s rho^n + tau f_j^{n-1} + G + g_j^bc): Eq. (sweep_to_obtain_f) with the
    tau M f^{n-1} term of Eq. (dg_discrete1) restored.  Returns (f [nv, ndof], its moment)."""
    mom, psi = sweep(p, s_iso=p.sig_s_dof * rho + p.source, s_dir=f_old, s_dir_scale=p.tau,
                     inflow=p.inflow if inflow is None else inflow, want_psi=True)
    return psi, mom
