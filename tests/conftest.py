import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a GB300 and the built CUDA library")
    config.addinivalue_line("markers", "slow: long-running CPU oracle case")


def oracle_quadrature(quad):
    """The oracle's own angular rule for a workload's quadrature descriptor."""
    from oracle import quadrature as q
    if quad[0] == "gl":
        return q.gl_slab(quad[1])
    return q.cl_hemisphere(quad[1], quad[2])


def cell_modes(x, degree):
    """A per-cell array as the unknowns of a piecewise-constant field: itself for Q0; for Q1
    the cell values in mode 0 (the cell average) and zero in the three linear modes."""
    x = np.asarray(x, dtype=float).ravel()
    return x.copy() if degree == 0 else np.concatenate([x, np.zeros(3 * x.size)])


def oracle_problem(wl, quad=None, degree=0):
    """oracle.transport.Problem from an inputs.Workload (both sides get the same arrays)."""
    from oracle.transport import Problem
    mu, eta, w = quad if quad is not None else oracle_quadrature(wl.quadrature)
    x0, x1, y0, y1 = wl.domain
    return Problem(wl.nx, wl.ny, x0, x1, y0, y1, mu, eta, w, wl.sigma_t.copy(),
                   wl.sigma_s.copy(), cell_modes(wl.source, degree), wl.c_dt,
                   np.array(wl.inflow, dtype=float), degree=degree)


@pytest.fixture
def rng():
    return np.random.default_rng(12345)
