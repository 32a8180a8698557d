"""Shared helpers of the GPU parity tests (test infrastructure)."""
import numpy as np

from conftest import oracle_problem, oracle_quadrature
from paper_2603_19647_gb300 import rte


def rel_l2(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def max_rel(a, b, floor=1e-3):
    """Largest element-wise relative error |a - b| / (|b| + floor max|b|): a bad value in one
    cell (a wrong tile edge, a dropped hand-off) shows here even where it hides in the L2
    norm of a large array.  The floor keeps values many orders below the field's maximum
    (deep in an absorber, where FP32 underflows first) from dominating."""
    a, b = np.asarray(a, float), np.asarray(b, float)
    scale = np.abs(b) + floor * (np.max(np.abs(b)) if b.size else 0.0)
    scale[scale == 0] = 1.0
    return float(np.max(np.abs(a - b) / scale)) if b.size else 0.0


def match_directions(h, quad_desc):
    """Permutation perm such that library direction d equals oracle direction perm[d]."""
    mu, eta, w = h.rte_get_quadrature()
    omu, oeta, ow = oracle_quadrature(quad_desc)
    perm = np.empty(mu.size, dtype=int)
    for d in range(mu.size):
        k = int(np.argmin((omu - mu[d]) ** 2 + (oeta - eta[d]) ** 2))
        perm[d] = k
    assert len(set(perm.tolist())) == mu.size
    return perm, (mu, eta, w), (omu, oeta, ow)


def lib_options(**kw):
    return rte.default_options(**kw)


def make_pair(wl, **opts):
    """Library handle and oracle problem for the same workload (options.degree on both)."""
    o = lib_options(**opts)
    h = rte.create_from_workload(wl, options=o)
    p = oracle_problem(wl, degree=opts.get("degree", 0))
    return h, p
