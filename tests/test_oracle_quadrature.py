"""Pins of the oracle's angular rules (Sec. 2.1, App. A) against closed forms."""
import math

import numpy as np
import pytest

from oracle import quadrature as q


def test_gl_two_point_closed_form():
    x, w = q.gauss_legendre(2)
    assert np.allclose(np.sort(x), [-1 / math.sqrt(3), 1 / math.sqrt(3)], atol=1e-15)
    assert np.allclose(w, [1.0, 1.0], atol=1e-15)


@pytest.mark.parametrize("n", [2, 4, 6, 8, 16])
def test_gl_polynomial_exactness(n):
    x, w = q.gauss_legendre(n)
    for k in range(2 * n):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.sum(w * x ** k) - exact) < 1e-13


def test_slab_rule_normalised():
    mu, eta, w = q.gl_slab(16)
    assert abs(w.sum() - 1) < 1e-14 and abs(np.sum(w * mu ** 2) - 1 / 3) < 1e-14
    assert np.all(eta == 0) and np.sum(mu > 0) == 8


def test_cl_full_sphere_indexing_and_moments():
    ox, oy, oz, w = q.chebyshev_legendre(8, 4)
    assert ox.size == 32
    # j = (j2-1) N_phi + j1: the first N_phi directions share the first GL node.
    assert np.allclose(oz[:8], oz[0]) and abs(w.sum() - 1) < 1e-14
    assert np.allclose(ox ** 2 + oy ** 2 + oz ** 2, 1.0, atol=1e-14)


@pytest.mark.parametrize("nphi,nvz,nv", [(32, 8, 128), (32, 16, 256), (16, 8, 64), (8, 2, 8)])
def test_cl_hemisphere_moments(nphi, nvz, nv):
    mu, eta, w = q.cl_hemisphere(nphi, nvz)
    assert mu.size == nv and abs(w.sum() - 1) < 1e-14
    # sphere averages of monomials: <x^2> = 1/3, <x^4> = 1/5, <x^2 y^2> = 1/15, odd = 0
    assert abs(np.sum(w * mu)) < 1e-14 and abs(np.sum(w * eta)) < 1e-14
    assert abs(np.sum(w * mu * eta)) < 1e-14
    assert abs(np.sum(w * mu ** 2) - 1 / 3) < 1e-14 and abs(np.sum(w * eta ** 2) - 1 / 3) < 1e-14
    if nphi >= 8 and nvz >= 4:
        assert abs(np.sum(w * mu ** 4) - 1 / 5) < 1e-13
        assert abs(np.sum(w * mu ** 2 * eta ** 2) - 1 / 15) < 1e-13
    # equal share per quadrant, no direction on an axis
    for sx in (1, -1):
        for sy in (1, -1):
            assert np.sum((np.sign(mu) == sx) & (np.sign(eta) == sy)) == nv // 4
    assert np.all(mu != 0) and np.all(eta != 0)
