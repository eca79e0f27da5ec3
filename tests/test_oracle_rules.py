"""Pins for the oracle's 1D rules and basis: closed forms, exactness and
partition of unity (Sec. 3.3 nodal GLL basis; Sec. 4.4 B^{1d})."""

import numpy as np
import pytest

from oracle import rules, lagrange


def test_gll_closed_forms():
    np.testing.assert_allclose(rules.gll_nodes(1), [0.0, 1.0], atol=0)
    np.testing.assert_allclose(rules.gll_nodes(2), [0.0, 0.5, 1.0], atol=1e-16)
    s5 = 0.5 / np.sqrt(5.0)
    np.testing.assert_allclose(rules.gll_nodes(3), [0.0, 0.5 - s5, 0.5 + s5, 1.0], atol=2e-16)
    s = 0.5 * np.sqrt(3.0 / 7.0)
    np.testing.assert_allclose(rules.gll_nodes(4), [0.0, 0.5 - s, 0.5, 0.5 + s, 1.0], atol=2e-16)


@pytest.mark.parametrize("p", range(1, 10))
def test_gll_are_roots_of_legendre_derivative(p):
    x = rules.gll_nodes(p)
    assert np.all(np.diff(x) > 0)
    np.testing.assert_allclose(x + x[::-1], 1.0, atol=1e-15)      # symmetric
    if p >= 2:
        # interior nodes: roots of P'_p on [-1,1]; P'_p(t) = sum of c_k P_k known via numpy
        t = 2 * x[1:-1] - 1
        dP = np.polynomial.legendre.Legendre.basis(p).deriv()(t)
        assert np.max(np.abs(dP)) < 1e-12 * max(1.0, p * p)


def test_gauss_closed_forms():
    x, w = rules.gauss_legendre(1)
    np.testing.assert_allclose(x, [0.5]); np.testing.assert_allclose(w, [1.0])
    x, w = rules.gauss_legendre(2)
    np.testing.assert_allclose(x, [0.5 - 0.5 / np.sqrt(3), 0.5 + 0.5 / np.sqrt(3)], atol=1e-16)
    np.testing.assert_allclose(w, [0.5, 0.5], atol=1e-16)
    x, w = rules.gauss_legendre(3)
    np.testing.assert_allclose(x, [0.5 - 0.5 * np.sqrt(0.6), 0.5, 0.5 + 0.5 * np.sqrt(0.6)], atol=1e-16)
    np.testing.assert_allclose(w, [5 / 18, 8 / 18, 5 / 18], atol=1e-16)


@pytest.mark.parametrize("q", range(1, 12))
def test_gauss_exactness(q):
    x, w = rules.gauss_legendre(q)
    assert abs(w.sum() - 1.0) < 1e-15
    for k in range(2 * q):
        assert abs((w * x ** k).sum() - 1.0 / (k + 1)) < 5e-16
    # and not exact one degree higher (the rule is exactly of degree 2q-1)
    # (the Gauss error for x^(2q) shrinks like 4^-2q, so check it while visible)
    k = 2 * q
    if q <= 8:
        assert abs((w * x ** k).sum() - 1.0 / (k + 1)) > 1e-13


@pytest.mark.parametrize("p", range(1, 9))
def test_lagrange_nodal_and_partition_of_unity(p):
    nodes = rules.gll_nodes(p)
    pts, _ = rules.gauss_legendre(p + 2)
    B, G = lagrange.basis_1d(nodes, pts)
    np.testing.assert_allclose(B.sum(axis=1), 1.0, atol=1e-13)
    np.testing.assert_allclose(G.sum(axis=1), 0.0, atol=1e-11)
    Bn, _ = lagrange.basis_1d(nodes, nodes)
    np.testing.assert_allclose(Bn, np.eye(p + 1), atol=1e-14)
    # exact interpolation of x^k (k <= p) and of its derivative
    for k in range(p + 1):
        np.testing.assert_allclose(B @ nodes ** k, pts ** k, atol=1e-13)
        np.testing.assert_allclose(G @ nodes ** k, k * pts ** max(k - 1, 0) if k else 0 * pts, atol=1e-11)


def test_gll_p2_1d_stiffness_closed_form():
    nodes = rules.gll_nodes(2)
    x, w = rules.gauss_legendre(4)
    B, G = lagrange.basis_1d(nodes, x)
    K1 = G.T @ np.diag(w) @ G
    np.testing.assert_allclose(K1, np.array([[7, -8, 1], [-8, 16, -8], [1, -8, 7]]) / 3.0, atol=1e-14)
    M1 = B.T @ np.diag(w) @ B
    np.testing.assert_allclose(M1, np.array([[4, 2, -1], [2, 16, 2], [-1, 2, 4]]) / 30.0, atol=1e-15)


def test_basis_3d_ordering():
    nodes = rules.gll_nodes(2)
    pts, _ = rules.gauss_legendre(3)
    B, G = lagrange.basis_1d(nodes, pts)
    phi, dphi = lagrange.basis_3d(B, G)
    Q, D = B.shape
    # point k = k1 + Q k2 + Q^2 k3, DOF i = i1 + D i2 + D^2 i3
    k1, k2, k3, i1, i2, i3 = 2, 0, 1, 1, 2, 0
    k = k1 + Q * (k2 + Q * k3)
    i = i1 + D * (i2 + D * i3)
    assert phi[k, i] == pytest.approx(B[k1, i1] * B[k2, i2] * B[k3, i3], abs=1e-16)
    assert dphi[k, 0, i] == pytest.approx(G[k1, i1] * B[k2, i2] * B[k3, i3], abs=1e-16)
    assert dphi[k, 1, i] == pytest.approx(B[k1, i1] * G[k2, i2] * B[k3, i3], abs=1e-16)
    assert dphi[k, 2, i] == pytest.approx(B[k1, i1] * B[k2, i2] * G[k3, i3], abs=1e-16)
