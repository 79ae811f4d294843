"""Pins of the oracle's 1D quadrature and nodal basis (Sec. 2.2.1, Sec. 2.2.3)."""
import math

import numpy as np
import pytest

from oracle.basis import basis_3d, cell_points, face_points, gauss_legendre_01, lagrange_1d, lgl_nodes_01


@pytest.mark.parametrize("nq", range(1, 12))
def test_gauss_exact_to_degree_2nq_minus_1(nq):
    x, w = gauss_legendre_01(nq)
    for j in range(2 * nq):
        assert abs((w * x ** j).sum() - 1.0 / (j + 1)) < 1e-15
    # and not exact one degree higher (the rule has exactly degree 2nq-1)
    assert abs((w * x ** (2 * nq)).sum() - 1.0 / (2 * nq + 1)) > 1e-14


@pytest.mark.parametrize("k", range(1, 10))
def test_lgl_nodes(k):
    x = lgl_nodes_01(k)
    assert len(x) == k + 1 and x[0] == 0.0 and x[-1] == 1.0
    assert np.all(np.diff(x) > 0)
    assert np.allclose(x + x[::-1], 1.0, atol=1e-15, rtol=0)
    # Closed-form LGL weights w_i = 2 / (k (k+1) P_k(t_i)^2) on [-1,1] give a rule exact to degree 2k-1.
    t = 2 * x - 1
    Pk = np.polynomial.legendre.Legendre.basis(k)(t)
    w = 0.5 * 2.0 / (k * (k + 1) * Pk ** 2)
    for j in range(2 * k):
        assert abs((w * x ** j).sum() - 1.0 / (j + 1)) < 1e-14


@pytest.mark.parametrize("k", range(1, 9))
def test_lagrange_properties(k):
    nodes = lgl_nodes_01(k)
    V, D = lagrange_1d(nodes, nodes)
    assert np.allclose(V, np.eye(k + 1), atol=1e-14)
    xs = np.linspace(-0.2, 1.3, 37)
    V, D = lagrange_1d(nodes, xs)
    assert np.allclose(V.sum(1), 1.0, atol=1e-12)
    assert np.allclose(D.sum(1), 0.0, atol=1e-10)
    rng = np.random.default_rng(k)
    c = rng.standard_normal(k + 1)
    p = np.polynomial.Polynomial(c)
    assert np.allclose(V @ p(nodes), p(xs), atol=1e-11)
    assert np.allclose(D @ p(nodes), p.deriv()(xs), atol=1e-9)


def test_basis_3d_tensor_structure_and_gradient():
    k = 3
    nodes = lgl_nodes_01(k)
    rng = np.random.default_rng(0)
    pts = rng.random((7, 3))
    phi, grad = basis_3d(nodes, pts)
    assert np.allclose(phi.sum(1), 1.0, atol=1e-13)
    # f(x) = x0^2 x1 + 3 x2^3 - x0 x1 x2 is in Q_3: interpolate and differentiate exactly
    n = k + 1
    i2, i1, i0 = np.meshgrid(range(n), range(n), range(n), indexing="ij")
    X = np.stack([nodes[i0.ravel()], nodes[i1.ravel()], nodes[i2.ravel()]], 1)
    f = lambda P: P[:, 0] ** 2 * P[:, 1] + 3 * P[:, 2] ** 3 - P[:, 0] * P[:, 1] * P[:, 2]
    df = lambda P: np.stack([2 * P[:, 0] * P[:, 1] - P[:, 1] * P[:, 2],
                             P[:, 0] ** 2 - P[:, 0] * P[:, 2],
                             9 * P[:, 2] ** 2 - P[:, 0] * P[:, 1]], 1)
    assert np.allclose(phi @ f(X), f(pts), atol=1e-13)
    assert np.allclose(np.einsum("pnb,n->pb", grad, f(X)), df(pts), atol=1e-12)


def test_point_sets():
    pts, w = cell_points(3)
    assert pts.shape == (27, 3) and abs(w.sum() - 1) < 1e-15
    x, _ = gauss_legendre_01(3)
    assert np.allclose(pts[1], [x[1], x[0], x[0]]) and np.allclose(pts[3], [x[0], x[1], x[0]])
    fp, fw = face_points(3, 1, 1)
    assert np.allclose(fp[:, 1], 1.0) and abs(fw.sum() - 1) < 1e-15
    assert np.allclose(fp[1], [x[1], 1.0, x[0]]) and np.allclose(fp[3], [x[0], 1.0, x[1]])


@pytest.mark.parametrize("nq", [13, 15, 16, 17, 23])
def test_gauss_exact_high_point_counts(nq):
    """The point counts of the high-degree rules (q = 13, 17, 23 of k = 8, 11, 15; 15 of the 2k+1 rule at
    k = 7): exact to degree 2 nq - 1, relative to each moment; symmetric about 1/2; weights sum to 1."""
    x, w = gauss_legendre_01(nq)
    assert np.all(np.diff(x) > 0) and np.all(w > 0)
    assert np.allclose(x + x[::-1], 1.0, atol=1e-15, rtol=0) and np.allclose(w, w[::-1], atol=1e-15, rtol=0)
    for j in range(2 * nq):
        assert abs((w * x ** j).sum() * (j + 1) - 1.0) < 1e-13, j


@pytest.mark.parametrize("k", [11, 15])
def test_lgl_nodes_high_degree(k):
    x = lgl_nodes_01(k)
    assert len(x) == k + 1 and x[0] == 0.0 and x[-1] == 1.0 and np.all(np.diff(x) > 0)
    assert np.allclose(x + x[::-1], 1.0, atol=1e-15, rtol=0)
    t = 2 * x - 1
    # interior nodes are the roots of P_k'
    assert np.abs(np.polynomial.legendre.Legendre.basis(k).deriv()(t[1:-1])).max() < 1e-9
    w = 1.0 / (k * (k + 1) * np.polynomial.legendre.Legendre.basis(k)(t) ** 2)
    for j in range(2 * k):
        assert abs((w * x ** j).sum() * (j + 1) - 1.0) < 1e-12, j


@pytest.mark.parametrize("k", [11, 15])
def test_lagrange_properties_high_degree(k):
    nodes = lgl_nodes_01(k)
    V, D = lagrange_1d(nodes, nodes)
    assert np.allclose(V, np.eye(k + 1), atol=1e-13)
    xs = np.linspace(0.0, 1.0, 41)
    V, D = lagrange_1d(nodes, xs)
    assert np.allclose(V.sum(1), 1.0, atol=1e-12)
    assert np.abs(D.sum(1)).max() < 1e-8
    rng = np.random.default_rng(k)
    p = np.polynomial.Legendre(rng.standard_normal(k + 1), domain=[0, 1])
    assert np.allclose(V @ p(nodes), p(xs), atol=1e-11)
    assert np.allclose(D @ p(nodes), p.deriv()(xs), atol=1e-7 * np.abs(p.deriv()(xs)).max())
