"""1D quadrature and nodal basis (oracle; test infrastructure only).

Sec. 2.2.1: reference element [0,1]^d, tensor-product nodal Lagrange basis on
Legendre--Gauss--Lobatto (LGL) support points.  Sec. 2.2.3: Gauss--Legendre
quadrature with n_q points, exact up to polynomial degree 2 n_q - 1.

Pinned by tests/test_oracle_basis.py (exactness on monomials, partition of
unity, exact derivatives of degree-k polynomials, node symmetry).
"""
import numpy as np


def gauss_legendre_01(nq):
    """Gauss--Legendre points and weights mapped from [-1,1] to [0,1] (Sec. 2.2.3)."""
    if nq < 1:
        raise ValueError("nq must be >= 1")
    x, w = np.polynomial.legendre.leggauss(nq)
    return 0.5 * (x + 1.0), 0.5 * w


def lgl_nodes_01(k):
    """k+1 Legendre--Gauss--Lobatto points on [0,1] (Sec. 2.2.1).

    The interior points are the roots of P_k'; numpy's companion-matrix roots
    are polished by three Newton steps on P_k'.
    """
    if k < 1:
        raise ValueError("k must be >= 1")
    pk = np.polynomial.legendre.Legendre.basis(k)
    d1, d2 = pk.deriv(1), pk.deriv(2)
    r = np.sort(np.real(d1.roots())) if k > 1 else np.zeros(0)
    for _ in range(3):
        if r.size:
            r = r - d1(r) / d2(r)
    x = np.concatenate([[-1.0], r, [1.0]])
    return 0.5 * (x + 1.0)


def lagrange_1d(nodes, x):
    """Values and first derivatives of the Lagrange polynomials l_i at points x.

    Returns (V, D) with V[p, i] = l_i(x_p) and D[p, i] = l_i'(x_p), written out
    from the product definition l_i(x) = prod_{j != i} (x - x_j)/(x_i - x_j).
    """
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(nodes)
    V = np.ones((len(x), n))
    D = np.zeros((len(x), n))
    for i in range(n):
        for j in range(n):
            if j != i:
                V[:, i] *= (x - nodes[j]) / (nodes[i] - nodes[j])
        for m in range(n):
            if m == i:
                continue
            t = np.full(len(x), 1.0 / (nodes[i] - nodes[m]))
            for j in range(n):
                if j != i and j != m:
                    t *= (x - nodes[j]) / (nodes[i] - nodes[j])
            D[:, i] += t
    return V, D


def basis_3d(nodes, pts):
    """Full 3D tensor-product basis at reference points pts [P,3].

    Node index i = i0 + n*i1 + n^2*i2 (x fastest).  Returns
    phi [P, n^3] and grad [P, n^3, 3] with grad[..., b] = d phi / d xi_b.
    """
    pts = np.asarray(pts, dtype=np.float64)
    n = len(nodes)
    V0, D0 = lagrange_1d(nodes, pts[:, 0])
    V1, D1 = lagrange_1d(nodes, pts[:, 1])
    V2, D2 = lagrange_1d(nodes, pts[:, 2])
    P = pts.shape[0]
    phi = np.einsum("pc,pb,pa->pcba", V2, V1, V0).reshape(P, n ** 3)
    g0 = np.einsum("pc,pb,pa->pcba", V2, V1, D0).reshape(P, n ** 3)
    g1 = np.einsum("pc,pb,pa->pcba", V2, D1, V0).reshape(P, n ** 3)
    g2 = np.einsum("pc,pb,pa->pcba", D2, V1, V0).reshape(P, n ** 3)
    return phi, np.stack([g0, g1, g2], axis=-1)


def cell_points(nq):
    """Tensor Gauss grid on [0,1]^3: points [nq^3, 3] (index p0 + nq p1 + nq^2 p2) and weights."""
    x, w = gauss_legendre_01(nq)
    p2, p1, p0 = np.meshgrid(np.arange(nq), np.arange(nq), np.arange(nq), indexing="ij")
    p0, p1, p2 = p0.ravel(), p1.ravel(), p2.ravel()
    pts = np.stack([x[p0], x[p1], x[p2]], axis=1)
    return pts, w[p0] * w[p1] * w[p2]


def face_points(nq, d, side):
    """Gauss grid on the face xi_d = side of [0,1]^3.

    The two tangential directions are the other two axes in increasing order
    (t1 < t2); point index a + nq*b runs over (xi_t1 = x_a, xi_t2 = x_b).
    Returns points [nq^2, 3] and weights [nq^2].
    """
    x, w = gauss_legendre_01(nq)
    t1, t2 = [a for a in range(3) if a != d]
    b, a = np.meshgrid(np.arange(nq), np.arange(nq), indexing="ij")
    a, b = a.ravel(), b.ravel()
    pts = np.zeros((nq * nq, 3))
    pts[:, d] = float(side)
    pts[:, t1] = x[a]
    pts[:, t2] = x[b]
    return pts, w[a] * w[b]
