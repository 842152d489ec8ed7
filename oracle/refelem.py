"""1D reference element on [-1, 1] (paper Sec. 2.2, "Volumetric DG spaces").

The DG basis is the tensor product of degree-p Lagrange polynomials whose nodes
are the p+1 Gauss-Lobatto-Legendre (GLL) points. Mass and stiffness matrices are
integrated exactly (the paper notes that the GLL mass matrix is not diagonal,
Sec. 4.1 "Structure of block-matrices", i.e. no nodal collocation), using
Gauss-Legendre quadrature with enough points for the polynomial degree.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).
"""
import numpy as np
from numpy.polynomial import legendre as npleg


def gll_nodes(p):
    """GLL nodes of degree p on [-1,1]: the endpoints and the roots of P_p' (the
    Gauss-Lobatto nodes of the DG basis, Sec. 2.2.1).

    Roots come from numpy's Legendre companion matrix and are polished with
    Newton's method on P_p' so that they are accurate to rounding.
    """
    if p < 1:
        raise ValueError("p >= 1 required")
    if p == 1:
        return np.array([-1.0, 1.0])
    c = np.zeros(p + 1)
    c[p] = 1.0
    d1 = npleg.legder(c)
    d2 = npleg.legder(d1)
    r = np.sort(npleg.legroots(d1).real)
    for _ in range(5):
        r = r - npleg.legval(r, d1) / npleg.legval(r, d2)
    return np.concatenate([[-1.0], r, [1.0]])


def gll_weights(p):
    """GLL quadrature weights w_j = 2 / (p (p+1) P_p(x_j)^2) (the lumped part of the
    GLL mass, Sec. 4.1 "Structure of block-matrices")."""
    x = gll_nodes(p)
    c = np.zeros(p + 1)
    c[p] = 1.0
    return 2.0 / (p * (p + 1) * npleg.legval(x, c) ** 2)


def gauss_legendre(m):
    """m-point Gauss-Legendre rule on [-1,1] (exact for degree 2m-1): the quadrature
    of every integral here and the nodes of the GL basis (Sec. 2.2.1, 6.4)."""
    return npleg.leggauss(m)


def lagrange_values(nodes, x):
    """V[i, k] = l_i(x_k) for the Lagrange basis on ``nodes`` (product formula; the
    tensor-product factors of the basis of Sec. 2.2.1)."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(nodes)
    V = np.ones((n, len(x)))
    for i in range(n):
        for m in range(n):
            if m != i:
                V[i] *= (x - nodes[m]) / (nodes[i] - nodes[m])
    return V


def lagrange_derivs(nodes, x):
    """D[i, k] = l_i'(x_k) for the basis of Sec. 2.2.1: derivative of the product
    formula by the product rule,
    l_i'(x) = sum_{k != i} 1/(x_i - x_k) prod_{m != i,k} (x - x_m)/(x_i - x_m)."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(nodes)
    D = np.zeros((n, len(x)))
    for i in range(n):
        for k in range(n):
            if k == i:
                continue
            term = np.full(len(x), 1.0 / (nodes[i] - nodes[k]))
            for m in range(n):
                if m != i and m != k:
                    term *= (x - nodes[m]) / (nodes[i] - nodes[m])
            D[i] += term
    return D


def basis_nodes(p, basis="gll"):
    """Nodes of the degree-p Lagrange basis: Gauss-Lobatto-Legendre ("gll", the
    paper's default) or Gauss-Legendre ("gl", Sec. 6.4: no nodes on the cell
    boundary, diagonal mass matrix)."""
    if basis == "gll":
        return gll_nodes(p)
    if basis == "gl":
        return gauss_legendre(p + 1)[0]
    raise ValueError(basis)


def mass_1d(p, basis="gll"):
    """Exact 1D mass matrix M[i,j] = int_{-1}^{1} l_i l_j (not diagonal with GLL
    nodes, Sec. 4.1 "Structure of block-matrices"; Gauss-Legendre, p+1 points)."""
    xg, wg = gauss_legendre(p + 1)
    V = lagrange_values(basis_nodes(p, basis), xg)
    return (V * wg) @ V.T


def stiffness_1d(p, basis="gll"):
    """Exact 1D stiffness matrix K[i,j] = int_{-1}^{1} l_i' l_j' (the 1D factor of the
    volume term of Eq. weak_form_IP)."""
    xg, wg = gauss_legendre(p + 1)
    D = lagrange_derivs(basis_nodes(p, basis), xg)
    return (D * wg) @ D.T


def endpoint_values(p, basis="gll"):
    """(e0, ep): values of each basis function at xi = -1 and xi = +1 (unit
    vectors for GLL, dense for GL): the value projection of Eq. solution_projection."""
    x = basis_nodes(p, basis)
    V = lagrange_values(x, np.array([-1.0, 1.0]))
    return V[:, 0].copy(), V[:, 1].copy()


def endpoint_derivs(p, basis="gll"):
    """(d0, dp): derivatives d/dxi of each basis function at xi = -1 and xi = +1: the
    derivative projection of Eq. gradient_projection."""
    x = basis_nodes(p, basis)
    D = lagrange_derivs(x, np.array([-1.0, 1.0]))
    return D[:, 0].copy(), D[:, 1].copy()
