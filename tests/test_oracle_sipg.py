"""Pins of the oracle's SIPG operator and block-Jacobi smoother.

The assembled route (quadrature of the weak form, facet by facet) and the
matrix-free facet route (Alg. 2 stages) share only the 1D reference element,
which is pinned separately; their agreement, symmetry, positivity, polynomial
consistency and the smoother's fixed point pin the operator (Sec. 2.3, 4.1)."""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse.linalg as spla

from oracle import sipg

CASES = [((3, 3), 1), ((3, 4), 2), ((3, 3), 3), ((2, 3), 5), ((2, 2, 2), 1), ((2, 3, 2), 2), ((2, 2, 2), 3)]


def _kappa(mesh, kind, seed=0):
    if kind == "one":
        return None
    return np.exp(np.random.default_rng(seed).normal(size=mesh.ncell))


@pytest.mark.parametrize("n,p", CASES)
@pytest.mark.parametrize("kind", ["one", "lognormal"])
def test_assembled_equals_facet_route(n, p, kind):
    mesh = sipg.Mesh(n, p)
    kap = _kappa(mesh, kind)
    A = sipg.assemble(mesh, kap)
    u = np.random.default_rng(1).normal(size=mesh.ndof)
    y1, y2 = A @ u, sipg.apply(mesh, u, kap)
    assert np.abs(y1 - y2).max() <= 1e-13 * np.abs(y1).max()


@pytest.mark.parametrize("n,p", CASES)
@pytest.mark.parametrize("kind", ["one", "lognormal"])
def test_symmetric_positive_definite(n, p, kind):
    mesh = sipg.Mesh(n, p)
    Ad = sipg.assemble(mesh, _kappa(mesh, kind)).toarray()
    assert np.abs(Ad - Ad.T).max() <= 1e-14 * np.abs(Ad).max()
    assert np.linalg.eigvalsh(0.5 * (Ad + Ad.T))[0] > 0.0


@pytest.mark.parametrize("n,p", CASES)
@pytest.mark.parametrize("kind", ["one", "lognormal"])
def test_block_diagonal_is_diagonal_of_assembled(n, p, kind):
    mesh = sipg.Mesh(n, p)
    kap = _kappa(mesh, kind)
    Ad = sipg.assemble(mesh, kap).toarray()
    B = sipg.block_diagonal(mesh, kap)
    nl = mesh.nloc
    for c in range(mesh.ncell):
        blk = Ad[c * nl:(c + 1) * nl, c * nl:(c + 1) * nl]
        assert np.abs(B[c] - blk).max() <= 1e-13 * np.abs(blk).max()


@pytest.mark.parametrize("d,p", [(2, 1), (2, 2), (2, 3), (2, 4), (3, 1), (3, 2), (3, 3)])
def test_polynomial_consistency(d, p):
    """For constant kappa and a global polynomial u of degree <= p per axis, the
    SIPG residual on cells away from the boundary equals the L2 projection of
    -kappa Lap u: (A u)_K = kappa M_K (-Lap u)_K (consistency of the method)."""
    n = (4,) * d
    mesh = sipg.Mesh(n, p)
    kap = 2.5
    rng = np.random.default_rng(d * 10 + p)
    C = rng.normal(size=(p + 1,) * d)                       # coefficients of x^a y^b z^c

    def poly(X, deriv=None):
        val = np.zeros(X.shape[0])
        for idx in np.ndindex(C.shape):
            term = np.full(X.shape[0], C[idx])
            for a in range(d):
                e = idx[a]
                if deriv == a:
                    term = term * (e * (e - 1) * X[:, a] ** max(e - 2, 0) if e >= 2 else 0.0)
                else:
                    term = term * X[:, a] ** e
            val += term
        return val

    X = mesh.node_coords()
    u = poly(X)
    lap = sum(poly(X, deriv=a) for a in range(d))
    Au = sipg.apply(mesh, u, np.full(mesh.ncell, kap))
    L = mesh.grid(-kap * lap)
    for a in range(d):
        L = sipg.apply_1d(mesh.M[a], L, mesh.node_axis(a))
    Mlap = mesh.flat(L)
    Au = Au.reshape(mesh.ncell, mesh.nloc)
    cells = np.indices(n[::-1]).reshape(d, -1)[::-1]
    inner = np.all([(cells[a] > 0) & (cells[a] < n[a] - 1) for a in range(d)], axis=0)
    scale = np.abs(Au).max()
    assert np.abs(Au[inner] - Mlap[inner]).max() <= 1e-11 * scale


@pytest.mark.parametrize("n,p", [((3, 4), 2), ((2, 2, 2), 2), ((3, 3), 4)])
@pytest.mark.parametrize("kind", ["one", "lognormal"])
def test_smoother_fixed_point_and_orders(n, p, kind):
    mesh = sipg.Mesh(n, p)
    kap = _kappa(mesh, kind)
    A = sipg.assemble(mesh, kap)
    rng = np.random.default_rng(3)
    b = rng.normal(size=mesh.ndof)
    xs = spla.spsolve(A.tocsc(), b)
    bj = sipg.BlockJacobi(mesh, kap)
    x1 = bj.step_alg2(xs, b, 0.8, 1)
    assert np.abs(x1 - xs).max() <= 1e-12 * np.abs(xs).max()
    # Alg. 4 (fused) == Alg. 2 (three sweeps) == dense u + omega D^-1 (b - A u)
    Ad = A.toarray()
    nl = mesh.nloc
    D = sla.block_diag(*[Ad[c * nl:(c + 1) * nl, c * nl:(c + 1) * nl] for c in range(mesh.ncell)])
    u0 = rng.normal(size=mesh.ndof)
    ud = u0.copy()
    for _ in range(3):
        ud = ud + 0.8 * np.linalg.solve(D, b - Ad @ ud)
    u2 = bj.step_alg2(u0, b, 0.8, 3)
    u4, proj = bj.step_alg4(u0, b, 0.8, 3)
    sc = np.abs(ud).max()
    assert np.abs(u2 - ud).max() <= 1e-12 * sc
    assert np.abs(u4 - ud).max() <= 1e-12 * sc
    # the returned projections are those of the returned iterate
    ref = sipg.project(mesh, mesh.grid(u4))
    for a in range(mesh.d):
        for f1, f2 in zip(proj[a], ref[a]):
            assert np.array_equal(f1, f2)


def test_load_vector_and_l2_error_closed_forms():
    for n, p in [((3, 2), 2), ((2, 2, 3), 3)]:
        mesh = sipg.Mesh(n, p)
        d = mesh.d
        one = lambda *X: np.ones_like(X[0])
        b = sipg.load_vector(mesh, one)
        assert abs(b.sum() - 1.0) < 1e-13                 # sum_i (1, phi_i) = |Omega|
        # polynomial f of degree <= p per axis: b = M f_nodal exactly
        f = lambda *X: sum((a + 1) * X[a] ** p for a in range(d)) + X[0] * X[-1]
        X = mesh.node_coords()
        F = mesh.grid(f(*[X[:, a] for a in range(d)]))
        for a in range(d):
            F = sipg.apply_1d(mesh.M[a], F, mesh.node_axis(a))
        assert np.allclose(sipg.load_vector(mesh, f), mesh.flat(F).reshape(-1), atol=1e-14)
        # interpolant of a degree-p polynomial has zero L2 error; ||0 - 1|| = 1
        u = f(*[X[:, a] for a in range(d)])
        assert sipg.l2_error(mesh, u, f) < 1e-13
        assert abs(sipg.l2_error(mesh, np.zeros(mesh.ndof), one) - 1.0) < 1e-13


@pytest.mark.parametrize("p", [1, 2, 3])
def test_harmonic_kappa_reading_stays_definite_at_high_contrast(p):
    """The kappa extension (every interior facet term scaled by the harmonic mean)
    keeps the operator positive definite at neighbour contrast 1000."""
    mesh = sipg.Mesh((4, 4), p)
    kap = np.array([1000.0 if (i + j) % 2 else 1.0 for j in range(4) for i in range(4)])
    assert np.linalg.eigvalsh(sipg.assemble(mesh, kap).toarray())[0] > 0.0


@pytest.mark.parametrize("n,p", [((4, 3, 5), 2), ((3, 4), 3), ((3, 3, 3), 3), ((5, 4), 1), ((3, 2, 3), 4)])
def test_diagonal_block_is_a_kronecker_sum_inverted_by_fast_diagonalisation(n, p):
    """The exact diagonal block A_KK of a cell (its volume term and the terms of
    its own facets) is the Kronecker sum sum_a M x .. x Kt_a x .. x M on an
    axis-aligned cell with cellwise kappa, with the 1D operator per axis
    Kt_a = kappa_K K + low face  kF_L (w_L (e0 d0^T + d0 e0^T) + gamma e0 e0^T)
                     + high face kF_R (-w_R (ep dp^T + dp ep^T) + gamma ep ep^T)
    (kF the harmonic mean with the neighbour and w = 1/2 on an interior facet,
    kF = kappa_K and w = 1 on the boundary). Then the generalised eigenpairs
    Kt_a S = M S Lambda, S^T M S = I, invert it exactly:
    A_KK^-1 = (S x S x S) (Lambda_x + Lambda_y + Lambda_z)^-1 (S x S x S)^T.
    Pinned against the oracle's block (the cell equation applied to unit
    vectors) and its dense inverse, on every cell of meshes with boundary,
    edge, corner and interior cells and lognormal kappa."""
    mesh = sipg.Mesh(n, p)
    d = mesh.d
    kap = np.exp(np.random.default_rng(12).normal(size=mesh.ncell))
    B = sipg.block_diagonal(mesh, kap)
    nn = list(mesh.n) + [1] * (3 - d)
    strides = [1, nn[0], nn[0] * nn[1]]
    for c in range(mesh.ncell):
        ci = [c % nn[0], (c // nn[0]) % nn[1], c // (nn[0] * nn[1])]
        kK = kap[c]
        Kt, S, lam = [], [], []
        for a in range(d):
            kL, wL, kR, wR = kK, 1.0, kK, 1.0
            if ci[a] > 0:
                kN = kap[c - strides[a]]
                kL, wL = 2 * kK * kN / (kK + kN), 0.5
            if ci[a] < nn[a] - 1:
                kN = kap[c + strides[a]]
                kR, wR = 2 * kK * kN / (kK + kN), 0.5
            e0, ep, d0, dp, g = mesh.e0, mesh.ep, mesh.d0[a], mesh.dp[a], mesh.gamma(a)
            Kt_a = (kK * mesh.K[a] + kL * (wL * (np.outer(e0, d0) + np.outer(d0, e0)) + g * np.outer(e0, e0))
                    + kR * (-wR * (np.outer(ep, dp) + np.outer(dp, ep)) + g * np.outer(ep, ep)))
            Kt.append(Kt_a)
            la, Sa = sla.eigh(Kt_a, mesh.M[a])
            S.append(Sa)
            lam.append(la)
        # node index i + q (j + q k): the slowest axis comes first in a Kronecker product
        A = np.zeros((mesh.nloc, mesh.nloc))
        for a in range(d):
            f = np.ones((1, 1))
            for b in reversed(range(d)):
                f = np.kron(f, Kt[a] if b == a else mesh.M[b])
            A += f
        Bc = B[c]
        assert np.abs(A - Bc).max() <= 1e-12 * np.abs(Bc).max()
        Sf, L = np.ones((1, 1)), np.zeros(1)
        for b in reversed(range(d)):
            Sf = np.kron(Sf, S[b])
            L = (L[:, None] + lam[b][None, :]).ravel()
        assert L.min() > 0
        Ainv = Sf @ np.diag(1.0 / L) @ Sf.T
        assert np.abs(Ainv - np.linalg.inv(Bc)).max() <= 1e-11 * np.abs(Ainv).max()


def _interior_kron_block(mesh):
    """Closed form of the diagonal block of a cell whose facets are all interior,
    for kappa = 1 on the cell and its neighbours: the Kronecker sum over axes of
    Kt_a = K + 1/2 (e0 d0^T + d0 e0^T) + gamma e0 e0^T - 1/2 (ep dp^T + dp ep^T)
    + gamma ep ep^T with 1D masses on the other axes (Sec. 4.1 block structure;
    every facet term of an interior facet carries the weight 1/2 of the averages)."""
    d = mesh.d
    Kt = []
    for a in range(d):
        e0, ep, d0, dp, g = mesh.e0, mesh.ep, mesh.d0[a], mesh.dp[a], mesh.gamma(a)
        Kt.append(mesh.K[a] + 0.5 * (np.outer(e0, d0) + np.outer(d0, e0)) + g * np.outer(e0, e0)
                  - 0.5 * (np.outer(ep, dp) + np.outer(dp, ep)) + g * np.outer(ep, ep))
    A = np.zeros((mesh.nloc, mesh.nloc))
    for a in range(d):
        f = np.ones((1, 1))
        for b in reversed(range(d)):
            f = np.kron(f, Kt[a] if b == a else mesh.M[b])
        A += f
    return A


@pytest.mark.parametrize("n,p", [((4, 3, 5), 2), ((3, 4), 3), ((3, 3, 3), 1), ((5, 3), 4)])
def test_interior_only_block_is_an_interior_cells_assembled_block(n, p):
    """Technique 4 (Sec. 4.1): every cell uses the diagonal block of an interior
    cell. With kappa = 1 that block is read off the assembled matrix (quadrature
    of the weak form, facet by facet) at a cell with no boundary facet, and it
    equals the closed-form Kronecker sum of the all-interior 1D operators."""
    mesh = sipg.Mesh(n, p)
    A = sipg.assemble(mesh).toarray()
    nn = list(mesh.n) + [1] * (3 - mesh.d)
    ci = [1, 1, 0 if mesh.d == 2 else 1]
    c = ci[0] + nn[0] * (ci[1] + nn[1] * ci[2])
    nl = mesh.nloc
    Aint = A[c * nl:(c + 1) * nl, c * nl:(c + 1) * nl]
    Kron = _interior_kron_block(mesh)
    assert np.abs(Kron - Aint).max() <= 1e-12 * np.abs(Aint).max()
    B = sipg.BlockJacobi(mesh, interior_only=True).B
    for k in range(mesh.ncell):
        assert np.abs(B[k] - Aint).max() <= 1e-12 * np.abs(Aint).max()


@pytest.mark.parametrize("n,p", [((4, 3, 5), 2), ((3, 4), 3), ((5, 3), 2)])
def test_interior_only_block_scales_with_the_cells_own_kappa(n, p):
    """With a lognormal kappa the Technique 4 block of every cell, boundary and
    corner cells included, is kappa_K times the kappa = 1 interior block (the
    reading of Technique 4 for cellwise kappa: the interior block with the
    cell's own coefficient on the cell and on all its facets). On a cell that
    touches the boundary it differs from the exact block, whose boundary facets
    carry the weight 1 instead of 1/2, and so does its inverse."""
    mesh = sipg.Mesh(n, p)
    kap = np.exp(np.random.default_rng(13).normal(size=mesh.ncell))
    Kron = _interior_kron_block(mesh)
    B = sipg.BlockJacobi(mesh, kap, interior_only=True).B
    exact = sipg.block_diagonal(mesh, kap)
    nn = list(mesh.n) + [1] * (3 - mesh.d)
    for k in range(mesh.ncell):
        ref = kap[k] * Kron
        assert np.abs(B[k] - ref).max() <= 1e-12 * np.abs(ref).max()
        ci = [k % nn[0], (k // nn[0]) % nn[1], k // (nn[0] * nn[1])]
        on_boundary = any(ci[a] in (0, nn[a] - 1) for a in range(mesh.d))
        if on_boundary:
            assert np.abs(B[k] - exact[k]).max() > 1e-3 * np.abs(exact[k]).max()
