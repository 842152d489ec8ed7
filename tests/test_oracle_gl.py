"""Gauss-Legendre basis (Sec. 6.4) in the oracle: the same SIPG problem in another
nodal basis. Every operator of the method (the bilinear form, the cellwise block
inverses, the Q1 transfer, which evaluates continuous functions at the nodes)
is basis-independent in function space, so a GL computation equals the GLL one
after the per-cell change of basis E (nodal values at the GL points)."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import hpmg, refelem, sipg


def _change_of_basis(mesh_gll):
    """E: GLL coefficients -> GL coefficients (values at the GL nodes), cellwise."""
    p, d = mesh_gll.p, mesh_gll.d
    E1 = refelem.lagrange_values(refelem.basis_nodes(p, "gll"), refelem.basis_nodes(p, "gl")).T   # [k][j]
    Ec = E1
    for _ in range(d - 1):
        Ec = np.kron(E1, Ec)
    return sp.kron(sp.identity(mesh_gll.ncell), sp.csr_matrix(Ec), format="csr")


@pytest.mark.parametrize("p", [1, 2, 4])
def test_gl_mass_is_diagonal_gauss_weights(p):
    M = refelem.mass_1d(p, "gl")
    w = refelem.gauss_legendre(p + 1)[1]
    assert np.abs(M - np.diag(w)).max() <= 1e-14
    e0, ep = refelem.endpoint_values(p, "gl")
    assert abs(e0.sum() - 1.0) <= 1e-13 and abs(ep.sum() - 1.0) <= 1e-13   # partition of unity
    assert np.count_nonzero(np.abs(e0) > 1e-12) == p + 1                     # dense, unlike GLL


@pytest.mark.parametrize("n,p", [((3, 2), 2), ((2, 2, 2), 2), ((3, 3), 3)])
def test_gl_operator_is_the_gll_operator_in_another_basis(n, p):
    kap = np.exp(np.random.default_rng(1).normal(size=int(np.prod(n))))
    mg, ml = sipg.Mesh(n, p), sipg.Mesh(n, p, basis="gl")
    E = _change_of_basis(mg).toarray()
    Ei = np.linalg.inv(E)
    A_gll = sipg.assemble(mg, kap).toarray()
    A_gl = sipg.assemble(ml, kap).toarray()
    assert np.abs(A_gl - Ei.T @ A_gll @ Ei).max() <= 1e-10 * np.abs(A_gl).max()
    # the matrix-free route agrees with the assembled GL matrix
    u = np.random.default_rng(2).normal(size=ml.ndof)
    assert np.abs(sipg.apply(ml, u, kap) - A_gl @ u).max() <= 1e-11 * np.abs(A_gl @ u).max()


def test_gl_mgmult_iterates_are_the_gll_iterates():
    """K cycles of MGMult in the GL basis give E times the GLL iterates (b_GL = E^-T b_GLL)."""
    n, p, K = (6, 5), 3, 4
    kap = np.exp(np.random.default_rng(3).normal(size=30))
    mg, ml = sipg.Mesh(n, p), sipg.Mesh(n, p, basis="gl")
    E = _change_of_basis(mg)
    b_gll = np.random.default_rng(4).normal(size=mg.ndof)
    b_gl = np.linalg.solve(E.toarray().T, b_gll)
    x_gll, _ = hpmg.mgmult(hpmg.Hierarchy(mg, kap), b_gll, eps=0.0, maxit=K)
    x_gl, _ = hpmg.mgmult(hpmg.Hierarchy(ml, kap), b_gl, eps=0.0, maxit=K)
    assert np.abs(x_gl - E @ x_gll).max() <= 1e-11 * np.abs(x_gl).max()
    # and with gradual p-coarsening
    x_gll, _ = hpmg.mgmult(hpmg.Hierarchy(mg, kap, gradual=True), b_gll, eps=0.0, maxit=K)
    x_gl, _ = hpmg.mgmult(hpmg.Hierarchy(ml, kap, gradual=True), b_gl, eps=0.0, maxit=K)
    assert np.abs(x_gl - E @ x_gll).max() <= 1e-11 * np.abs(x_gl).max()


def test_two_peak_rhs_is_minus_laplacian():
    """The closed-form f of the "two-peak" solution equals -Lap u by fourth-order
    central differences, and u vanishes on the boundary of the unit square."""
    from paper_2510_00998_gb300 import workloads as w
    rng = np.random.default_rng(5)
    x, y = rng.uniform(0.05, 0.95, 200), rng.uniform(0.05, 0.95, 200)
    h = 1e-3
    u = lambda a, b: w.two_peak_u(a, b)

    def d2(fm2, fm1, f0, fp1, fp2):
        return (-fm2 + 16 * fm1 - 30 * f0 + 16 * fp1 - fp2) / (12 * h * h)

    lap = d2(u(x - 2 * h, y), u(x - h, y), u(x, y), u(x + h, y), u(x + 2 * h, y)) + \
        d2(u(x, y - 2 * h), u(x, y - h), u(x, y), u(x, y + h), u(x, y + 2 * h))
    f = w.two_peak_f(x, y)
    assert np.abs(f + lap).max() <= 1e-6 * np.abs(f).max()
    t = np.linspace(0, 1, 11)
    for a, b in ((t, 0 * t), (t, 0 * t + 1), (0 * t, t), (0 * t + 1, t)):
        assert np.abs(w.two_peak_u(a, b)).max() == 0.0


@pytest.mark.parametrize("n,p", [((5, 4), 2), ((3, 4, 3), 2)])
def test_gl_interior_only_block_is_the_gll_one_in_another_basis(n, p):
    """Technique 4's block (an interior cell's block, own kappa) transforms like
    the exact blocks: B_GL = E^-T B_GLL E^-1 per cell."""
    kap = np.exp(np.random.default_rng(6).normal(size=int(np.prod(n))))
    mg, ml = sipg.Mesh(n, p), sipg.Mesh(n, p, basis="gl")
    E = _change_of_basis(mg).toarray()[:mg.nloc, :mg.nloc]
    Ei = np.linalg.inv(E)
    for interior_only in (False, True):
        Bg = sipg.BlockJacobi(mg, kap, interior_only=interior_only).B
        Bl = sipg.BlockJacobi(ml, kap, interior_only=interior_only).B
        for c in range(mg.ncell):
            assert np.abs(Bl[c] - Ei.T @ Bg[c] @ Ei).max() <= 1e-10 * np.abs(Bl[c]).max()
