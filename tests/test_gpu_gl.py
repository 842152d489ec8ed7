"""The Gauss-Legendre nodal basis (Sec. 6.4) on the GPU: every stage of the path
against the oracle in the GL basis, the basis invariance of the discrete
solution (GPU against GPU, no oracle), and the shape of Table 5."""
import os

import numpy as np
import pytest

from oracle import hpmg, refelem, sipg

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

DEV = "cuda:0"
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
CASES = [((7, 5), 1), ((9, 6), 2), ((5, 7), 4), ((4, 3), 6), ((5, 4, 3), 1), ((6, 5, 7), 2), ((5, 4, 6), 3),
         ((3, 4, 5), 4), ((3, 3, 2), 5), ((4, 3, 3), 6)]


@pytest.fixture(scope="module")
def dgmg():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2510_00998_gb300 import dgmg as m
    assert torch.cuda.is_available()
    return m


def _kappa(n, seed=0):
    return np.exp(np.random.default_rng(seed).normal(size=int(np.prod(n))))


def _t(x):
    return torch.tensor(np.asarray(x, dtype=np.float64), device=DEV)


def _np(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _ctx(dgmg, n, p, kap=None, **kw):
    return dgmg.Context(n, p, kap, basis=dgmg.DGMG_BASIS_GL, **kw)


def test_nodes_and_invalid_basis(dgmg):
    ctx = _ctx(dgmg, (4, 4), 3)
    assert np.abs(ctx.gll_nodes() - refelem.gauss_legendre(4)[0]).max() <= 1e-15
    with pytest.raises(dgmg.DGMGError):
        dgmg.Context((4, 4), 2, basis=2)
    with pytest.raises(dgmg.DGMGError):
        dgmg.Batch([((4, 4, 4), 2, None)], basis=dgmg.DGMG_BASIS_GL)


@pytest.mark.parametrize("n,p", CASES)
def test_apply_and_residual(dgmg, n, p):
    """y = A u in the GL basis (dense cell-to-facet projection) to rounding."""
    kap = _kappa(n)
    mesh = sipg.Mesh(n, p, basis="gl")
    ctx = _ctx(dgmg, n, p, kap)
    rng = np.random.default_rng(1)
    u, b = rng.normal(size=mesh.ndof), rng.normal(size=mesh.ndof)
    y = torch.empty(mesh.ndof, dtype=torch.float64, device=DEV)
    ctx.apply(_t(u), y)
    assert _rel(_np(y), sipg.apply(mesh, u, kap)) <= 1e-12
    r = torch.empty_like(y)
    ctx.residual(_t(u), _t(b), r)
    assert _rel(_np(r), sipg.residual(mesh, u, b, kap)) <= 1e-12


def _oracle_traces(mesh, u):
    """Oracle projections (values e^T u and derivatives d^T u along each axis at
    both ends) in the library's layout [cell][face][value, derivative][node]."""
    U = mesh.grid(u)
    d, q = mesh.d, mesh.q
    out = np.zeros((mesh.ncell, 2 * d, 2, q ** (d - 1)))
    for a in range(d):
        na = mesh.node_axis(a)
        for side, (ev, dv) in enumerate([(mesh.e0, mesh.d0[a]), (mesh.ep, mesh.dp[a])]):
            out[:, 2 * a + side, 0, :] = np.tensordot(U, ev, axes=([na], [0])).reshape(mesh.ncell, -1)
            out[:, 2 * a + side, 1, :] = np.tensordot(U, dv, axes=([na], [0])).reshape(mesh.ncell, -1)
    return out.reshape(-1)


@pytest.mark.parametrize("n,p", CASES)
def test_project_with_and_without_prolongation(dgmg, n, p):
    mesh = sipg.Mesh(n, p, basis="gl")
    ctx = _ctx(dgmg, n, p)
    rng = np.random.default_rng(2)
    u = rng.normal(size=mesh.ndof)
    ut = _t(u)
    tr = torch.empty(ctx.trace_size(), dtype=torch.float64, device=DEV)
    ctx.project(ut, None, tr)
    assert _rel(_np(tr), _oracle_traces(mesh, u)) <= 1e-13
    e = rng.normal(size=hpmg.interior_vertex_count(n))
    ctx.project(ut, _t(e), tr)
    u2 = u + hpmg.p_prolongation(mesh) @ e
    assert _rel(_np(ut), u2) <= 1e-14
    assert _rel(_np(tr), _oracle_traces(mesh, u2)) <= 1e-13


@pytest.mark.parametrize("n,p", CASES)
def test_smooth_matches_alg4(dgmg, n, p):
    kap = _kappa(n, 3)
    mesh = sipg.Mesh(n, p, basis="gl")
    ctx = _ctx(dgmg, n, p, kap, omega_dg=0.7)
    rng = np.random.default_rng(3)
    u, b = rng.normal(size=mesh.ndof), rng.normal(size=mesh.ndof)
    ut = _t(u)
    ctx.smooth(ut, _t(b), 3)
    ref, _ = sipg.BlockJacobi(mesh, kap).step_alg4(u, b, 0.7, 3)
    assert _rel(_np(ut), ref) <= 1e-11


@pytest.mark.parametrize("n,p", [((9, 6), 2), ((5, 4, 6), 3)])
def test_smooth_interior_only_block(dgmg, n, p):
    kap = _kappa(n, 4)
    mesh = sipg.Mesh(n, p, basis="gl")
    ctx = _ctx(dgmg, n, p, kap, block_inverse=dgmg.DGMG_BLOCK_INTERIOR_ONLY)
    rng = np.random.default_rng(5)
    u, b = rng.normal(size=mesh.ndof), rng.normal(size=mesh.ndof)
    ut = _t(u)
    ctx.smooth(ut, _t(b), 2)
    ref = sipg.BlockJacobi(mesh, kap, interior_only=True).step_alg2(u, b, 0.8, 2)
    assert _rel(_np(ut), ref) <= 1e-11


@pytest.mark.parametrize("n,p", [((9, 6), 2), ((5, 4, 6), 3), ((3, 4, 5), 4)])
def test_residual_restrict(dgmg, n, p):
    kap = _kappa(n, 6)
    mesh = sipg.Mesh(n, p, basis="gl")
    ctx = _ctx(dgmg, n, p, kap)
    rng = np.random.default_rng(6)
    u, b = rng.normal(size=mesh.ndof), rng.normal(size=mesh.ndof)
    ut, bt = _t(u), _t(b)
    tr = torch.empty(ctx.trace_size(), dtype=torch.float64, device=DEV)
    ctx.project(ut, None, tr)
    r = torch.empty_like(ut)
    rc = torch.empty(ctx.cg_size(0), dtype=torch.float64, device=DEV)
    ctx.residual_restrict(ut, bt, tr, r, rc)
    ref = sipg.residual(mesh, u, b, kap)
    assert _rel(_np(r), ref) <= 1e-12
    assert _rel(_np(rc), hpmg.p_prolongation(mesh).T @ ref) <= 1e-12


@pytest.mark.parametrize("n,p,prec,gradual", [((16, 16), 2, 0, 0), ((6, 5, 7), 2, 0, 0), ((4, 4, 4), 4, 0, 0),
                                              ((5, 6, 7), 3, 1, 0), ((7, 6, 5), 4, 1, 0), ((9, 7), 3, 0, 1),
                                              ((5, 4, 5), 4, 0, 1), ((5, 4, 5), 4, 1, 1)])
def test_vcycle(dgmg, n, p, prec, gradual):
    """FP64 to rounding (1e-11), FP32 within the V-cycle's FP32 bound (2e-5)."""
    kap = _kappa(n, 8)
    mesh = sipg.Mesh(n, p, basis="gl")
    ctx = _ctx(dgmg, n, p, kap, precision=prec, p_coarsening=gradual)
    hier = hpmg.Hierarchy(mesh, kap, gradual=bool(gradual))
    r = np.random.default_rng(9).normal(size=mesh.ndof)
    e = torch.empty(mesh.ndof, dtype=torch.float64, device=DEV)
    ctx.vcycle(_t(r), e)
    assert _rel(_np(e), hier.vcycle(r)) <= (1e-11 if prec == 0 else 2e-5)
    assert dgmg.wait_timeouts() == 0


@pytest.mark.parametrize("n,p,prec,outer", [((8, 8, 8), 2, 0, 0), ((6, 5, 4), 3, 0, 0), ((8, 8, 8), 3, 1, 0),
                                            ((12, 10), 4, 1, 1), ((10, 9, 8), 4, 1, 2)])
def test_solve_matches_oracle(dgmg, n, p, prec, outer):
    kap = _kappa(n, 10)
    mesh = sipg.Mesh(n, p, basis="gl")
    ctx = _ctx(dgmg, n, p, kap, precision=prec, outer=outer)
    b = np.random.default_rng(12).normal(size=mesh.ndof)
    x = torch.zeros(mesh.ndof, dtype=torch.float64, device=DEV)
    st, _ = ctx.solve(_t(b), x)
    assert st.rel_residual <= 1e-10
    x_ref, _, _ = hpmg.pcg(hpmg.Hierarchy(mesh, kap), b, rtol=1e-13)
    assert np.linalg.norm(_np(x) - x_ref) <= 1e-9 * np.linalg.norm(x_ref)


def _gll_to_gl(x, n, p):
    """Per cell, the GLL coefficients mapped to the values at the GL nodes."""
    E = torch.tensor(refelem.lagrange_values(refelem.basis_nodes(p, "gll"), refelem.basis_nodes(p, "gl")).T,
                     device=DEV)
    q, d = p + 1, len(n)
    X = x.view(-1, *([q] * d))          # [cell][(k)][j][i], x fastest
    if d == 2:
        return torch.einsum("ai,bj,cji->cba", E, E, X).reshape(-1)
    return torch.einsum("ai,bj,ck,dkji->dcba", E, E, E, X).reshape(-1)


@pytest.mark.parametrize("n,p", [((24, 20), 3), ((10, 9, 8), 2), ((7, 6, 8), 4)])
def test_solution_is_basis_invariant(dgmg, n, p):
    """The same load f gives the same discrete function in both bases: x_GL = E
    x_GLL, with E the GLL basis evaluated at the GL nodes (Sec. 6.4: the basis
    changes the algebra, not the discrete solution). GPU against GPU."""
    from paper_2510_00998_gb300 import workloads
    kap = _kappa(n, 11)
    xs = []
    for basis in (dgmg.DGMG_BASIS_GLL, dgmg.DGMG_BASIS_GL):
        ctx = dgmg.Context(n, p, kap, basis=basis, rtol=1e-11, maxit=400)
        b = workloads.sine_rhs(ctx, DEV)
        x = torch.zeros_like(b)
        st, _ = ctx.solve(b, x)
        assert st.rel_residual <= 1e-11
        xs.append(x)
    ref = _gll_to_gl(xs[0], n, p)
    assert float((xs[1] - ref).abs().max() / ref.abs().max()) <= 1e-8


@pytest.mark.parametrize("n,p,gradual", [((9, 9), 2, 0), ((12, 10), 3, 0), ((6, 5, 4), 2, 0), ((9, 9), 4, 1)])
def test_mgmult_iterates_match_oracle(dgmg, n, p, gradual):
    K, nu = 4, 3
    kap = _kappa(n, 13)
    mesh = sipg.Mesh(n, p, basis="gl")
    b = np.random.default_rng(17).normal(size=mesh.ndof)
    hier = hpmg.Hierarchy(mesh, kap, factor=3, nu_pre=nu, nu_post=nu, gradual=bool(gradual))
    u_ref, _ = hpmg.mgmult(hier, b, eps=0.0, maxit=K)
    ctx = _ctx(dgmg, n, p, kap, outer=dgmg.DGMG_OUTER_MGMULT, coarsening=3, nu_pre=nu, nu_post=nu, rtol=1e-30,
               maxit=K, p_coarsening=gradual)
    x = torch.zeros(mesh.ndof, dtype=torch.float64, device=DEV)
    st, _ = ctx.solve(_t(b), x, allow_notconverged=True)
    assert st.iterations == K
    assert _rel(_np(x), u_ref) <= 1e-11


@pytest.mark.parametrize("n,p", [((9, 9), 2), ((9, 9), 3), ((27, 27), 2)])
def test_table5_cycle_counts_match_oracle(dgmg, n, p):
    """Two-peak solution in the GL basis: both exit criteria take the oracle's
    number of cycles (+-1 where the ratio lands at the threshold)."""
    from paper_2510_00998_gb300 import workloads
    nu = 3
    mesh = sipg.Mesh(n, p, basis="gl")
    b = sipg.load_vector(mesh, lambda x, y: workloads.two_peak_f(x, y))
    hier = hpmg.Hierarchy(mesh, factor=3, nu_pre=nu, nu_post=nu)
    _, k_un = hpmg.mgmult(hier, b, eps=1e-7)
    _, k_pr = hpmg.mgmult(hier, b, eps=1e-7, residual_kind="prec")
    for outer, k_ref in ((dgmg.DGMG_OUTER_MGMULT, k_un), (dgmg.DGMG_OUTER_MGMULT_PREC, k_pr)):
        ctx = _ctx(dgmg, n, p, outer=outer, coarsening=3, nu_pre=nu, nu_post=nu, rtol=1e-7, maxit=300)
        bt = workloads.two_peak_rhs_2d(ctx, DEV)
        assert _rel(_np(bt), b) <= 1e-12          # the library's load vector is the oracle's
        x = torch.zeros_like(bt)
        st, _ = ctx.solve(bt, x)
        assert abs(st.iterations - k_ref) <= 1, (outer, st.iterations, k_ref)


def test_table5_shape(dgmg):
    """A comparison under a reading, not a pin (omega, nu and the penalty of
    Tables 3-5 are not stated;
    nu = 4, omega = 0.8 is the reading that reproduces them best): on 9^2, 27^2,
    81^2 and p = 2..4 the GL cycle counts lie between 0.7x the count of Table 5
    and one cycle above it, and, as Sec. 6.4 reports, stay close to the GLL
    counts of the same two-peak problem: the unpreconditioned count at or a
    little above the GLL one, the preconditioned one within a cycle."""
    from paper_2510_00998_gb300 import workloads
    rows = np.loadtxt(os.path.join(GOLDEN, "table5_two_peak_cycles.txt"))
    meshes, degrees = (9, 27, 81), (2, 3, 4)
    gll = workloads.tables34(meshes=meshes, degrees=degrees, rhs="two_peak", basis=0)
    gl = workloads.tables34(meshes=meshes, degrees=degrees, rhs="two_peak", basis=1)
    for n, p, _, _, gl_un, gl_pr in rows:
        key = (int(n), int(p))
        if key not in gl:
            continue
        k_un, k_pr = gl[key]
        assert 0.7 * gl_un <= k_un <= gl_un + 1, (key, k_un, gl_un)
        assert 0.7 * gl_pr <= k_pr <= gl_pr + 1, (key, k_pr, gl_pr)
        assert gll[key][0] <= k_un <= 1.1 * gll[key][0] + 1, (key, gl[key], gll[key])
        assert abs(k_pr - gll[key][1]) <= 1, (key, gl[key], gll[key])
