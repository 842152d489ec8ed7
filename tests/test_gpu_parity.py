"""GPU parity: every stage of the path through the C ABI against the FP64 oracle.

Sizes span several CTAs (a CTA holds 128/q^(d-1) cells) and ragged tails
(cell counts not divisible by the CTA size, unequal n per axis)."""
import numpy as np
import pytest

from oracle import hpmg, sipg

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def dgmg():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2510_00998_gb300 import dgmg as m
    assert torch.cuda.is_available()
    return m


DEV = "cuda:0"
CASES = [((7, 5), 1), ((9, 6), 2), ((5, 7), 4), ((4, 3), 6), ((5, 4, 3), 1), ((6, 5, 7), 2), ((5, 4, 6), 3),
         ((3, 4, 5), 4), ((3, 3, 2), 5)]
KINDS = ["one", "lognormal"]


def _kappa(n, kind, seed=0):
    if kind == "one":
        return None
    return np.exp(np.random.default_rng(seed).normal(size=int(np.prod(n))))


def _t(x):
    return torch.tensor(np.asarray(x, dtype=np.float64), device=DEV)


def _np(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("n,p", CASES)
@pytest.mark.parametrize("kind", KINDS)
def test_apply_and_residual(dgmg, n, p, kind):
    kap = _kappa(n, kind)
    mesh = sipg.Mesh(n, p)
    ctx = dgmg.Context(n, p, kap)
    rng = np.random.default_rng(1)
    u, b = rng.normal(size=mesh.ndof), rng.normal(size=mesh.ndof)
    ut, bt = _t(u), _t(b)
    y = torch.empty_like(ut)
    ctx.apply(ut, y)
    assert _rel(_np(y), sipg.apply(mesh, u, kap)) <= 1e-12
    r = torch.empty_like(ut)
    ctx.residual(ut, bt, r)
    ref = sipg.residual(mesh, u, b, kap)
    assert _rel(_np(r), ref) <= 1e-12


def _oracle_traces(mesh, u):
    """Oracle projections rearranged to the library's per-cell trace layout:
    [cell][face = 2 axis + side][value, d/d(+axis)][tangential node]."""
    U = mesh.grid(u)
    d, q = mesh.d, mesh.q
    out = np.zeros((mesh.ncell, 2 * d, 2, q ** (d - 1)))
    for a in range(d):
        na = mesh.node_axis(a)
        for side, (ev, dv) in enumerate([(mesh.e0, mesh.d0[a]), (mesh.ep, mesh.dp[a])]):
            val = np.tensordot(U, ev, axes=([na], [0]))       # removes the node axis
            der = np.tensordot(U, dv, axes=([na], [0]))
            # remaining node axes are ordered highest axis first; flatten to lowest fastest
            out[:, 2 * a + side, 0, :] = val.reshape(mesh.ncell, -1)
            out[:, 2 * a + side, 1, :] = der.reshape(mesh.ncell, -1)
    return out.reshape(-1)


@pytest.mark.parametrize("n,p", CASES)
def test_project_with_and_without_prolongation(dgmg, n, p):
    mesh = sipg.Mesh(n, p)
    ctx = dgmg.Context(n, p)
    rng = np.random.default_rng(2)
    u = rng.normal(size=mesh.ndof)
    ut = _t(u)
    tr = torch.empty(ctx.trace_size(), dtype=torch.float64, device=DEV)
    ctx.project(ut, None, tr)
    assert _rel(_np(tr), _oracle_traces(mesh, u)) <= 1e-13
    assert np.array_equal(_np(ut), u)
    e = rng.normal(size=hpmg.interior_vertex_count(n))
    ctx.project(ut, _t(e), tr)
    u2 = u + hpmg.p_prolongation(mesh) @ e
    assert _rel(_np(ut), u2) <= 1e-14
    assert _rel(_np(tr), _oracle_traces(mesh, u2)) <= 1e-13


@pytest.mark.parametrize("n,p", CASES)
@pytest.mark.parametrize("kind", KINDS)
def test_smooth_matches_alg4(dgmg, n, p, kind):
    kap = _kappa(n, kind)
    mesh = sipg.Mesh(n, p)
    ctx = dgmg.Context(n, p, kap, omega_dg=0.7)
    rng = np.random.default_rng(3)
    u, b = rng.normal(size=mesh.ndof), rng.normal(size=mesh.ndof)
    ut = _t(u)
    ctx.smooth(ut, _t(b), 3)
    ref, _ = sipg.BlockJacobi(mesh, kap).step_alg4(u, b, 0.7, 3)
    assert _rel(_np(ut), ref) <= 1e-11


@pytest.mark.parametrize("n,p", [((9, 6), 2), ((5, 4, 6), 3)])
def test_smooth_interior_only_block(dgmg, n, p):
    kap = _kappa(n, "lognormal", 4)
    mesh = sipg.Mesh(n, p)
    ctx = dgmg.Context(n, p, kap, block_inverse=dgmg.DGMG_BLOCK_INTERIOR_ONLY)
    rng = np.random.default_rng(5)
    u, b = rng.normal(size=mesh.ndof), rng.normal(size=mesh.ndof)
    ut = _t(u)
    ctx.smooth(ut, _t(b), 2)
    ref = sipg.BlockJacobi(mesh, kap, interior_only=True).step_alg2(u, b, 0.8, 2)
    assert _rel(_np(ut), ref) <= 1e-11


@pytest.mark.parametrize("n,p", CASES)
@pytest.mark.parametrize("kind", KINDS)
def test_residual_restrict(dgmg, n, p, kind):
    kap = _kappa(n, kind)
    mesh = sipg.Mesh(n, p)
    ctx = dgmg.Context(n, p, kap)
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


@pytest.mark.parametrize("n,f", [((16, 16), 2), ((13, 11), 2), ((9, 10), 3), ((8, 7, 6), 2), ((9, 9, 5), 3)])
def test_cg_levels(dgmg, n, f):
    kap = _kappa(n, "lognormal", 7)
    mesh = sipg.Mesh(n, 1)
    ctx = dgmg.Context(n, 1, kap, coarsening=f, omega_cg=0.7)
    hier = hpmg.Hierarchy(mesh, kap, factor=f, omega_cg=0.7)
    assert ctx.info.nlevels_cg == hier.nlevels
    rng = np.random.default_rng(8)
    for lvl in range(hier.nlevels):
        nv = hier.A[lvl].shape[0]
        assert ctx.cg_size(lvl) == nv
        u, b = rng.normal(size=nv), rng.normal(size=nv)
        r = torch.empty(nv, dtype=torch.float64, device=DEV)
        ctx.cg_residual(lvl, _t(u), _t(b), r)
        assert _rel(_np(r), b - hier.A[lvl] @ u) <= 1e-12
        ut = _t(u)
        ctx.cg_smooth(lvl, ut, _t(b), 3)
        assert _rel(_np(ut), hier.cg_jacobi(lvl, u, b, 3)) <= 1e-12
        if lvl + 1 < hier.nlevels:
            nc = hier.A[lvl + 1].shape[0]
            rc = torch.empty(nc, dtype=torch.float64, device=DEV)
            ctx.h_restrict(lvl, _t(u), rc)
            assert _rel(_np(rc), hier.Ph[lvl].T @ u) <= 1e-13
            ec = rng.normal(size=nc)
            uf = _t(b)
            ctx.h_prolong(lvl, _t(ec), uf)
            assert _rel(_np(uf), b + hier.Ph[lvl] @ ec) <= 1e-13
    nc = hier.A[-1].shape[0]
    rr = rng.normal(size=nc)
    e = torch.empty(nc, dtype=torch.float64, device=DEV)
    ctx.coarse_solve(_t(rr), e)
    assert _rel(_np(e), hier.coarse_solve(rr)) <= 1e-12


@pytest.mark.parametrize("n,p", [((16, 16), 2), ((9, 6), 3), ((6, 5, 7), 2), ((4, 4, 4), 3), ((5, 3, 4), 4)])
@pytest.mark.parametrize("kind", KINDS)
def test_vcycle_fp64(dgmg, n, p, kind):
    kap = _kappa(n, kind)
    mesh = sipg.Mesh(n, p)
    ctx = dgmg.Context(n, p, kap)
    hier = hpmg.Hierarchy(mesh, kap)
    r = np.random.default_rng(9).normal(size=mesh.ndof)
    e = torch.empty(mesh.ndof, dtype=torch.float64, device=DEV)
    ctx.vcycle(_t(r), e)
    assert _rel(_np(e), hier.vcycle(r)) <= 1e-11


@pytest.mark.parametrize("n,p", [((16, 16), 2), ((6, 5, 7), 2), ((4, 4, 4), 4), ((5, 6, 7), 3), ((7, 6, 5), 4),
                                 ((5, 4, 3), 1), ((4, 3, 5), 5), ((9, 8, 7), 4)])
def test_vcycle_mixed_fp32(dgmg, n, p):
    """FP32 V-cycle: every stage in FP32 except the FP64 coarsest solve; bound on
    the relative max error derived from FP32 rounding through ~10 stages of
    O(q) sums each: 2e-5 (measured well below)."""
    kap = _kappa(n, "lognormal")
    mesh = sipg.Mesh(n, p)
    ctx = dgmg.Context(n, p, kap, precision=dgmg.DGMG_MIXED_FP32)
    hier = hpmg.Hierarchy(mesh, kap)
    r = np.random.default_rng(10).normal(size=mesh.ndof)
    e = torch.empty(mesh.ndof, dtype=torch.float64, device=DEV)
    ctx.vcycle(_t(r), e)
    assert _rel(_np(e), hier.vcycle(r)) <= 2e-5
    assert dgmg.wait_timeouts() == 0


@pytest.mark.parametrize("n,p,kind,prec,outer", [((16, 16), 2, "one", 0, 0), ((8, 8, 8), 2, "lognormal", 0, 0),
                                                 ((6, 5, 4), 3, "lognormal", 0, 0),
                                                 ((8, 8, 8), 3, "lognormal", 1, 0), ((12, 10), 4, "lognormal", 1, 0),
                                                 ((8, 8, 8), 3, "lognormal", 1, 1), ((12, 10), 4, "lognormal", 1, 1),
                                                 ((10, 9, 8), 4, "lognormal", 1, 2)])
def test_solve_matches_oracle(dgmg, n, p, kind, prec, outer):
    """FP64 PCG, mixed precision with FP64 PCG around the FP32 V-cycle, and the
    reliable-update FP32 CG (outer 0 = the precision's default)."""
    kap = _kappa(n, kind)
    mesh = sipg.Mesh(n, p)
    ctx = dgmg.Context(n, p, kap, precision=prec, outer=outer)
    b = np.random.default_rng(12).normal(size=mesh.ndof)
    x = torch.zeros(mesh.ndof, dtype=torch.float64, device=DEV)
    st, _ = ctx.solve(_t(b), x)
    assert st.rel_residual <= 1e-10
    x_ref, _, _ = hpmg.pcg(hpmg.Hierarchy(mesh, kap), b, rtol=1e-13)
    assert np.linalg.norm(_np(x) - x_ref) <= 1e-9 * np.linalg.norm(x_ref)


def test_solve_config_2d_16_p2(dgmg):
    """2D unit square, 16x16, p=2, manufactured u = sin(pi x) sin(pi y)."""
    n, p = (16, 16), 2
    mesh = sipg.Mesh(n, p)
    uex = lambda x, y: np.sin(np.pi * x) * np.sin(np.pi * y)
    f = lambda x, y: 2 * np.pi ** 2 * uex(x, y)
    b = sipg.load_vector(mesh, f)
    ctx = dgmg.Context(n, p)
    # the library's own load vector from f at its quadrature points
    mq = p + 2
    xq = torch.empty(mesh.ncell * mq ** 2 * 2, dtype=torch.float64, device=DEV)
    ctx.quad_points(xq)
    X = _np(xq).reshape(-1, 2)
    fq = _t(f(X[:, 0], X[:, 1]))
    bt = torch.empty(mesh.ndof, dtype=torch.float64, device=DEV)
    ctx.load_vector(fq, bt)
    assert _rel(_np(bt), b) <= 1e-13
    x = torch.zeros_like(bt)
    st, _ = ctx.solve(bt, x)
    assert st.rel_residual <= 1e-10
    x_ref, _, _ = hpmg.pcg(hpmg.Hierarchy(mesh), b, rtol=1e-13)
    assert np.linalg.norm(_np(x) - x_ref) <= 1e-9 * np.linalg.norm(x_ref)
    assert sipg.l2_error(mesh, _np(x), uex) < 1e-3


def test_solve_host_entry(dgmg):
    n, p = (6, 6, 5), 2
    mesh = sipg.Mesh(n, p)
    ctx = dgmg.Context(n, p)
    b = np.random.default_rng(13).normal(size=mesh.ndof)
    bh = torch.tensor(b).pin_memory()
    xh = torch.zeros(mesh.ndof, dtype=torch.float64).pin_memory()
    st = ctx.solve_host(bh, xh)
    assert st.rel_residual <= 1e-10
    x_ref, _, _ = hpmg.pcg(hpmg.Hierarchy(mesh), b, rtol=1e-13)
    assert np.linalg.norm(xh.numpy() - x_ref) <= 1e-9 * np.linalg.norm(x_ref)


def test_invalid_arguments_fail_loudly(dgmg):
    with pytest.raises(dgmg.DGMGError):
        dgmg.Context((4, 4), 0)
    with pytest.raises(dgmg.DGMGError):
        dgmg.Context((1, 4), 2)
    with pytest.raises(dgmg.DGMGError):
        dgmg.Context((4, 4), 2, kappa=np.array([1.0] * 15 + [-1.0]))
    ctx = dgmg.Context((4, 4), 2)
    with pytest.raises(dgmg.DGMGError):
        ctx.h_restrict(5, torch.zeros(9, dtype=torch.float64, device=DEV), torch.zeros(1, dtype=torch.float64,
                                                                                     device=DEV))


def test_nonfinite_rhs_reported(dgmg):
    ctx = dgmg.Context((4, 4), 2)
    b = torch.zeros(ctx.ndof, dtype=torch.float64, device=DEV)
    b[3] = float("nan")
    x = torch.zeros_like(b)
    with pytest.raises(dgmg.DGMGError) as ei:
        ctx.solve(b, x)
    assert ei.value.code == dgmg.DGMG_ENONFINITE


@pytest.mark.parametrize("n,p", [((2, 2), 1), ((2, 2), 6), ((2, 3), 3), ((2, 2, 2), 1), ((2, 2, 2), 4),
                                 ((2, 3, 2), 6)])
def test_minimum_meshes_and_degree_extremes(dgmg, n, p):
    """Smallest meshes (two cells per axis, one Q1 unknown per axis) and the
    lowest and highest supported degrees: apply, smoothing, V-cycle, solve."""
    kap = _kappa(n, "lognormal", 9)
    mesh = sipg.Mesh(n, p)
    ctx = dgmg.Context(n, p, kap)
    rng = np.random.default_rng(14)
    u, b = rng.normal(size=mesh.ndof), rng.normal(size=mesh.ndof)
    y = torch.empty(mesh.ndof, dtype=torch.float64, device=DEV)
    ctx.apply(_t(u), y)
    assert _rel(_np(y), sipg.apply(mesh, u, kap)) <= 1e-12
    ut = _t(u)
    ctx.smooth(ut, _t(b), 2)
    ref, _ = sipg.BlockJacobi(mesh, kap).step_alg4(u, b, 0.8, 2)
    assert _rel(_np(ut), ref) <= 1e-11
    hier = hpmg.Hierarchy(mesh, kap)
    e = torch.empty_like(y)
    ctx.vcycle(_t(b), e)
    assert _rel(_np(e), hier.vcycle(b)) <= 1e-11
    x = torch.zeros_like(y)
    st, _ = ctx.solve(_t(b), x)
    assert st.rel_residual <= 1e-10


def test_zero_rhs_returns_zero(dgmg):
    ctx = dgmg.Context((4, 5, 3), 2)
    b = torch.zeros(ctx.ndof, dtype=torch.float64, device=DEV)
    x = torch.zeros_like(b)
    st, _ = ctx.solve(b, x)
    assert st.iterations == 0 and float(x.abs().max()) == 0.0


@pytest.mark.parametrize("prec", [0, 1])
def test_maxit_exhaustion_reports_not_converged(dgmg, prec):
    """maxit reached: DGMG_ENOTCONVERGED, x holds a finite last iterate whose
    residual is below the initial one."""
    n, p = (8, 8, 8), 3
    ctx = dgmg.Context(n, p, _kappa(n, "lognormal", 2), precision=prec, maxit=3)
    b = torch.tensor(np.random.default_rng(15).normal(size=ctx.ndof), device=DEV)
    x = torch.zeros_like(b)
    with pytest.raises(dgmg.DGMGError) as ei:
        ctx.solve(b, x)
    assert ei.value.code == dgmg.DGMG_ENOTCONVERGED
    assert bool(torch.isfinite(x).all())
    r = torch.empty_like(b)
    ctx.residual(x, b, r)
    assert float(r.norm()) < float(b.norm())


@pytest.mark.parametrize("n,p,prec", [((8, 8, 8), 3, 0), ((9, 8, 7), 4, 1), ((12, 10), 4, 0)])
def test_autotuned_tiles(dgmg, n, p, prec):
    """The tile autotuner only changes how cells are grouped into CTAs (and which
    of two smoothing kernels with different summation orders runs): FP64
    results agree with the default tiles to rounding; every solve meets the
    oracle bound. The chosen tiles are reported by dgmg_info."""
    kap = _kappa(n, "lognormal")
    mesh = sipg.Mesh(n, p)
    b = np.random.default_rng(21).normal(size=mesh.ndof)
    xs = []
    for tune in (0, 1):
        ctx = dgmg.Context(n, p, kap, precision=prec, autotune=tune)
        tiles = list(ctx.info.tiles)
        assert all(t >= 0 for t in tiles) and tiles[0] > 0   # 0: the one-thread-per-cell kernel
        if prec == 0:
            assert tiles[3:] == [0, 0, 0]
        x = torch.zeros(mesh.ndof, dtype=torch.float64, device=DEV)
        st, _ = ctx.solve(_t(b), x)
        assert st.rel_residual <= 1e-10
        xs.append(_np(x))
    if prec == 0:
        assert np.abs(xs[0] - xs[1]).max() <= 1e-12 * np.abs(xs[0]).max()
    x_ref, _, _ = hpmg.pcg(hpmg.Hierarchy(mesh, kap), b, rtol=1e-13)
    for x in xs:
        assert np.linalg.norm(x - x_ref) <= 1e-9 * np.linalg.norm(x_ref)


@pytest.mark.parametrize("n,p,prec,gradual", [((8, 7, 6), 3, 0, 0), ((9, 8, 7), 4, 1, 0), ((12, 10), 4, 0, 1),
                                              ((6, 6, 5), 3, 1, 1)])
def test_update_kappa_equals_fresh_context(dgmg, n, p, prec, gradual):
    """dgmg_update_kappa (factors recomputed on the device, Q1 operators on the
    host, no allocation) gives the context of the new kappa: the V-cycle equals a
    fresh context's to rounding, the solve meets the oracle bound."""
    kap1, kap2 = _kappa(n, "lognormal", 31), _kappa(n, "lognormal", 32)
    mesh = sipg.Mesh(n, p)
    ctx = dgmg.Context(n, p, kap1, precision=prec, p_coarsening=gradual)
    ctx.update_kappa(kap2)
    fresh = dgmg.Context(n, p, kap2, precision=prec, p_coarsening=gradual)
    assert ctx.info.device_bytes == fresh.info.device_bytes
    r = np.random.default_rng(33).normal(size=mesh.ndof)
    e1, e2 = (torch.empty(mesh.ndof, dtype=torch.float64, device=DEV) for _ in range(2))
    ctx.vcycle(_t(r), e1)
    fresh.vcycle(_t(r), e2)
    assert _rel(_np(e1), _np(e2)) <= (1e-13 if prec == 0 else 1e-6)
    b = np.random.default_rng(34).normal(size=mesh.ndof)
    x = torch.zeros(mesh.ndof, dtype=torch.float64, device=DEV)
    st, _ = ctx.solve(_t(b), x)
    assert st.rel_residual <= 1e-10
    x_ref, _, _ = hpmg.pcg(hpmg.Hierarchy(mesh, kap2), b, rtol=1e-13)
    assert np.linalg.norm(_np(x) - x_ref) <= 1e-9 * np.linalg.norm(x_ref)
    with pytest.raises(dgmg.DGMGError):
        ctx.update_kappa(-kap2)


@pytest.mark.parametrize("n,p,nu,prec", [((24, 20, 18), 1, (2, 2), 0), ((24, 20, 18), 1, (3, 1), 0),
                                         ((17, 33, 9), 1, (1, 2), 0), ((70, 52), 1, (2, 2), 0),
                                         ((61, 45), 2, (0, 3), 0), ((24, 20, 18), 1, (2, 2), 1),
                                         ((48, 44, 40), 1, (2, 2), 0)])
def test_vcycle_q1_one_launch(dgmg, n, p, nu, prec):
    """The Q1 levels of a V-cycle run as one cooperative launch: the finer
    levels on the whole grid with grid-wide barriers, the small levels (up to 512
    vertices in FP32; in FP64 only a one-vertex coarsest level) and the coarsest
    solve in one block. Meshes
    with several grid-wide
    levels, odd and even numbers of Jacobi steps (the result buffer flips with
    their parity) and nu_pre = 0 (no pre-smoothing: a zeroed iterate)."""
    kap = _kappa(n, "lognormal", 4)
    mesh = sipg.Mesh(n, p)
    ctx = dgmg.Context(n, p, kap, nu_pre=nu[0], nu_post=nu[1],
                       precision=dgmg.DGMG_MIXED_FP32 if prec else dgmg.DGMG_FP64)
    hier = hpmg.Hierarchy(mesh, kap, nu_pre=nu[0], nu_post=nu[1])
    assert hier.A[0].shape[0] > 512                 # at least one level on the whole grid
    r = np.random.default_rng(11).normal(size=mesh.ndof)
    e = torch.empty(mesh.ndof, dtype=torch.float64, device=DEV)
    ctx.vcycle(_t(r), e)
    torch.cuda.synchronize()
    before = dgmg.kernel_launches()
    ctx.vcycle(_t(r), e)
    torch.cuda.synchronize()
    launches = dgmg.kernel_launches() - before
    # a launch per step would take 7 or more for each of the hier.nlevels - 1 levels
    assert launches <= sum(nu) + 8 < sum(nu) + 1 + 7 * (hier.nlevels - 1)
    assert _rel(_np(e), hier.vcycle(r)) <= (2e-5 if prec else 1e-11)
    assert dgmg.wait_timeouts() == 0


def test_binding_rejects_short_vectors(dgmg):
    """Every method checks that its tensors hold the lengths the library reads
    or writes (DG vectors, traces, Q1 levels), before anything is launched."""
    ctx = dgmg.Context((4, 4, 4), 2)

    def z(n, dtype=torch.float64):
        return torch.zeros(max(n, 0), dtype=dtype, device=DEV)
    nd, nt, n0 = ctx.ndof, ctx.trace_size(), ctx.cg_size(0)
    short = z(nd - 1)
    calls = [lambda: ctx.apply(short, z(nd)), lambda: ctx.apply(z(nd), short),
             lambda: ctx.residual(z(nd), z(nd), short), lambda: ctx.smooth(short, z(nd), 1),
             lambda: ctx.vcycle(z(nd), short), lambda: ctx.solve(short, z(nd)),
             lambda: ctx.project(z(nd), z(n0 - 1), z(nt)), lambda: ctx.project(z(nd), None, z(nt - 1)),
             lambda: ctx.residual_restrict(z(nd), z(nd), z(nt), z(nd), z(n0 - 1)),
             lambda: ctx.cg_residual(0, z(n0), z(n0), z(n0 - 1)),
             lambda: ctx.h_restrict(0, z(n0), z(ctx.cg_size(1) - 1)),
             lambda: ctx.h_prolong(0, z(ctx.cg_size(1) - 1), z(n0)),
             lambda: ctx.coarse_solve(z(int(ctx.info.ncoarse) - 1), z(int(ctx.info.ncoarse))),
             lambda: ctx.solve_host(torch.zeros(nd - 1, dtype=torch.float64), torch.zeros(nd, dtype=torch.float64))]
    launches = dgmg.kernel_launches()
    for call in calls:
        with pytest.raises(ValueError):
            call()
    assert dgmg.kernel_launches() == launches
    ctx32 = dgmg.Context((4, 4, 4), 4, precision=dgmg.DGMG_MIXED_FP32)
    with pytest.raises(ValueError):
        ctx32.apply_f32(z(ctx32.ndof - 1, torch.float32), z(ctx32.ndof, torch.float32))
    batch = dgmg.Batch([((4, 4, 4), 2, None), ((5, 4, 3), 3, None)])
    with pytest.raises(ValueError):
        batch.solve([z(nd), z(60 * 64 - 1)], [z(nd), z(60 * 64)])
