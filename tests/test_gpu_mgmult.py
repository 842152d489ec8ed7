"""The stationary hp-multigrid iteration (Alg. 7, MGMult) on the GPU against the
oracle's own MGMult, and the shape of the paper's Tables 3-4 (cycles to reduce
the residual by 1e-7 on 2D meshes refined by factor 3)."""
import os

import numpy as np
import pytest

from oracle import hpmg, sipg

torch = pytest.importorskip("torch")

DEV = "cuda:0"
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def dgmg():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2510_00998_gb300 import dgmg as m
    assert torch.cuda.is_available()
    return m


def _kappa(n, kind):
    if kind == "one":
        return None
    return np.exp(np.random.default_rng(7).normal(size=int(np.prod(n))))


def _sin_product_rhs(mesh):
    f = lambda x, y: 8 * np.pi ** 2 * np.sin(2 * np.pi * x) * np.sin(2 * np.pi * y)
    return sipg.load_vector(mesh, f)


@pytest.mark.gpu
@pytest.mark.parametrize("n,p,factor,kind", [((9, 9), 2, 3, "one"), ((12, 10), 3, 2, "lognormal"),
                                             ((6, 5, 4), 2, 2, "lognormal"), ((9, 9, 9), 1, 3, "one"),
                                             ((7, 6), 4, 2, "lognormal")])
def test_mgmult_iterates_match_oracle(dgmg, n, p, factor, kind):
    """After K cycles the GPU iterate equals the oracle's MGMult iterate."""
    K, nu = 5, 3
    kap = _kappa(n, kind)
    mesh = sipg.Mesh(n, p)
    b = np.random.default_rng(17).normal(size=mesh.ndof)
    hier = hpmg.Hierarchy(mesh, kap, factor=factor, nu_pre=nu, nu_post=nu)
    u_ref, k = hpmg.mgmult(hier, b, eps=0.0, maxit=K)
    assert k == K
    ctx = dgmg.Context(n, p, kap, outer=dgmg.DGMG_OUTER_MGMULT, coarsening=factor, nu_pre=nu, nu_post=nu,
                       rtol=1e-30, maxit=K)
    x = torch.zeros(mesh.ndof, dtype=torch.float64, device=DEV)
    st, rc = ctx.solve(torch.tensor(b, device=DEV), x, allow_notconverged=True)
    assert rc == dgmg.DGMG_ENOTCONVERGED and st.iterations == K
    xg = x.cpu().numpy()
    assert np.abs(xg - u_ref).max() <= 1e-11 * np.abs(u_ref).max()
    # the reported residual is the true residual of the returned iterate
    res = np.linalg.norm(b - sipg.apply(mesh, xg, kap)) / np.linalg.norm(b)
    assert abs(st.rel_residual - res) <= 1e-9 * res


@pytest.mark.gpu
@pytest.mark.parametrize("n,p", [((9, 9), 2), ((9, 9), 3), ((27, 27), 2)])
def test_mgmult_cycle_counts_match_oracle(dgmg, n, p):
    """Both exit criteria of Sec. 6.3 (unpreconditioned and preconditioned
    residual, 1e-7) take the oracle's number of cycles (+-1 where the ratio
    lands at the threshold)."""
    nu = 3
    mesh = sipg.Mesh(n, p)
    b = _sin_product_rhs(mesh)
    hier = hpmg.Hierarchy(mesh, factor=3, nu_pre=nu, nu_post=nu)
    _, k_un = hpmg.mgmult(hier, b, eps=1e-7)
    _, k_pr = hpmg.mgmult(hier, b, eps=1e-7, residual_kind="prec")
    bt = torch.tensor(b, device=DEV)
    for outer, k_ref in ((dgmg.DGMG_OUTER_MGMULT, k_un), (dgmg.DGMG_OUTER_MGMULT_PREC, k_pr)):
        ctx = dgmg.Context(n, p, outer=outer, coarsening=3, nu_pre=nu, nu_post=nu, rtol=1e-7, maxit=200)
        x = torch.zeros_like(bt)
        st, _ = ctx.solve(bt, x)
        assert abs(st.iterations - k_ref) <= 1, (outer, st.iterations, k_ref)
        if outer == dgmg.DGMG_OUTER_MGMULT:
            assert st.rel_residual <= 1e-7
        else:
            assert st.prec_residual <= 1e-7


@pytest.mark.gpu
def test_mgmult_tables_3_4_shape(dgmg):
    """A comparison under a reading, not a pin (the paper states neither
    omega, nu nor the penalty for
    Tables 3-4): on 9^2 ... 243^2 with factor-3 coarsening, nu = 4 and omega = 0.8
    (the reading that reproduces the printed tables best) the cycle counts are
    h-robust (unpreconditioned: within 1.5x across the meshes; preconditioned: not
    growing with refinement), grow with p, and lie between 0.7x the printed
    count and one cycle above it."""
    from paper_2510_00998_gb300 import workloads
    rows = np.loadtxt(os.path.join(GOLDEN, "table3_4_cycles.txt"))
    got = workloads.tables34(meshes=(9, 27, 81, 243), degrees=(2, 3))
    for p in (2, 3):
        un = [got[(n, p)][0] for n in (9, 27, 81, 243)]
        pr = [got[(n, p)][1] for n in (9, 27, 81, 243)]
        assert max(un) <= 1.5 * min(un), un
        assert all(pr[i + 1] <= pr[i] + 1 for i in range(3)), pr
    for n in (9, 27, 81, 243):
        assert got[(n, 3)][0] > got[(n, 2)][0]
    for n, p, unprec, prec in rows:
        if (int(n), int(p)) in got:
            k_un, k_pr = got[(int(n), int(p))]
            assert 0.7 * unprec <= k_un <= unprec + 1, (n, p, k_un, unprec)
            assert 0.7 * prec <= k_pr <= prec + 1, (n, p, k_pr, prec)
