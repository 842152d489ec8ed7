"""Gradual p-coarsening (DG p -> p-1 -> ... -> 1 -> Q1) on the GPU against the
oracle's gradual hierarchy."""
import numpy as np
import pytest

from oracle import hpmg, sipg

torch = pytest.importorskip("torch")

DEV = "cuda:0"


@pytest.fixture(scope="module")
def dgmg():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2510_00998_gb300 import dgmg as m
    assert torch.cuda.is_available()
    return m


def _kappa(n, seed=0):
    return np.exp(np.random.default_rng(seed).normal(size=int(np.prod(n))))


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.gpu
@pytest.mark.parametrize("n,p,prec", [((9, 7), 3, 0), ((6, 5, 4), 2, 0), ((5, 4, 5), 4, 0), ((4, 3, 3), 5, 0),
                                      ((8, 6), 6, 0), ((5, 4, 5), 4, 1), ((9, 7), 3, 1), ((4, 3, 3), 5, 1)])
def test_gradual_vcycle_matches_oracle(dgmg, n, p, prec):
    """FP64 to rounding (1e-11), FP32 within the V-cycle's FP32 bound (2e-5)."""
    kap = _kappa(n)
    mesh = sipg.Mesh(n, p)
    ctx = dgmg.Context(n, p, kap, p_coarsening=1, precision=prec)
    assert ctx.info.dg_levels == p
    hier = hpmg.Hierarchy(mesh, kap, gradual=True)
    r = np.random.default_rng(9).normal(size=mesh.ndof)
    e = torch.empty(mesh.ndof, dtype=torch.float64, device=DEV)
    ctx.vcycle(torch.tensor(r, device=DEV), e)
    assert _rel(e.cpu().numpy(), hier.vcycle(r)) <= (1e-11 if prec == 0 else 2e-5)


@pytest.mark.gpu
@pytest.mark.parametrize("n,p,prec", [((8, 8, 8), 3, 0), ((6, 6, 5), 4, 1), ((12, 10), 5, 0)])
def test_gradual_solve_matches_oracle(dgmg, n, p, prec):
    kap = _kappa(n, 1)
    mesh = sipg.Mesh(n, p)
    b = np.random.default_rng(12).normal(size=mesh.ndof)
    ctx = dgmg.Context(n, p, kap, p_coarsening=1, precision=prec)
    x = torch.zeros(mesh.ndof, dtype=torch.float64, device=DEV)
    st, _ = ctx.solve(torch.tensor(b, device=DEV), x)
    assert st.rel_residual <= 1e-10
    x_ref, _, _ = hpmg.pcg(hpmg.Hierarchy(mesh, kap), b, rtol=1e-13)
    assert np.linalg.norm(x.cpu().numpy() - x_ref) <= 1e-9 * np.linalg.norm(x_ref)


@pytest.mark.gpu
def test_gradual_mgmult_matches_oracle_and_is_p_robust(dgmg):
    """MGMult iterates equal the oracle's gradual MGMult after K cycles; on 9x9 the
    cycle counts stay flat in p (direct coarsening grows with p)."""
    n, p, K = (9, 9), 4, 4
    mesh = sipg.Mesh(n, p)
    kap = _kappa(n, 2)
    b = np.random.default_rng(3).normal(size=mesh.ndof)
    u_ref, _ = hpmg.mgmult(hpmg.Hierarchy(mesh, kap, factor=3, nu_pre=3, nu_post=3, gradual=True), b, eps=0.0,
                           maxit=K)
    ctx = dgmg.Context(n, p, kap, outer=dgmg.DGMG_OUTER_MGMULT, coarsening=3, nu_pre=3, nu_post=3, rtol=1e-30,
                       maxit=K, p_coarsening=1)
    x = torch.zeros(mesh.ndof, dtype=torch.float64, device=DEV)
    ctx.solve(torch.tensor(b, device=DEV), x, allow_notconverged=True)
    assert _rel(x.cpu().numpy(), u_ref) <= 1e-11
    from paper_2510_00998_gb300 import workloads
    direct = workloads.tables34(meshes=(9,), degrees=(2, 4, 6))
    gradual = workloads.tables34(meshes=(9,), degrees=(2, 4, 6), p_coarsening=1)
    assert gradual[(9, 6)][0] < 0.5 * direct[(9, 6)][0]
    assert max(v[0] for v in gradual.values()) <= 1.5 * min(v[0] for v in gradual.values())


@pytest.mark.gpu
@pytest.mark.parametrize("n,p,prec", [((6, 5, 4), 3, 0), ((6, 5, 4), 4, 1), ((10, 9), 5, 1)])
def test_gradual_estimate_bytes_exact(dgmg, n, p, prec):
    est = dgmg.estimate_bytes(n, p, p_coarsening=1, precision=prec)
    ctx = dgmg.Context(n, p, p_coarsening=1, precision=prec)
    assert est == ctx.info.device_bytes
