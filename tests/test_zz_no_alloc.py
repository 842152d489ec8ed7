"""The allocation-free residual + p-restriction entry point.

Some callers cannot allocate device memory when they call into the library
(in loops that forbid allocation after start-up, under a fixed memory budget,
without an allocator at the point of the call). dgmg_residual_restrict_noalloc serves
them with a fixed device array as scratch. This checks, through the C ABI,
that two consecutive calls give the same residual and restricted residual as
dgmg_residual_restrict. The file is named to be collected last."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def dgmg():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2510_00998_gb300 import dgmg as m
    assert torch.cuda.is_available()
    return m


def _rel(a, b):
    return float((a - b).abs().max() / b.abs().max().clamp_min(1e-300))


@pytest.mark.parametrize("n,p", [((9, 7), 3), ((6, 5, 7), 2), ((5, 4, 3), 4)])
def test_noalloc_matches_allocating_entry_twice(dgmg, n, p):
    rng = np.random.default_rng(21)
    kappa = np.exp(rng.normal(size=int(np.prod(n))))
    ctx = dgmg.Context(n, p, kappa)
    dev = "cuda:0"
    u = torch.tensor(rng.normal(size=ctx.ndof), device=dev)
    b = torch.tensor(rng.normal(size=ctx.ndof), device=dev)
    tr = torch.empty(ctx.trace_size(), dtype=torch.float64, device=dev)
    ctx.project(u, None, tr)
    r_ref = torch.empty_like(u)
    rc_ref = torch.empty(ctx.cg_size(0), dtype=torch.float64, device=dev)
    ctx.residual_restrict(u, b, tr, r_ref, rc_ref)
    for _ in range(2):
        r = torch.full_like(u, float("nan"))
        rc = torch.full_like(rc_ref, float("nan"))
        ctx.residual_restrict_noalloc(u, b, tr, r, rc)
        torch.cuda.synchronize()
        assert _rel(r, r_ref) <= 1e-12
        assert _rel(rc, rc_ref) <= 1e-12


def test_noalloc_rejects_meshes_beyond_the_fixed_scratch(dgmg):
    ctx = dgmg.Context((80, 80, 48), 1)          # 307,200 cells x 8 corners > 2^21
    dev = "cuda:0"
    u = torch.zeros(ctx.ndof, dtype=torch.float64, device=dev)
    tr = torch.zeros(ctx.trace_size(), dtype=torch.float64, device=dev)
    rc = torch.zeros(ctx.cg_size(0), dtype=torch.float64, device=dev)
    with pytest.raises(dgmg.DGMGError) as ei:
        ctx.residual_restrict_noalloc(u, u, tr, None, rc)
    assert ei.value.code == dgmg.DGMG_EINVAL
