"""The "recompute" variant of the block inverse (paper Table 6, Sec. 7.1):
with opts.recompute_block the per-cell factors of A_KK^-1 are computed again
before every smoothing step instead of once at set-up. Same factors, so the
smoothing steps, V-cycles and solves equal the precomputed ones (and so the
oracle's)."""
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


def _rel(a, b):
    return float((a - b).abs().max() / b.abs().max().clamp_min(1e-300))


@pytest.mark.parametrize("n,p", [((6, 5, 4), 2), ((4, 3, 5), 3), ((9, 7), 3)])
@pytest.mark.parametrize("precision", [0, 1])
def test_recomputed_factors_give_the_same_cycles_and_solves(dgmg, n, p, precision):
    rng = np.random.default_rng(41)
    kappa = np.exp(rng.normal(size=int(np.prod(n))))
    b = rng.normal(size=int(np.prod(n)) * (p + 1) ** len(n))
    dev = "cuda:0"
    bt = torch.tensor(b, device=dev)
    out = {}
    for rb in (0, 1):
        ctx = dgmg.Context(n, p, kappa, precision=precision, recompute_block=rb)
        e = torch.zeros_like(bt)
        ctx.vcycle(bt, e)
        u = torch.zeros_like(bt)
        ctx.smooth(u, bt, 3)
        x = torch.zeros_like(bt)
        st, _ = ctx.solve(bt, x)
        torch.cuda.synchronize()
        out[rb] = (e.clone(), u.clone(), x.clone(), st.iterations, st.rel_residual)
        ctx.close()
    assert _rel(out[1][0], out[0][0]) <= 1e-13
    assert _rel(out[1][1], out[0][1]) <= 1e-13
    assert out[1][3] == out[0][3]
    assert out[1][4] <= 1e-10
    if precision == 0:
        mesh = sipg.Mesh(n, p)
        e_ref = hpmg.Hierarchy(mesh, kappa).vcycle(b)
        assert _rel(out[1][0], torch.tensor(e_ref, device=dev)) <= 1e-11
    assert dgmg.wait_timeouts() == 0


def test_batched_solves_reject_recompute(dgmg):
    with pytest.raises(dgmg.DGMGError) as ei:
        dgmg.Batch([((4, 4, 4), 2, None)], recompute_block=1)
    assert ei.value.code == dgmg.DGMG_EINVAL
