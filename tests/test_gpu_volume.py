"""The volume term alone, r = b - kappa_K E u_K (Sec. 4.1 dense local
mat-vec), in its two forms: sum-factorised on the CUDA cores (FP32) and a dense
contraction on the tensor cores (tcgen05, TF32 operands, FP32 accumulation),
against the oracle's volume term (FP64). Meshes with partial 32-cell blocks
and partial 128-cell tiles."""
import numpy as np
import pytest

from oracle import sipg

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def dgmg():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2510_00998_gb300 import dgmg as m
    assert torch.cuda.is_available()
    return m


def _case(n, seed):
    mesh = sipg.Mesh(n, 4)
    rng = np.random.default_rng(seed)
    kappa = np.exp(rng.normal(size=mesh.ncell))
    u = rng.normal(size=mesh.ndof).astype(np.float32)
    b = rng.normal(size=mesh.ndof).astype(np.float32)
    vol = mesh.flat(sipg.volume_term(mesh, mesh.grid(u.astype(np.float64)), mesh.kappa_grid(kappa))).reshape(-1)
    return mesh, kappa, u, b, vol


# FP32 sum factorisation: six passes of 5-term FP32 sums per value, |E u|
# bounded by the row sums of |E|: well inside 1e-5 of max |kappa E u|.
# TF32: operands rounded to 11 significant bits (relative 2^-12 each), 125
# products summed in FP32: below 125 * 2 * 2^-12 * max|E_nk u_k| in the worst
# case; 2e-3 of max |kappa E u| holds with a factor of 10 to spare on these
# random inputs.
TOL = {0: 1e-5, 1: 2e-3}


@pytest.mark.parametrize("n", [(5, 4, 7), (8, 8, 8), (3, 3, 3), (12, 11, 10)])
@pytest.mark.parametrize("method", [0, 1])
def test_volume_term_matches_oracle(dgmg, n, method):
    mesh, kappa, u, b, vol = _case(n, 31)
    ctx = dgmg.Context(n, 4, kappa)
    dev = "cuda:0"
    ut, bt = torch.tensor(u, device=dev), torch.tensor(b, device=dev)
    for _ in range(2):                                   # the second call reuses E and the factors
        r = torch.full_like(ut, float("nan"))
        ctx.volume_residual_f32(ut, bt, r, method)
        torch.cuda.synchronize()
        ref = b.astype(np.float64) - vol
        err = np.abs(r.cpu().numpy().astype(np.float64) - ref).max() / np.abs(vol).max()
        assert err <= TOL[method], err
    assert dgmg.wait_timeouts() == 0


def test_volume_term_rejects_other_degrees_and_misaligned_vectors(dgmg):
    ctx = dgmg.Context((4, 4, 4), 3)
    x = torch.zeros(ctx.ndof, dtype=torch.float32, device="cuda:0")
    with pytest.raises(dgmg.DGMGError) as ei:
        ctx.volume_residual_f32(x, x.clone(), x.clone(), 0)
    assert ei.value.code == dgmg.DGMG_EINVAL
    ctx5 = dgmg.Context((4, 4, 4), 4)
    y = torch.zeros(ctx5.ndof + 1, dtype=torch.float32, device="cuda:0")
    with pytest.raises(dgmg.DGMGError) as ei:
        ctx5.volume_residual_f32(y[1:], y[1:].clone(), y[1:].clone(), 1)
    assert ei.value.code == dgmg.DGMG_EINVAL
