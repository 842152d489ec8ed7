"""The FP32 operator of the reliable-update CG recurrences, y = A u (Eq.
matrix_form_IP; the cell equation of Alg. 2 stage 3 with b = 0), in its three
forms: per pencil, one thread per cell with A_KK u in the direct
sum-factorised form, and one thread per cell through the fast-diagonalisation
factors, each against the oracle's FP64 apply. Meshes with partial 32-cell
blocks, boundary faces on every side and lognormal kappa; degrees 1 to 4."""
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


# FP32: every output is a sum of at most a few hundred products whose sizes are
# bounded by |A| |u|; the error is a few units of 2^-24 of that bound. 2e-6 of
# the norm of A u (and 2e-5 of its largest entry, elementwise) leaves a factor
# of about ten over what these random inputs show.
TOL_NORM, TOL_MAX = 2e-6, 2e-5


@pytest.mark.parametrize("n,p", [((5, 4, 7), 4), ((8, 8, 8), 4), ((3, 3, 3), 3), ((12, 11, 10), 3),
                                 ((6, 5, 4), 2), ((7, 3, 5), 1), ((33, 2, 2), 4)])
@pytest.mark.parametrize("form", [0, 1, 2])
def test_fp32_operator_matches_oracle(dgmg, n, p, form):
    mesh = sipg.Mesh(n, p)
    rng = np.random.default_rng(17)
    kappa = np.exp(rng.normal(size=mesh.ncell))
    u = rng.normal(size=mesh.ndof).astype(np.float32)
    ref = sipg.apply(mesh, u.astype(np.float64), kappa)
    ctx = dgmg.Context(n, p, kappa, precision=dgmg.DGMG_MIXED_FP32)
    ut = torch.tensor(u, device="cuda:0")
    y = torch.full_like(ut, float("nan"))
    ctx.apply_f32(ut, y, form)
    torch.cuda.synchronize()
    yv = y.cpu().numpy().astype(np.float64)
    assert np.isfinite(yv).all()
    assert np.linalg.norm(yv - ref) <= TOL_NORM * np.linalg.norm(ref)
    assert np.abs(yv - ref).max() <= TOL_MAX * np.abs(ref).max()
    assert dgmg.wait_timeouts() == 0


def test_direct_form_rounds_like_the_per_pencil_form(dgmg):
    """The direct one-thread-per-cell form evaluates the same sum-factorised
    expression as the per-pencil kernel; its difference from it stays at the
    size of the per-pencil form's own FP32 error against the oracle."""
    n, p = (16, 16, 16), 4
    mesh = sipg.Mesh(n, p)
    rng = np.random.default_rng(5)
    kappa = np.exp(rng.normal(size=mesh.ncell))
    x = (np.arange(mesh.ndof) % 97) / 97.0
    u = (np.sin(3.0 * x) + 1e-3 * rng.normal(size=mesh.ndof)).astype(np.float32)
    ref = sipg.apply(mesh, u.astype(np.float64), kappa)
    ctx = dgmg.Context(n, p, kappa, precision=dgmg.DGMG_MIXED_FP32)
    ut = torch.tensor(u, device="cuda:0")
    out = {}
    for form in (0, 1):
        y = torch.empty_like(ut)
        ctx.apply_f32(ut, y, form)
        out[form] = y.cpu().numpy().astype(np.float64)
    e_pencil = np.linalg.norm(out[1] - ref)
    assert np.linalg.norm(out[0] - out[1]) <= 3.0 * e_pencil + 1e-30
    assert np.linalg.norm(out[0] - ref) <= 3.0 * e_pencil + 1e-30


def test_fp32_operator_rejects_fp64_ctx_and_bad_arguments(dgmg):
    ctx64 = dgmg.Context((4, 4, 4), 2)
    x = torch.zeros(ctx64.ndof, dtype=torch.float32, device="cuda:0")
    with pytest.raises(dgmg.DGMGError) as ei:
        ctx64.apply_f32(x, x.clone(), 0)
    assert ei.value.code == dgmg.DGMG_EINVAL
    ctx = dgmg.Context((4, 4, 4), 2, precision=dgmg.DGMG_MIXED_FP32)
    with pytest.raises(dgmg.DGMGError) as ei:
        ctx.apply_f32(x, x, 0)
    assert ei.value.code == dgmg.DGMG_EINVAL
    with pytest.raises(dgmg.DGMGError) as ei:
        ctx.apply_f32(x, x.clone(), 3)
    assert ei.value.code == dgmg.DGMG_EINVAL


def test_fp32_operator_with_interior_only_blocks(dgmg):
    """Technique 4 contexts: forms 0 and 1 never use the block factors and still
    give A u; form 2 (A_KK u from the per-cell factors, which there factor the
    interior cell's block, not A_KK) is rejected."""
    n, p = (5, 4, 6), 4
    mesh = sipg.Mesh(n, p)
    rng = np.random.default_rng(23)
    kappa = np.exp(rng.normal(size=mesh.ncell))
    u = rng.normal(size=mesh.ndof).astype(np.float32)
    ref = sipg.apply(mesh, u.astype(np.float64), kappa)
    ctx = dgmg.Context(n, p, kappa, precision=dgmg.DGMG_MIXED_FP32,
                       block_inverse=dgmg.DGMG_BLOCK_INTERIOR_ONLY)
    ut = torch.tensor(u, device="cuda:0")
    for form in (0, 1):
        y = torch.full_like(ut, float("nan"))
        ctx.apply_f32(ut, y, form)
        torch.cuda.synchronize()
        yv = y.cpu().numpy().astype(np.float64)
        assert np.linalg.norm(yv - ref) <= TOL_NORM * np.linalg.norm(ref)
    with pytest.raises(dgmg.DGMGError) as ei:
        ctx.apply_f32(ut, torch.empty_like(ut), 2)
    assert ei.value.code == dgmg.DGMG_EINVAL
    assert dgmg.wait_timeouts() == 0
