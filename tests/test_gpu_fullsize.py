"""Parity at the full workload sizes, in the launch configuration bench.py uses.

32^3 cells, p = 3, kappa = 1 (the bench workload) and 64^3 cells, p = 4,
lognormal kappa (mixed precision). The oracle applies the operator to the whole
mesh; block inverses are formed for sampled cells only, on a window of at
most 3 cells per axis around each sampled cell with the same boundary status,
neighbour kappa and cell size (the diagonal block depends on nothing else)."""
import numpy as np
import pytest

from oracle import sipg

torch = pytest.importorskip("torch")

DEV = "cuda:0"


@pytest.fixture(scope="module")
def dgmg():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2510_00998_gb300 import dgmg as m
    assert torch.cuda.is_available()
    return m


def _window_block(mesh, kappa, cell):
    """A_KK of `cell` from a window mesh of at most 3 cells per axis."""
    d = mesh.d
    ci = [(cell // int(np.prod(mesh.n[:a]))) % mesh.n[a] for a in range(d)]
    lo = [max(0, ci[a] - 1) for a in range(d)]
    hi = [min(mesh.n[a] - 1, ci[a] + 1) for a in range(d)]
    wn = tuple(hi[a] - lo[a] + 1 for a in range(d))
    w = sipg.Mesh(wn, mesh.p)
    # the window keeps the full mesh's cell size and the boundary status of
    # `cell`: window faces that are not domain faces must not be boundary facets
    # for the centre cell -- guaranteed because the window extends one cell past
    # the centre wherever the full mesh does
    w.h = mesh.h
    w.M, w.K, w.d0, w.dp = mesh.M, mesh.K, mesh.d0, mesh.dp
    kw = None
    if kappa is not None:
        kg = np.asarray(kappa).reshape(mesh.n[::-1])
        sl = tuple(slice(lo[a], hi[a] + 1) for a in range(d))[::-1]
        kw = kg[sl].reshape(-1)
    B = sipg.block_diagonal(w, kw)
    wc = sum((ci[a] - lo[a]) * int(np.prod(wn[:a])) for a in range(d))
    return B[wc]


@pytest.mark.gpu
@pytest.mark.parametrize("case", ["bench_32_p3", "mixed_64_p4"])
def test_full_size_apply_smooth_solve(dgmg, case):
    if case == "bench_32_p3":
        n, p, kappa, prec = (32, 32, 32), 3, None, 0
    else:
        n, p, prec = (64, 64, 64), 4, 1
        kappa = np.exp(np.random.default_rng(3).normal(size=int(np.prod(n))))
    mesh = sipg.Mesh(n, p)
    ctx = dgmg.Context(n, p, kappa, precision=prec)
    rng = np.random.default_rng(31)
    u = rng.normal(size=mesh.ndof)
    b = rng.normal(size=mesh.ndof)
    ut, bt = torch.tensor(u, device=DEV), torch.tensor(b, device=DEV)
    # apply: every output against the oracle
    y = torch.empty_like(ut)
    ctx.apply(ut, y)
    y_ref = sipg.apply(mesh, u, kappa)
    assert np.abs(y.cpu().numpy() - y_ref).max() <= 1e-12 * np.abs(y_ref).max()
    # one FP64 smoothing step, checked on sampled cells (incl. corners and faces)
    r_ref = b - y_ref
    us = ut.clone()
    ctx.smooth(us, bt, 1)
    us = us.cpu().numpy().reshape(mesh.ncell, mesh.nloc)
    nc = mesh.ncell
    sample = sorted(set([0, nc - 1, n[0] - 1, nc // 2, nc // 3 + 7] + list(rng.integers(0, nc, size=12))))
    omega = ctx.info.omega_dg
    for c in sample:
        B = _window_block(mesh, kappa, int(c))
        ref = u.reshape(nc, -1)[c] + omega * np.linalg.solve(B, r_ref.reshape(nc, -1)[c])
        assert np.abs(us[c] - ref).max() <= 1e-11 * np.abs(ref).max()
    # full solve: the true residual of the GPU solution, recomputed by the oracle
    x = torch.zeros_like(bt)
    st, _ = ctx.solve(bt, x)
    assert st.rel_residual <= 1e-10
    res = b - sipg.apply(mesh, x.cpu().numpy(), kappa)
    assert np.linalg.norm(res) <= 1.05e-10 * np.linalg.norm(b)


def test_window_block_matches_full_block_on_small_mesh():
    """The windowed diagonal block equals the block of the whole mesh (pins the
    sampling helper itself)."""
    n, p = (5, 4, 6), 2
    mesh = sipg.Mesh(n, p)
    kappa = np.exp(np.random.default_rng(0).normal(size=mesh.ncell))
    full = sipg.block_diagonal(mesh, kappa)
    for c in [0, 7, 33, mesh.ncell - 1, 61]:
        assert np.abs(_window_block(mesh, kappa, c) - full[c]).max() <= 1e-13 * np.abs(full[c]).max()


@pytest.mark.gpu
def test_full_size_fp32_vcycle_against_fp64():
    """64^3, p = 4, lognormal kappa: the FP32 V-cycle of the mixed-precision
    context (one-thread-per-cell smoothing and residual kernels at the bench's
    launch configuration) against the FP64 V-cycle of an FP64 context, whose
    kernels match the oracle on smaller meshes; every output within the FP32
    V-cycle bound of the small-mesh tests (2e-5 of the maximum)."""
    import __graft_entry__
    __graft_entry__.build()
    from paper_2510_00998_gb300 import dgmg as m
    n, p = (64, 64, 64), 4
    kappa = np.exp(np.random.default_rng(3).normal(size=int(np.prod(n))))
    r = torch.tensor(np.random.default_rng(41).normal(size=int(np.prod(n)) * (p + 1) ** 3), device=DEV)
    outs = []
    for prec in (m.DGMG_FP64, m.DGMG_MIXED_FP32):
        ctx = m.Context(n, p, kappa, precision=prec, autotune=1)
        e = torch.empty_like(r)
        ctx.vcycle(r, e)
        torch.cuda.synchronize()
        outs.append(e)
        ctx.close()
    assert float((outs[1] - outs[0]).abs().max() / outs[0].abs().max()) <= 2e-5
    assert m.wait_timeouts() == 0
