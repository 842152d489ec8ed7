"""Batched solves (one launch per stage for many independent problems) against
the oracle, problem by problem."""
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


def _problem(n, p, seed, kind):
    rng = np.random.default_rng(seed)
    kappa = None if kind == "one" else np.exp(rng.normal(size=int(np.prod(n))))
    mesh = sipg.Mesh(n, p)
    b = rng.normal(size=mesh.ndof)
    return mesh, kappa, b


MIX3 = [((5, 6, 4), 2, "lognormal"), ((8, 8, 8), 1, "one"), ((7, 5, 6), 3, "lognormal"), ((6, 6, 6), 2, "one"),
        ((6, 5, 7), 3, "lognormal"), ((4, 4, 4), 4, "lognormal"), ((9, 8, 7), 2, "lognormal")]


@pytest.mark.gpu
@pytest.mark.parametrize("mix,prec", [("3d", 0), ("2d", 0), ("3d", 1), ("2d", 1)])
def test_batch_solutions_match_oracle(dgmg, mix, prec):
    """Every problem of a mixed batch (sizes, degrees 1-4, kappa fields) reaches
    its own residual bound, and its solution is the oracle's, with the FP64 and
    with the FP32 V-cycle."""
    spec = MIX3 if mix == "3d" else [((12, 10), 2, "lognormal"), ((9, 9), 4, "one"), ((16, 7), 3, "lognormal"),
                                     ((6, 11), 2, "one")]
    probs = [_problem(n, p, 40 + i, kind) for i, (n, p, kind) in enumerate(spec)]
    batch = dgmg.Batch([(n, p, kap) for (n, p, _), (_, kap, _) in zip(spec, probs)], precision=prec)
    bs = [torch.tensor(b, device=DEV) for _, _, b in probs]
    xs = [torch.zeros_like(b) for b in bs]
    stats, _ = batch.solve(bs, xs)
    for (mesh, kap, b), x, st in zip(probs, xs, stats):
        xn = x.cpu().numpy()
        res = np.linalg.norm(b - sipg.apply(mesh, xn, kap)) / np.linalg.norm(b)
        assert st.rel_residual <= 1e-10 and res <= 1.05e-10
        assert abs(st.rel_residual - res) <= 1e-3 * res + 1e-15
        x_ref, _, _ = hpmg.pcg(hpmg.Hierarchy(mesh, kap), b, rtol=1e-13)
        assert np.linalg.norm(xn - x_ref) <= 1e-9 * np.linalg.norm(x_ref)
    assert batch.info().groups == len({p for _, p, _ in spec})


@pytest.mark.gpu
def test_batch_single_problem_equals_context_solve(dgmg):
    """A batch of one problem runs the context's own algorithm: same iterations,
    same solution to rounding. In a mixed batch every problem takes the
    iterations it takes alone."""
    n, p = (7, 6, 5), 3
    mesh, kap, b = _problem(n, p, 3, "lognormal")
    bt = torch.tensor(b, device=DEV)
    ctx = dgmg.Context(n, p, kap)
    x1 = torch.zeros_like(bt)
    st1, _ = ctx.solve(bt, x1)
    batch = dgmg.Batch([(n, p, kap)])
    x2 = torch.zeros_like(bt)
    (st2,), _ = batch.solve([bt], [x2])
    assert st2.iterations == st1.iterations
    assert (x1 - x2).abs().max().item() <= 1e-11 * x1.abs().max().item()
    spec = [((5, 6, 4), 2, "lognormal"), ((8, 8, 8), 1, "one"), ((6, 5, 7), 3, "lognormal")]
    probs = [_problem(n, p, 60 + i, kind) for i, (n, p, kind) in enumerate(spec)]
    bs = [torch.tensor(b, device=DEV) for _, _, b in probs]
    alone = []
    for (n, p, _), (_, kap, _), bt in zip(spec, probs, bs):
        st, _ = dgmg.Context(n, p, kap).solve(bt, torch.zeros_like(bt))
        alone.append(st.iterations)
    batch = dgmg.Batch([(n, p, kap) for (n, p, _), (_, kap, _) in zip(spec, probs)])
    stats, _ = batch.solve(bs, [torch.zeros_like(b) for b in bs])
    assert [s.iterations for s in stats] == alone


@pytest.mark.gpu
def test_batch_launches_do_not_grow_with_count(dgmg):
    """One launch per stage: a batch of twice as many problems of the same
    shapes launches the same kernels per iteration; repeated solves reuse the
    captured iteration."""
    base = [((6, 5, 4), 2), ((5, 5, 5), 3), ((8, 6, 6), 2)]
    kpi = []
    for reps in (1, 2):
        spec = [(n, p, np.exp(np.random.default_rng(k).normal(size=int(np.prod(n)))))
                for k, (n, p) in enumerate(base * reps)]
        batch = dgmg.Batch(spec)
        bs = [torch.randn(int(np.prod(n)) * (p + 1) ** 3, dtype=torch.float64, device=DEV) for n, p, _ in spec]
        for _ in range(2):
            xs = [torch.zeros_like(b) for b in bs]
            stats, _ = batch.solve(bs, xs)
            assert max(s.rel_residual for s in stats) <= 1e-10
        kpi.append(batch.info().kernels_per_iteration)
    assert kpi[0] > 0 and kpi[0] == kpi[1]


@pytest.mark.gpu
def test_batch_autotuned_tiles_same_results(dgmg):
    """Tuned tiles regroup cells into CTAs (and may switch the smoothing kernel):
    the solutions agree with the default tiles to rounding."""
    spec = [((6, 5, 4), 2, "lognormal"), ((5, 5, 5), 3, "one"), ((4, 5, 6), 4, "lognormal")]
    probs = [_problem(n, p, 80 + i, kind) for i, (n, p, kind) in enumerate(spec)]
    bs = [torch.tensor(b, device=DEV) for _, _, b in probs]
    out = []
    for tune in (0, 1):
        batch = dgmg.Batch([(n, p, kap) for (n, p, _), (_, kap, _) in zip(spec, probs)], autotune=tune)
        xs = [torch.zeros_like(b) for b in bs]
        stats, _ = batch.solve(bs, xs)
        assert max(s.rel_residual for s in stats) <= 1e-10
        inf = batch.info()
        # 0: the one-thread-per-cell kernel (smoothing step and residual)
        assert all(inf.group_tiles[k][0] > 0 and min(inf.group_tiles[k]) >= 0 for k in range(inf.groups))
        out.append([x.cpu().numpy() for x in xs])
    for a, b in zip(*out):
        assert np.abs(a - b).max() <= 1e-9 * np.abs(a).max()


@pytest.mark.gpu
def test_batch_invalid_arguments(dgmg):
    with pytest.raises(dgmg.DGMGError):
        dgmg.Batch([((4, 4, 4), 2, None)], precision=7)
    with pytest.raises(dgmg.DGMGError):
        dgmg.Batch([((4, 4, 4), 2, None), ((5, 5), 2, None)])
    with pytest.raises(dgmg.DGMGError):
        dgmg.Batch([((4, 4, 4), 2, None)], nu_pre=0)
    with pytest.raises(dgmg.DGMGError):
        dgmg.Batch([((4, 4, 4), 9, None)])
