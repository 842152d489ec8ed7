"""The solve server: continuous batching of independent solves.

Each request's result must be the same whether it is solved alone
(dgmg_solve on its own context) or in a mix with other requests that arrive
while it runs; the HBM budget must bound admission; resident hierarchies are
reused for repeated problems."""
import time

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


DEV = "cuda:0"


def _problem(n, p, seed, kind):
    rng = np.random.default_rng(seed)
    ncell = int(np.prod(n))
    kappa = None if kind == "one" else np.exp(rng.normal(size=ncell))
    ndof = ncell * (p + 1) ** len(n)
    b = torch.tensor(rng.normal(size=ndof), device=DEV)
    return kappa, b


def _wait(srv, tickets, timeout=120.0):
    t0 = time.time()
    out = {}
    seen_active = 0
    while len(out) < len(tickets):
        seen_active = max(seen_active, srv.info().active)
        for t in tickets:
            if t in out:
                continue
            st, stats = srv.poll(t)
            if st == 2:
                out[t] = stats
        assert time.time() - t0 < timeout
        time.sleep(0.0005)
    return out, seen_active


MIX = [((8, 7, 6), 2, "lognormal"), ((10, 10), 3, "one"), ((6, 6, 6), 3, "lognormal"), ((12, 9), 4, "lognormal"),
       ((9, 8, 7), 1, "one"), ((7, 7, 7), 2, "one"), ((16, 16), 2, "lognormal"), ((5, 6, 7), 4, "lognormal")]


@pytest.mark.parametrize("precision", [0, 1])
def test_results_in_the_mix_equal_results_alone(dgmg, precision):
    probs = [(n, p, _problem(n, p, 100 + i, kind)) for i, (n, p, kind) in enumerate(MIX)]
    # alone
    alone = []
    for n, p, (kappa, b) in probs:
        ctx = dgmg.Context(n, p, kappa, precision=precision)
        x = torch.zeros_like(b)
        st, _ = ctx.solve(b, x)
        assert st.rel_residual <= 1e-10
        alone.append(x.cpu().numpy())
    # in the mix: staggered arrivals while earlier requests are running
    srv = dgmg.Server(8 << 30, 4, precision=precision)
    xs, tickets = [], []
    for k, (n, p, (kappa, b)) in enumerate(probs):
        x = torch.zeros_like(b)
        # stream (not device-wide) synchronisation: the server may be capturing
        # a CUDA graph on another stream meanwhile
        torch.cuda.current_stream().synchronize()
        tickets.append(srv.submit(n, p, b, x, kappa))
        xs.append(x)
        if k % 3 == 2:
            time.sleep(0.002)
    res, seen_active = _wait(srv, tickets)
    torch.cuda.synchronize()
    for k, t in enumerate(tickets):
        assert res[t].rel_residual <= 1e-10
        assert res[t].seconds >= res[t].queue_seconds >= 0.0
        xm = xs[k].cpu().numpy()
        assert np.abs(xm - alone[k]).max() <= 1e-12 * np.abs(alone[k]).max()
    assert seen_active >= 2          # work of several requests was on the GPU together
    inf = srv.info()
    assert inf.done == len(probs) and inf.failed == 0
    # a finished request is reported once; its record is then released
    for t in tickets:
        with pytest.raises(dgmg.DGMGError) as ei:
            srv.poll(t)
        assert ei.value.code == dgmg.DGMG_EINVAL
    srv.close()


def test_budget_bounds_admission_and_evicts(dgmg):
    n, p = (8, 8, 8), 2
    one = dgmg.estimate_bytes(n, p)
    srv = dgmg.Server(int(one * 1.5), 4)          # room for one hierarchy at a time
    probs = [_problem(n, p, 200 + i, "lognormal") for i in range(3)]
    xs, tickets = [], []
    for kappa, b in probs:
        x = torch.zeros_like(b)
        # stream (not device-wide) synchronisation: the server may be capturing
        # a CUDA graph on another stream meanwhile
        torch.cuda.current_stream().synchronize()
        tickets.append(srv.submit(n, p, b, x, kappa))
        xs.append(x)
    res, seen_active = _wait(srv, tickets)
    assert seen_active == 1
    inf = srv.info()
    assert inf.done == 3 and inf.evictions >= 2 and inf.bytes_in_use <= inf.budget
    for k, (kappa, b) in enumerate(probs):
        ctx = dgmg.Context(n, p, kappa)
        x = torch.zeros_like(b)
        ctx.solve(b, x)
        assert torch.allclose(xs[k], x, rtol=0, atol=1e-12 * float(x.abs().max()))
    srv.close()


def test_request_larger_than_budget_fails(dgmg):
    srv = dgmg.Server(1 << 20, 2)
    kappa, b = _problem((8, 8, 8), 3, 5, "one")
    x = torch.zeros_like(b)
    t = srv.submit((8, 8, 8), 3, b, x, kappa)
    for _ in range(2000):
        try:
            status, _ = srv.poll(t)
        except dgmg.DGMGError as e:
            assert e.code == dgmg.DGMG_EBUDGET
            break
        time.sleep(0.001)
    else:
        pytest.fail("request was not rejected")
    srv.close()


def test_repeated_problem_reuses_resident_hierarchy(dgmg):
    srv = dgmg.Server(4 << 30, 2)
    kappa, b = _problem((9, 9, 9), 2, 7, "lognormal")
    x1, x2 = torch.zeros_like(b), torch.zeros_like(b)
    t1 = srv.submit((9, 9, 9), 2, b, x1, kappa)
    _wait(srv, [t1])
    t2 = srv.submit((9, 9, 9), 2, b, x2, kappa)
    res, _ = _wait(srv, [t2])
    inf = srv.info()
    assert inf.cache_hits == 1 and inf.cache_misses == 1
    assert torch.equal(x1, x2)
    srv.close()


@pytest.mark.parametrize("n,p,prec", [((8, 8, 8), 2, 0), ((16, 12), 4, 1), ((7, 9, 5), 3, 1)])
def test_estimate_bytes_matches_allocation(dgmg, n, p, prec):
    ctx = dgmg.Context(n, p, precision=prec)
    assert dgmg.estimate_bytes(n, p, precision=prec) == ctx.info.device_bytes
