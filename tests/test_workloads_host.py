"""Host side of the seeded synthetic workloads (no GPU): the request streams of
the batch and serving measurements follow their stated recipe and are
reproducible, the two-phase coefficient is a half-space split of the cube, and
the one-at-a-time FIFO latency model is exact on a hand-worked trace."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2510_00998_gb300 import workloads as W  # noqa: E402


def test_batch_stream_recipe():
    reqs = W.request_stream("batch", 256, 4)
    assert len(reqs) == 256
    for r in reqs:
        nn = r["n"][0]
        assert r["n"] == (nn, nn, nn) and 8 <= nn <= 24 and r["p"] in (2, 3, 4)
        assert r["kappa_kind"] == "lognormal" and r["kappa"].shape == (nn ** 3,) and (r["kappa"] > 0).all()
        assert r["coeffs"].shape == (8,) and r["waves"].shape == (8, 3)
        assert r["waves"].min() >= 1 and r["waves"].max() <= 4
    # the size of the 256-solve batch: about 3.8e5 DoF per problem, 9.7e7 in all
    ndof = sum(r["n"][0] ** 3 * (r["p"] + 1) ** 3 for r in reqs)
    assert 8.5e7 <= ndof <= 1.1e8
    # reproducible from the seed
    again = W.request_stream("batch", 256, 4)
    assert all(a["n"] == b["n"] and a["p"] == b["p"] and np.array_equal(a["kappa"], b["kappa"])
               for a, b in zip(reqs, again))


def test_serve_stream_recipe():
    reqs = W.request_stream("serve", 300, 5)
    kinds = {r["kappa_kind"] for r in reqs}
    assert kinds == {"one", "lognormal", "two-phase"}
    for r in reqs:
        nn = r["n"][0]
        assert 8 <= nn <= 48 and 2 <= r["p"] <= 5
        if r["kappa_kind"] == "one":
            assert r["kappa"] is None
        else:
            assert r["kappa"].shape == (nn ** 3,)


@pytest.mark.parametrize("seed", range(6))
def test_two_phase_kappa_is_a_half_space_split(seed):
    n = (9, 7, 8)
    k = W.two_phase_kappa(n, np.random.default_rng(seed))
    assert set(np.unique(k)) <= {1.0, 100.0}
    # a half-space: some plane separates the cell centres of the two phases,
    # i.e. w.x - b >= 1 on one and <= -1 on the other is feasible (a linear program)
    c = np.stack(np.meshgrid(*[(np.arange(v) + 0.5) / v for v in n[::-1]], indexing="ij")[::-1], -1).reshape(-1, 3)
    hi, lo = c[k == 100.0], c[k == 1.0]
    if len(hi) and len(lo):
        from scipy.optimize import linprog
        A = np.vstack([-np.hstack([hi, -np.ones((len(hi), 1))]), np.hstack([lo, -np.ones((len(lo), 1))])])
        res = linprog(np.zeros(4), A_ub=A, b_ub=-np.ones(len(A)), bounds=[(None, None)] * 4, method="highs")
        assert res.status == 0


def test_fifo_latencies_hand_worked():
    # arrivals 0, 0, 5 with service 1, 2, 1: done at 1, 3, 6
    assert W.fifo_latencies([0.0, 0.0, 5.0], [1.0, 2.0, 1.0]) == [1.0, 3.0, 1.0]
    assert W.pct([1.0, 2.0, 3.0, 4.0], 50) == 2.5


def test_fourier_rhs_values_on_the_host():
    X = torch.tensor([[0.25, 0.5, 0.125], [0.5, 0.5, 0.5]], dtype=torch.float64)
    f = W.fourier_rhs_values(X, [2.0, -1.0], [(1, 1, 1), (2, 1, 4)])
    x = X.numpy()
    ref = (2.0 * np.prod(np.sin(np.pi * x), axis=1)
           - np.sin(2 * np.pi * x[:, 0]) * np.sin(np.pi * x[:, 1]) * np.sin(4 * np.pi * x[:, 2]))
    assert np.allclose(f.numpy(), ref, rtol=0, atol=1e-15)
