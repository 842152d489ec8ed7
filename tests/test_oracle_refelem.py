"""Pins of the oracle's 1D reference element (paper Sec. 2.2) against closed forms."""
import numpy as np
import pytest

from oracle import refelem


GLL_CLOSED = {
    1: [-1.0, 1.0],
    2: [-1.0, 0.0, 1.0],
    3: [-1.0, -1.0 / np.sqrt(5.0), 1.0 / np.sqrt(5.0), 1.0],
    4: [-1.0, -np.sqrt(3.0 / 7.0), 0.0, np.sqrt(3.0 / 7.0), 1.0],
    5: [-1.0, -np.sqrt(1.0 / 3.0 + 2.0 * np.sqrt(7.0) / 21.0), -np.sqrt(1.0 / 3.0 - 2.0 * np.sqrt(7.0) / 21.0),
        np.sqrt(1.0 / 3.0 - 2.0 * np.sqrt(7.0) / 21.0), np.sqrt(1.0 / 3.0 + 2.0 * np.sqrt(7.0) / 21.0), 1.0],
}


@pytest.mark.parametrize("p", sorted(GLL_CLOSED))
def test_gll_nodes_closed_form(p):
    assert np.allclose(refelem.gll_nodes(p), GLL_CLOSED[p], atol=1e-15, rtol=0)


def test_gll_weights_closed_form():
    assert np.allclose(refelem.gll_weights(2), [1 / 3, 4 / 3, 1 / 3], atol=1e-15)
    assert np.allclose(refelem.gll_weights(3), [1 / 6, 5 / 6, 5 / 6, 1 / 6], atol=1e-15)
    for p in range(1, 9):
        assert abs(refelem.gll_weights(p).sum() - 2.0) < 1e-14


@pytest.mark.parametrize("p", range(1, 8))
def test_lagrange_cardinal_and_derivative_exact(p):
    x = refelem.gll_nodes(p)
    assert np.allclose(refelem.lagrange_values(x, x), np.eye(p + 1), atol=1e-14)
    rng = np.random.default_rng(p)
    c = rng.normal(size=p + 1)                      # random polynomial of degree p
    f = np.polynomial.polynomial.Polynomial(c)
    t = rng.uniform(-1, 1, 7)
    interp = f(x) @ refelem.lagrange_values(x, t)
    deriv = f(x) @ refelem.lagrange_derivs(x, t)
    assert np.allclose(interp, f(t), atol=1e-12)
    assert np.allclose(deriv, f.deriv()(t), atol=1e-11)


@pytest.mark.parametrize("p", range(1, 8))
def test_mass_stiffness_exact_on_monomials(p):
    x = refelem.gll_nodes(p)
    M, K = refelem.mass_1d(p), refelem.stiffness_1d(p)
    assert np.allclose(M.sum(axis=1), refelem.gll_weights(p), atol=1e-14)   # int l_i
    assert np.allclose(K @ np.ones(p + 1), 0.0, atol=1e-12)
    assert abs(x @ K @ x - 2.0) < 1e-12
    for a in range(p + 1):
        for b in range(p + 1):
            s = a + b
            exact_m = 2.0 / (s + 1) if s % 2 == 0 else 0.0
            assert abs(x ** a @ M @ x ** b - exact_m) < 1e-13
            sk = a + b - 2
            exact_k = (a * b * 2.0 / (sk + 1) if sk % 2 == 0 else 0.0) if a > 0 and b > 0 else 0.0
            assert abs(x ** a @ K @ x ** b - exact_k) < 1e-11


def test_endpoint_tables_gll():
    for p in range(1, 7):
        e0, ep = refelem.endpoint_values(p)
        assert np.allclose(e0, np.eye(p + 1)[0]) and np.allclose(ep, np.eye(p + 1)[p])
        d0, dp = refelem.endpoint_derivs(p)
        x = refelem.gll_nodes(p)
        assert abs(d0 @ x - 1.0) < 1e-12 and abs(dp @ x - 1.0) < 1e-12
        if p >= 2:
            assert abs(d0 @ x ** 2 - (-2.0)) < 1e-12 and abs(dp @ x ** 2 - 2.0) < 1e-12


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6])
def test_gll_mass_is_lumped_plus_rank_one(p):
    """The exact GLL mass equals the lumped (row-sum) mass plus sigma l l^T with
    l_i = 1 / prod_{m != i} (x_i - x_m), the leading coefficient of the basis
    function l_i, and sigma < 0: the q-point GLL rule is exact to degree 2p - 1,
    so its error on l_i l_j is proportional to the product of leading
    coefficients. The smoothing kernels apply the facet masses in this form."""
    M = refelem.mass_1d(p)
    x = refelem.gll_nodes(p)
    w = M.sum(axis=1)
    assert np.abs(w - refelem.gll_weights(p)).max() <= 1e-14      # row sums = the GLL weights
    lc = np.array([1.0 / np.prod([x[i] - x[m] for m in range(p + 1) if m != i]) for i in range(p + 1)])
    sigma = (M[0, 0] - w[0]) / lc[0] ** 2
    assert sigma < 0
    assert np.abs(M - np.diag(w) - sigma * np.outer(lc, lc)).max() <= 1e-13
