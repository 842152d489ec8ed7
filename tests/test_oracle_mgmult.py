"""Pin of the oracle's MGMult (Alg. 7): each cycle is nu block-Jacobi steps
followed by the coarse-grid correction of Alg. 6 (one h-V-cycle on the Q1
levels), so the error after k cycles is E^k times the initial error with the
dense cycle matrix E = (I - P B_0 P^T A) J^nu, built here from the assembled
matrix (J = I - omega D^-1 A with D its diagonal blocks, B_0 the dense h-cycle
on the Q1 levels). The two exit criteria of Sec. 6.3 are checked against norms
of these dense iterates. (The cycle counts of Tables 3-5 depend on parameters
the paper does not state; the iteration itself is pinned here.)"""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import hpmg, sipg


def _dense_cycle(hier, Ad):
    """E of one MGMult cycle, from dense matrices only."""
    def level_B(level):
        A = hier.A[level].toarray()
        if level == hier.nlevels - 1:
            return np.linalg.inv(A)
        J = np.eye(len(A)) - hier.omega_cg * A / hier.D[level][:, None]
        Ph = hier.Ph[level].toarray()
        E = (np.linalg.matrix_power(J, hier.nu_post) @ (np.eye(len(A)) - Ph @ level_B(level + 1) @ Ph.T @ A)
             @ np.linalg.matrix_power(J, hier.nu_pre))
        return (np.eye(len(A)) - E) @ np.linalg.inv(A)
    nl = hier.mesh.nloc
    D = sla.block_diag(*[Ad[c * nl:(c + 1) * nl, c * nl:(c + 1) * nl] for c in range(hier.mesh.ncell)])
    J = np.eye(len(Ad)) - hier.omega_dg * np.linalg.solve(D, Ad)
    P = hier.P.toarray()
    return (np.eye(len(Ad)) - P @ level_B(0) @ P.T @ Ad) @ np.linalg.matrix_power(J, hier.nu_pre)


@pytest.mark.parametrize("n,p,nu", [((6, 5), 2, 2), ((6, 6), 1, 4), ((4, 3, 4), 1, 3)])
def test_mgmult_iterates_follow_the_dense_cycle(n, p, nu):
    mesh = sipg.Mesh(n, p)
    kap = np.exp(np.random.default_rng(21).normal(size=mesh.ncell))
    hier = hpmg.Hierarchy(mesh, kap, nu_pre=nu)
    assert hier.nlevels >= 2
    Ad = sipg.assemble(mesh, kap).toarray()
    E = _dense_cycle(hier, Ad)
    rng = np.random.default_rng(22)
    b, u0 = rng.normal(size=mesh.ndof), rng.normal(size=mesh.ndof)
    xs = np.linalg.solve(Ad, b)
    e = u0 - xs
    for k in (1, 2, 5):
        u, cycles = hpmg.mgmult(hier, b, u0=u0, eps=1e-300, maxit=k)
        assert cycles == k
        ek = np.linalg.matrix_power(E, k) @ e
        assert np.abs((u - xs) - ek).max() <= 1e-10 * np.abs(e).max()
    # the cycle contracts
    assert np.max(np.abs(np.linalg.eigvals(E))) < 1.0


@pytest.mark.parametrize("kind", ["unprec", "prec"])
def test_mgmult_exit_criteria(kind):
    """'unprec' stops at the first k with ||b - A u_k|| < eps ||b - A u_0||;
    'prec' at the first k with ||u_k - u_(k-1)|| < eps ||u_1 - u_0||."""
    n, p = (6, 5), 2
    mesh = sipg.Mesh(n, p)
    kap = np.exp(np.random.default_rng(23).normal(size=mesh.ncell))
    hier = hpmg.Hierarchy(mesh, kap, nu_pre=2)
    Ad = sipg.assemble(mesh, kap).toarray()
    E = _dense_cycle(hier, Ad)
    b = np.random.default_rng(24).normal(size=mesh.ndof)
    xs = np.linalg.solve(Ad, b)
    us = [np.zeros(mesh.ndof)]
    for _ in range(60):
        us.append(xs + E @ (us[-1] - xs))
    eps = 1e-6
    if kind == "unprec":
        r0 = np.linalg.norm(b - Ad @ us[0])
        want = next(k for k in range(1, 61) if np.linalg.norm(b - Ad @ us[k]) < eps * r0)
    else:
        d1 = np.linalg.norm(us[1] - us[0])
        want = next(k for k in range(1, 61) if np.linalg.norm(us[k] - us[k - 1]) < eps * d1)
    u, cycles = hpmg.mgmult(hier, b, eps=eps, maxit=200, residual_kind=kind)
    assert cycles == want
    assert np.abs(u - us[want]).max() <= 1e-9 * np.abs(xs).max()
