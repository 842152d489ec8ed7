"""Mistakes planted in the oracle, on the CPU, each of which one of the pins
must catch: a wrong sign, a wrong mean, a dropped term, a wrong weight or a lost
smoothing step anywhere in the operator, the transfers, the smoother or the
V-cycle makes the named pin fail. (Each plant is undone after its test.)"""
import numpy as np
import pytest
import scipy.sparse as sp

import test_oracle_hpmg as H
import test_oracle_refelem as R
import test_oracle_sipg as S
import test_oracle_traffic as T
from oracle import hpmg, refelem, sipg, traffic


def _fails(pin, *args):
    with pytest.raises(AssertionError):
        pin(*args)


def test_theta_sign(monkeypatch):
    # the non-symmetric form in the matrix-free route (Sec. 2.3.1 sign convention;
    # the term vanishes for continuous u, so the consistency pin cannot see it:
    # the independent assembled route does)
    monkeypatch.setattr(sipg, "THETA", +1.0)
    _fails(S.test_assembled_equals_facet_route, (3, 4), 2, "one")


def test_arithmetic_facet_kappa(monkeypatch):
    # the arithmetic instead of the harmonic mean of kappa on interior facets
    def arithmetic(mesh, kappa_grid, direction):
        ca, nd, k = mesh.cell_axis(direction), mesh.n[direction], kappa_grid
        shape = list(k.shape)
        shape[ca] = nd + 1
        kF = np.zeros(shape)
        kF[sipg._sl(mesh.d, ca, slice(1, nd))] = 0.5 * (k[sipg._sl(mesh.d, ca, slice(0, nd - 1))]
                                                       + k[sipg._sl(mesh.d, ca, slice(1, nd))])
        kF[sipg._sl(mesh.d, ca, slice(0, 1))] = k[sipg._sl(mesh.d, ca, slice(0, 1))]
        kF[sipg._sl(mesh.d, ca, slice(nd, nd + 1))] = k[sipg._sl(mesh.d, ca, slice(nd - 1, nd))]
        return kF.reshape(kF.shape + (1,) * mesh.d)
    monkeypatch.setattr(sipg, "facet_kappa", arithmetic)
    _fails(S.test_assembled_equals_facet_route, (3, 4), 2, "lognormal")


def test_dropped_volume_axis(monkeypatch):
    # the volume term of the last axis dropped from the cell equation
    def partial(mesh, U, kappa_grid):
        Y = np.zeros_like(U)
        for direction in range(mesh.d - 1):
            T = U
            for a in range(mesh.d):
                T = sipg.apply_1d(mesh.K[a] if a == direction else mesh.M[a], T, mesh.node_axis(a))
            Y += T
        return Y * kappa_grid.reshape(kappa_grid.shape + (1,) * mesh.d)
    monkeypatch.setattr(sipg, "volume_term", partial)
    _fails(S.test_assembled_equals_facet_route, (3, 4), 2, "one")


def test_wrong_block_inverse(monkeypatch):
    # a block inverse off by one percent: the smoother is no longer Alg. 2 / Alg. 4
    orig = sipg.BlockJacobi.apply_inverse
    monkeypatch.setattr(sipg.BlockJacobi, "apply_inverse", lambda self, r: 1.01 * orig(self, r))
    _fails(S.test_smoother_fixed_point_and_orders, (3, 4), 2, "one")


def test_p_prolongation_weight(monkeypatch):
    # one hat of the p-prolongation (Sec. 5.1) with half its weight
    orig = hpmg.p_prolongation

    def halved(mesh):
        P = orig(mesh).tolil(copy=True)
        P[:, 0] = 0.5 * P[:, 0].toarray()
        return P.tocsr()
    monkeypatch.setattr(hpmg, "p_prolongation", halved)
    _fails(H.test_p_prolongation_is_q1_interpolation, (4, 3), 2)
    _fails(H.test_galerkin_p_coarse_operator_is_q1_stiffness, (4, 4), 2)


def test_h_prolongation_mirrored_weights(monkeypatch):
    # the 1D interpolation taken from the wrong end of the axis (the short
    # coarse cell of an odd mesh at the start instead of the end)
    orig = hpmg.interp_1d
    monkeypatch.setattr(hpmg, "interp_1d", lambda n, f: sp.csr_matrix(orig(n, f).toarray()[::-1, ::-1]))
    _fails(H.test_h_prolongation_is_nested_q1_interpolation, (13, 7), 2)


def test_lost_q1_smoothing_step(monkeypatch):
    # one Q1 Jacobi step lost on every call (pre- and post-smoothing)
    orig = hpmg.Hierarchy.cg_jacobi
    monkeypatch.setattr(hpmg.Hierarchy, "cg_jacobi",
                        lambda self, level, u, b, nsteps: orig(self, level, u, b, max(nsteps - 1, 0)))
    _fails(H.test_vcycle_matches_dense_error_propagation, (6, 5), 2, "lognormal")


def test_table1_coefficient(monkeypatch):
    # 6d instead of 7d facet values per cell in the access model of Table 1
    def wrong(d, p, standalone=False):
        return (5 if standalone else 3) * (p + 1) ** d + 6 * d * (p + 1) ** (d - 1)
    monkeypatch.setattr(traffic, "accesses_alg2", wrong)
    _fails(T.test_table1_memory_accesses)


def test_lumped_mass(monkeypatch):
    # the GLL-lumped mass diag(w) in place of the exact 1D mass (Sec. 4.1: with
    # GLL nodes the exact mass is not diagonal)
    monkeypatch.setattr(refelem, "mass_1d", lambda p, basis="gll": np.diag(refelem.gll_weights(p)))
    _fails(R.test_mass_stiffness_exact_on_monomials, 3)


def test_gll_weight_formula(monkeypatch):
    # P_p(x_j) to the first instead of the second power in the GLL weights
    import numpy.polynomial.legendre as npleg

    def wrong(p):
        c = np.zeros(p + 1)
        c[p] = 1.0
        return 2.0 / (p * (p + 1) * np.abs(npleg.legval(refelem.gll_nodes(p), c)))
    monkeypatch.setattr(refelem, "gll_weights", wrong)
    _fails(R.test_gll_weights_closed_form)


def test_too_few_load_vector_points(monkeypatch):
    # p points per axis: exact only to degree 2p - 1, below the 2p of (f, phi_i)
    orig = sipg.load_vector
    monkeypatch.setattr(sipg, "load_vector", lambda mesh, f, nquad=None: orig(mesh, f, mesh.q - 1))
    _fails(S.test_load_vector_and_l2_error_closed_forms)


def test_technique4_wrong_centre_cell(monkeypatch):
    # the Technique 4 block taken from the cell before the centre of the 3^d
    # helper mesh (a cell with a boundary facet) instead of the centre cell
    orig = sipg.block_diagonal
    monkeypatch.setattr(sipg, "block_diagonal", lambda mesh, kappa=None: np.roll(orig(mesh, kappa), 1, axis=0))
    _fails(S.test_interior_only_block_is_an_interior_cells_assembled_block, (3, 4), 3)


def test_mgmult_lost_smoothing_step(monkeypatch):
    # MGMult (Alg. 7) with one block-Jacobi step per cycle lost
    import test_oracle_mgmult as G
    orig = sipg.BlockJacobi.step_alg2
    monkeypatch.setattr(sipg.BlockJacobi, "step_alg2",
                        lambda self, u, b, omega, nsteps=1: orig(self, u, b, omega, max(nsteps - 1, 0)))
    _fails(G.test_mgmult_iterates_follow_the_dense_cycle, (6, 5), 2, 2)
