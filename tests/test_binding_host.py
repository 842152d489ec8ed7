"""Argument checks of the Python binding that run before any library call:
vector lengths from the mesh and degree, one coefficient per cell, tensors on
the device (CPU only: nothing here reaches a kernel)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def dgmg():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2510_00998_gb300 import dgmg as m
    return m


def test_sizes_from_mesh_and_degree(dgmg):
    assert dgmg._ncell((4, 5, 6)) == 120
    assert dgmg._ndof((4, 5, 6), 3) == 120 * 64
    assert dgmg._ndof((7, 3), 4) == 21 * 25


def test_kappa_needs_one_value_per_cell(dgmg):
    k = dgmg._kappa([[1.0, 2.0], [3.0, 4.0]], (2, 2))
    assert k.dtype == np.float64 and k.flags["C_CONTIGUOUS"] and k.tolist() == [1.0, 2.0, 3.0, 4.0]
    with pytest.raises(ValueError):
        dgmg._kappa(np.ones(15), (4, 4))
    with pytest.raises(ValueError):
        dgmg.Context((4, 4), 2, kappa=np.ones(17))      # rejected before the context is created


def test_pointer_checks(dgmg):
    with pytest.raises(TypeError):
        dgmg._ptr(np.zeros(4))
    with pytest.raises(ValueError):
        dgmg._ptr(torch.zeros(4, dtype=torch.float64))  # host tensor
    assert dgmg._ptr(None) is None


def test_missing_library_fails_loudly(dgmg, monkeypatch, tmp_path):
    """No fallback: without libdgmg.so every entry of the binding raises."""
    monkeypatch.setattr(dgmg, "_lib", None)
    missing = str(tmp_path / "libdgmg.so")
    with pytest.raises(OSError):
        dgmg.load(missing)
    monkeypatch.setattr(dgmg, "LIB_PATH", missing)
    monkeypatch.setattr(dgmg.load, "__defaults__", (missing,))
    with pytest.raises(OSError):
        dgmg.Context((4, 4), 2)
    with pytest.raises(OSError):
        dgmg.kernel_launches()


def test_estimate_bytes_on_the_host(dgmg):
    """dgmg_estimate_bytes (the server's admission size; equal to a context's
    allocations, checked on the GPU) is host arithmetic: it validates its
    arguments and grows with the problem as its arrays do."""
    for bad in [((4, 4), 0), ((4, 4), 7), ((1, 4), 2), ((4, 4, 4, 4), 2)]:
        with pytest.raises(dgmg.DGMGError) as ei:
            dgmg.estimate_bytes(*bad)
        assert ei.value.code == dgmg.DGMG_EINVAL
    with pytest.raises(dgmg.DGMGError):
        dgmg.estimate_bytes((8, 8, 8), 3, coarsening=4)
    b16, b32 = dgmg.estimate_bytes((16, 16, 16), 3), dgmg.estimate_bytes((32, 32, 32), 3)
    ndof = 32 ** 3 * 64
    # at least the five FP64 solver vectors, the DG iterate's table and two trace buffers
    assert b32 >= (5 + 1) * 8 * ndof + 2 * 8 * 32 ** 3 * 6 * 2 * 16
    assert 7.5 <= b32 / b16 <= 8.1                      # linear in the cells (the coarse inverse is small)
    mixed = dgmg.estimate_bytes((32, 32, 32), 3, precision=dgmg.DGMG_MIXED_FP32)
    assert b32 < mixed < 2 * b32                         # FP32 copies of the DG and Q1 levels on top
    assert dgmg.estimate_bytes((32, 32, 32), 3, p_coarsening=1) > b32


def test_default_options_are_the_documented_ones(dgmg):
    """dgmg_default_opts fills the defaults the header states (the readings of
    the unstated parameters: omega 0.8 on both level kinds, V(2,2), exact
    blocks, coarsening factor 2, rtol 1e-10)."""
    o = dgmg.default_opts()
    assert (o.omega_dg, o.omega_cg, o.nu_pre, o.nu_post) == (0.8, 0.8, 2, 2)
    assert o.precision == dgmg.DGMG_FP64 and o.block_inverse == dgmg.DGMG_BLOCK_EXACT
    assert (o.coarsening, o.rtol, o.maxit, o.delta) == (2, 1e-10, 200, 0.01)
    assert (o.autotune, o.p_coarsening, o.basis, o.recompute_block) == (0, 0, dgmg.DGMG_BASIS_GLL, 0)
    assert b"sm_103a" in dgmg.load().dgmg_version()
