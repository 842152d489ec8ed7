"""The library's host set-up of the 1D reference element (GLL or GL nodes, the
exact mass and stiffness, the end-point values and derivatives, the Cholesky
factor inverse of the mass, Gauss-Legendre rules; Sec. 2.2 and 6.5), built on
the CPU from its own source and compared with the oracle's reference element."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import refelem

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2510_00998_gb300", "csrc")


def _compiler():
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    nvcc = os.path.join(cuda, "bin", "nvcc")
    if os.path.exists(nvcc):
        return [nvcc, "-x", "cu"], cuda
    if shutil.which("nvcc"):
        return ["nvcc", "-x", "cu"], cuda
    pytest.skip("nvcc not available")


@pytest.fixture(scope="module")
def dump(tmp_path_factory):
    cc, cuda = _compiler()
    exe = str(tmp_path_factory.mktemp("refelem") / "refelem_dump")
    cmd = cc + ["-std=c++17", "-O2", "-I" + os.path.join(ROOT, "include"), "-I" + CSRC,
                os.path.join(ROOT, "tests", "refelem_dump.cpp"), os.path.join(CSRC, "refelem.cpp"), "-o", exe]
    p = subprocess.run(cmd, capture_output=True, text=True)
    assert p.returncode == 0, p.stdout + p.stderr
    out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    tables = {}
    for line in out.splitlines():
        f = line.split()
        tables[(f[0], int(f[1]), int(f[2]))] = np.array([float(v) for v in f[3:]])
    return tables


BASES = {0: "gll", 1: "gl"}


@pytest.mark.parametrize("basis", [0, 1])
@pytest.mark.parametrize("p", range(1, 7))
def test_reference_element_matches_oracle(dump, p, basis):
    q, b = p + 1, BASES[basis]
    nodes = dump[("nodes", p, basis)]
    assert np.abs(nodes - refelem.basis_nodes(p, b)).max() <= 1e-15
    M, K = dump[("M", p, basis)].reshape(q, q), dump[("K", p, basis)].reshape(q, q)
    Mo, Ko = refelem.mass_1d(p, b), refelem.stiffness_1d(p, b)
    assert np.abs(M - Mo).max() <= 1e-14 * np.abs(Mo).max()
    assert np.abs(K - Ko).max() <= 1e-13 * np.abs(Ko).max()
    e0, ep = refelem.endpoint_values(p, b)
    d0, dp = refelem.endpoint_derivs(p, b)
    assert np.abs(dump[("e0", p, basis)] - e0).max() <= 1e-14
    assert np.abs(dump[("ep", p, basis)] - ep).max() <= 1e-14
    assert np.abs(dump[("d0", p, basis)] - d0).max() <= 1e-12 * np.abs(d0).max()
    assert np.abs(dump[("dp", p, basis)] - dp).max() <= 1e-12 * np.abs(dp).max()
    if basis == 0:
        # GLL: the end values are exactly the unit vectors (the kernels rely on it)
        assert np.array_equal(dump[("e0", p, basis)], np.eye(q)[0])
        assert np.array_equal(dump[("ep", p, basis)], np.eye(q)[-1])
    else:
        # GL: the exact mass is the diagonal of the Gauss weights (Sec. 6.4)
        assert np.abs(M - np.diag(refelem.gauss_legendre(q)[1])).max() <= 1e-14


@pytest.mark.parametrize("basis", [0, 1])
@pytest.mark.parametrize("p", range(1, 7))
def test_cholesky_inverse_of_the_mass(dump, p, basis):
    # L^-1 lower triangular with L^-1 M L^-T = I (the factors' generalised
    # eigenproblem is reduced with it)
    q = p + 1
    Li = dump[("Linv", p, basis)].reshape(q, q)
    M = dump[("M", p, basis)].reshape(q, q)
    assert np.array_equal(np.tril(Li), Li)
    assert np.abs(Li @ M @ Li.T - np.eye(q)).max() <= 1e-13


@pytest.mark.parametrize("m", range(1, 10))
def test_gauss_legendre_rules(dump, m):
    x, w = dump[("glx", m, 0)], dump[("glw", m, 0)]
    xo, wo = refelem.gauss_legendre(m)
    assert np.abs(x - xo).max() <= 1e-15 and np.abs(w - wo).max() <= 1e-14
    # exact for every monomial of degree <= 2m - 1
    for k in range(2 * m):
        exact = 2.0 / (k + 1) if k % 2 == 0 else 0.0
        assert abs(w @ x ** k - exact) <= 1e-14
