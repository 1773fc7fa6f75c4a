"""The library's HYP arithmetic (the per-link code its kernels run,
csrc/hyp.cuh) compiled for the host by a test harness and compared with the
oracle without a GPU: the polar-iteration projection against the oracle's
eigendecomposition, the fat links and the block HYP action."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import gauge, hyp, lattice
from tests import seeded

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    out = str(tmp_path_factory.mktemp("hyp") / "libhyp_harness.so")
    subprocess.run([nvcc, "-O2", "-std=c++17", "-shared", "-Xcompiler", "-fPIC", "-o", out,
                    os.path.join(HERE, "hyp_harness.cu")], check=True, capture_output=True)
    lib = ctypes.CDLL(out)
    for f in (lib.hyp_smear_host, lib.hyp_block_action_host, lib.hyp_project_host):
        f.restype = None
    return lib


def _c(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def _smear(lib, U, alpha):
    U = _c(U)
    out = np.empty_like(U)
    L = (ctypes.c_int * 4)(*U.shape[:4])
    lib.hyp_smear_host(U.ctypes.data, L, (ctypes.c_double * 3)(*alpha), out.ctypes.data)
    return out


def test_projection_matches_oracle(harness):
    M = np.stack([seeded.complex_matrix(3, s) for s in range(50)] +
                 [np.eye(3) + 0.1 * seeded.complex_matrix(3, 100 + s) for s in range(50)])
    M = _c(M)
    out = np.empty_like(M)
    harness.hyp_project_host(M.ctypes.data, len(M), out.ctypes.data)
    assert np.abs(out - hyp.project_su3(M)).max() < 1e-12


@pytest.mark.parametrize("dims,alpha", [((4, 4, 4, 4), hyp.ALPHA), ((4, 6, 4, 2), hyp.ALPHA),
                                        ((4, 4, 4, 4), (0.5, 0.9, 0.1))])
def test_fat_links_match_oracle(harness, dims, alpha):
    U = gauge.generate_links(dims, 0.6, 31)
    assert np.abs(_smear(harness, U, alpha) - hyp.smear(U, alpha)).max() < 1e-12


def test_block_action_matches_oracle(harness):
    geom = lattice.Geometry((6, 6, 6, 6), (3, 3, 3, 3))
    U = gauge.generate_links(geom.dims, 0.5, 32)
    V = _smear(harness, U, hyp.ALPHA)
    out = np.empty(geom.n_blocks)
    harness.hyp_block_action_host(V.ctypes.data, (ctypes.c_int * 4)(*geom.dims), (ctypes.c_int * 4)(*geom.block),
                                  out.ctypes.data)
    assert np.abs(out - hyp.block_hyp_action(U, geom)).max() < 1e-11
