"""Host-side planning of the estimators' batched interpolation steps
(csrc/interp_plan.hpp), compiled for the host: the coefficients (a_k, b_k)
with which the whole-lattice FP32 solves form system k's links from the two
shared endpoint fields are the oracle's Eq. (gfparam) weights of the
operator pair of that interpolation step (both operators, every chunk
offset, the independent mode), and the chunk sizes split N into equal
chunks within the budget."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import estimator

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    out = str(tmp_path_factory.mktemp("plan") / "libinterp_plan_harness.so")
    subprocess.run([cxx, "-O2", "-std=c++17", "-shared", "-fPIC", "-o", out,
                    os.path.join(HERE, "interp_plan_harness.cpp")], check=True, capture_output=True)
    h = ctypes.CDLL(out)
    h.balanced_chunk_host.restype = ctypes.c_int
    return h


def _coefs(lib, N, i0, n, shift, independent):
    ab = np.zeros(2 * n, dtype=np.float32)
    lib.interp_coefs_host(N, i0, n, shift, int(independent), ab.ctypes.data_as(ctypes.POINTER(ctypes.c_float)))
    return ab.reshape(n, 2).astype(np.float64)


@pytest.mark.parametrize("N,i0,n", [(12, 0, 12), (24, 6, 6), (24, 18, 6), (3, 2, 1), (48, 0, 48)])
def test_coefficients_are_the_oracle_pair_weights(lib, N, i0, n):
    # the oracle's pair with the endpoints as basis vectors returns the
    # weights of U and U' of both operators of interpolation step i
    e0, e1 = np.array([1.0, 0.0]), np.array([0.0, 1.0])
    for shift in (0, 1):
        got = _coefs(lib, N, i0, n, shift, False)
        for k in range(n):
            ref = estimator.pair(e0, e1, i0 + k, N, "interp")[shift]
            assert np.abs(got[k] - ref).max() <= 6e-8, (shift, k)
        if i0 == 0 and shift == 0:
            assert np.array_equal(got[0], [1.0, 0.0])      # U itself
        if i0 + n == N and shift == 1:
            assert np.array_equal(got[-1], [0.0, 1.0])     # U' itself


def test_independent_mode_pairs_u_with_u_prime(lib):
    e0, e1 = np.array([1.0, 0.0]), np.array([0.0, 1.0])
    for shift in (0, 1):
        got = _coefs(lib, 7, 3, 4, shift, True)
        ref = estimator.pair(e0, e1, 0, 7, "independent")[shift]
        assert np.array_equal(got, np.tile(ref, (4, 1)))


@pytest.mark.parametrize("N,k", [(12, 11), (24, 6), (24, 7), (12, 12), (12, 100), (5, 1), (3, 2), (1, 0), (48, 14)])
def test_balanced_chunks(lib, N, k):
    c = lib.balanced_chunk_host(N, k)
    kk = min(max(k, 1), N)
    chunks = [min(c, N - i0) for i0 in range(0, N, c)]
    assert sum(chunks) == N
    assert c <= kk                                   # within the budget
    assert len(chunks) == -(-N // kk)                # no more chunks than the budget needs
    assert max(chunks) - min(chunks) <= 1            # equal sizes
