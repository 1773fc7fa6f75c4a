"""The shared-memory layout and the descriptors of the MLP's tensor-core
GEMM (csrc/tc_layout.hpp), compiled for the host: the operand tile is the
canonical no-swizzle K-major layout of tcgen05.mma (8 x 16-byte core
matrices), the strides written into the shared-memory descriptor describe
that same layout, each K = 16 slice the kernel hands to one MMA has it too,
and the descriptor fields sit where the PTX ISA puts them."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    out = str(tmp_path_factory.mktemp("tclayout") / "libtc_layout_harness.so")
    subprocess.run([cxx, "-O2", "-std=c++17", "-shared", "-fPIC", "-o", out,
                    os.path.join(HERE, "tc_layout_harness.cpp")], check=True, capture_output=True)
    h = ctypes.CDLL(out)
    h.tc_smem_desc_host.restype = ctypes.c_uint64
    h.tc_smem_desc_host.argtypes = [ctypes.c_uint32] * 3
    h.tc_instr_desc_host.restype = ctypes.c_uint32
    h.tc_instr_desc_host.argtypes = [ctypes.c_int]
    return h


def _consts(lib):
    c = (ctypes.c_int * 4)()
    lib.tc_constants_host(c)
    return tuple(c)


def _offsets(lib, rows):
    tm, tk, _, _ = _consts(lib)
    out = np.zeros(rows * tk, dtype=np.uint32)
    lib.tc_canon_off_host(rows, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)))
    return out.reshape(rows, tk).astype(np.int64)


@pytest.mark.parametrize("rows", [128, 64, 256])
def test_tile_layout_is_the_canonical_k_major_one(lib, rows):
    tm, tk, lbo, sbo = _consts(lib)
    off = _offsets(lib, rows)
    # a bijection onto the tile's 2-byte elements
    assert np.array_equal(np.sort(off.ravel()), np.arange(0, rows * tk * 2, 2))
    r, k = np.meshgrid(np.arange(rows), np.arange(tk), indexing="ij")
    # core matrix (r/8, k/8) is 128 contiguous bytes: 8 rows of 16 bytes,
    # 8 consecutive K elements per row
    core = off // 128
    assert np.array_equal(core, (r // 8) * (tk // 8) + k // 8)
    assert np.array_equal(off % 128, (r % 8) * 16 + (k % 8) * 2)
    # the strides of the descriptor: core matrices LBO apart along K, groups
    # of 8 rows SBO apart
    assert np.array_equal(off, (k // 8) * lbo + (r // 8) * sbo + (r % 8) * 16 + (k % 8) * 2)


def test_each_mma_slice_has_the_same_layout(lib):
    """MMA j of a chunk reads K = 16j .. 16j + 15 from the descriptor start
    tile + 2 j LBO: relative to that start, the slice is laid out as slice 0."""
    tm, tk, lbo, sbo = _consts(lib)
    off = _offsets(lib, tm)
    for j in range(tk // 16):
        assert np.array_equal(off[:, 16 * j:16 * j + 16] - 2 * j * lbo, off[:, :16])


def test_shared_memory_descriptor_fields(lib):
    tm, tk, lbo, sbo = _consts(lib)
    for addr in (0, 16, 0x3FFF0, 98304 + 256):
        d = lib.tc_smem_desc_host(addr, lbo, sbo)
        assert d & 0x3FFF == (addr >> 4) & 0x3FFF
        assert (d >> 16) & 0x3FFF == lbo >> 4
        assert (d >> 32) & 0x3FFF == sbo >> 4
        assert (d >> 46) & 0x7 == 1          # descriptor version
        assert (d >> 49) & 0x7 == 0          # base offset
        assert (d >> 52) & 0x1 == 0          # relative leading-offset mode
        assert (d >> 61) & 0x7 == 0          # no swizzle
        assert (d >> 14) & 0x3 == 0 and (d >> 30) & 0x3 == 0


@pytest.mark.parametrize("tn", [256, 64])
def test_instruction_descriptor_fields(lib, tn):
    tm, _, _, _ = _consts(lib)
    d = lib.tc_instr_desc_host(tn)
    assert d & 0x7 == 0                      # dense, no sparsity selector
    assert (d >> 3) & 1 == 0                 # no saturation
    assert (d >> 4) & 0x3 == 1               # FP32 accumulator
    assert (d >> 7) & 0x7 == 1               # A: BF16
    assert (d >> 10) & 0x7 == 1              # B: BF16
    assert (d >> 13) & 0xF == 0              # no negation, both K-major
    assert (d >> 17) & 0x3F == tn // 8       # N / 8
    assert (d >> 23) & 1 == 0
    assert (d >> 24) & 0x1F == tm // 16      # M / 16
    assert d >> 29 == 0
