"""Per-thread arithmetic of the library's kernels compiled for the host by a
test harness (tests/kernel_math_harness.cu) and compared with the oracle
without a GPU: the HYP smearing (csrc/hyp.cuh: the polar-iteration
projection against the oracle's eigendecomposition, the fat links, the
block HYP action) and the per-block plaquette-action change with its block
scan (csrc/block_action.cuh)."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import dirac, filter as ofilter, gauge, hyp, lattice
from tests import seeded

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    out = str(tmp_path_factory.mktemp("kmath") / "libkernel_math_harness.so")
    subprocess.run([nvcc, "-O2", "-std=c++17", "-shared", "-Xcompiler", "-fPIC", "-o", out,
                    os.path.join(HERE, "kernel_math_harness.cu")], check=True, capture_output=True)
    lib = ctypes.CDLL(out)
    for f in (lib.hyp_smear_host, lib.hyp_block_action_host, lib.hyp_project_host, lib.block_change_host,
              lib.outer_faces_host, lib.outer_crossing_host):
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


def _su3_exp(omega, eps):
    return gauge.expm_i_hermitian(gauge.hermitian_generators(omega), eps)


@pytest.mark.parametrize("dims,block,which", [((6, 6, 6, 6), (3, 3, 3, 3), "active"),
                                              ((4, 4, 4, 4), (2, 2, 2, 2), "active"),
                                              ((4, 4, 4, 4), (2, 2, 2, 2), "random"),
                                              ((4, 8, 4, 4), (4, 2, 2, 2), "random")])
def test_block_action_change_matches_oracle(harness, dims, block, which):
    """dS_w,b with the first-changed-link attribution: proposals on the
    active links (blocks of extent 3 and 2) and on a random subset of all
    links, including a direction spanned by one block."""
    geom = lattice.Geometry(dims, block)
    U = gauge.generate_links(dims, 0.5, 40)
    g = np.random.default_rng(41)
    sel = geom.active_links() if which == "active" else g.random(dims + (4,)) < 0.15
    Up = np.where(sel[..., None, None], U @ _su3_exp(g.standard_normal(dims + (4, 8)), 0.4), U)
    out = np.empty(geom.n_blocks)
    harness.block_change_host(_c(U).ctypes.data, _c(Up).ctypes.data, (ctypes.c_int * 4)(*dims),
                              (ctypes.c_int * 4)(*block), out.ctypes.data)
    ref = ofilter.per_block_action_change(U, Up, geom)
    assert np.abs(out - ref).max() < 1e-11
    assert abs(out.sum() - (gauge.wilson_action(Up) - gauge.wilson_action(U))) < 1e-9


def _projector_from_faces(info):
    """Per-site spin projector from (colour, faces, mu, sign) as the kernels
    apply it: (1 + t gamma_mu)/2 for one face, 1 for more, 0 otherwise."""
    from oracle.gamma import GAMMA
    P = np.zeros(info.shape[:-1] + (4, 4), dtype=np.complex128)
    col, nf, mu, t = (info[..., k] for k in range(4))
    one = (col == 0) & (nf == 1)
    for m in range(4):
        for sg in (1, -1):
            sel = one & (mu == m) & (t == sg)
            P[sel] = 0.5 * (np.eye(4) + sg * GAMMA[m])
    P[(col == 0) & (nf >= 2)] = np.eye(4)
    return P


@pytest.mark.parametrize("dims,outer,inner", [((16, 8, 8, 8), (8, 4, 4, 4), (4, 2, 2, 2)),
                                              ((8, 8, 8, 8), (4, 4, 4, 4), (2, 2, 2, 2))])
def test_outer_projectors_and_masks_match_oracle(harness, dims, outer, inner):
    """The recursive decomposition's face logic: the SUB projector equals
    the oracle's P_b on every outer block, the OUTER projector the oracle's
    projector of the outer blocks, and the masked links are exactly those
    whose hop leaves an outer block."""
    from oracle import recursive
    nest = recursive.Nested(dims, outer, inner)
    L, l, B = (ctypes.c_int * 4)(*dims), (ctypes.c_int * 4)(*inner), (ctypes.c_int * 4)(*outer)
    info = np.empty(dims + (4,), dtype=np.int32)
    harness.outer_faces_host(L, l, B, 0, info.ctypes.data)
    Psub = _projector_from_faces(info)
    Pb = recursive.sub_projector(nest)
    for b in range(nest.outer.n_blocks):
        assert np.array_equal(dirac.extract_block(Psub, nest.outer, b), Pb)
    harness.outer_faces_host(L, l, B, 1, info.ctypes.data)
    assert np.array_equal(_projector_from_faces(info), nest.outer.projector())
    cr = np.empty(dims + (4,), dtype=np.int32)
    harness.outer_crossing_host(L, B, cr.ctypes.data)
    for mu in range(4):
        assert np.array_equal(cr[..., mu].astype(bool), ~nest.outer.fwd_intra(mu))
