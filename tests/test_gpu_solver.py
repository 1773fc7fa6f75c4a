"""GPU parity of the Krylov solves (whole lattice and Dirichlet blocks) with
the oracle: the solution matches the oracle's CGNR solution and the true
residual, recomputed with the oracle's D, meets the tolerance."""
import functools

import numpy as np
import pytest
import torch

import paper_1204_1306_gb300 as ps
from oracle import dirac, estimator, gauge, lattice, linalg
from tests import seeded
from tests.gpu_util import canonical, native, rel_err

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("solver", [ps.SOLVER_CGNR, ps.SOLVER_BICGSTAB])
@pytest.mark.parametrize("inner", [ps.PREC_F64, ps.PREC_F32, ps.PREC_BF16])
def test_full_solve_parity(inner, solver):
    dims, block, kappa = (4, 4, 4, 4), (2, 2, 2, 2), 0.15
    ctx = ps.psms_create(dims, block, kappa, 1)
    ps.psms_full_solver(ctx, solver)
    ps.psms_gauge_init(ctx, 0, 0.3, 0x50534D53)
    U = gauge.generate_links(dims, 0.3, 0x50534D53)
    b = seeded.spinor(dims, 1)
    x = torch.zeros_like(native(ctx, b))
    info = ps.psms_solve(ctx, 0, ps.OP_FULL, native(ctx, b), x, 1e-13, 20000, inner)
    got = canonical(ctx, x)
    ref, _, _ = linalg.cgnr(lambda v: dirac.apply_D(U, v, kappa), lambda v: dirac.apply_D(U, v, kappa, dagger=True),
                            b, tol=1e-14)
    r = b - dirac.apply_D(U, got, kappa)
    assert np.sqrt(linalg.norm2(r) / linalg.norm2(b)) <= 1e-13
    assert info["true_residual"] <= 1e-13
    assert rel_err(got, ref) < 1e-11


@pytest.mark.parametrize("solver", [ps.SOLVER_CGNR, ps.SOLVER_BICGSTAB])
def test_full_solve_16x4_config(solver):
    """16^4, kappa = 0.156, eps = 0.5 links: mixed FP32 inner iterations in FP64
    defect correction to 1e-10 (true residual checked with the oracle's D),
    with either inner Krylov method."""
    dims, block, kappa = (16, 16, 16, 16), (4, 4, 4, 4), 0.156
    ctx = ps.psms_create(dims, block, kappa, 1)
    ps.psms_full_solver(ctx, solver)
    ps.psms_gauge_init(ctx, 0, 0.5, 0x50534D53 + 1)
    U = gauge.generate_links(dims, 0.5, 0x50534D53 + 1)
    b = seeded.spinor(dims, 2)
    x = torch.zeros_like(native(ctx, b))
    info = ps.psms_solve(ctx, 0, ps.OP_FULL, native(ctx, b), x, 1e-10, 20000, ps.PREC_F32)
    got = canonical(ctx, x)
    r = b - dirac.apply_D(U, got, kappa)
    assert np.sqrt(linalg.norm2(r) / linalg.norm2(b)) <= 1e-10
    assert info["outer_iters"] >= 1


@pytest.mark.parametrize("krylov", [ps.SOLVER_CGNR, ps.SOLVER_BICGSTAB])
@pytest.mark.parametrize("inner", [ps.PREC_F64, ps.PREC_F32])
@pytest.mark.parametrize("dims,block", [((4, 4, 4, 4), (2, 2, 2, 2)), ((8, 8, 8, 8), (4, 4, 4, 4)),
                                        ((8, 8, 8, 8), (8, 8, 8, 4))])
def test_block_solve_parity(dims, block, inner, krylov):
    kappa = 0.156
    geom = lattice.Geometry(dims, block)
    ctx = ps.psms_create(dims, block, kappa, 1)
    ps.psms_block_krylov(ctx, krylov)
    ps.psms_gauge_init(ctx, 0, 0.5, 5)
    U = gauge.generate_links(dims, 0.5, 5)
    b = seeded.spinor(dims, 6)
    x = torch.zeros_like(native(ctx, b))
    ps.psms_solve(ctx, 0, ps.OP_BLOCKS, native(ctx, b), x, 1e-13, 20000, inner)
    got = canonical(ctx, x)
    blocks = sorted({0, geom.n_blocks // 3, geom.n_blocks - 1})
    ref = estimator.solve_blocks(U, b, geom, kappa, blocks, 1e-14)
    for bb in blocks:
        g = dirac.extract_block(got, geom, bb)
        assert rel_err(g, dirac.extract_block(ref, geom, bb)) < 1e-11
    # true residual of the whole block-diagonal system
    r = b - dirac.apply_D(U, got, kappa, geom, mode="block")
    assert np.sqrt(linalg.norm2(r) / linalg.norm2(b)) <= 1e-13
    # single block: zero outside
    x1 = torch.zeros_like(x)
    ps.psms_solve(ctx, 0, blocks[-1], native(ctx, b), x1, 1e-13, 20000, inner)
    g1 = canonical(ctx, x1)
    mask = (geom.block_index == blocks[-1])[..., None, None]
    assert np.abs(g1 * ~mask).max() == 0.0
    assert rel_err(g1 * mask, ref * mask) < 1e-11


def test_bicgstab_batched_global_estimates_match():
    """The global level (batched whole-lattice solves of the Schur estimator)
    gives the same estimates with either inner method (both to 1e-13)."""
    dims, block, kappa = (8, 8, 8, 8), (4, 4, 4, 4), 0.156
    ctx = ps.psms_create(dims, block, kappa, 2)
    ps.psms_gauge_init(ctx, 0, 0.5, 9)
    ps.psms_gauge_copy(ctx, 1, 0)
    ps.psms_gauge_sweep(ctx, 1, ps.ACTIVE_BLOCKS, 1, 1, 5.3, 3, 0)
    got = []
    for solver in (ps.SOLVER_CGNR, ps.SOLVER_BICGSTAB):
        ps.psms_full_solver(ctx, solver)
        got.append(ps.psms_logdet_ratio(ctx, ps.LEVEL_GLOBAL, 0, 1, 4, ps.EST_INTERP, 5, 0, 1e-13, ps.PREC_F32))
    assert np.abs(got[0] - got[1]).max() < 1e-8
    with pytest.raises(ps.PsmsError):
        ps.psms_full_solver(ctx, 7)


def test_solver_reports_non_convergence():
    dims, block = (4, 4, 4, 4), (2, 2, 2, 2)
    ctx = ps.psms_create(dims, block, 0.15, 1)
    ps.psms_gauge_init(ctx, 0, 0.3, 1)
    b = seeded.spinor(dims, 3)
    x = torch.zeros_like(native(ctx, b))
    with pytest.raises(ps.PsmsError) as e:
        ps.psms_solve(ctx, 0, ps.OP_FULL, native(ctx, b), x, 1e-13, 3, ps.PREC_F64)
    assert e.value.status == 4
    with pytest.raises(ps.PsmsError) as e:
        ps.psms_solve(ctx, 0, ps.OP_BLOCKS, native(ctx, b), x, 1e-13, 2, ps.PREC_F64)
    assert e.value.status == 4


_VARIANT_CASE = dict(dims=(8, 8, 8, 16), block=(8, 8, 8, 8), kappa=0.156)


@functools.lru_cache(maxsize=1)
def _variant_reference():
    """The oracle's solution on block 1 of the variant test (computed once)."""
    c = _VARIANT_CASE
    geom = lattice.Geometry(c["dims"], c["block"])
    U = gauge.generate_links(c["dims"], 0.5, 15)
    b = seeded.spinor(c["dims"], 16)
    ref = estimator.solve_blocks(U, b, geom, c["kappa"], [1], 1e-14)
    return geom, U, b, dirac.extract_block(ref, geom, 1)


@pytest.mark.parametrize("variant", range(18))
def test_block_solver_cluster_variants(variant):
    """Every (cluster size, register cap) variant of the block solver gives the
    oracle's solution (8^4 blocks: one block is shared by up to 8 CTAs of a
    thread-block cluster)."""
    c = _VARIANT_CASE
    geom, U, b, ref1 = _variant_reference()
    ctx = ps.psms_create(c["dims"], c["block"], c["kappa"], 1)
    ps.psms_gauge_init(ctx, 0, 0.5, 15)
    ps.psms_autotune(ctx, False, variant)
    for inner in (ps.PREC_F32, ps.PREC_F64):
        x = torch.zeros_like(native(ctx, b))
        ps.psms_solve(ctx, 0, ps.OP_BLOCKS, native(ctx, b), x, 1e-13, 20000, inner)
        got = canonical(ctx, x)
        r = b - dirac.apply_D(U, got, c["kappa"], geom, mode="block")
        assert np.sqrt(linalg.norm2(r) / linalg.norm2(b)) <= 1e-13
        assert rel_err(dirac.extract_block(got, geom, 1), ref1) < 1e-11


_SMEM_CASE = dict(dims=(8, 8, 8, 8), block=(4, 4, 4, 4), kappa=0.156)


@functools.lru_cache(maxsize=1)
def _smem_reference():
    """The oracle's block solutions on blocks 0 and 9 of the 4^4-block case."""
    c = _SMEM_CASE
    geom = lattice.Geometry(c["dims"], c["block"])
    U = gauge.generate_links(c["dims"], 0.5, 25)
    b = seeded.spinor(c["dims"], 26)
    ref = estimator.solve_blocks(U, b, geom, c["kappa"], [0, 9], 1e-14)
    return geom, U, b, {bb: dirac.extract_block(ref, geom, bb) for bb in (0, 9)}


@pytest.mark.parametrize("variant", [18, 19, 20])
def test_block_solver_shared_memory_link_variants(variant):
    """The variants that stage each block's FP32 links in shared memory once
    per solve (4^4 blocks) give the oracle's solution, alone and batched
    over several right-hand sides."""
    c = _SMEM_CASE
    geom, U, b, refs = _smem_reference()
    ctx = ps.psms_create(c["dims"], c["block"], c["kappa"], 1)
    ps.psms_gauge_init(ctx, 0, 0.5, 25)
    ps.psms_autotune(ctx, False, variant)
    x = torch.zeros_like(native(ctx, b))
    info = ps.psms_solve(ctx, 0, ps.OP_BLOCKS, native(ctx, b), x, 1e-13, 20000, ps.PREC_F32)
    got = canonical(ctx, x)
    r = b - dirac.apply_D(U, got, c["kappa"], geom, mode="block")
    assert np.sqrt(linalg.norm2(r) / linalg.norm2(b)) <= 1e-13
    for bb, ref in refs.items():
        assert rel_err(dirac.extract_block(got, geom, bb), ref) < 1e-11
    # batched over interpolation steps (the block level): the same estimates
    # as the default variant, to the solve tolerance
    c2 = ps.psms_create(c["dims"], c["block"], c["kappa"], 2)
    ps.psms_gauge_init(c2, 0, 0.5, 25)
    ps.psms_gauge_copy(c2, 1, 0)
    ps.psms_gauge_sweep(c2, 1, ps.ACTIVE_BLOCKS, 1, 1, 5.3, 3, 0)
    ps.psms_autotune(c2, False, 0)
    ref = ps.psms_logdet_ratio(c2, ps.LEVEL_BLOCK, 0, 1, 3, ps.EST_INTERP, 5, 0, 1e-13, ps.PREC_F32)
    ps.psms_autotune(c2, False, variant)
    got = ps.psms_logdet_ratio(c2, ps.LEVEL_BLOCK, 0, 1, 3, ps.EST_INTERP, 5, 0, 1e-13, ps.PREC_F32)
    assert np.abs(got - ref).max() < 1e-8


def test_profile_precision_filter_and_inner_reduction():
    """The hop profile counts only the launches of the storage precision
    asked for (FP32 inner iterations and FP64 true residuals add up to all
    launches), and a smaller inner reduction per defect-correction step
    reaches the same FP64 true residual in no more outer steps."""
    dims, block, kappa = (8, 8, 8, 8), (4, 4, 4, 4), 0.15
    ctx = ps.psms_create(dims, block, kappa, 1)
    ps.psms_gauge_init(ctx, 0, 0.3, 0x50534D53)
    b = native(ctx, seeded.spinor(dims, 2))
    ps.psms_solve(ctx, 0, ps.OP_FULL, b, torch.zeros_like(b), 1e-12, 20000, ps.PREC_F32)  # variants tuned
    counts = {}
    for mode in (1, 10 + ps.PREC_F32, 10 + ps.PREC_F64):
        ps.psms_profile_enable(ctx, mode)
        ps.psms_solve(ctx, 0, ps.OP_FULL, b, torch.zeros_like(b), 1e-12, 20000, ps.PREC_F32)
        counts[mode] = ps.psms_profile_read(ctx)
        ps.psms_profile_enable(ctx, 0)
    (n_all, _, by_all), (n32, _, by32), (n64, _, by64) = counts[1], counts[10 + ps.PREC_F32], counts[10 + ps.PREC_F64]
    assert n64 >= 1 and n32 > n64 and n32 + n64 == n_all
    assert by32 + by64 == pytest.approx(by_all, rel=1e-12)
    outer, xs = {}, {}
    for delta in (1e-4, 1e-6):
        ps.psms_inner_reduction(ctx, delta)
        x = torch.zeros_like(b)
        info = ps.psms_solve(ctx, 0, ps.OP_FULL, b, x, 1e-12, 20000, ps.PREC_F32)
        assert info["true_residual"] <= 1e-12
        outer[delta], xs[delta] = info["outer_iters"], canonical(ctx, x)
    assert outer[1e-6] < outer[1e-4]
    assert rel_err(xs[1e-6], xs[1e-4]) < 1e-10
    with pytest.raises(ps.PsmsError):
        ps.psms_inner_reduction(ctx, 0.9)
    ps.psms_inner_reduction(ctx, 0.0)
