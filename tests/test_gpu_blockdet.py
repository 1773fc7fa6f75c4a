"""GPU parity of the exact block determinants (Sec. 3: LU of the small
blocks; Tables 1-2 put coefficients on this exact action): ln|det D_b| by
the device's batched FP64 LU of the even-odd reduced block operator against
the oracle's dense LU of the full block operator (relative 1e-10), and
filter steps with the exact block level and the global-level coefficient of
its action (identical decisions, Delta within 1e-8, links within 1e-12)."""
import numpy as np
import pytest

import paper_1204_1306_gb300 as ps
from oracle import filter as ofilter, gauge, lattice
from tests.gpu_util import get_links, set_links

pytestmark = pytest.mark.gpu

SEED = 0x50534D53
# Table 1 (Sec. 5): the block-determinant action's coefficients at the
# block level (1.644) and at the global level (-0.644)
TABLE1_DET = dict(exact_block=True, block_det_coef=1.644, beta_global_blockdet=-0.644)


def _ctx(dims, block, kappa, eps, seed, sweep=True):
    ctx = ps.psms_create(dims, block, kappa, 2)
    ps.psms_gauge_init(ctx, 0, eps, seed)
    if sweep:
        ps.psms_gauge_sweep(ctx, 0, ps.ACTIVE_ALL, 1, 1, 5.3, SEED, 1 << 40)
    return ctx


def test_block_logdet_parity_2x4_blocks():
    dims, block, kappa = (4, 4, 4, 8), (2, 2, 2, 2), 0.15
    geom = lattice.Geometry(dims, block)
    ctx = _ctx(dims, block, kappa, 0.5, 31)
    U = get_links(ctx, 0)
    got = ps.psms_block_logdet(ctx, 0)
    ref = np.array([ofilter.block_logdet(U, geom, b, kappa) for b in range(geom.n_blocks)])
    assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max()


@pytest.mark.parametrize("chunk", [0, 3])
def test_block_logdet_parity_4x4_blocks(chunk):
    """4^4 blocks (1536-dim reduced operators), a sample of blocks against
    the oracle's 3072-dim dense LU; chunk 3 factorises the 16 blocks in
    batches of 3 (ragged last batch)."""
    dims, block, kappa = (8, 8, 8, 8), (4, 4, 4, 4), 0.156
    geom = lattice.Geometry(dims, block)
    ctx = _ctx(dims, block, kappa, 0.5, 32)
    ps.psms_max_chunk(ctx, chunk)
    U = get_links(ctx, 0)
    got = ps.psms_block_logdet(ctx, 0)
    sample = [0, 7, 15] if chunk else [3, 12]
    ref = np.array([ofilter.block_logdet(U, geom, b, kappa) for b in sample])
    assert np.abs(got[sample] - ref).max() <= 1e-10 * np.abs(ref).max()
    # every block's determinant differs (the field is rough)
    assert len(np.unique(np.round(got, 6))) == geom.n_blocks


def test_filter_step_exact_block_sum_decision():
    """4^4 lattice, 2^4 blocks: exact block level with Table 1's coefficient
    structure (one decision on the sum), global level with the block action's
    coefficient; three chained steps."""
    dims, block, kappa = (4, 4, 4, 4), (2, 2, 2, 2), 0.15
    geom = lattice.Geometry(dims, block)
    ctx = ps.psms_create(dims, block, kappa, 1)
    ps.psms_gauge_init(ctx, 0, 0.3, SEED)
    U = get_links(ctx, 0)
    prm = ofilter.FilterParams(kappa=kappa, beta0=5.3, n_iter=1, n_or=0, n_block=2, n_global=2, tol=1e-13,
                               exact_block=True, block_det_coef=1.644, beta_global_blockdet=-0.644)
    for step in range(3):
        r = ps.psms_filter_step(ctx, 0, beta0=5.3, n_iter=1, n_or=0, n_block=2, n_global=2, tol=1e-13,
                                inner_prec=ps.PREC_F64, seed=SEED, step=step, exact_block=True, beta_block_det=1.644,
                                beta_global_blockdet=-0.644)
        U, rec = ofilter.filter_step(U, geom, prm, SEED, step)
        assert np.array_equal(r["accept_block"], rec["accept_block"])
        assert abs(r["delta_block_sum"] - rec["delta_block"].sum()) < 1e-8
        assert r["accept_global"] == rec["accept_global"]
        if r["n_accept_blocks"] > 0:
            assert abs(r["delta_global"] - rec["delta_global"]) < 1e-8
        assert np.abs(get_links(ctx, 0) - U).max() < 1e-12


def test_filter_step_exact_block_per_block_decisions():
    """8^4 lattice, 4^4 blocks (per-block decisions): an external proposal
    moves the active links of three blocks; the others keep their
    determinants (Delta_b = 0 exactly on both sides)."""
    dims, block, kappa = (8, 8, 8, 8), (4, 4, 4, 4), 0.156
    geom = lattice.Geometry(dims, block)
    ctx = _ctx(dims, block, kappa, 0.5, 33)
    U = get_links(ctx, 0)
    ps.psms_gauge_copy(ctx, 1, 0)
    ps.psms_gauge_sweep(ctx, 1, ps.ACTIVE_BLOCKS, 1, 1, 5.3, SEED, 5)
    Usw = get_links(ctx, 1)
    moved = [1, 6, 11]
    sel = np.isin(geom.block_index, moved)[..., None] & geom.active_links()
    prop = U.copy()
    prop[sel] = Usw[sel]
    set_links(ctx, 1, prop)
    step = 9
    kw = dict(exact_block=True, beta_block_det=1.0, beta_global_blockdet=0.0, beta_block=0.2)
    r = ps.psms_filter_step(ctx, 0, beta0=5.3, n_block=1, n_global=1, tol=1e-13, inner_prec=ps.PREC_F32,
                            seed=SEED, step=step, proposal_field=1, **kw)
    prm = ofilter.FilterParams(kappa=kappa, beta0=5.3, n_block=1, n_global=1, tol=1e-13, exact_block=True,
                               beta_block=0.2)
    U2, rec = ofilter.filter_step(U, geom, prm, SEED, step, proposal=prop)
    assert np.abs(r["delta_block"] - rec["delta_block"]).max() < 1e-8
    still = np.setdiff1d(np.arange(geom.n_blocks), moved)
    assert np.all(r["delta_block"][still] == 0.0)
    assert np.array_equal(r["accept_block"], rec["accept_block"])
    assert r["accept_global"] == rec["accept_global"]
    if r["n_accept_blocks"] > 0:
        assert abs(r["delta_global"] - rec["delta_global"]) < 1e-8
    assert np.abs(get_links(ctx, 0) - U2).max() < 1e-12
