"""GPU parity of the stochastic determinant-ratio estimates, the domain
sweep and the filter step with the oracle, on identical Philox draws.
Estimates: within 1e-8 absolute with both sides solved to 1e-13; heatbath
links within 1e-12; identical accept/reject decisions."""
import numpy as np
import pytest
import torch

import paper_1204_1306_gb300 as ps
from oracle import estimator, filter as ofilter, gauge, lattice
from tests.gpu_util import get_links, set_links

pytestmark = pytest.mark.gpu

SEED = 0x50534D53


def _pair(dims, block, kappa, eps, seed, sweep_beta=5.3):
    """U from the link generator and U' = one domain sweep of U (both sides)."""
    geom = lattice.Geometry(dims, block)
    ctx = ps.psms_create(dims, block, kappa, 2)
    ps.psms_gauge_init(ctx, 0, eps, seed)
    ps.psms_gauge_copy(ctx, 1, 0)
    ps.psms_gauge_sweep(ctx, 1, ps.ACTIVE_BLOCKS, 1, 0, sweep_beta, seed, 0)
    U = gauge.generate_links(dims, eps, seed)
    Up, _, _ = gauge.domain_sweep(U, geom, sweep_beta, 1, 0, seed, 0)
    return ctx, geom, U, Up


@pytest.mark.parametrize("dims,block,n_or", [((4, 4, 4, 4), (2, 2, 2, 2), 0), ((8, 8, 8, 8), (4, 4, 4, 4), 1),
                                             ((8, 4, 8, 4), (4, 4, 4, 4), 2)])
def test_domain_sweep_parity(dims, block, n_or):
    geom = lattice.Geometry(dims, block)
    ctx = ps.psms_create(dims, block, 0.15, 1)
    ps.psms_gauge_init(ctx, 0, 0.5, 9)
    failed = ps.psms_gauge_sweep(ctx, 0, ps.ACTIVE_BLOCKS, 1, n_or, 5.3, 77, 40)
    got = get_links(ctx, 0)
    U = gauge.generate_links(dims, 0.5, 9)
    ref, _, f = gauge.domain_sweep(U, geom, 5.3, 1, n_or, 77, 40)
    assert failed == f == 0
    assert np.abs(got - ref).max() < 1e-12


def test_all_link_sweep_parity():
    dims, block = (4, 4, 4, 8), (2, 2, 2, 2)
    geom = lattice.Geometry(dims, block)
    ctx = ps.psms_create(dims, block, 0.15, 1)
    ps.psms_gauge_init(ctx, 0, 0.3, 19)
    ps.psms_gauge_sweep(ctx, 0, ps.ACTIVE_ALL, 2, 1, 5.3, 5, 0)
    U = gauge.generate_links(dims, 0.3, 19)
    subsets = [(mu, geom.parity == p) for mu in range(4) for p in (0, 1)]
    s = 0
    for _ in range(2):
        gauge.one_sweep(U, geom, subsets, 5.3, "hb", 5, s)
        gauge.one_sweep(U, geom, subsets, 5.3, "or", 5, s + 1)
        gauge.one_sweep(U, geom, subsets[::-1], 5.3, "or", 5, s + 2)
        gauge.one_sweep(U, geom, subsets[::-1], 5.3, "hb", 5, s + 3)
        s += 4
    U = gauge.reunitarise(U)
    assert np.abs(get_links(ctx, 0) - U).max() < 1e-12


@pytest.mark.parametrize("mode", [ps.EST_INTERP, ps.EST_INDEPENDENT])
@pytest.mark.parametrize("inner", [ps.PREC_F64, ps.PREC_F32])
def test_block_level_parity(mode, inner):
    dims, block, kappa = (4, 4, 4, 4), (2, 2, 2, 2), 0.15
    ctx, geom, U, Up = _pair(dims, block, kappa, 0.3, SEED)
    N = 4
    got = ps.psms_logdet_ratio(ctx, ps.LEVEL_BLOCK, 0, 1, N, mode, SEED, 3, 1e-13, inner)
    ref = estimator.block_level(U, Up, geom, kappa, N, SEED, 3, tol=1e-13,
                                mode="interp" if mode == ps.EST_INTERP else "independent")
    assert np.abs(got - ref).max() < 1e-8


def test_block_level_parity_4x4_blocks():
    dims, block, kappa = (8, 8, 8, 8), (4, 4, 4, 4), 0.156
    ctx, geom, U, Up = _pair(dims, block, kappa, 0.5, SEED + 1)
    N = 3
    got = ps.psms_logdet_ratio(ctx, ps.LEVEL_BLOCK, 0, 1, N, ps.EST_INTERP, SEED, 5, 1e-13, ps.PREC_F32)
    blocks = [0, 5, 10, 15]
    ref = estimator.block_level(U, Up, geom, kappa, N, SEED, 5, tol=1e-13, blocks=blocks)
    assert np.abs(got[blocks] - ref[blocks]).max() < 1e-8
    # blocks without active-link changes have Delta = 0 up to rounding: none here
    assert np.all(np.abs(got) > 0)


def test_block_level_parity_16x4_sampled():
    """The 16^4 workload's block level (256 blocks of 4^4, batched with the
    batch split into chunks of two interpolation steps): three sampled
    blocks against the oracle."""
    dims, block, kappa = (16, 16, 16, 16), (4, 4, 4, 4), 0.156
    ctx, geom, U, Up = _pair(dims, block, kappa, 0.5, SEED + 9)
    N = 3
    ps.psms_max_chunk(ctx, 2)
    got = ps.psms_logdet_ratio(ctx, ps.LEVEL_BLOCK, 0, 1, N, ps.EST_INTERP, SEED, 8, 1e-13, ps.PREC_F32)
    blocks = [0, 117, 255]
    ref = estimator.block_level(U, Up, geom, kappa, N, SEED, 8, tol=1e-13, blocks=blocks)
    assert np.abs(got[blocks] - ref[blocks]).max() < 1e-8


@pytest.mark.parametrize("inner", [ps.PREC_F64, ps.PREC_F32])
def test_global_level_parity(inner):
    dims, block, kappa = (4, 4, 4, 4), (2, 2, 2, 2), 0.15
    ctx, geom, U, Up = _pair(dims, block, kappa, 0.3, SEED)
    N = 2
    got = ps.psms_logdet_ratio(ctx, ps.LEVEL_GLOBAL, 0, 1, N, ps.EST_INTERP, SEED, 4, 1e-13, inner)
    ref = estimator.global_level(U, Up, geom, kappa, N, SEED, 4, tol=1e-13)
    assert np.abs(got - ref).max() < 1e-8


def test_global_level_parity_with_projector():
    """8^4 lattice with 4^4 blocks: rank-2 spin projectors on one-face sites."""
    dims, block, kappa = (8, 8, 8, 8), (4, 4, 4, 4), 0.156
    ctx, geom, U, Up = _pair(dims, block, kappa, 0.5, SEED + 2)
    got = ps.psms_logdet_ratio(ctx, ps.LEVEL_GLOBAL, 0, 1, 1, ps.EST_INTERP, SEED, 6, 1e-13, ps.PREC_F32)
    ref = estimator.global_level(U, Up, geom, kappa, 1, SEED, 6, tol=1e-13)
    assert np.abs(got - ref).max() < 1e-8


def test_filter_step_parity_4x4_2x4_blocks():
    """4^4 lattice, 2^4 blocks, kappa 0.15, eps 0.3, beta 5.3, N = 4 (3 steps):
    identical decisions, estimates within 1e-8, identical links."""
    dims, block, kappa = (4, 4, 4, 4), (2, 2, 2, 2), 0.15
    geom = lattice.Geometry(dims, block)
    ctx = ps.psms_create(dims, block, kappa, 1)
    ps.psms_gauge_init(ctx, 0, 0.3, SEED)
    U = gauge.generate_links(dims, 0.3, SEED)
    prm = ofilter.FilterParams(kappa=kappa, beta0=5.3, n_iter=1, n_or=0, n_block=4, n_global=4, tol=1e-13)
    for step in range(3):
        r = ps.psms_filter_step(ctx, 0, beta0=5.3, n_iter=1, n_or=0, n_block=4, n_global=4, tol=1e-13,
                                inner_prec=ps.PREC_F64, seed=SEED, step=step)
        U, rec = ofilter.filter_step(U, geom, prm, SEED, step)
        assert r["accept_global"] == rec["accept_global"]
        assert np.array_equal(r["accept_block"], rec["accept_block"])
        assert abs(r["delta_global"] - rec["delta_global"]) < 1e-8
        assert abs(r["delta_block_sum"] - rec["delta_block"].sum()) < 1e-8
        assert tuple(r["shift"]) == tuple(rec["shift"])
        assert np.abs(get_links(ctx, 0) - U).max() < 1e-12


def test_filter_step_parity_per_block_decisions():
    """8^4 lattice with 4^4 blocks: per-block decisions (active links of
    different blocks share no plaquette)."""
    dims, block, kappa = (8, 8, 8, 8), (4, 4, 4, 4), 0.156
    geom = lattice.Geometry(dims, block)
    ctx = ps.psms_create(dims, block, kappa, 1)
    ps.psms_gauge_init(ctx, 0, 0.5, SEED + 3)
    # thermalise all links first so that some blocks accept
    ps.psms_gauge_sweep(ctx, 0, ps.ACTIVE_ALL, 3, 2, 5.3, SEED, 1 << 40)
    U = get_links(ctx, 0)
    prm = ofilter.FilterParams(kappa=kappa, beta0=5.3, n_iter=1, n_or=1, n_block=2, n_global=1, tol=1e-13)
    r = ps.psms_filter_step(ctx, 0, beta0=5.3, n_iter=1, n_or=1, n_block=2, n_global=1, tol=1e-13,
                            inner_prec=ps.PREC_F32, seed=SEED, step=7)
    U, rec = ofilter.filter_step(U, geom, prm, SEED, 7)
    assert np.array_equal(r["accept_block"], rec["accept_block"])
    assert np.abs(r["delta_block"] - rec["delta_block"]).max() < 1e-8
    assert r["accept_global"] == rec["accept_global"]
    assert abs(r["delta_global"] - rec["delta_global"]) < 1e-8
    assert np.abs(get_links(ctx, 0) - U).max() < 1e-12
