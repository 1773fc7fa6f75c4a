"""GPU parity of the parametrised levels (App. C; Sec. 5; Tables 1-2) with the
FP64 oracle: one level of HYP smearing (fat links within 1e-12), the block
HYP plaquette action and the per-block plaquette-action change (within
1e-11), and filter steps with the HYP level and the App. C beta terms of the
block and global levels (identical decisions, Delta within 1e-8, links
within 1e-12)."""
import numpy as np
import pytest
import torch

import paper_1204_1306_gb300 as ps
from oracle import filter as ofilter, gauge, hyp, lattice
from tests.gpu_util import from_dev, get_links, set_links

pytestmark = pytest.mark.gpu

SEED = 0x50534D53
# Table 1 (Sec. 5): level 1 (HYP level) and the plaquette / HYP coefficients
# of the block (level 2) and global (level 3) filters
TABLE1 = dict(hyp_level=(-0.0196, 0.0963), beta_block=-0.1187, beta_block_hyp=-0.0614, beta_global=0.0465,
              beta_global_hyp=-0.0349)


def _smeared(ctx, field, alpha=None):
    out = torch.empty(ctx.V * 4 * 9 * 2, dtype=torch.float64, device="cuda")
    ps.psms_hyp_smear(ctx, field, out, alpha)
    torch.cuda.synchronize()
    return from_dev(out, ctx.dims + (4, 3, 3))


@pytest.mark.parametrize("dims,block,alpha", [((4, 4, 4, 8), (2, 2, 2, 4), None),
                                              ((8, 8, 8, 8), (4, 4, 4, 4), None),
                                              ((8, 4, 4, 4), (4, 2, 2, 2), (0.5, 0.4, 0.2))])
def test_hyp_smear_parity(dims, block, alpha):
    ctx = ps.psms_create(dims, block, 0.15, 1)
    ps.psms_gauge_init(ctx, 0, 0.5, 21)
    got = _smeared(ctx, 0, alpha)
    ref = hyp.smear(gauge.generate_links(dims, 0.5, 21), hyp.ALPHA if alpha is None else alpha)
    assert np.abs(got - ref).max() < 1e-12
    # SU(3) output
    eye = np.eye(3)
    assert np.abs(got @ np.conj(np.swapaxes(got, -1, -2)) - eye).max() < 1e-12


@pytest.mark.parametrize("dims,block", [((8, 8, 8, 8), (4, 4, 4, 4)), ((4, 4, 4, 4), (2, 2, 2, 2)),
                                        ((8, 8, 8, 4), (4, 4, 4, 4))])
def test_hyp_block_action_parity(dims, block):
    geom = lattice.Geometry(dims, block)
    ctx = ps.psms_create(dims, block, 0.15, 1)
    ps.psms_gauge_init(ctx, 0, 0.5, 22)
    ps.psms_gauge_sweep(ctx, 0, ps.ACTIVE_ALL, 1, 1, 5.3, SEED, 1 << 40)
    U = get_links(ctx, 0)
    got = ps.psms_hyp_block_action(ctx, 0)
    ref = hyp.block_hyp_action(U, geom)
    assert np.abs(got - ref).max() < 1e-11


@pytest.mark.parametrize("dims,block,active", [((8, 8, 8, 8), (4, 4, 4, 4), ps.ACTIVE_BLOCKS),
                                               ((4, 4, 4, 4), (2, 2, 2, 2), ps.ACTIVE_BLOCKS),
                                               ((8, 8, 8, 8), (4, 4, 4, 4), ps.ACTIVE_ALL),
                                               ((8, 8, 8, 4), (4, 4, 4, 4), ps.ACTIVE_BLOCKS)])
def test_block_action_change_parity(dims, block, active):
    """dS_w,b by plaquette attribution: proposals on the active links, on
    every link (plaquettes shared by blocks), and with one block spanning a
    direction; the block sums add up to dS_w."""
    geom = lattice.Geometry(dims, block)
    ctx = ps.psms_create(dims, block, 0.15, 2)
    ps.psms_gauge_init(ctx, 0, 0.5, 23)
    ps.psms_gauge_copy(ctx, 1, 0)
    ps.psms_gauge_sweep(ctx, 1, active, 1, 1, 5.3, SEED, 7)
    U, Up = get_links(ctx, 0), get_links(ctx, 1)
    got = ps.psms_block_action_change(ctx, 0, 1)
    ref = ofilter.per_block_action_change(U, Up, geom)
    assert np.abs(got - ref).max() < 1e-11
    assert abs(got.sum() - (gauge.wilson_action(Up) - gauge.wilson_action(U))) < 1e-9


def _thermalised_ctx(dims, block, kappa, seed):
    ctx = ps.psms_create(dims, block, kappa, 2)
    ps.psms_gauge_init(ctx, 0, 0.5, seed)
    ps.psms_gauge_sweep(ctx, 0, ps.ACTIVE_ALL, 3, 2, 5.3, SEED, 1 << 40)
    return ctx, get_links(ctx, 0)


@pytest.mark.parametrize("coefs", [TABLE1, dict(TABLE1, hyp_level=(1.0, 1.0))], ids=["table1", "strong"])
def test_filter_step_hyp_level_parity(coefs):
    """8^4 lattice, 4^4 blocks: HYP level (per-block decisions, counter
    (step, 5, b)), block level with beta_block dS_w,b + beta_block_hyp
    dS_HYP,b, global level with beta_global dS_w + beta_global_hyp dS_HYP."""
    dims, block, kappa = (8, 8, 8, 8), (4, 4, 4, 4), 0.156
    geom = lattice.Geometry(dims, block)
    ctx, U = _thermalised_ctx(dims, block, kappa, SEED + 5)
    step = 13
    r = ps.psms_filter_step(ctx, 0, beta0=5.3, n_iter=1, n_or=1, n_block=2, n_global=1, tol=1e-13,
                            inner_prec=ps.PREC_F32, seed=SEED, step=step, **coefs)
    prm = ofilter.FilterParams(kappa=kappa, beta0=5.3, n_iter=1, n_or=1, n_block=2, n_global=1, tol=1e-13, **coefs)
    U2, rec = ofilter.filter_step(U, geom, prm, SEED, step)
    assert r["n_accept_hyp"] == int(rec["accept_hyp"].sum())
    assert np.abs(ps.psms_filter_record(ctx, ps.REC_DELTA_HYP) - rec["delta_hyp"]).max() < 1e-10
    assert np.array_equal(r["accept_block"], rec["accept_block"])
    passed = rec["accept_hyp"]
    if passed.any():
        assert np.abs(r["delta_block"][passed] - rec["delta_block"][passed]).max() < 1e-8
    assert r["accept_global"] == rec["accept_global"]
    if "delta_global" in rec and r["n_accept_blocks"] > 0:
        assert abs(r["delta_global"] - rec["delta_global"]) < 1e-8
    assert tuple(r["shift"]) == tuple(rec["shift"])
    assert np.abs(get_links(ctx, 0) - U2).max() < 1e-12
    if coefs is not TABLE1:
        assert 0 < r["n_accept_hyp"] < geom.n_blocks


def test_filter_step_hyp_level_sum_decision():
    """4^4 lattice, 2^4 blocks: the HYP level and the block level take one
    decision on the sum (counters (step, 5, 0) and (step, 1, 0))."""
    dims, block, kappa = (4, 4, 4, 4), (2, 2, 2, 2), 0.15
    geom = lattice.Geometry(dims, block)
    ctx = ps.psms_create(dims, block, kappa, 1)
    ps.psms_gauge_init(ctx, 0, 0.3, SEED)
    U = get_links(ctx, 0)
    prm = ofilter.FilterParams(kappa=kappa, beta0=5.3, n_iter=1, n_or=0, n_block=2, n_global=2, tol=1e-13,
                               **TABLE1)
    for step in range(3):
        r = ps.psms_filter_step(ctx, 0, beta0=5.3, n_iter=1, n_or=0, n_block=2, n_global=2, tol=1e-13,
                                inner_prec=ps.PREC_F64, seed=SEED, step=step, **TABLE1)
        U, rec = ofilter.filter_step(U, geom, prm, SEED, step)
        assert r["n_accept_hyp"] == int(rec["accept_hyp"].sum())
        assert np.array_equal(r["accept_block"], rec["accept_block"])
        assert r["accept_global"] == rec["accept_global"]
        if "delta_global" in rec and r["n_accept_blocks"] > 0:
            assert abs(r["delta_global"] - rec["delta_global"]) < 1e-8
        assert np.abs(get_links(ctx, 0) - U).max() < 1e-12


def test_filter_step_beta_block_only_parity():
    """beta_block != 0 without the HYP level (the App. C plaquette term of the
    block level alone)."""
    dims, block, kappa = (8, 8, 8, 8), (4, 4, 4, 4), 0.156
    geom = lattice.Geometry(dims, block)
    ctx, U = _thermalised_ctx(dims, block, kappa, SEED + 6)
    step = 4
    kw = dict(beta_block=0.35, beta_global=-0.2)
    r = ps.psms_filter_step(ctx, 0, beta0=5.3, n_iter=1, n_or=1, n_block=2, n_global=1, tol=1e-13,
                            inner_prec=ps.PREC_F32, seed=SEED, step=step, **kw)
    prm = ofilter.FilterParams(kappa=kappa, beta0=5.3, n_iter=1, n_or=1, n_block=2, n_global=1, tol=1e-13, **kw)
    U2, rec = ofilter.filter_step(U, geom, prm, SEED, step)
    assert np.array_equal(r["accept_block"], rec["accept_block"])
    assert np.abs(r["delta_block"] - rec["delta_block"]).max() < 1e-8
    assert r["accept_global"] == rec["accept_global"]
    assert np.abs(get_links(ctx, 0) - U2).max() < 1e-12
