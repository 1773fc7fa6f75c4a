"""GPU parity of the recursive domain decomposition (Eq. (ddrec), Eq. (4step);
the 5-step filter of Sec. 5) with oracle/recursive.py on identical Philox
draws: the stage-2 estimates of the outer blocks' Schur complements, the
global level of the outer decomposition, and filter steps with one level of
recursion (identical decisions, Delta within 1e-8, links within 1e-12)."""
import numpy as np
import pytest
import torch

import paper_1204_1306_gb300 as ps
from oracle import estimator, gauge, lattice, recursive
from tests.gpu_util import get_links, set_links

pytestmark = pytest.mark.gpu

SEED = 0x50534D53
# 8^4 lattice, 4^4 outer blocks of 2^4 inner blocks (16 outer, 256 inner)
DIMS, OUTER, INNER, KAPPA = (8, 8, 8, 8), (4, 4, 4, 4), (2, 2, 2, 2), 0.156


def _pair(dims, outer, inner, kappa, seed, n_or=1):
    """U (thermalised on every link) and U' = one domain sweep of U on the
    inner blocks' active links; both sides get the same fields."""
    ctx = ps.psms_create(dims, inner, kappa, 3)
    ps.psms_set_outer_blocks(ctx, outer)
    ps.psms_gauge_init(ctx, 0, 0.5, seed)
    ps.psms_gauge_sweep(ctx, 0, ps.ACTIVE_ALL, 2, 1, 5.3, SEED, 1 << 40)
    ps.psms_gauge_copy(ctx, 1, 0)
    ps.psms_gauge_sweep(ctx, 1, ps.ACTIVE_BLOCKS, 1, n_or, 5.3, seed, 3)
    return ctx, get_links(ctx, 0), get_links(ctx, 1)


@pytest.mark.parametrize("mode,inner", [(ps.EST_INTERP, ps.PREC_F64), (ps.EST_INTERP, ps.PREC_F32),
                                        (ps.EST_INDEPENDENT, ps.PREC_F32)])
def test_sub_level_parity(mode, inner):
    """Stage 2: Delta_b of every outer block (projector P_b on the inner-block
    faces inside b, noise stream level 4)."""
    nest = recursive.Nested(DIMS, OUTER, INNER)
    ctx, U, Up = _pair(DIMS, OUTER, INNER, KAPPA, SEED + 11)
    N = 2
    got = ps.psms_logdet_ratio(ctx, ps.LEVEL_SUB, 0, 1, N, mode, SEED, 3, 1e-13, inner)
    ref = recursive.sub_level(U, Up, nest, KAPPA, N, SEED, 3, tol=1e-13,
                              mode="interp" if mode == ps.EST_INTERP else "independent")
    assert got.shape == ref.shape == (nest.outer.n_blocks, N)
    assert np.abs(got - ref).max() < 1e-8
    assert np.all(np.abs(got) > 1e-6)   # every outer block changed


@pytest.mark.parametrize("inner,shared", [(ps.PREC_F32, 1), (ps.PREC_F32, 0)])
def test_outer_global_level_parity(inner, shared):
    """Global Schur complement of the outer decomposition = the oracle's
    global level with the outer blocks as blocks (FP32 inner iterations on
    shared-endpoint or materialised FP32 links)."""
    nest = recursive.Nested(DIMS, OUTER, INNER)
    ctx, U, Up = _pair(DIMS, OUTER, INNER, KAPPA, SEED + 12)
    ps.psms_shared_links(ctx, shared)
    N = 2
    got = ps.psms_logdet_ratio(ctx, ps.LEVEL_OUTER_GLOBAL, 0, 1, N, ps.EST_INTERP, SEED, 4, 1e-13, inner)
    ref = estimator.global_level(U, Up, nest.outer, KAPPA, N, SEED, 4, tol=1e-13)
    assert np.abs(got - ref).max() < 1e-8


def test_outer_global_level_every_shared_link_hop_variant():
    """Every form of the shared-endpoint-link hop (register caps, branch-free
    or general, flagged or unconditional endpoint reads), forced one by one,
    gives the oracle's global level of the outer decomposition."""
    nest = recursive.Nested(DIMS, OUTER, INNER)
    ctx, U, Up = _pair(DIMS, OUTER, INNER, KAPPA, SEED + 15)
    ref = estimator.global_level(U, Up, nest.outer, KAPPA, 2, SEED, 8, tol=1e-12)
    n = ps.psms_hop_variant(ctx, 0)
    for v in range(n):
        ps.psms_hop_variant(ctx, v)
        got = ps.psms_logdet_ratio(ctx, ps.LEVEL_OUTER_GLOBAL, 0, 1, 2, ps.EST_INTERP, SEED, 8, 1e-12, ps.PREC_F32)
        assert np.abs(got - ref).max() < 1e-8, v
    ps.psms_hop_variant(ctx, -1)


def test_global_level_ignores_outer_blocks():
    """PSMS_LEVEL_GLOBAL is the Schur complement of the context's blocks
    whether or not outer blocks are set."""
    nest = recursive.Nested(DIMS, OUTER, INNER)
    ctx, U, Up = _pair(DIMS, OUTER, INNER, KAPPA, SEED + 13)
    got = ps.psms_logdet_ratio(ctx, ps.LEVEL_GLOBAL, 0, 1, 1, ps.EST_INTERP, SEED, 5, 1e-13, ps.PREC_F32)
    ref = estimator.global_level(U, Up, nest.inner, KAPPA, 1, SEED, 5, tol=1e-13)
    assert np.abs(got - ref).max() < 1e-8


def test_sub_level_chunked_parity():
    """Interpolation steps split over several launches (chunk offsets i0 > 0)
    give the same stage-2 and outer-global estimates."""
    nest = recursive.Nested(DIMS, OUTER, INNER)
    ctx, U, Up = _pair(DIMS, OUTER, INNER, KAPPA, SEED + 14)
    N = 3
    ps.psms_max_chunk(ctx, 2)
    got = ps.psms_logdet_ratio(ctx, ps.LEVEL_SUB, 0, 1, N, ps.EST_INTERP, SEED, 6, 1e-13, ps.PREC_F32)
    ref = recursive.sub_level(U, Up, nest, KAPPA, N, SEED, 6, tol=1e-13, blocks=[0, 15])
    assert np.abs(got[[0, 15]] - ref[[0, 15]]).max() < 1e-8
    ps.psms_max_chunk(ctx, 1)
    got = ps.psms_logdet_ratio(ctx, ps.LEVEL_OUTER_GLOBAL, 0, 1, 2, ps.EST_INTERP, SEED, 7, 1e-13, ps.PREC_F32)
    ref = estimator.global_level(U, Up, nest.outer, KAPPA, 2, SEED, 7, tol=1e-13)
    assert np.abs(got - ref).max() < 1e-8


@pytest.mark.parametrize("coefs,steps", [(dict(), 2), (dict(beta_block=0.3, beta_sub=-0.4, beta_global=0.2), 1)],
                         ids=["plain", "beta"])
def test_filter_step_recursive_parity(coefs, steps):
    """8^4 lattice, 4^4 outer / 2^4 inner blocks: chained 5-step filter steps
    (domain sweep, inner blocks, outer-block Schur complements, global
    Schur complement of the outer blocks, translation); one decision on the
    sum at stages 1 and 2 (inner extent 2)."""
    nest = recursive.Nested(DIMS, OUTER, INNER)
    ctx = ps.psms_create(DIMS, INNER, KAPPA, 1)
    ps.psms_set_outer_blocks(ctx, OUTER)
    ps.psms_gauge_init(ctx, 0, 0.5, SEED + 15)
    ps.psms_gauge_sweep(ctx, 0, ps.ACTIVE_ALL, 2, 1, 5.3, SEED, 1 << 40)
    U = get_links(ctx, 0)
    prm = recursive.RecursiveParams(kappa=KAPPA, beta0=5.3, n_iter=1, n_or=1, n_block=1, n_sub=2, n_global=1,
                                    tol=1e-13, **coefs)
    for step in range(steps):
        r = ps.psms_filter_step(ctx, 0, beta0=5.3, n_iter=1, n_or=1, n_block=1, n_sub=2, n_global=1, tol=1e-13,
                                inner_prec=ps.PREC_F32, seed=SEED, step=step, **coefs)
        U, rec = recursive.filter_step(U, nest, prm, SEED, step)
        assert np.array_equal(ps.psms_filter_record(ctx, ps.REC_ACCEPT_BLOCK).astype(bool), rec["accept_block"])
        assert abs(r["delta_block_sum"] - rec["delta_block"].sum()) < 1e-8
        if rec["changed_sub"].any():
            assert np.abs(ps.psms_filter_record(ctx, ps.REC_DELTA_SUB) - rec["delta_sub"]).max() < 1e-8
            assert np.array_equal(ps.psms_filter_record(ctx, ps.REC_ACCEPT_SUB).astype(bool), rec["accept_sub"])
        assert np.array_equal(r["accept_block"], rec["accept_after_sub"])
        assert r["accept_global"] == rec["accept_global"]
        if r["n_accept_blocks"] > 0:
            assert abs(r["delta_global"] - rec["delta_global"]) < 1e-8
        assert tuple(r["shift"]) == tuple(rec["shift"])
        assert np.abs(get_links(ctx, 0) - U).max() < 1e-12


def test_filter_step_recursive_per_outer_block_decisions():
    """16^4 lattice, 8^4 outer blocks of 4^4 inner blocks (Sec. 5's nesting):
    per-inner-block decisions at stage 1 and per-outer-block decisions at
    stage 2 (counter (step, 4, b)).  An external proposal moves the active
    links of three inner blocks, two in outer block 0 and one in outer block
    9, so that the oracle estimates only those; the global level is off."""
    dims, outer, inner = (16, 16, 16, 16), (8, 8, 8, 8), (4, 4, 4, 4)
    nest = recursive.Nested(dims, outer, inner)
    ctx = ps.psms_create(dims, inner, KAPPA, 2)
    ps.psms_set_outer_blocks(ctx, outer)
    ps.psms_gauge_init(ctx, 0, 0.5, SEED + 16)
    ps.psms_gauge_sweep(ctx, 0, ps.ACTIVE_ALL, 2, 1, 5.3, SEED, 1 << 40)
    U = get_links(ctx, 0)
    ps.psms_gauge_copy(ctx, 1, 0)
    ps.psms_gauge_sweep(ctx, 1, ps.ACTIVE_BLOCKS, 1, 1, 5.3, SEED, 99)
    Usw = get_links(ctx, 1)
    geo = nest.inner
    moved = [b for b in range(geo.n_blocks) if nest.outer_of_inner[b] == 0][:2]
    moved += [b for b in range(geo.n_blocks) if nest.outer_of_inner[b] == 9][:1]
    sel = np.isin(geo.block_index, moved)[..., None] & geo.active_links()
    prop = U.copy()
    prop[sel] = Usw[sel]
    set_links(ctx, 1, prop)
    step = 21
    r = ps.psms_filter_step(ctx, 0, beta0=5.3, n_block=1, n_sub=1, n_global=1, global_level=False, tol=1e-13,
                            inner_prec=ps.PREC_F32, seed=SEED, step=step, proposal_field=1)
    prm = recursive.RecursiveParams(kappa=KAPPA, beta0=5.3, n_block=1, n_sub=1, n_global=1, tol=1e-13,
                                    global_level=False)
    U2, rec = recursive.filter_step(U, nest, prm, SEED, step, proposal=prop, skip_unchanged=True)
    acc1 = ps.psms_filter_record(ctx, ps.REC_ACCEPT_BLOCK).astype(bool)
    assert np.array_equal(acc1, rec["accept_block"])
    assert np.abs(r["delta_block"][moved] - rec["delta_block"][moved]).max() < 1e-8
    still = np.setdiff1d(np.arange(geo.n_blocks), moved)
    assert np.abs(r["delta_block"][still]).max() < 1e-8            # M = 1 there
    dsub = ps.psms_filter_record(ctx, ps.REC_DELTA_SUB)
    assert np.abs(dsub - rec["delta_sub"]).max() < 1e-8
    assert np.array_equal(ps.psms_filter_record(ctx, ps.REC_ACCEPT_SUB).astype(bool), rec["accept_sub"])
    assert set(np.nonzero(rec["changed_sub"])[0]) <= {0, 9}
    assert np.array_equal(r["accept_block"], rec["accept_after_sub"])
    assert tuple(r["shift"]) == tuple(rec["shift"])
    assert np.abs(get_links(ctx, 0) - U2).max() < 1e-12


def test_filter_step_recursive_learned_gauge_fixed():
    """The recursive filter with the learned level and relative gauge fixing
    (the hierarchy the 32^3 x 64 workload runs): 16^4 lattice, 8^4 outer
    blocks of 4^4 inner blocks, an external proposal moving four inner
    blocks (two in outer block 0, two in outer block 9).  Both sides decide
    on the device's in-step h and its FP32 gauge transformations; stage 2
    interpolates between the stage-1 endpoints merged on the accepted inner
    blocks."""
    from oracle import mlp
    dims, outer, inner = (16, 16, 16, 16), (8, 8, 8, 8), (4, 4, 4, 4)
    nest = recursive.Nested(dims, outer, inner)
    geo = nest.inner
    ctx = ps.psms_create(dims, inner, KAPPA, 4)
    ps.psms_set_outer_blocks(ctx, outer)
    ps.psms_gauge_init(ctx, 0, 0.5, SEED + 17)
    ps.psms_gauge_sweep(ctx, 0, ps.ACTIVE_ALL, 2, 1, 5.3, SEED, 1 << 40)
    U = get_links(ctx, 0)
    ps.psms_gauge_copy(ctx, 1, 0)
    ps.psms_gauge_sweep(ctx, 1, ps.ACTIVE_BLOCKS, 1, 1, 5.3, SEED, 77)
    Usw = get_links(ctx, 1)
    moved = [b for b in range(geo.n_blocks) if nest.outer_of_inner[b] == 0][:2]
    moved += [b for b in range(geo.n_blocks) if nest.outer_of_inner[b] == 9][:2]
    sel = np.isin(geo.block_index, moved)[..., None] & geo.active_links()
    prop = U.copy()
    prop[sel] = Usw[sel]
    set_links(ctx, 1, prop)
    # a random antisymmetric surrogate whose h rejects some blocks
    p = mlp.init_params(11)
    p["ys"] = 30.0
    flat = np.concatenate([p["W1"].ravel(), p["b1"], p["W2"].ravel(), p["b2"], p["w3"], [p["b3"]], p["mu"],
                           p["sigma"], [p["ys"]]]).astype(np.float32)
    ps.psms_mlp_params(ctx, flat)
    # the device's transformations of this pair (FP32 iteration, as in the step)
    g = torch.zeros(2 * ctx.V * 9 * 2, dtype=torch.float64, device="cuda")
    ps.psms_relative_gauge_fix(ctx, 0, 1, 2, 3, g_dev=g, prec=ps.PREC_F32)
    gg = g.cpu().numpy().view(np.complex128).reshape((2,) + dims + (3, 3))
    step = 23
    r = ps.psms_filter_step(ctx, 0, beta0=5.3, n_block=1, n_sub=1, n_global=1, global_level=False, tol=1e-13,
                            inner_prec=ps.PREC_F32, seed=SEED, step=step, proposal_field=1, learned=True,
                            gauge_fix={"prec": ps.PREC_F32})
    h = ps.psms_filter_record(ctx, ps.REC_H)
    prm = recursive.RecursiveParams(kappa=KAPPA, beta0=5.3, n_block=1, n_sub=1, n_global=1, tol=1e-13,
                                    global_level=False, learned=p)
    U2, rec = recursive.filter_step(U, nest, prm, SEED, step, proposal=prop, skip_unchanged=True, h_override=h,
                                    gf_override=(gg[0], gg[1]))
    assert r["gf_steps"] > 0
    assert r["n_accept_learned"] == int(rec["passed_learned"].sum())
    assert np.any(h[moved] != 0)
    assert np.array_equal(ps.psms_filter_record(ctx, ps.REC_ACCEPT_BLOCK).astype(bool), rec["accept_block"])
    assert np.abs(r["delta_block"][moved] - rec["delta_block"][moved]).max() < 1e-8
    assert np.abs(ps.psms_filter_record(ctx, ps.REC_DELTA_SUB) - rec["delta_sub"]).max() < 1e-8
    assert np.array_equal(ps.psms_filter_record(ctx, ps.REC_ACCEPT_SUB).astype(bool), rec["accept_sub"])
    assert np.array_equal(r["accept_block"], rec["accept_after_sub"])
    assert np.abs(get_links(ctx, 0) - U2).max() < 1e-12
