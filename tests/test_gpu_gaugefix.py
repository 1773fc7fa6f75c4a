"""GPU parity of the relative gauge fixing (Sec. 4.2, App. B) with the
oracle: FP64 iteration against the oracle's transformations, the FP32
iteration by the properties that fix it (exact swap symmetry, SU(3)
transformations, gauge-invariant endpoints, recovery of a pure gauge
transformation, distance reached), and the filter step with gauge-fixed
interpolation (identical decisions)."""
import numpy as np
import pytest
import torch

import paper_1204_1306_gb300 as ps
from oracle import filter as ofilter, gauge, gaugefix, lattice
from tests.gpu_util import from_dev, get_links, set_links

pytestmark = pytest.mark.gpu

SEED = 0x50534D53


def _pair(dims, block, seed, therm=2):
    """Thermalised U in slot 0 and a domain-sweep proposal U' in slot 1."""
    ctx = ps.psms_create(dims, block, 0.156, 4)
    ps.psms_gauge_init(ctx, 0, 0.5, seed)
    ps.psms_gauge_sweep(ctx, 0, ps.ACTIVE_ALL, therm, 1, 5.3, SEED, 1 << 40)
    ps.psms_gauge_copy(ctx, 1, 0)
    ps.psms_gauge_sweep(ctx, 1, ps.ACTIVE_BLOCKS, 1, 1, 5.3, SEED, 3 << 20)
    return ctx


def _g(ctx, **kw):
    g = torch.empty(2 * ctx.V * 9 * 2, dtype=torch.float64, device="cuda")
    info = ps.psms_relative_gauge_fix(ctx, 0, 1, 2, 3, g_dev=g, **kw)
    torch.cuda.synchronize()
    gg = from_dev(g, (2,) + ctx.dims + (3, 3))
    return gg[0], gg[1], info


@pytest.mark.parametrize("dims,block", [((8, 8, 8, 8), (4, 4, 4, 4)), ((8, 8, 8, 16), (8, 8, 8, 8))])
def test_fp64_iteration_parity(dims, block):
    geom = lattice.Geometry(dims, block)
    ctx = _pair(dims, block, SEED + 5)
    U, Up = get_links(ctx, 0), get_links(ctx, 1)
    g1, g2, info = _g(ctx, prec=ps.PREC_F64)
    r1, r2, rinfo = gaugefix.relative_gauge_fix(U, Up, geom)
    assert np.array_equal(info["swapped"], rinfo["swapped"])
    assert np.array_equal(info["steps"], rinfo["steps"])
    assert np.array_equal(info["alpha"], rinfo["alpha"])
    assert np.abs(info["theta"] - rinfo["theta"]).max() <= 1e-9 * max(1.0, rinfo["theta"].max())
    assert np.abs(g1 - r1).max() < 1e-10 and np.abs(g2 - r2).max() < 1e-10
    # the endpoints are the transforms of the inputs
    assert np.abs(get_links(ctx, 2) - gaugefix.transform(U, g1)).max() < 1e-13
    assert np.abs(get_links(ctx, 3) - gaugefix.transform(Up, g2)).max() < 1e-13


@pytest.mark.parametrize("prec", [ps.PREC_F32, ps.PREC_F64])
def test_swap_symmetry_exact(prec):
    """The reverse move gets exactly the swapped transformations and endpoints."""
    dims, block = (8, 8, 8, 16), (8, 8, 8, 8)
    ctx = _pair(dims, block, SEED + 6)
    g1, g2, i1 = _g(ctx, prec=prec)
    e0, eN = get_links(ctx, 2), get_links(ctx, 3)
    g = torch.empty(2 * ctx.V * 9 * 2, dtype=torch.float64, device="cuda")
    i2 = ps.psms_relative_gauge_fix(ctx, 1, 0, 3, 2, g_dev=g, prec=prec)
    torch.cuda.synchronize()
    h = from_dev(g, (2,) + ctx.dims + (3, 3))
    assert np.array_equal(h[0], g2) and np.array_equal(h[1], g1)
    assert np.array_equal(i1["steps"], i2["steps"]) and np.array_equal(i1["swapped"], ~i2["swapped"])
    assert np.array_equal(get_links(ctx, 2), e0) and np.array_equal(get_links(ctx, 3), eN)


def test_fp32_iteration_properties():
    """FP32 steps: converged blocks, SU(3) transformations (FP64 reunitarised)
    that leave gauge-invariant quantities unchanged, and a fixed distance
    within the FP64 oracle's."""
    dims, block = (8, 8, 8, 16), (8, 8, 8, 8)
    geom = lattice.Geometry(dims, block)
    ctx = _pair(dims, block, SEED + 7)
    U, Up = get_links(ctx, 0), get_links(ctx, 1)
    g1, g2, info = _g(ctx, prec=ps.PREC_F32)
    assert np.all(info["theta"] < 1e-3)
    inside = gaugefix.interior_mask(geom)
    for g in (g1, g2):
        assert np.abs(g @ gauge.dag(g) - np.eye(3)).max() < 1e-14
        assert np.abs(np.linalg.det(g) - 1).max() < 1e-14
        assert np.array_equal(g[~inside], np.broadcast_to(np.eye(3), g[~inside].shape))
    e0, eN = get_links(ctx, 2), get_links(ctx, 3)
    for a, b in ((e0, U), (eN, Up)):
        for mu in range(4):
            for nu in range(mu + 1, 4):
                pa = np.trace(gauge.plaquette_field(a, mu, nu), axis1=-2, axis2=-1)
                pb = np.trace(gauge.plaquette_field(b, mu, nu), axis1=-2, axis2=-1)
                assert np.abs(pa - pb).max() < 1e-13
    r1, r2, _ = gaugefix.relative_gauge_fix(U, Up, geom)
    d_dev = gaugefix.sprod(e0, eN)
    d_ref = gaugefix.sprod(gaugefix.transform(U, r1), gaugefix.transform(Up, r2))
    assert d_dev < 0.9 * gaugefix.sprod(U, Up)
    assert abs(d_dev - d_ref) <= 0.02 * d_ref


@pytest.mark.parametrize("prec", [ps.PREC_F32, ps.PREC_F64])
def test_recovers_pure_gauge(prec):
    """U' = U^k with k on the block interiors: the fixed pair coincides."""
    dims, block = (8, 8, 8, 8), (4, 4, 4, 4)
    geom = lattice.Geometry(dims, block)
    ctx = ps.psms_create(dims, block, 0.156, 4)
    ps.psms_gauge_init(ctx, 0, 0.5, SEED + 8)
    U = get_links(ctx, 0)
    om = np.random.default_rng(5).standard_normal(geom.dims + (8,))
    k = gauge.expm_i_hermitian(gauge.hermitian_generators(om), 0.6)
    k = np.where(gaugefix.interior_mask(geom)[..., None, None], k, np.eye(3))
    set_links(ctx, 1, gaugefix.transform(U, k))
    tol = 1e-9 if prec == ps.PREC_F32 else 1e-20
    g1, g2, info = _g(ctx, prec=prec, alpha0=0.1, alpha_min=0.1, theta_tol=tol, max_iter=3000)
    assert np.all(info["theta"] < tol)
    d = gaugefix.sprod(get_links(ctx, 2), get_links(ctx, 3))
    assert d < (1e-9 if prec == ps.PREC_F32 else 1e-12), d


def test_identical_fields_and_small_blocks():
    ctx = ps.psms_create((8, 8, 8, 8), (4, 4, 4, 4), 0.156, 4)
    ps.psms_gauge_init(ctx, 0, 0.5, SEED + 9)
    ps.psms_gauge_copy(ctx, 1, 0)
    g1, g2, info = _g(ctx)
    assert np.all(info["steps"] == 0)
    assert np.array_equal(get_links(ctx, 2), get_links(ctx, 0))
    ctx2 = ps.psms_create((4, 4, 4, 4), (2, 2, 2, 2), 0.15, 4)
    ps.psms_gauge_init(ctx2, 0, 0.3, SEED)
    ps.psms_gauge_copy(ctx2, 1, 0)
    ps.psms_gauge_sweep(ctx2, 1, ps.ACTIVE_BLOCKS, 1, 0, 5.3, SEED, 0)
    info = ps.psms_relative_gauge_fix(ctx2, 0, 1, 2, 3)
    assert np.all(info["steps"] == 0)
    assert np.array_equal(get_links(ctx2, 3), get_links(ctx2, 1))
    with pytest.raises(ps.PsmsError):
        ps.psms_relative_gauge_fix(ctx, 0, 1, 1, 3)
    with pytest.raises(ps.PsmsError):
        ps.psms_relative_gauge_fix(ctx, 0, 1, 2, 3, alpha0=0.1, alpha_min=0.2)


@pytest.mark.parametrize("prec", [ps.PREC_F64, ps.PREC_F32])
def test_filter_step_with_gauge_fixing_parity(prec):
    """8^4 lattice, 4^4 blocks: levels 1 and 2 interpolate between gauge-fixed
    endpoints.  FP64 iteration: the oracle fixes the gauge itself; FP32: the
    oracle takes the device's transformations (computed for the same
    proposal), so both sides decide on the same numbers."""
    dims, block, kappa = (8, 8, 8, 8), (4, 4, 4, 4), 0.156
    geom = lattice.Geometry(dims, block)
    ctx = ps.psms_create(dims, block, kappa, 4)
    ps.psms_gauge_init(ctx, 0, 0.5, SEED + 3)
    ps.psms_gauge_sweep(ctx, 0, ps.ACTIVE_ALL, 3, 2, 5.3, SEED, 1 << 40)
    U = get_links(ctx, 0)
    step = 7
    gf = {"prec": prec}
    override = None
    if prec == ps.PREC_F32:
        ps.psms_gauge_copy(ctx, 1, 0)
        ps.psms_gauge_sweep(ctx, 1, ps.ACTIVE_BLOCKS, 1, 1, 5.3, SEED, step << 20)
        g1, g2, _ = _g(ctx, prec=prec)
        override = (g1, g2)
    r = ps.psms_filter_step(ctx, 0, beta0=5.3, n_iter=1, n_or=1, n_block=3, n_global=1, tol=1e-13,
                            inner_prec=ps.PREC_F32, seed=SEED, step=step, gauge_fix=gf)
    prm = ofilter.FilterParams(kappa=kappa, beta0=5.3, n_iter=1, n_or=1, n_block=3, n_global=1, tol=1e-13,
                               gauge_fix={} if override is None else None)
    U2, rec = ofilter.filter_step(U, geom, prm, SEED, step, gf_override=override)
    assert r["gf_steps"] > 0
    if override is None:
        assert r["gf_steps"] == int(rec["gauge_fix"]["steps"].sum())
    assert np.array_equal(r["accept_block"], rec["accept_block"])
    assert np.abs(r["delta_block"] - rec["delta_block"]).max() < 1e-8
    assert r["accept_global"] == rec["accept_global"]
    if r["n_accept_blocks"] > 0:
        assert abs(r["delta_global"] - rec["delta_global"]) < 1e-8
    assert np.abs(get_links(ctx, 0) - U2).max() < 1e-12
