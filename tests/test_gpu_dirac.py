"""GPU parity of the Wilson-Dirac operator, the link generator and the gauge
helpers against the FP64 oracle (relative 1e-12 for FP64 D_w)."""
import numpy as np
import pytest
import torch

import paper_1204_1306_gb300 as ps
from oracle import dirac, gauge, lattice
from tests import seeded
from tests.gpu_util import canonical, get_links, native, rel_err, set_links

pytestmark = pytest.mark.gpu

GEOMS = [
    ((4, 4, 4, 4), (2, 2, 2, 2)),      # 4^4 lattice, 2^4 blocks
    ((6, 4, 4, 2), (2, 2, 2, 2)),      # ragged: V/2 = 96 < one CTA
    ((8, 8, 8, 8), (4, 4, 4, 4)),
    ((12, 12, 12, 12), (4, 4, 4, 4)),  # odd block count, no colouring
    ((16, 16, 16, 16), (4, 4, 4, 4)),  # 16^4, 4^4 blocks
]


@pytest.mark.parametrize("dims,block", GEOMS)
@pytest.mark.parametrize("eps", [0.3, 0.5])
def test_link_generator_parity(dims, block, eps):
    ctx = ps.psms_create(dims, block, 0.15, 1)
    ps.psms_gauge_init(ctx, 0, eps, 0x50534D53 + 7)
    U = get_links(ctx, 0)
    ref = gauge.generate_links(dims, eps, 0x50534D53 + 7)
    assert np.abs(U - ref).max() < 5e-14


@pytest.mark.parametrize("dims,block", GEOMS)
def test_dw_fp64_parity(dims, block):
    kappa = 0.156
    ctx = ps.psms_create(dims, block, kappa, 1)
    ps.psms_gauge_init(ctx, 0, 0.5, 11)
    U = gauge.generate_links(dims, 0.5, 11)
    psi = seeded.spinor(dims, 12)
    out = torch.zeros_like(native(ctx, psi))
    ps.psms_dw_apply(ctx, 0, ps.OP_FULL, native(ctx, psi), out, ps.PREC_F64)
    got = canonical(ctx, out)
    ref = dirac.apply_D(U, psi, kappa)
    assert rel_err(got, ref) < 1e-12


def test_dw_haar_field_and_edges():
    """Haar-random SU(3) links set through the canonical layout; zero input
    gives zero output; a delta source reproduces one column of D."""
    dims, block = (4, 4, 2, 4), (2, 2, 2, 2)
    ctx = ps.psms_create(dims, block, 0.13, 1)
    U = seeded.gauge_field(dims, 5)
    set_links(ctx, 0, U)
    zero = np.zeros(dims + (4, 3), dtype=complex)
    out = torch.zeros_like(native(ctx, zero))
    ps.psms_dw_apply(ctx, 0, ps.OP_FULL, native(ctx, zero), out, ps.PREC_F64)
    assert np.abs(canonical(ctx, out)).max() == 0.0
    delta = zero.copy()
    delta[0, 0, 0, 0, 2, 1] = 1.0
    ps.psms_dw_apply(ctx, 0, ps.OP_FULL, native(ctx, delta), out, ps.PREC_F64)
    assert rel_err(canonical(ctx, out), dirac.apply_D(U, delta, 0.13)) < 1e-13


@pytest.mark.parametrize("dims,block", [((4, 4, 4, 4), (2, 2, 2, 2)), ((8, 8, 8, 8), (4, 4, 4, 4)),
                                        ((8, 4, 4, 8), (4, 2, 2, 4))])
def test_block_operators(dims, block):
    """PSMS_OP_BLOCKS = D_bb + D_ww and a single D_b (Eq. (domdec))."""
    from oracle import lattice
    geom = lattice.Geometry(dims, block)
    kappa = 0.15
    ctx = ps.psms_create(dims, block, kappa, 1)
    ps.psms_gauge_init(ctx, 0, 0.5, 3)
    U = gauge.generate_links(dims, 0.5, 3)
    psi = seeded.spinor(dims, 4)
    out = torch.zeros_like(native(ctx, psi))
    ps.psms_dw_apply(ctx, 0, ps.OP_BLOCKS, native(ctx, psi), out, ps.PREC_F64)
    assert rel_err(canonical(ctx, out), dirac.apply_D(U, psi, kappa, geom, mode="block")) < 1e-12
    b = geom.n_blocks - 1
    ps.psms_dw_apply(ctx, 0, b, native(ctx, psi), out, ps.PREC_F64)
    got = canonical(ctx, out)
    ref = np.zeros_like(psi)
    dirac.insert_block(ref, geom, b, dirac.apply_D_open(dirac.extract_block(U, geom, b),
                                                         dirac.extract_block(psi, geom, b), kappa))
    assert rel_err(got, ref) < 1e-12


@pytest.mark.parametrize("prec,tol", [(ps.PREC_F32, 2e-6), (ps.PREC_BF16, 2e-2)])
def test_dw_low_precision(prec, tol):
    """FP32 arithmetic with FP32 or BF16 spinor storage (FP32 links)."""
    dims, block = (8, 8, 8, 8), (4, 4, 4, 4)
    kappa = 0.157
    ctx = ps.psms_create(dims, block, kappa, 1)
    ps.psms_gauge_init(ctx, 0, 0.5, 21)
    U = gauge.generate_links(dims, 0.5, 21)
    psi = seeded.spinor(dims, 22)
    nat = native(ctx, psi, prec)
    out = torch.zeros_like(nat)
    ps.psms_dw_apply(ctx, 0, ps.OP_FULL, nat, out, prec)
    assert rel_err(canonical(ctx, out, prec), dirac.apply_D(U, psi, kappa)) < tol


@pytest.mark.parametrize("prec,tol", [(ps.PREC_F32, 2e-6), (ps.PREC_BF16, 2e-2)])
def test_dw_every_hop_variant(prec, tol):
    """Every autotuned Wilson-hop variant (register caps, branch-free
    whole-lattice specialisation), forced one by one: whole-lattice D_w with
    the antiperiodic time boundary, and the Dirichlet block operator."""
    dims, block = (8, 8, 4, 8), (4, 4, 4, 4)
    geom = lattice.Geometry(dims, block)
    kappa = 0.157
    ctx = ps.psms_create(dims, block, kappa, 1)
    ps.psms_gauge_init(ctx, 0, 0.5, 23)
    U = gauge.generate_links(dims, 0.5, 23)
    psi = seeded.spinor(dims, 24)
    nat = native(ctx, psi, prec)
    ref_full = dirac.apply_D(U, psi, kappa)
    ref_blk = dirac.apply_D(U, psi, kappa, geom, mode="block")
    n = ps.psms_hop_variant(ctx, 0)
    for v in range(n):
        ps.psms_hop_variant(ctx, v)
        out = torch.zeros_like(nat)
        ps.psms_dw_apply(ctx, 0, ps.OP_FULL, nat, out, prec)
        assert rel_err(canonical(ctx, out, prec), ref_full) < tol, v
        out = torch.zeros_like(nat)
        ps.psms_dw_apply(ctx, 0, ps.OP_BLOCKS, nat, out, prec)
        assert rel_err(canonical(ctx, out, prec), ref_blk) < tol, v
    # the single-parity launches of the even-odd whole-lattice solver with
    # each whole-lattice variant forced (two threads per site: 8, 9; staged
    # with per-thread copies: 10, 11, with bulk copies: 12, 13): the FP64
    # defect correction reaches its true residual only if the inner
    # operator is right
    b = native(ctx, seeded.spinor(dims, 25))
    for v in (5, 8, 9, 10, 11, 12, 13):
        ps.psms_hop_variant(ctx, v)
        x = torch.zeros_like(b)
        info = ps.psms_solve(ctx, 0, ps.OP_FULL, b, x, 1e-11, 4000, ps.PREC_F32)
        assert info["true_residual"] <= 1e-11 and info["outer_iters"] <= 6, (v, info)
    ps.psms_hop_variant(ctx, -1)
    with pytest.raises(ps.PsmsError):
        ps.psms_hop_variant(ctx, n)


def test_plaquette_and_translation():
    from oracle import lattice
    dims, block = (8, 4, 4, 8), (4, 2, 2, 4)
    ctx = ps.psms_create(dims, block, 0.15, 1)
    ps.psms_gauge_init(ctx, 0, 0.5, 31)
    U = gauge.generate_links(dims, 0.5, 31)
    plaq, sw = ps.psms_plaquette(ctx, 0)
    assert abs(plaq - gauge.mean_plaquette(U)) < 1e-13
    assert abs(sw - gauge.wilson_action(U)) < 1e-10 * abs(sw)
    s = (3, 1, 2, 5)
    before = get_links(ctx, 0)
    ps.psms_gauge_translate(ctx, 0, s)
    assert np.array_equal(get_links(ctx, 0), lattice.Geometry(dims, block).translate(before, s))


def test_geometry_info():
    from oracle import lattice
    for dims, block in [((8, 8, 8, 8), (4, 4, 4, 4)), ((16, 16, 16, 16), (4, 4, 4, 4)), ((4, 4, 4, 4), (2, 2, 2, 2))]:
        ctx = ps.psms_create(dims, block, 0.15, 1)
        nb, dimP, nact = ps.psms_geometry_info(ctx)
        geom = lattice.Geometry(dims, block)
        assert nb == geom.n_blocks
        assert dimP == geom.dim_projector()
        assert nact == int(geom.active_links().sum())


def test_invalid_arguments_are_reported():
    with pytest.raises(ps.PsmsError):
        ps.psms_create((6, 6, 6, 6), (3, 3, 3, 3), 0.15, 1)
    ctx = ps.psms_create((4, 4, 4, 4), (2, 2, 2, 2), 0.15, 1)
    with pytest.raises(ps.PsmsError):
        ps.psms_gauge_init(ctx, 5, 0.3, 1)
    buf = torch.zeros(ps.psms_spinor_bytes(ctx, ps.PREC_F64), dtype=torch.uint8, device="cuda")
    with pytest.raises(ps.PsmsError):
        ps.psms_dw_apply(ctx, 0, ps.OP_FULL, buf, buf, ps.PREC_F64)
    with pytest.raises(ps.PsmsError):
        ps.psms_dw_apply(ctx, 0, 99, buf, torch.zeros_like(buf), ps.PREC_F64)


def test_nonfinite_inputs_and_allocation_failure():
    """NaN / infinite inputs are rejected with PSMS_EINVAL before anything is
    written; a lattice larger than the device memory fails with PSMS_ENOMEM
    (a real allocation failure, no fault)."""
    dims = (4, 4, 4, 4)
    ctx = ps.psms_create(dims, (2, 2, 2, 2), 0.15, 1)
    ps.psms_gauge_init(ctx, 0, 0.3, 1)
    before = get_links(ctx, 0)
    U = gauge.generate_links(dims, 0.3, 2)
    U[1, 2, 3, 0, 1, 0, 2] = np.nan
    with pytest.raises(ps.PsmsError) as e:
        set_links(ctx, 0, U)
    assert e.value.status == 1
    assert np.array_equal(get_links(ctx, 0), before)
    psi = seeded.spinor(dims, 3)
    psi[0, 0, 0, 1, 2, 1] = np.inf
    with pytest.raises(ps.PsmsError) as e:
        native(ctx, psi)
    assert e.value.status == 1
    b = native(ctx, seeded.spinor(dims, 4))
    bad = b.view(torch.float64).clone()
    bad[17] = float("nan")
    x = torch.zeros_like(b)
    with pytest.raises(ps.PsmsError) as e:
        ps.psms_solve(ctx, 0, ps.OP_FULL, bad.view(torch.uint8), x, 1e-10, 100, ps.PREC_F64)
    assert e.value.status == 1
    # 128^4 sites, two FP64 link slots of 155 GB each: above the device's
    # memory, so the second allocation fails and everything is freed
    with pytest.raises(ps.PsmsError) as e:
        ps.psms_create((128, 128, 128, 128), (8, 8, 8, 8), 0.15, 2)
    assert e.value.status == 2
    # the library stays usable
    ps.psms_dw_apply(ctx, 0, ps.OP_FULL, b, x, ps.PREC_F64)
