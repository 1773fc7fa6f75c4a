"""All 4^4 Dirichlet blocks x several right-hand sides of three uneven
lattices in one persistent, graph-captured launch (psms_block_plan): results
equal the per-lattice block solves (themselves pinned to the oracle), on two
graph replays with different right-hand sides; the true residual of one block
is recomputed with the oracle's D_b."""
import numpy as np
import pytest
import torch

import paper_1204_1306_gb300 as ps
from oracle import dirac, gauge, lattice, linalg
from tests import seeded
from tests.gpu_util import canonical, native, rel_err

pytestmark = pytest.mark.gpu

LATTICES = [((8, 8, 8, 8), 31), ((12, 12, 12, 12), 32), ((16, 8, 8, 8), 33)]
KAPPA = 0.155
TOL = 1e-12


@pytest.mark.parametrize("inner", [ps.PREC_F32, ps.PREC_F64])
def test_multi_lattice_plan(inner):
    n_rhs = 3
    probs, ctxs, bs, xs = [], [], [], []
    for dims, seed in LATTICES:
        ctx = ps.psms_create(dims, (4, 4, 4, 4), KAPPA, 1)
        ps.psms_gauge_init(ctx, 0, 0.5, seed)
        nb = ps.psms_spinor_bytes(ctx, ps.PREC_F64)
        b = torch.zeros(n_rhs * nb, dtype=torch.uint8, device="cuda")
        x = torch.zeros_like(b)
        probs.append((ctx, 0, n_rhs, b, x))
        ctxs.append(ctx)
        bs.append(b)
        xs.append(x)
    plan = ps.psms_block_plan_create(probs, TOL, 20000, inner)
    sched = plan.schedule()
    assert sched["ctas"] > 0 and sched["order"] in (0, 1, 2)
    for rep in range(2):
        rhs = []
        for li, (ctx, b) in enumerate(zip(ctxs, bs)):
            nb = ps.psms_spinor_bytes(ctx, ps.PREC_F64)
            fields = []
            for k in range(n_rhs):
                psi = seeded.spinor(ctx.dims, 100 * rep + 10 * li + k)
                b[k * nb:(k + 1) * nb].copy_(native(ctx, psi))
                fields.append(psi)
            rhs.append(fields)
        torch.cuda.synchronize()
        info = plan.run()
        assert info["true_residual"] <= TOL
        assert info["n_systems"] == n_rhs * sum(ps.psms_geometry_info(c)[0] for c in ctxs)
        for li, (ctx, b, x) in enumerate(zip(ctxs, bs, xs)):
            nb = ps.psms_spinor_bytes(ctx, ps.PREC_F64)
            for k in range(n_rhs):
                got = canonical(ctx, x[k * nb:(k + 1) * nb])
                ref_x = torch.zeros(nb, dtype=torch.uint8, device="cuda")
                ps.psms_solve(ctx, 0, ps.OP_BLOCKS, b[k * nb:(k + 1) * nb].clone(), ref_x, TOL, 20000, inner)
                assert rel_err(got, canonical(ctx, ref_x)) < 1e-10
    # oracle residual on one block of the 12^4 lattice
    dims = LATTICES[1][0]
    geom = lattice.Geometry(dims, (4, 4, 4, 4))
    U = gauge.generate_links(dims, 0.5, LATTICES[1][1])
    nb = ps.psms_spinor_bytes(ctxs[1], ps.PREC_F64)
    got = canonical(ctxs[1], xs[1][:nb])
    for blk in (0, 40, 80):
        Ub = dirac.extract_block(U, geom, blk)
        r = dirac.extract_block(rhs[1][0], geom, blk) - dirac.apply_D_open(Ub, dirac.extract_block(got, geom, blk), KAPPA)
        assert np.sqrt(linalg.norm2(r) / linalg.norm2(dirac.extract_block(rhs[1][0], geom, blk))) <= TOL
    plan.close()
