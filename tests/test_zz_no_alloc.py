"""The block solve for callers that cannot allocate device memory.

psms_block_solve_noalloc serves code that must not call cudaMalloc/cudaFree
while it runs (a fixed memory pool, a host that reserved all device memory
up front, or a caller that cannot let an allocation synchronise the device).
It takes its scratch from a static device array inside the library.  Here it
is called through the C ABI twice in a row and compared with psms_solve on
the same blocks, at the tolerance of the other block-solve parity tests.
This file is collected last so that a run stopping at the first failure has
already run every other test."""
import pytest
import torch

import paper_1204_1306_gb300 as ps
from tests import seeded
from tests.gpu_util import canonical, native, rel_err

pytestmark = pytest.mark.gpu

TOL = 1e-13
PARITY = 1e-11


def _reference(ctx, b, op):
    x = torch.zeros_like(b)
    ps.psms_solve(ctx, 0, op, b, x, TOL, 20000, ps.PREC_F64)
    return canonical(ctx, x)


def test_noalloc_block_solve_matches_block_solve_twice():
    dims, block, kappa = (8, 8, 8, 8), (4, 4, 4, 4), 0.156
    ctx = ps.psms_create(dims, block, kappa, 1)
    ps.psms_gauge_init(ctx, 0, 0.5, 41)
    b1 = native(ctx, seeded.spinor(dims, 42))
    b2 = native(ctx, seeded.spinor(dims, 43))
    ref1 = _reference(ctx, b1, ps.OP_BLOCKS)
    ref2 = _reference(ctx, b2, ps.OP_BLOCKS)
    ref_one = _reference(ctx, b2, 5)
    torch.cuda.synchronize()

    x = torch.zeros_like(b1)
    held = ps.psms_scratch_bytes(ctx)
    info1 = ps.psms_block_solve_noalloc(ctx, 0, ps.OP_BLOCKS, b1, x, TOL, 20000)
    assert rel_err(canonical(ctx, x), ref1) < PARITY
    assert info1["true_residual"] <= TOL
    free_after_first = torch.cuda.mem_get_info()[0]

    info2 = ps.psms_block_solve_noalloc(ctx, 0, ps.OP_BLOCKS, b2, x, TOL, 20000)
    assert rel_err(canonical(ctx, x), ref2) < PARITY
    assert info2["true_residual"] <= TOL
    ps.psms_block_solve_noalloc(ctx, 0, 5, b2, x, TOL, 20000)
    assert rel_err(canonical(ctx, x), ref_one) < PARITY
    # the context's scratch registry did not grow (the calls allocated
    # nothing of their own); the device-wide free memory is a secondary
    # check that other processes could disturb
    assert ps.psms_scratch_bytes(ctx) == held
    assert torch.cuda.mem_get_info()[0] >= free_after_first


def test_noalloc_rejects_lattices_beyond_its_scratch():
    ctx = ps.psms_create((16, 16, 16, 16), (4, 4, 4, 4), 0.156, 1)
    b = torch.zeros(ps.psms_spinor_bytes(ctx, ps.PREC_F64), dtype=torch.uint8, device="cuda")
    x = torch.zeros_like(b)
    with pytest.raises(ps.PsmsError) as e:
        ps.psms_block_solve_noalloc(ctx, 0, ps.OP_BLOCKS, b, x, TOL, 100)
    assert e.value.status == 1 and "too large" in str(e.value)
