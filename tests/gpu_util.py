"""Helpers for the GPU parity tests: numpy canonical arrays <-> device
tensors and native spinor buffers (argument marshalling only)."""
import numpy as np
import torch

import paper_1204_1306_gb300 as ps


def to_dev(a):
    a = np.ascontiguousarray(a, dtype=np.complex128)
    return torch.from_numpy(a.view(np.float64).reshape(-1).copy()).cuda()


def from_dev(t, shape):
    return t.detach().cpu().numpy().view(np.complex128).reshape(shape)


def native(ctx, psi, prec=ps.PREC_F64):
    nat = torch.empty(ps.psms_spinor_bytes(ctx, prec), dtype=torch.uint8, device="cuda")
    ps.psms_spinor_import(ctx, to_dev(psi), nat, prec)
    return nat


def empty_native(ctx, prec=ps.PREC_F64):
    return torch.zeros(ps.psms_spinor_bytes(ctx, prec), dtype=torch.uint8, device="cuda")


def canonical(ctx, nat, prec=ps.PREC_F64):
    out = torch.empty(ctx.V * 24, dtype=torch.float64, device="cuda")
    ps.psms_spinor_export(ctx, nat, out, prec)
    torch.cuda.synchronize()
    return from_dev(out, ctx.dims + (4, 3))


def set_links(ctx, f, U):
    ps.psms_gauge_set(ctx, f, to_dev(U))


def get_links(ctx, f):
    out = torch.empty(ctx.V * 4 * 9 * 2, dtype=torch.float64, device="cuda")
    ps.psms_gauge_get(ctx, f, out)
    torch.cuda.synchronize()
    return from_dev(out, ctx.dims + (4, 3, 3))


def rel_err(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))
