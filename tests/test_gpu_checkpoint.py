"""Checkpoint / resume of the Markov chain: a chain saved after some filter
steps and resumed in a fresh context continues bit-identically (all random
numbers are counter-based, so the field, step and seed are the whole state),
and the learned level's parameters travel with it."""
import numpy as np
import pytest
import torch

import paper_1204_1306_gb300 as ps
from tests.gpu_util import get_links

pytestmark = pytest.mark.gpu

SEED = 0x50534D53
DIMS, BLOCK, KAPPA = (8, 8, 8, 8), (4, 4, 4, 4), 0.156
STEP = dict(beta0=5.3, n_iter=1, n_or=1, n_block=2, n_global=2, tol=1e-12, inner_prec=ps.PREC_F32, seed=SEED)


def _ctx():
    ctx = ps.psms_create(DIMS, BLOCK, KAPPA, 1)
    ps.psms_gauge_init(ctx, 0, 0.5, SEED + 9)
    return ctx


def test_resume_is_bit_identical(tmp_path):
    a = _ctx()
    ps.psms_mlp_init(a, 4)
    for s in range(2):
        ps.psms_filter_step(a, 0, step=s, **STEP)
    path = tmp_path / "chain.ckpt"
    ps.psms_checkpoint_save(a, 0, path, 2, SEED)
    rest = [ps.psms_filter_step(a, 0, step=s, learned=True, **STEP) for s in (2, 3)]
    ua = get_links(a, 0)

    b = ps.psms_create(DIMS, BLOCK, KAPPA, 1)
    step, seed = ps.psms_checkpoint_load(b, 0, path)
    assert (step, seed) == (2, SEED)
    assert np.array_equal(ps.psms_mlp_params(a), ps.psms_mlp_params(b))
    again = [ps.psms_filter_step(b, 0, step=s, learned=True, **STEP) for s in range(step, step + 2)]
    for r, q in zip(rest, again):
        assert np.array_equal(r["accept_block"], q["accept_block"])
        assert r["accept_global"] == q["accept_global"]
        assert np.array_equal(r["delta_block"], q["delta_block"])
    assert np.array_equal(get_links(b, 0), ua)


def test_checkpoint_rejects_other_lattice_and_damage(tmp_path):
    a = _ctx()
    path = tmp_path / "chain.ckpt"
    ps.psms_checkpoint_save(a, 0, path, 0, SEED)
    other = ps.psms_create(DIMS, (4, 4, 4, 8), KAPPA, 1)
    with pytest.raises(ps.PsmsError) as e:
        ps.psms_checkpoint_load(other, 0, path)
    assert e.value.status == 1
    data = path.read_bytes()
    bad = tmp_path / "short.ckpt"
    bad.write_bytes(data[:len(data) // 2])
    with pytest.raises(ps.PsmsError) as e:
        ps.psms_checkpoint_load(a, 0, bad)
    assert e.value.status == 1
    with pytest.raises(ps.PsmsError):
        ps.psms_checkpoint_load(a, 0, tmp_path / "missing.ckpt")
    # the field is untouched by a failed load
    u0 = get_links(a, 0)
    ps.psms_checkpoint_load(a, 0, path)
    assert np.array_equal(get_links(a, 0), u0)
