"""GPU parity of the learned delayed-acceptance level with the FP64 oracle:
domain features (FP32 output of FP64 arithmetic), the BF16 tensor-core MLP
forward and gradients (BF16 tolerance), training, and the filter step with
the learned level inserted (identical decisions on the kernel's h)."""
import numpy as np
import pytest
import torch

import paper_1204_1306_gb300 as ps
from oracle import filter as ofilter, gauge, lattice, mlp
from tests.gpu_util import get_links

pytestmark = pytest.mark.gpu

SEED = 0x50534D53


def _params(seed):
    g = np.random.default_rng(seed)
    p = mlp.init_params(seed)
    p["b1"] = g.standard_normal(256) * 0.1
    p["b2"] = g.standard_normal(256) * 0.1
    p["b3"] = 0.3
    mu = g.standard_normal(32) * 0.2
    sg = 0.5 + g.random(32)
    p["mu"] = np.concatenate([mu, mu])
    p["sigma"] = np.concatenate([sg, sg])
    p["ys"] = 2.5
    return p


def _flat(p):
    return np.concatenate([p["W1"].ravel(), p["b1"], p["W2"].ravel(), p["b2"], p["w3"], [p["b3"]], p["mu"],
                           p["sigma"], [p["ys"]]]).astype(np.float32)


def _rounded(p):
    """The parameters as the device holds them (FP32)."""
    return mlp.unflatten(_flat(p))


@pytest.mark.parametrize("dims,block", [((8, 8, 8, 8), (4, 4, 4, 4)), ((8, 8, 8, 16), (8, 8, 8, 8)),
                                        ((4, 4, 4, 4), (2, 2, 2, 2))])
def test_domain_features_parity(dims, block):
    geom = lattice.Geometry(dims, block)
    ctx = ps.psms_create(dims, block, 0.15, 1)
    ps.psms_gauge_init(ctx, 0, 0.5, 12)
    out = torch.zeros(geom.n_blocks * 32, dtype=torch.float32, device="cuda")
    ps.psms_domain_features(ctx, 0, out)
    got = out.cpu().numpy().reshape(geom.n_blocks, 32).astype(np.float64)
    ref = mlp.domain_features(gauge.generate_links(dims, 0.5, 12), geom)
    assert np.abs(got - ref).max() <= 2e-6 * max(1.0, np.abs(ref).max())


def test_pair_features_parity():
    """[f(U_b), f(U'_b)] with the block distance of Eq. (sprodgf) in slots 18, 50."""
    dims, block = (8, 8, 8, 8), (4, 4, 4, 4)
    geom = lattice.Geometry(dims, block)
    ctx = ps.psms_create(dims, block, 0.15, 2)
    ps.psms_gauge_init(ctx, 0, 0.5, 12)
    ps.psms_gauge_copy(ctx, 1, 0)
    ps.psms_gauge_sweep(ctx, 1, ps.ACTIVE_BLOCKS, 1, 1, 5.3, 3, 0)
    out = torch.zeros(geom.n_blocks * 64, dtype=torch.float32, device="cuda")
    ps.psms_domain_features_pair(ctx, 0, 1, out)
    got = out.cpu().numpy().reshape(geom.n_blocks, 64).astype(np.float64)
    U = gauge.generate_links(dims, 0.5, 12)
    Up, _, _ = gauge.domain_sweep(U, geom, 5.3, 1, 1, 3, 0)
    ref = mlp.pair_features(U, Up, geom)
    assert np.abs(got - ref).max() <= 2e-6 * max(1.0, np.abs(ref).max())
    assert np.all(ref[:, 18] > 0) and np.array_equal(ref[:, 18], ref[:, 50])


def test_mlp_forward_and_gradient_parity():
    ctx = ps.psms_create((4, 4, 4, 4), (2, 2, 2, 2), 0.15, 1)
    p = _params(5)
    ps.psms_mlp_params(ctx, _flat(p))
    q = _rounded(p)
    g = np.random.default_rng(9)
    B = 300
    z = np.concatenate([q["mu"][:32] + g.standard_normal((B, 32)), q["mu"][:32] + g.standard_normal((B, 32))], axis=1)
    zd = torch.from_numpy(z.astype(np.float32)).cuda()
    h = torch.zeros(B, dtype=torch.float32, device="cuda")
    ps.psms_mlp_predict(ctx, zd, B, h)
    z32 = z.astype(np.float32).astype(np.float64)
    got = h.cpu().numpy().astype(np.float64)
    # at the device's precision (BF16 operands, FP32 accumulation): tight
    ref_r = mlp.antisym_rounded(q, z32)
    assert np.linalg.norm(got - ref_r) <= 2e-3 * np.linalg.norm(ref_r)
    # against the FP64 definition: BF16 rounding (2^-8 relative per operand)
    # of n(f,f') and n(f',f) is amplified by their cancellation in h
    ref = mlp.antisym(q, z32)
    assert np.linalg.norm(got - ref) <= 0.25 * np.linalg.norm(ref)
    y = g.standard_normal(B) * 3.0
    loss, grad = ps.psms_mlp_grad(ctx, zd, torch.from_numpy(y).cuda(), B)
    ref_loss_r, ref_g_r = mlp.loss_and_grad_rounded(q, z32, y)
    ref_flat_r = mlp.flatten_grads(ref_g_r)
    assert abs(loss - ref_loss_r) <= 1e-3 * ref_loss_r
    o = 0
    for k, n in (("W1", 256 * 64), ("b1", 256), ("W2", 256 * 256), ("b2", 256), ("w3", 256)):
        a, b = grad[o:o + n], ref_flat_r[o:o + n]
        assert np.linalg.norm(a - b) <= 1e-2 * np.linalg.norm(b) + 1e-6, k
        o += n
    ref_loss, ref_g = mlp.loss_and_grad(q, z32, y)
    ref_flat = mlp.flatten_grads(ref_g)
    assert abs(loss - ref_loss) <= 0.1 * ref_loss
    assert np.linalg.norm(grad - ref_flat) <= 0.25 * np.linalg.norm(ref_flat)


def test_mlp_training_fits_an_antisymmetric_target():
    ctx = ps.psms_create((4, 4, 4, 4), (2, 2, 2, 2), 0.15, 1)
    ps.psms_mlp_init(ctx, 3)
    g = np.random.default_rng(4)
    n = 4096
    fa, fb = g.standard_normal((n, 32)), g.standard_normal((n, 32))
    y = 20.0 * (fb[:, 0] - fa[:, 0]) + 5.0 * (fb[:, 3] ** 2 - fa[:, 3] ** 2) + 3.0 * np.tanh(fb[:, 7] - fa[:, 7])
    z = np.concatenate([fa, fb], axis=1).astype(np.float32)
    zd, yd = torch.from_numpy(z).cuda(), torch.from_numpy(y).cuda()
    losses = ps.psms_mlp_train(ctx, zd, yd, n, epochs=30, batch=256, lr=2e-3, seed=1)
    assert losses[-1] < 0.05 * losses[0]
    h = torch.zeros(n, dtype=torch.float32, device="cuda")
    ps.psms_mlp_predict(ctx, zd, n, h)
    hv = h.cpu().numpy()
    assert np.corrcoef(hv, y)[0, 1] > 0.97
    # antisymmetry of the deployed surrogate
    zs = np.concatenate([z[:, 32:], z[:, :32]], axis=1)
    hs = torch.zeros(n, dtype=torch.float32, device="cuda")
    ps.psms_mlp_predict(ctx, torch.from_numpy(zs).cuda(), n, hs)
    assert np.abs(hs.cpu().numpy() + hv).max() <= 1e-5 * np.abs(hv).max()


def test_filter_step_with_learned_level_parity():
    """8^4 lattice, 4^4 blocks: learned level, then the stochastic block level
    on the blocks that passed with Delta_b - h_b; both sides decide on the
    kernel's h."""
    dims, block, kappa = (8, 8, 8, 8), (4, 4, 4, 4), 0.156
    geom = lattice.Geometry(dims, block)
    ctx = ps.psms_create(dims, block, kappa, 1)
    ps.psms_gauge_init(ctx, 0, 0.5, SEED + 3)
    ps.psms_gauge_sweep(ctx, 0, ps.ACTIVE_ALL, 3, 2, 5.3, SEED, 1 << 40)
    U = get_links(ctx, 0)
    p = _params(8)
    p["ys"] = 40.0
    ps.psms_mlp_params(ctx, _flat(p))
    q = _rounded(p)
    step = 11
    Up, _, _ = gauge.domain_sweep(U, geom, 5.3, 1, 1, SEED, step << 20)
    z = mlp.pair_features(U, Up, geom).astype(np.float32)
    hd = torch.zeros(geom.n_blocks, dtype=torch.float32, device="cuda")
    ps.psms_mlp_predict(ctx, torch.from_numpy(z).cuda(), geom.n_blocks, hd)
    h_dev = hd.cpu().numpy().astype(np.float64)
    r = ps.psms_filter_step(ctx, 0, beta0=5.3, n_iter=1, n_or=1, n_block=2, n_global=1, tol=1e-13,
                            inner_prec=ps.PREC_F32, seed=SEED, step=step, learned=True)
    prm = ofilter.FilterParams(kappa=kappa, beta0=5.3, n_iter=1, n_or=1, n_block=2, n_global=1, tol=1e-13,
                               learned=q)
    # both sides decide on the h the device computed inside the step
    h_step = ps.psms_filter_record(ctx, ps.REC_H)
    assert np.abs(h_step - h_dev).max() <= 1e-3 * max(1.0, np.abs(h_dev).max())
    U2, rec = ofilter.filter_step(U, geom, prm, SEED, step, h_override=h_step)
    assert r["n_accept_learned"] == int(rec["passed_learned"].sum())
    assert 0 < r["n_accept_learned"] < geom.n_blocks
    assert np.array_equal(r["accept_block"], rec["accept_block"])
    passed = rec["passed_learned"]
    assert np.abs(r["delta_block"][passed] - rec["delta_block"][passed]).max() < 1e-8
    assert r["accept_global"] == rec["accept_global"]
    assert np.abs(get_links(ctx, 0) - U2).max() < 1e-12
    # features the device computed inside the step equal the oracle's (h agrees)
    h_ref = mlp.antisym_rounded(q, z.astype(np.float64))
    assert np.linalg.norm(h_dev - h_ref) <= 2e-3 * np.linalg.norm(h_ref)
