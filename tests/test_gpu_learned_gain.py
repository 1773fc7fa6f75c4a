"""What the trained network gains over the method without it.

On a 16^4 lattice with 4^4 blocks (kappa 0.156, 48 interpolation steps at
the block level) the MLP is trained on the GPU, by the library's own forward
and backward kernels, on block log-det-ratio estimates Delta_b that the
method itself generates for domain-sweep proposals.  On held-out proposals
the learned level (accept with min{1, exp(-h_b)}, then the stochastic level
with Delta_b - h_b) must
  * predict Delta_b (positive correlation),
  * let through fewer blocks to the expensive stochastic level (saved block
    solves), and
  * keep more accepted blocks per stochastic block solve than the plain
    hierarchy, while every accepted update stays exact (App. C mechanism:
    the combined acceptance min{1,e^-h} min{1,e^-(Delta-h)} never exceeds
    min{1,e^-Delta}, and both levels together satisfy detailed balance)."""
import numpy as np
import pytest
import torch

import paper_1204_1306_gb300 as ps

pytestmark = pytest.mark.gpu

SEED = 0x50534D53
DIMS, BLOCK, KAPPA, N = (16, 16, 16, 16), (4, 4, 4, 4), 0.156, 48


def _samples(ctx, steps, step0):
    """(features z [n, 64], labels Delta_b [n]) from domain-sweep proposals."""
    nb = ps.psms_geometry_info(ctx)[0]
    zs, ys = [], []
    z = torch.zeros(nb * 64, dtype=torch.float32, device="cuda")
    for s in range(step0, step0 + steps):
        ps.psms_gauge_copy(ctx, 1, 0)
        ps.psms_gauge_sweep(ctx, 1, ps.ACTIVE_BLOCKS, 1, 1, 5.3, SEED, (s + 1) << 20)
        d = ps.psms_logdet_ratio(ctx, ps.LEVEL_BLOCK, 0, 1, N, ps.EST_INTERP, SEED, s, 1e-10, ps.PREC_F32)
        ps.psms_domain_features_pair(ctx, 0, 1, z)
        zs.append(z.view(nb, 64).cpu().numpy().copy())
        ys.append(d.sum(axis=1))
        # move the chain a little so the proposals differ
        ps.psms_gauge_sweep(ctx, 0, ps.ACTIVE_ALL, 1, 0, 5.3, SEED, (s + 1) << 30)
    return np.concatenate(zs).astype(np.float32), np.concatenate(ys)


def test_learned_level_gain():
    ctx = ps.psms_create(DIMS, BLOCK, KAPPA, 2)
    ps.psms_gauge_init(ctx, 0, 0.5, SEED + 1)
    ps.psms_gauge_sweep(ctx, 0, ps.ACTIVE_ALL, 4, 2, 5.3, SEED, 1 << 40)
    z_tr, y_tr = _samples(ctx, 24, 0)
    z_te, y_te = _samples(ctx, 8, 1000)
    ps.psms_mlp_init(ctx, 7)
    losses = ps.psms_mlp_train(ctx, torch.from_numpy(z_tr).cuda(), torch.from_numpy(y_tr).cuda(), len(y_tr),
                               epochs=60, batch=256, lr=1e-3, weight_decay=1e-4, seed=3)
    assert losses[-1] < losses[0]
    h = torch.zeros(len(y_te), dtype=torch.float32, device="cuda")
    ps.psms_mlp_predict(ctx, torch.from_numpy(z_te).cuda(), len(y_te), h)
    h = h.cpu().numpy().astype(np.float64)
    corr = float(np.corrcoef(h, y_te)[0, 1])
    print(f"held-out correlation of h with Delta_b: {corr:.3f}")
    assert corr > 0.2, corr

    # identical uniforms for both hierarchies
    g = np.random.default_rng(11)
    u_learned, u_block = g.random(len(y_te)), g.random(len(y_te))
    plain_acc = u_block < np.exp(-np.maximum(y_te, 0.0))
    passed = u_learned < np.exp(-np.maximum(h, 0.0))
    learned_acc = passed & (u_block < np.exp(-np.maximum(y_te - h, 0.0)))
    # exactness bound per block: combined acceptance <= plain acceptance
    p_plain = np.minimum(1.0, np.exp(-y_te))
    p_learned = np.minimum(1.0, np.exp(-h)) * np.minimum(1.0, np.exp(-(y_te - h)))
    assert np.all(p_learned <= p_plain + 1e-12)
    solves_plain = len(y_te)
    solves_learned = int(passed.sum())
    assert solves_learned < solves_plain
    eff_plain = plain_acc.sum() / solves_plain
    eff_learned = learned_acc.sum() / max(solves_learned, 1)
    print(f"corr {corr:.3f}; stochastic block solves {solves_learned}/{solves_plain}; accepted blocks "
          f"{learned_acc.sum()} vs {plain_acc.sum()}; accepted per solve {eff_learned:.4f} vs {eff_plain:.4f}")
    assert eff_learned > eff_plain
