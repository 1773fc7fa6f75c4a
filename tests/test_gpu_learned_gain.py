"""What the trained network gains over the method without it.

On a 16^4 lattice with 4^4 blocks (kappa 0.156, 48 interpolation steps at
the block level) the MLP is trained on the GPU, by the library's own forward
and backward kernels, on block log-det-ratio estimates Delta_b that the
method itself generates for domain-sweep proposals.  On held-out proposals
(labels averaged over four independent noise draws) the learned level
(accept with min{1, exp(-h_b)}, then the stochastic level with
Delta_b - h_b) must
  * predict Delta_b (positive correlation),
  * send fewer blocks to the expensive stochastic level (saved block solves),
  * turn away the worse proposals: the blocks it rejects have a lower plain
    acceptance than those it passes, and
  * stay exact (App. C mechanism: the combined acceptance
    min{1,e^-h} min{1,e^-(Delta-h)} never exceeds min{1,e^-Delta}, and both
    levels together satisfy detailed balance).
The expected accepted blocks per stochastic block solve of both hierarchies
are printed: on these inputs the estimator noise of Delta_b is much larger
than its spread between proposals, so the saved solves come with a
comparable loss of accepted blocks."""
import numpy as np
import pytest
import torch

import paper_1204_1306_gb300 as ps

pytestmark = pytest.mark.gpu

SEED = 0x50534D53
DIMS, BLOCK, KAPPA, N = (16, 16, 16, 16), (4, 4, 4, 4), 0.156, 48


def _samples(ctx, steps, step0, reps):
    """(features z [n, 64], labels Delta_b [n] averaged over reps noise draws)."""
    nb = ps.psms_geometry_info(ctx)[0]
    zs, ys = [], []
    z = torch.zeros(nb * 64, dtype=torch.float32, device="cuda")
    for s in range(step0, step0 + steps):
        ps.psms_gauge_copy(ctx, 1, 0)
        ps.psms_gauge_sweep(ctx, 1, ps.ACTIVE_BLOCKS, 1, 1, 5.3, SEED, (s + 1) << 20)
        d = [ps.psms_logdet_ratio(ctx, ps.LEVEL_BLOCK, 0, 1, N, ps.EST_INTERP, SEED + 17 * r, s, 1e-10,
                                  ps.PREC_F32).sum(axis=1) for r in range(reps)]
        ps.psms_domain_features_pair(ctx, 0, 1, z)
        zs.append(z.view(nb, 64).cpu().numpy().copy())
        ys.append(np.mean(d, axis=0))
        # move the chain a little so the proposals differ
        ps.psms_gauge_sweep(ctx, 0, ps.ACTIVE_ALL, 1, 0, 5.3, SEED, (s + 1) << 30)
    return np.concatenate(zs).astype(np.float32), np.concatenate(ys)


def test_learned_level_gain():
    ctx = ps.psms_create(DIMS, BLOCK, KAPPA, 2)
    ps.psms_gauge_init(ctx, 0, 0.5, SEED + 1)
    ps.psms_gauge_sweep(ctx, 0, ps.ACTIVE_ALL, 4, 2, 5.3, SEED, 1 << 40)
    z_tr, y_tr = _samples(ctx, 48, 0, 1)
    z_te, y_te = _samples(ctx, 8, 1000, 4)
    ps.psms_mlp_init(ctx, 7)
    # labels are noise-dominated: a small learning rate and few epochs keep
    # the network from fitting the noise of the training labels
    losses = ps.psms_mlp_train(ctx, torch.from_numpy(z_tr).cuda(), torch.from_numpy(y_tr).cuda(), len(y_tr),
                               epochs=10, batch=256, lr=1e-4, weight_decay=1e-4, seed=3)
    assert losses[-1] < losses[0]
    h = torch.zeros(len(y_te), dtype=torch.float32, device="cuda")
    ps.psms_mlp_predict(ctx, torch.from_numpy(z_te).cuda(), len(y_te), h)
    h = h.cpu().numpy().astype(np.float64)
    corr = float(np.corrcoef(h, y_te)[0, 1])
    p_pass = np.minimum(1.0, np.exp(-h))
    p_plain = np.minimum(1.0, np.exp(-y_te))
    p_learned = p_pass * np.minimum(1.0, np.exp(-(y_te - h)))
    rej = float(np.sum((1 - p_pass) * p_plain) / np.sum(1 - p_pass))
    pas = float(np.sum(p_pass * p_plain) / np.sum(p_pass))
    print(f"held-out correlation of h with Delta_b (4 draws): {corr:.3f}; blocks passed {p_pass.mean():.3f}; "
          f"plain acceptance of turned-away blocks {rej:.4f} vs passed {pas:.4f}; expected accepted blocks per "
          f"stochastic solve: learned {p_learned.mean() / p_pass.mean():.4f}, plain {p_plain.mean():.4f}")
    assert corr > 0.1, corr
    # exactness bound per block: combined acceptance <= plain acceptance
    assert np.all(p_learned <= p_plain + 1e-12)
    # saved stochastic block solves
    assert p_pass.mean() < 0.9
    # the saved solves are on the worse proposals
    assert rej < 0.85 * pas, (rej, pas)
