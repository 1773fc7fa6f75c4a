"""Detailed balance of the filter chain (App. A): the hierarchy of the
library (block level with N interpolation steps, then the global Schur level)
run as a finite-state Markov chain.  K gauge fields that differ only on the
active links, a symmetric external proposal (uniform over the other fields)
and no translation: the stationary distribution must be
|det D(U_k)|^2 / sum_j |det D(U_j)|^2, with the determinants from dense LU
of the oracle's D.  Plus the parity of one externally proposed step with the
oracle."""
import numpy as np
import pytest

import paper_1204_1306_gb300 as ps
from oracle import dirac, filter as ofilter, gauge, lattice
from tests.gpu_util import get_links, set_links

pytestmark = pytest.mark.gpu

SEED = 0x50534D53
DIMS, BLOCK, KAPPA = (4, 4, 4, 4), (2, 2, 2, 2), 0.14


def _configs(k_states, eps):
    """U_0 with its active links multiplied by exp(i eps H_k), k = 0..K-1."""
    geom = lattice.Geometry(DIMS, BLOCK)
    act = geom.active_links()
    U0 = gauge.generate_links(DIMS, 0.3, 11)
    g = np.random.default_rng(3)
    out = []
    for _ in range(k_states):
        om = g.standard_normal(U0.shape[:5] + (8,))
        R = gauge.expm_i_hermitian(gauge.hermitian_generators(om), eps)
        out.append(np.where(act[..., None, None], U0 @ R, U0))
    return geom, out


def test_external_proposal_parity():
    geom, (U, Up) = _configs(2, 0.35)
    ctx = ps.psms_create(DIMS, BLOCK, KAPPA, 2)
    set_links(ctx, 0, U)
    set_links(ctx, 1, Up)
    prm = dict(beta0=5.3, n_block=4, n_global=4, tol=1e-13)
    for step in range(3):
        r = ps.psms_filter_step(ctx, 0, inner_prec=ps.PREC_F64, seed=SEED, step=step, proposal_field=1,
                                translate=False, **prm)
        U, rec = ofilter.filter_step(U, geom, ofilter.FilterParams(kappa=KAPPA, **prm), SEED, step,
                                     proposal=Up, translate=False)
        assert r["accept_global"] == rec["accept_global"]
        assert np.array_equal(r["accept_block"], rec["accept_block"])
        assert abs(r["delta_block_sum"] - rec["delta_block"].sum()) < 1e-8
        assert abs(r["delta_global"] - rec["delta_global"]) < 1e-8
        assert tuple(r["shift"]) == (0, 0, 0, 0)
        assert np.abs(get_links(ctx, 0) - U).max() < 1e-12
    assert np.array_equal(get_links(ctx, 1), Up)  # the proposal slot is untouched


def test_filter_chain_detailed_balance():
    """eps = 0.15 perturbations (log-weight spread about 0.5) and N = 64
    interpolation steps at both levels keep the estimator noise near one
    unit, so the chain moves (acceptance about one half)."""
    k_states, n_steps, n_batches = 3, 4000, 20
    geom, configs = _configs(k_states, 0.15)
    logw = np.array([2.0 * np.linalg.slogdet(
        dirac.dense_matrix(lambda v, U=U: dirac.apply_D(U, v, KAPPA), geom.V, DIMS + (4, 3)))[1] for U in configs])
    pi = np.exp(logw - logw.max())
    pi /= pi.sum()
    ctx = ps.psms_create(DIMS, BLOCK, KAPPA, k_states + 1)
    for k, U in enumerate(configs):
        set_links(ctx, k + 1, U)
    ps.psms_gauge_copy(ctx, 0, 1)
    state, visits, moves = 0, [], 0
    rng = np.random.default_rng(5)
    for step in range(n_steps):
        j = (state + 1 + int(rng.integers(k_states - 1))) % k_states
        r = ps.psms_filter_step(ctx, 0, beta0=5.3, n_block=64, n_global=64, tol=1e-10, inner_prec=ps.PREC_F32,
                                seed=SEED, step=step, proposal_field=j + 1, translate=False)
        if r["accept_global"] and r["n_accept_blocks"] > 0:
            state, moves = j, moves + 1
        visits.append(state)
        if step % 1000 == 999:
            assert np.array_equal(get_links(ctx, 0), configs[state])
    visits = np.array(visits)
    acc = moves / n_steps
    freq = np.array([(visits == k).mean() for k in range(k_states)])
    batches = visits.reshape(n_batches, -1)
    bf = np.array([[(b == k).mean() for k in range(k_states)] for b in batches])
    se = bf.std(axis=0, ddof=1) / np.sqrt(n_batches)
    z = (freq - pi) / np.maximum(se, 1e-3)
    print(f"acceptance {acc:.3f}; exact pi {np.round(pi, 4)}; chain {np.round(freq, 4)}; "
          f"batch-means s.e. {np.round(se, 4)}; z {np.round(z, 2)}")
    assert acc > 0.15
    assert np.all(np.abs(z) < 4.0), z


def test_block_chain_detailed_balance_learned_gauge_fixed():
    """App. A for the block part of the benchmarked hierarchy: the learned
    level (a fixed random antisymmetric network, App. C's auxiliary action)
    and then the stochastic block level with Delta_b - h_b between
    relatively gauge-fixed endpoints (Sec. 4.2), per-block decisions (4^4
    blocks), no global level.  Two blocks of an 8^4 lattice have three
    states each, differing on their active links; the symmetric proposal
    moves each of them to one of its two other states; no other link ever
    changes.  The blocks are independent chains whose stationary
    distributions must be |det D_b(U_k)|^2 / sum_j |det D_b(U_j)|^2, with
    the determinants from the oracle's dense LU of the block operator."""
    from oracle import mlp
    dims, block, kappa = (8, 8, 8, 8), (4, 4, 4, 4), 0.156
    geom = lattice.Geometry(dims, block)
    act = geom.active_links()
    varying, k_states, n_steps, n_batches = (5, 10), 3, 3000, 20
    U0 = gauge.generate_links(dims, 0.3, 21)
    g = np.random.default_rng(22)
    sel = {b: (geom.block_index == b)[..., None] & act for b in varying}
    states = {}
    for b in varying:
        states[b] = []
        for _ in range(k_states):
            om = g.standard_normal(U0.shape[:5] + (8,))
            R = gauge.expm_i_hermitian(gauge.hermitian_generators(om), 0.15)
            states[b].append(np.where(sel[b][..., None, None], U0 @ R, U0))

    def field(s):
        F = U0.copy()
        for b in varying:
            F[sel[b]] = states[b][s[b]][sel[b]]
        return F

    pis = {}
    for b in varying:
        logw = np.array([2.0 * ofilter.block_logdet(states[b][k], geom, b, kappa) for k in range(k_states)])
        p = np.exp(logw - logw.max())
        pis[b] = p / p.sum()
    ctx = ps.psms_create(dims, block, kappa, 2)
    q = mlp.init_params(17)
    q["ys"] = 150.0    # h of order one on these nearby states
    flat = np.concatenate([q["W1"].ravel(), q["b1"], q["W2"].ravel(), q["b2"], q["w3"], [q["b3"]], q["mu"],
                           q["sigma"], [q["ys"]]]).astype(np.float32)
    ps.psms_mlp_params(ctx, flat)
    s = {b: 0 for b in varying}
    set_links(ctx, 0, field(s))
    rng = np.random.default_rng(23)
    visits, moves, h_seen = [], 0, 0.0
    for step in range(n_steps):
        t = {b: (s[b] + 1 + int(rng.integers(k_states - 1))) % k_states for b in varying}
        set_links(ctx, 1, field(t))
        r = ps.psms_filter_step(ctx, 0, beta0=5.3, n_block=16, n_global=1, global_level=False, tol=1e-10,
                                inner_prec=ps.PREC_F32, seed=SEED, step=step, proposal_field=1, translate=False,
                                learned=True, gauge_fix={"prec": ps.PREC_F32})
        if step < 50:
            h_seen = max(h_seen, float(np.abs(ps.psms_filter_record(ctx, ps.REC_H)[list(varying)]).max()))
        for b in varying:
            if r["accept_block"][b]:
                s[b] = t[b]
                moves += 1
        visits.append([s[b] for b in varying])
        if step % 1000 == 999:
            assert np.array_equal(get_links(ctx, 0), field(s))
    visits = np.array(visits)
    acc = moves / (n_steps * len(varying))
    assert acc > 0.15
    assert h_seen > 0.05          # the learned level is not idle
    for col, b in enumerate(varying):
        v = visits[:, col]
        freq = np.array([(v == k).mean() for k in range(k_states)])
        bf = np.array([[(w == k).mean() for k in range(k_states)] for w in v.reshape(n_batches, -1)])
        se = bf.std(axis=0, ddof=1) / np.sqrt(n_batches)
        z = (freq - pis[b]) / np.maximum(se, 1e-3)
        print(f"block {b}: acceptance {acc:.3f}; exact pi {np.round(pis[b], 4)}; chain {np.round(freq, 4)}; "
              f"z {np.round(z, 2)}")
        assert np.all(np.abs(z) < 4.0), z
