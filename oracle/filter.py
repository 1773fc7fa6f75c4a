"""Accept/reject and one hierarchical filter step.  TEST INFRASTRUCTURE ONLY.

Eq. (hierarchy): after the proposal T_0, level i accepts with
min{1, exp(-Delta_i)}; the result of a level is the proposal of the next.
Decision rule: one uniform u per decision (draw map TAG_ACCEPT, counter =
filter step, level, block), accept iff Delta <= 0 or u < exp(-Delta).

One step of the 3-level filter (domain sweep -> block det ratios -> global
Schur det ratio), Sec. 3, Eq. (4step) with one DD level and App. C:

 0) U' = domain sweep of U on the active links at coupling beta0
    (sweep ids start at step * 2^20).
 1) per block b: Delta_b = beta_block * dS_w,b + sum_i (|M_{b,i} xi|^2 - |xi|^2)
    accepted block by block (blocks with extent >= 3, where the active links
    of different blocks share no plaquette and the proposal factorises); for
    smaller blocks one decision on sum_b Delta_b.  Rejected blocks get their
    old links back.
 2) Delta = beta_global * dS_w + Schur estimate between U and the field after
    level 1; accepted or rejected as a whole.
 3) the field is translated by a random vector (after the global step).

dS_w,b attributes every plaquette to the block of the first changed link in
the order (x,mu), (x+mu,nu), (x+nu,mu), (x,nu); a link belongs to the block of
its starting site.
"""
from dataclasses import dataclass

import numpy as np

from . import philox
from .estimator import block_level, global_level
from .gauge import domain_sweep, plaquette_field, wilson_action
from .lattice import gauge_shift

SWEEP_STRIDE = 1 << 20


@dataclass
class FilterParams:
    kappa: float
    beta0: float
    n_iter: int = 1
    n_or: int = 0
    n_block: int = 4
    n_global: int = 4
    beta_block: float = 0.0
    beta_global: float = 0.0
    tol: float = 1e-13
    global_level: bool = True
    learned: object = None   # MLP parameter dict (oracle.mlp) or None
    gauge_fix: object = None  # relative gauge fixing (Sec. 4.2): dict of oracle.gaugefix parameters, or None
    exact_block: bool = False    # block level with exact determinants (Sec. 3, dense LU) instead of Eq. (staccN)
    block_det_coef: float = 1.0  # coefficient of the exact block-determinant action at the block level (Table 1: 1.644)
    beta_global_blockdet: float = 0.0  # coefficient of the block-determinant action at the global level (App. C)
    hyp_level: object = None  # (beta_1^(0), beta_1^(1)) of the HYP plaquette level (App. C), or None
    beta_block_hyp: float = 0.0   # beta^(1) of the block level (HYP action)
    beta_global_hyp: float = 0.0  # beta^(1) of the global level (HYP action)


def gaussian_acceptance(sigma2):
    """Eq. (acceptance): <P_acc> = erfc(sqrt(Sigma^2 / 8)) for Gaussian Delta."""
    from math import erfc, sqrt
    return erfc(sqrt(sigma2 / 8.0))


def stochastic_acceptance(lam):
    """App. A.2: acceptance probability of one stochastic step in terms of the
    eigenvalues lam of M^dagger M,
    P_acc = sum_i min(1, 1/lam_i) prod_{j != i} (lam_i - 1)/(lam_i - lam_j),
    evaluated with 60-digit mpmath arithmetic (distinct eigenvalues)."""
    import mpmath as mp
    with mp.workdps(60):
        lam = [mp.mpf(float(x)) for x in lam]
        tot = mp.mpf(0)
        for i, li in enumerate(lam):
            term = min(mp.mpf(1), 1 / li)
            for j, lj in enumerate(lam):
                if j != i:
                    term *= (li - 1) / (li - lj)
            tot += term
        return float(tot)


def accept(delta, u):
    return bool(delta <= 0.0 or u < np.exp(-delta))


def block_logdet(U, geom, b, kappa):
    """ln|det D_b(U)| of one Dirichlet block, by LU of its dense matrix."""
    from .dirac import apply_D_open, dense_matrix, extract_block
    Ub = extract_block(U, geom, b)
    Db = dense_matrix(lambda v: apply_D_open(Ub, v, kappa), geom.Vb, geom.block + (4, 3))
    return float(np.linalg.slogdet(Db)[1])


def exact_block_change(U, Up, geom, kappa, blocks=None):
    """Change of the block-determinant action S_b = -2 ln|det D_b| (so that
    exp(-S_b) is the block's fermion weight |det D_b|^2, N_f = 2) from U to
    U' for the listed blocks (others 0): the exact value of the stochastic
    block estimate, E[exp(-Delta_b)] = exp(-dS_b) (Sec. 4.1)."""
    out = np.zeros(geom.n_blocks)
    # a block whose links did not change keeps its determinant: 0 exactly
    moved = np.zeros(geom.n_blocks, dtype=bool)
    np.logical_or.at(moved, geom.block_index.ravel(), np.any(U != Up, axis=(-1, -2, -3)).ravel())
    for b in (range(geom.n_blocks) if blocks is None else blocks):
        if moved[b]:
            out[b] = 2.0 * (block_logdet(U, geom, b, kappa) - block_logdet(Up, geom, b, kappa))
    return out


def per_block_action_change(U, Up, geom):
    """dS_w,b (without beta) for every block, by plaquette attribution."""
    changed = np.any(U != Up, axis=(-1, -2))              # [dims, 4]
    out = np.zeros(geom.n_blocks)
    bidx = geom.block_index
    for mu in range(4):
        for nu in range(mu + 1, 4):
            d = -(np.real(np.trace(plaquette_field(Up, mu, nu), axis1=-2, axis2=-1))
                  - np.real(np.trace(plaquette_field(U, mu, nu), axis1=-2, axis2=-1))) / 3.0
            cands = [
                (changed[..., mu], bidx),
                (gauge_shift(changed[..., nu], mu, +1), gauge_shift(bidx, mu, +1)),
                (gauge_shift(changed[..., mu], nu, +1), gauge_shift(bidx, nu, +1)),
                (changed[..., nu], bidx),
            ]
            owner = np.full(geom.dims, -1)
            for ch, bi in cands:
                sel = (owner < 0) & ch
                owner[sel] = bi[sel]
            m = owner >= 0
            out += np.bincount(owner[m], weights=d[m], minlength=geom.n_blocks)
    return out


def _merge(U, V, acc_b, geom, active):
    """U with the active links of accepted blocks taken from V."""
    out = U.copy()
    sel = acc_b[geom.block_index][..., None] & active
    out[sel] = V[sel]
    return out


def filter_step(U, geom, prm, seed, step, h_override=None, gf_override=None, proposal=None, translate=True):
    """Returns (new field, record dict).

    With prm.exact_block the block level uses block_det_coef times the exact
    change of the block-determinant action (dense LU, the paper's own method
    for blocks of up to about 6^4 sites, Sec. 3) instead of the stochastic
    estimate; that action may then also enter the global level with
    beta_global_blockdet (Tables 1 and 2 carry coefficients at both levels,
    summing to the action's target 1; App. C allows coefficients only on
    exactly evaluated actions).

    With prm.hyp_level = (b0, b1) a parametrised level precedes the others
    (App. C; the first filter of Tables 1 and 2): per block,
    Delta_b = b0 dS_w,b + b1 dS_HYP,b with the block HYP action of
    oracle.hyp, counter (step, 5, b), or one decision on the sum for blocks
    of extent <= 2 (counter (step, 5, 0)).  Blocks it rejects keep their
    links and skip the later block levels.  beta_block_hyp and
    beta_global_hyp add the HYP action's change to the block and global
    levels.

    With prm.learned (per-block decisions only) a learned level precedes
    level 1: h_b from the surrogate (or h_override, the values a device
    computed, so that both sides decide on the same numbers), accepted with
    min{1, exp(-h_b)} (counter (step, 3, b)); level 1 runs on the blocks that
    passed, with Delta_b - h_b.

    With prm.gauge_fix the interpolations of levels 1 and 2 (Eq. (gfparam))
    run between U^{g_1} and U'^{g_2} (Sec. 4.2): level 1 between the fixed
    pair of (U, U'), level 2 between U and the field after level 1, whose
    fixed pair equals the level-1 one on accepted blocks and (U, U) on the
    others (the blocks decouple).  gf_override = (g_1, g_2) replaces the
    oracle's own transformations with a device's.

    proposal: an external proposal (differing from U on active links only,
    drawn symmetrically) replaces the domain sweep; translate=False skips
    the translation (both for detailed-balance tests of the chain)."""
    active = geom.active_links()
    if proposal is None:
        Unew, _, failed = domain_sweep(U, geom, prm.beta0, prm.n_iter, prm.n_or, seed, step * SWEEP_STRIDE)
    else:
        Unew, failed = np.array(proposal, copy=True), 0
    per_block = min(geom.block) >= 3
    passed = np.ones(geom.n_blocks, dtype=bool)
    use_hyp = prm.hyp_level is not None or prm.beta_block_hyp != 0.0 or prm.beta_global_hyp != 0.0
    ds_hyp = None
    rec_hyp = None
    if use_hyp:
        from .hyp import block_hyp_change
        ds_hyp = block_hyp_change(U, Unew, geom)
    if prm.hyp_level is not None:
        b0, b1 = prm.hyp_level
        d_hyp = b0 * per_block_action_change(U, Unew, geom) + b1 * ds_hyp
        if per_block:
            passed = np.array([accept(d_hyp[b], philox.accept_uniform(seed, step, 5, b)) for b in range(geom.n_blocks)])
        else:
            passed = np.full(geom.n_blocks, accept(d_hyp.sum(), philox.accept_uniform(seed, step, 5, 0)))
        rec_hyp = (d_hyp, passed.copy())
    h = np.zeros(geom.n_blocks)
    rec_h = None
    if prm.learned is not None:
        from .mlp import antisym, pair_features
        assert per_block
        z = pair_features(U, Unew, geom)
        h = antisym(prm.learned, z) if h_override is None else np.asarray(h_override, dtype=np.float64)
        passed = passed & np.array([accept(h[b], philox.accept_uniform(seed, step, 3, b))
                                    for b in range(geom.n_blocks)])
        rec_h = h

    E0, EN = U, Unew
    rec_gf = None
    if prm.gauge_fix is not None or gf_override is not None:
        from .gaugefix import relative_gauge_fix, transform
        if gf_override is None:
            g1, g2, rec_gf = relative_gauge_fix(U, Unew, geom, **prm.gauge_fix)
        else:
            g1, g2 = gf_override
        E0, EN = transform(U, g1), transform(Unew, g2)

    blocks = [b for b in range(geom.n_blocks) if passed[b]]
    d_blk = np.zeros(geom.n_blocks)
    ds_det = None
    if prm.exact_block or prm.beta_global_blockdet != 0.0:
        ds_det = exact_block_change(U, Unew, geom, prm.kappa)
    if blocks and prm.exact_block:
        d_blk[blocks] = prm.block_det_coef * ds_det[blocks]
    elif blocks:
        d_all = block_level(E0, EN, geom, prm.kappa, prm.n_block, seed, step, tol=prm.tol, blocks=blocks)
        d_blk[blocks] = d_all[blocks].sum(axis=1)
    if prm.beta_block != 0.0:
        d_blk = d_blk + prm.beta_block * per_block_action_change(U, Unew, geom)
    if prm.beta_block_hyp != 0.0:
        d_blk = d_blk + prm.beta_block_hyp * ds_hyp
    d_blk = d_blk - h
    if per_block:
        acc_b = np.array([passed[b] and accept(d_blk[b], philox.accept_uniform(seed, step, 1, b))
                          for b in range(geom.n_blocks)])
    else:
        a = bool(passed.all()) and accept(d_blk.sum(), philox.accept_uniform(seed, step, 1, 0))
        acc_b = np.full(geom.n_blocks, a)

    Umid = _merge(U, Unew, acc_b, geom, active)

    rec = {"delta_block": d_blk, "accept_block": acc_b, "hb_failed": failed, "h": rec_h,
           "passed_learned": passed, "gauge_fix": rec_gf,
           "delta_hyp": None if rec_hyp is None else rec_hyp[0],
           "accept_hyp": None if rec_hyp is None else rec_hyp[1]}
    Ufin = Umid
    if prm.global_level:
        G0, GN = U, Umid
        if E0 is not U:
            G0, GN = _merge(U, E0, acc_b, geom, active), _merge(U, EN, acc_b, geom, active)
        dg = global_level(G0, GN, geom, prm.kappa, prm.n_global, seed, step, tol=prm.tol)
        d = float(dg.sum())
        if prm.beta_global != 0.0:
            d += prm.beta_global * (wilson_action(Umid) - wilson_action(U))
        if prm.beta_global_hyp != 0.0:
            d += prm.beta_global_hyp * float(ds_hyp[acc_b].sum())
        if prm.beta_global_blockdet != 0.0:
            d += prm.beta_global_blockdet * float(ds_det[acc_b].sum())
        acc_g = accept(d, philox.accept_uniform(seed, step, 2, 0))
        rec["delta_global"] = d
        rec["delta_global_terms"] = dg
        rec["accept_global"] = acc_g
        if not acc_g:
            Ufin = U.copy()
    s = philox.shift_vector(seed, step, geom.dims) if translate else (0, 0, 0, 0)
    rec["shift"] = s
    return geom.translate(Ufin, s), rec
