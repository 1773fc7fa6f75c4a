"""Recursive domain decomposition (Eq. (ddrec)) and the filter step with one
level of recursion (Eq. (4step); the 5-step PSMS algorithm of Sec. 5).
TEST INFRASTRUCTURE ONLY: imported by tests, the package's smoke check and
the benchmark's CPU baseline, never by the product path.

Nested blocks.  The lattice is tiled by outer blocks b of extent B_mu (the
blocks of the global Schur step), and every outer block by inner blocks b'
of extent l_mu (the smallest blocks, whose determinants enter stage 1);
l_mu divides B_mu and B_mu divides L_mu.  The global step needs an even
number of outer blocks in every direction (Sec. 3).  Inside an outer block
the inner blocks are coloured by the parity of their coordinates within the
outer block; this needs an even number of inner blocks per direction, or
exactly one (then no hop in that direction joins two inner blocks of the
same outer block).  With even counts everywhere this colouring is the
lattice's own checkerboard of inner blocks.

Eq. (ddrec): det D_b = prod_{b' in C_b} det D_b' * det D-hat_b, where D_b is
the Dirichlet operator of outer block b (Eq. (Dw) with the hops that leave b
dropped), split like Eq. (domdec) into its black and white inner blocks,
D_b = [[D_bb, D_bw], [D_wb, D_ww]], and
D-hat_b = 1 - D_bb^-1 D_bw D_ww^-1 D_wb.  D-hat_b depends on the links inside
b only (it obeys Dirichlet boundary conditions, Sec. 3).

Projector P_b (Eq. (detschur) restated for an outer block): on a site of a
black inner block, the spin projector onto range((1 + gamma_mu)/2) for every
+mu face of its inner block that is not on the +mu face of the outer block,
range((1 - gamma_mu)/2) for every such -mu face, the whole spin space for
two or more such faces, and zero elsewhere.  A face on the outer block's
boundary carries no hop, so it adds nothing to P_b;
det(1 - Q_b) = det(1 - P_b Q_b) on range(P_b) as in Sec. 4.4.

Stage 2 (Eq. (staccN) for D-hat_b): Delta_b = sum_i |M_{b,i} xi_i|^2 - |xi_i|^2,
M_{b,i} = (1 - P_b Q_b(U_{i+1}))^-1 (1 - P_b Q_b(U_i)) on range(P_b), with
Eq. (inverseschur) applied to D_b:
(1 - P_b Q_b)^-1 s = s - P_b [D_b^-1 (0, D_wb s)]_black.
Noise: one field on the whole lattice per i (draw map TAG_NOISE, stream
(LEVEL_SUB << 32) | i); outer block b takes its own sites, projected by P_b.
Accept/reject counter: (step, LEVEL_SUB, b).
"""
from dataclasses import dataclass

import numpy as np

from . import philox
from .dirac import apply_D_open, extract_block, mass_from_kappa
from .dirac import _colour, _colour_dag, _spin
from .estimator import block_level, global_level, noise, pair, project, solve_blocks
from .filter import SWEEP_STRIDE, _merge, accept, per_block_action_change
from .gamma import GAMMA, ONE4
from .gauge import domain_sweep, wilson_action
from .lattice import Geometry
from .linalg import cgnr, norm2

LEVEL_SUB = 4


class Nested:
    """Outer blocks (extent `outer`) tiled by inner blocks (extent `inner`)."""

    def __init__(self, dims, outer, inner):
        self.dims = tuple(int(d) for d in dims)
        self.outer = Geometry(self.dims, outer)
        self.inner = Geometry(self.dims, inner)
        self.sub = Geometry(tuple(int(b) for b in outer), inner)   # one outer block, as a lattice
        if not self.outer.colouring_ok:
            raise ValueError("the global Schur step needs an even number of outer blocks per direction")
        for n in self.sub.nb:
            if n != 1 and n % 2:
                raise ValueError("an outer block needs one or an even number of inner blocks per direction")
        # outer block of every inner block (inner block index order)
        first = [tuple(B[m] * self.inner.block[m] for m in range(4))
                 for B in np.ndindex(*self.inner.nb)]
        self.outer_of_inner = np.array([self.outer.block_index[x] for x in first])

    def sub_colours(self):
        """colour (0 black, 1 white) of the inner blocks of one outer block."""
        return self.sub.block_colours()


def sub_projector(nest):
    """P_b per site of one outer block, shape outer + (4, 4) (the same for
    every outer block)."""
    sub = nest.sub
    B = sub.dims
    P = np.zeros(B + (4, 4), dtype=np.complex128)
    single = np.zeros(B + (4, 4), dtype=np.complex128)
    nface = np.zeros(B, dtype=int)
    for mu in range(4):
        plus = (sub.local[mu] == sub.block[mu] - 1) & (sub.x[mu] != B[mu] - 1)
        minus = (sub.local[mu] == 0) & (sub.x[mu] != 0)
        for mask, sgn in ((plus, +1.0), (minus, -1.0)):
            nface += mask
            single[mask] = 0.5 * (ONE4 + sgn * GAMMA[mu])
    black = sub.black_sites()
    P[black & (nface == 1)] = single[black & (nface == 1)]
    P[black & (nface >= 2)] = ONE4
    return P


def apply_D_outer(Ub, psi, kappa, sub, mode="full", dagger=False):
    """D_b of one outer block (array [B0..B3, ...], Dirichlet in every
    direction) and its pieces, with the inner blocks of `sub`:
    'full'  -- D_b (= apply_D_open);
    'block' -- the inner-block Dirichlet operators D_b' (D_bb + D_ww);
    'inter' -- hops between different inner blocks (D_bw + D_wb), no
               diagonal term."""
    m0 = mass_from_kappa(kappa)
    s = -1.0 if dagger else 1.0
    out = np.zeros_like(psi) if mode == "inter" else (4.0 + m0) * psi
    for mu in range(4):
        Pm = ONE4 - s * GAMMA[mu]
        Pp = ONE4 + s * GAMMA[mu]
        Umu = Ub[..., mu, :, :]
        n = psi.shape[mu]
        lo = tuple(slice(0, n - 1) if m == mu else slice(None) for m in range(4))
        hi = tuple(slice(1, n) if m == mu else slice(None) for m in range(4))
        fwd = np.zeros_like(psi)
        bwd = np.zeros_like(psi)
        fwd[lo] = _colour(Umu[lo], _spin(Pm, psi[hi]))
        bwd[hi] = _colour_dag(Umu[lo], _spin(Pp, psi[lo]))
        if mode != "full":
            keep_f = sub.fwd_intra(mu)
            keep_b = sub.bwd_intra(mu)
            if mode == "inter":
                keep_f, keep_b = ~keep_f, ~keep_b
            fwd = fwd * keep_f[..., None, None]
            bwd = bwd * keep_b[..., None, None]
        out = out - 0.5 * (fwd + bwd)
    return out


def solve_outer(Ub, rhs, kappa, tol):
    """D_b x = rhs on one outer block."""
    x, _, _ = cgnr(lambda v: apply_D_open(Ub, v, kappa),
                   lambda v: apply_D_open(Ub, v, kappa, dagger=True), rhs, tol=tol)
    return x


def sub_one_minus_PQ(Ub, xi, nest, kappa, P, tol):
    """(1 - P_b Q_b) xi on one outer block, xi supported on black inner blocks."""
    sub = nest.sub
    black = sub.black_sites()[..., None, None]
    white = ~black
    col = nest.sub_colours()
    blacks = [b for b in range(sub.n_blocks) if col[b] == 0]
    whites = [b for b in range(sub.n_blocks) if col[b] == 1]
    t1 = apply_D_outer(Ub, xi * black, kappa, sub, "inter") * white    # D_wb xi
    t2 = solve_blocks(Ub, t1, sub, kappa, whites, tol)                 # D_ww^-1
    t3 = apply_D_outer(Ub, t2, kappa, sub, "inter") * black            # D_bw
    t4 = solve_blocks(Ub, t3, sub, kappa, blacks, tol)                 # D_bb^-1
    return xi - project(P, t4)


def sub_inv_one_minus_PQ(Ub, s, nest, kappa, P, tol):
    """(1 - P_b Q_b)^-1 s = s - P_b [D_b^-1 (0, D_wb s)]_black (Eq. (inverseschur)
    for the outer block)."""
    sub = nest.sub
    black = sub.black_sites()[..., None, None]
    y = apply_D_outer(Ub, s * black, kappa, sub, "inter") * ~black
    z = solve_outer(Ub, y, kappa, tol)
    return s - project(P, z * black)


def sub_level(U, Up, nest, kappa, N, seed, counter, tol=1e-13, mode="interp", blocks=None):
    """Delta contributions [n_outer, N] of stage 2: entry (b, i) =
    |M_{b,i} xi_i|^2 - |xi_i|^2.  Outer blocks not listed are NaN."""
    geo = nest.outer
    if blocks is None:
        blocks = range(geo.n_blocks)
    blocks = list(blocks)
    P = sub_projector(nest)
    out = np.full((geo.n_blocks, N), np.nan)
    for i in range(N):
        Ua, Ub = pair(U, Up, i, N, mode)
        xi_all = noise(geo, seed, counter, LEVEL_SUB, i)
        for b in blocks:
            xi = project(P, extract_block(xi_all, geo, b))
            v = sub_one_minus_PQ(extract_block(Ua, geo, b), xi, nest, kappa, P, tol)
            w = sub_inv_one_minus_PQ(extract_block(Ub, geo, b), v, nest, kappa, P, tol)
            out[b, i] = norm2(w) - norm2(xi)
    return out


@dataclass
class RecursiveParams:
    kappa: float
    beta0: float
    n_iter: int = 1
    n_or: int = 0
    n_block: int = 4
    n_sub: int = 4
    n_global: int = 4
    beta_block: float = 0.0
    beta_sub: float = 0.0
    beta_global: float = 0.0
    tol: float = 1e-13
    global_level: bool = True
    learned: object = None    # MLP parameter dict (oracle.mlp) of the learned level before stage 1, or None
    gauge_fix: object = None  # relative gauge fixing of the inner blocks (dict of oracle.gaugefix parameters), or None


def filter_step(U, nest, prm, seed, step, proposal=None, translate=True, skip_unchanged=False, h_override=None,
                gf_override=None):
    """One step of the filter with one level of recursion (Eq. (4step)).
    Returns (new field, record dict).

     0) U' = domain sweep of U on the active links of the inner blocks at
        beta0 (sweep ids from step * 2^20), or the external `proposal`;
     1) per inner block b': Delta_b' = beta_block dS_w,b' + block estimate
        (counter (step, 1, b')), as in the filter without recursion:
        decisions per inner block when every inner extent is >= 3, else one
        decision on the sum (counter (step, 1, 0));
     2) per outer block b holding an accepted inner block whose links
        changed in stage 1:
        Delta_b = beta_sub sum_{b' in b} dS_w,b' + stage-2 estimate between U
        and the field after stage 1 (counter (step, LEVEL_SUB, b)); outer
        blocks without a change keep Delta_b = 0 and are not drawn.  Per
        outer block under the same extent rule as stage 1, else one decision
        on the sum (counter (step, LEVEL_SUB, 0)).  A rejected outer block
        gets all its old links back;
     3) Delta = beta_global dS_w + global Schur estimate with the outer
        blocks (counter (step, 2, 0)) between U and the field after stage 2;
     4) translation by a random vector.

    skip_unchanged: stage 1 estimates only the inner blocks whose links
    changed and gives the others Delta = 0, the exact value of their
    estimate (M = 1); for external proposals that move few blocks.

    prm.learned (per-inner-block decisions only): the learned level of
    oracle.filter precedes stage 1 -- h_b of the inner block (or
    h_override), accepted with min{1, exp(-h_b)} (counter (step, 3, b));
    stage 1 runs on the blocks that passed with Delta_b - h_b.
    prm.gauge_fix (or gf_override = (g_1, g_2)): every interpolation runs
    between relatively gauge-fixed endpoints (Sec. 4.2) of the inner
    blocks' interiors: stage 1 between U^{g_1} and U'^{g_2}; stage 2 and
    the global level between the fixed pair of (U, field after the stage
    before), which (the inner blocks decouple) is the stage-1 pair merged
    on the accepted inner blocks (U elsewhere)."""
    inner, outer = nest.inner, nest.outer
    active = inner.active_links()
    if proposal is None:
        Unew, _, failed = domain_sweep(U, inner, prm.beta0, prm.n_iter, prm.n_or, seed, step * SWEEP_STRIDE)
    else:
        Unew, failed = np.array(proposal, copy=True), 0
    per_block = min(inner.block) >= 3

    link_changed = np.any(U != Unew, axis=(-1, -2))            # [dims, 4]
    block_moved = np.zeros(inner.n_blocks, dtype=bool)
    np.logical_or.at(block_moved, inner.block_index.ravel(), link_changed.any(axis=-1).ravel())

    # learned level (before stage 1)
    passed = np.ones(inner.n_blocks, dtype=bool)
    h = np.zeros(inner.n_blocks)
    if prm.learned is not None:
        from .mlp import antisym, pair_features
        assert per_block
        h = (antisym(prm.learned, pair_features(U, Unew, inner)) if h_override is None
             else np.asarray(h_override, dtype=np.float64))
        passed = np.array([accept(h[b], philox.accept_uniform(seed, step, 3, b)) for b in range(inner.n_blocks)])

    # relatively gauge-fixed endpoints of the interpolations
    E0, EN = U, Unew
    if prm.gauge_fix is not None or gf_override is not None:
        from .gaugefix import relative_gauge_fix, transform
        g1, g2 = (relative_gauge_fix(U, Unew, inner, **prm.gauge_fix)[:2] if gf_override is None
                  else gf_override)
        E0, EN = transform(U, g1), transform(Unew, g2)
    fixed = E0 is not U

    # stage 1: inner blocks
    todo = [b for b in range(inner.n_blocks) if passed[b] and (block_moved[b] or not skip_unchanged)]
    d_in = np.zeros(inner.n_blocks)
    if todo:
        d_in[todo] = block_level(E0, EN, inner, prm.kappa, prm.n_block, seed, step, tol=prm.tol,
                                 blocks=todo)[todo].sum(axis=1)
    ds_in = per_block_action_change(U, Unew, inner) if (prm.beta_block or prm.beta_sub) else np.zeros(inner.n_blocks)
    d_in = d_in + prm.beta_block * ds_in - h
    if per_block:
        acc_in = np.array([passed[b] and accept(d_in[b], philox.accept_uniform(seed, step, 1, b))
                           for b in range(inner.n_blocks)])
    else:
        acc_in = np.full(inner.n_blocks, accept(d_in.sum(), philox.accept_uniform(seed, step, 1, 0)))
    U1 = _merge(U, Unew, acc_in, inner, active)

    # stage 2: Schur complements of the outer blocks.  An outer block changes
    # when one of its accepted inner blocks changed a link; det D-hat_b of
    # the others is unchanged (it depends on the links inside b only).
    changed = np.zeros(outer.n_blocks, dtype=bool)
    for b in range(inner.n_blocks):
        if acc_in[b] and block_moved[b]:
            changed[nest.outer_of_inner[b]] = True
    d_sub = np.zeros(outer.n_blocks)
    blocks = [b for b in range(outer.n_blocks) if changed[b]]
    if blocks:
        S0, S1 = U, U1
        if fixed:
            S0, S1 = _merge(U, E0, acc_in, inner, active), _merge(U, EN, acc_in, inner, active)
        d_all = sub_level(S0, S1, nest, prm.kappa, prm.n_sub, seed, step, tol=prm.tol, blocks=blocks)
        d_sub[blocks] = d_all[blocks].sum(axis=1)
    if prm.beta_sub != 0.0:
        d_sub = d_sub + prm.beta_sub * np.bincount(nest.outer_of_inner, weights=ds_in * acc_in,
                                                   minlength=outer.n_blocks)
    if per_block:
        acc_out = np.array([(not changed[b]) or accept(d_sub[b], philox.accept_uniform(seed, step, LEVEL_SUB, b))
                            for b in range(outer.n_blocks)])
    else:
        a = (not changed.any()) or accept(d_sub.sum(), philox.accept_uniform(seed, step, LEVEL_SUB, 0))
        acc_out = np.full(outer.n_blocks, a)
    acc2 = acc_in & acc_out[nest.outer_of_inner]
    U2 = _merge(U, Unew, acc2, inner, active)

    rec = {"delta_block": d_in, "accept_block": acc_in, "delta_sub": d_sub, "accept_sub": acc_out,
           "changed_sub": changed, "accept_after_sub": acc2, "hb_failed": failed, "h": h,
           "passed_learned": passed}
    Ufin = U2
    if prm.global_level:
        G0, G1 = U, U2
        if fixed:
            G0, G1 = _merge(U, E0, acc2, inner, active), _merge(U, EN, acc2, inner, active)
        dg = global_level(G0, G1, outer, prm.kappa, prm.n_global, seed, step, tol=prm.tol)
        d = float(dg.sum())
        if prm.beta_global != 0.0:
            d += prm.beta_global * (wilson_action(U2) - wilson_action(U))
        acc_g = accept(d, philox.accept_uniform(seed, step, 2, 0))
        rec["delta_global"] = d
        rec["delta_global_terms"] = dg
        rec["accept_global"] = acc_g
        if not acc_g:
            Ufin = U.copy()
    s = philox.shift_vector(seed, step, nest.dims) if translate else (0, 0, 0, 0)
    rec["shift"] = s
    return outer.translate(Ufin, s), rec
