"""Pins of the recursive domain decomposition (Eq. (ddrec)) and of the
filter step with one level of recursion (Eq. (4step)).

The outer-block Schur complement is compared with dense linear algebra
(determinant factorisation by LU, Schur complements from dense blocks); its
projector with a rank counted from the block geometry and with the range of
the dense hopping matrix; the 5-step filter with the 4-step one it reduces
to when every outer block is a single inner block."""
from math import comb

import numpy as np
import pytest

from oracle import dirac, estimator, filter as ofilter, gauge, lattice, recursive
from oracle.gamma import GAMMA
from tests import seeded

K = 0.156


def _perturbed(U, eps, seed):
    g = np.random.default_rng(seed)
    om = g.standard_normal(U.shape[:-2] + (8,))
    return U @ gauge.expm_i_hermitian(gauge.hermitian_generators(om), eps)


def _dense(apply, shape):
    return dirac.dense_matrix(apply, int(np.prod(shape[:4])), shape)


def _proj_dense(P, sel):
    """Dense matrix of the site-diagonal spin projector on the sites `sel`."""
    Ps = P.reshape(-1, 4, 4)[sel.reshape(-1)]
    n = Ps.shape[0]
    out = np.zeros((n * 12, n * 12), dtype=np.complex128)
    for k in range(n):
        out[k * 12:(k + 1) * 12, k * 12:(k + 1) * 12] = np.kron(Ps[k], np.eye(3))
    return out


def _range_basis(P):
    """Orthonormal basis of range(P) as spinor fields on the array of P."""
    basis = []
    for x in np.ndindex(*P.shape[:4]):
        w, v = np.linalg.eigh(P[x])
        for k in np.nonzero(w > 0.5)[0]:
            for c in range(3):
                f = np.zeros(P.shape[:4] + (4, 3), dtype=np.complex128)
                f[x][:, c] = v[:, k]
                basis.append(f)
    return basis


# --- geometry ------------------------------------------------------------------

def test_nested_geometry():
    nest = recursive.Nested((8, 8, 8, 8), (4, 4, 4, 4), (2, 2, 2, 2))
    # with even counts the colouring inside an outer block is the lattice's
    # checkerboard of inner blocks
    col_in = nest.inner.block_colours()
    col_sub = nest.sub_colours().reshape(nest.sub.nb)
    for b, I in enumerate(np.ndindex(*nest.inner.nb)):
        assert col_in[b] == col_sub[tuple(i % 2 for i in I)]
        O = tuple(i // 2 for i in I)
        assert nest.outer_of_inner[b] == np.ravel_multi_index(O, nest.outer.nb)
    recursive.Nested((4, 4, 2, 2), (2, 2, 1, 1), (2, 1, 1, 1))   # one inner block per direction is allowed
    with pytest.raises(ValueError):
        recursive.Nested((12, 4, 4, 4), (4, 2, 2, 2), (2, 1, 1, 1))   # three outer blocks in time
    with pytest.raises(ValueError):
        recursive.Nested((12, 4, 4, 4), (6, 2, 2, 2), (2, 1, 1, 1))   # three inner blocks per outer block
    with pytest.raises(ValueError):
        recursive.Nested((8, 8, 8, 8), (4, 4, 4, 4), (3, 4, 4, 4))


@pytest.mark.parametrize("l", [2, 3, 4])
def test_sub_projector_rank_by_counting(l):
    """Outer blocks of (2l)^4 in inner blocks of l^4 (l = 4: the 8^4 / 4^4
    decomposition of Sec. 5): each inner block has one inner face per
    direction; a site on k of them lies in C(4,k) (l-1)^(4-k) places, and
    carries spin rank 2 for k = 1, 4 for k >= 2 (Sec. 4.4).  Eight of the
    sixteen inner blocks are black."""
    nest = recursive.Nested((4 * l,) * 4, (2 * l,) * 4, (l,) * 4)
    P = recursive.sub_projector(nest)
    assert np.abs(P @ P - P).max() < 1e-15
    assert np.abs(P - np.conj(np.swapaxes(P, -1, -2))).max() < 1e-15
    rank = int(round(np.real(np.trace(P, axis1=-2, axis2=-1)).sum())) * 3
    one = comb(4, 1) * (l - 1) ** 3
    many = sum(comb(4, k) * (l - 1) ** (4 - k) for k in range(2, 5))
    assert rank == 8 * 3 * (2 * one + 4 * many)
    if l == 4:
        assert rank == 11616


def _all_faces_projector(nest):
    """The projector a torus of inner blocks would have: every face of a
    black inner block counted, including faces on the outer boundary (a
    plausible mistake the next pin must catch)."""
    sub = nest.sub
    P = np.zeros(sub.dims + (4, 4), dtype=np.complex128)
    single = np.zeros_like(P)
    nface = np.zeros(sub.dims, dtype=int)
    for mu in range(4):
        for mask, sgn in ((sub.local[mu] == sub.block[mu] - 1, 1.0), (sub.local[mu] == 0, -1.0)):
            nface += mask
            single[mask] = 0.5 * (np.eye(4) + sgn * GAMMA[mu])
    black = sub.black_sites()
    P[black & (nface == 1)] = single[black & (nface == 1)]
    P[black & (nface >= 2)] = np.eye(4)
    return P


@pytest.mark.parametrize("outer,inner", [((4, 4, 2, 2), (2, 2, 2, 2)), ((6, 4, 2, 2), (3, 2, 2, 2)),
                                         ((4, 2, 2, 2), (2, 2, 1, 1))])
def test_sub_projector_is_the_range_seen_by_D_wb(outer, inner):
    """D_wb (1 - P_b) = 0 and D_wb is injective on range(P_b), from the dense
    hopping matrix of the outer block's Dirichlet operator.  Where faces on
    the outer boundary exist, counting them too gives a projector on which
    D_wb is not injective."""
    dims = tuple(2 * o for o in outer)
    nest = recursive.Nested(dims, outer, inner)
    Ub = seeded.gauge_field(outer, 71)
    D = _dense(lambda v: dirac.apply_D_open(Ub, v, K), outer + (4, 3))
    Dblk = _dense(lambda v: recursive.apply_D_outer(Ub, v, K, nest.sub, "block"), outer + (4, 3))
    black = nest.sub.black_sites()
    bl = np.repeat(black.reshape(-1), 12)
    A = (D - Dblk)[np.ix_(~bl, bl)]                       # D_wb, dense
    Pb, Pall = recursive.sub_projector(nest), _all_faces_projector(nest)
    cases = [(Pb, True)] + ([(Pall, False)] if np.abs(Pb - Pall).max() > 0 else [])
    assert len(cases) == (2 if inner[2] == 2 else 1)
    for P, minimal in cases:
        Pm = _proj_dense(P, black)
        assert np.abs(A @ (np.eye(len(Pm)) - Pm)).max() < 1e-14
        r = int(round(np.real(np.trace(Pm))))
        sv = np.linalg.svd(A @ Pm, compute_uv=False)
        assert (int(np.sum(sv > 1e-10)) == r) == minimal


def test_sub_operator_pieces_dense():
    """'block' + 'inter' = D_b; 'block' is block diagonal in the inner blocks,
    each diagonal block the inner Dirichlet operator; 'inter' only joins
    inner blocks of different colour."""
    outer, inner = (4, 4, 2, 2), (2, 2, 1, 1)
    nest = recursive.Nested((8, 8, 4, 4), outer, inner)
    Ub = seeded.gauge_field(outer, 72)
    D = _dense(lambda v: dirac.apply_D_open(Ub, v, K), outer + (4, 3))
    Db = _dense(lambda v: recursive.apply_D_outer(Ub, v, K, nest.sub, "block"), outer + (4, 3))
    Di = _dense(lambda v: recursive.apply_D_outer(Ub, v, K, nest.sub, "inter"), outer + (4, 3))
    assert np.abs(Db + Di - D).max() < 1e-15
    bidx = np.repeat(nest.sub.block_index.reshape(-1), 12)
    col = np.repeat(nest.sub.colour.reshape(-1), 12)
    assert np.all(Db[bidx[:, None] != bidx[None, :]] == 0)
    assert np.all(Di[col[:, None] == col[None, :]] == 0)
    for b in range(nest.sub.n_blocks):
        sel = bidx == b
        ref = _dense(lambda v: dirac.apply_D_open(dirac.extract_block(Ub, nest.sub, b), v, K), inner + (4, 3))
        assert np.abs(Db[np.ix_(sel, sel)] - ref).max() < 1e-15


# --- Eq. (ddrec) ---------------------------------------------------------------

@pytest.mark.parametrize("dims,outer,inner", [((8, 4, 4, 4), (4, 2, 2, 2), (2, 1, 1, 1)),
                                              ((4, 4, 2, 2), (2, 2, 1, 1), (2, 1, 1, 1))])
def test_ddrec_factorisation(dims, outer, inner):
    """log|det D_b| = sum_b' log|det D_b'| + log|det (1 - P_b Q_b)| on range(P_b),
    with the Schur factor from the oracle's (1 - P_b Q_b) applied to a basis
    of range(P_b) and the determinants by dense LU."""
    nest = recursive.Nested(dims, outer, inner)
    U = gauge.generate_links(dims, 0.4, 73)
    P = recursive.sub_projector(nest)
    basis = _range_basis(P)
    B = np.stack([f.reshape(-1) for f in basis], axis=1)
    for b in (0, nest.outer.n_blocks - 1):
        Ub = dirac.extract_block(U, nest.outer, b)
        lhs = np.linalg.slogdet(_dense(lambda v: dirac.apply_D_open(Ub, v, K), outer + (4, 3)))[1]
        blocks = sum(np.linalg.slogdet(_dense(
            lambda v: dirac.apply_D_open(dirac.extract_block(Ub, nest.sub, c), v, K), inner + (4, 3)))[1]
            for c in range(nest.sub.n_blocks))
        S = np.stack([recursive.sub_one_minus_PQ(Ub, f, nest, K, P, 1e-14).reshape(-1) for f in basis], axis=1)
        schur = np.linalg.slogdet(B.conj().T @ S)[1]
        assert abs(lhs - blocks - schur) < 1e-10 * abs(lhs), (lhs, blocks, schur)
        assert abs(schur) > 1e-3          # the Schur factor is not trivial here


def test_ddrec_with_global_schur():
    """Eqs. (ddfactor) and (ddrec) together on a whole lattice:
    log|det D| = sum_b' log|det D_b'| + sum_b log|det D-hat_b| + log|det D-hat|,
    D-hat the global Schur complement of the outer blocks (dense)."""
    dims, outer, inner = (4, 4, 2, 2), (2, 2, 1, 1), (2, 1, 1, 1)
    nest = recursive.Nested(dims, outer, inner)
    U = gauge.generate_links(dims, 0.4, 74)
    D = _dense(lambda v: dirac.apply_D(U, v, K), dims + (4, 3))
    lhs = np.linalg.slogdet(D)[1]
    bl = np.repeat(nest.outer.black_sites().reshape(-1), 12)
    Dbb, Dbw = D[np.ix_(bl, bl)], D[np.ix_(bl, ~bl)]
    Dwb, Dww = D[np.ix_(~bl, bl)], D[np.ix_(~bl, ~bl)]
    glob = np.linalg.slogdet(np.eye(bl.sum()) - np.linalg.solve(Dbb, Dbw @ np.linalg.solve(Dww, Dwb)))[1]
    inner_dets = sum(np.linalg.slogdet(_dense(
        lambda v: dirac.apply_D_open(dirac.extract_block(U, nest.inner, c), v, K), inner + (4, 3)))[1]
        for c in range(nest.inner.n_blocks))
    P = recursive.sub_projector(nest)
    basis = _range_basis(P)
    B = np.stack([f.reshape(-1) for f in basis], axis=1)
    subs = 0.0
    for b in range(nest.outer.n_blocks):
        Ub = dirac.extract_block(U, nest.outer, b)
        S = np.stack([recursive.sub_one_minus_PQ(Ub, f, nest, K, P, 1e-14).reshape(-1) for f in basis], axis=1)
        subs += np.linalg.slogdet(B.conj().T @ S)[1]
    assert abs(lhs - inner_dets - subs - glob) < 1e-9 * abs(lhs)


# --- stage-2 estimator -----------------------------------------------------------

@pytest.mark.parametrize("mode,N", [("independent", 2), ("interp", 3)])
def test_sub_estimator_equals_dense(mode, N):
    """Delta_{b,i} = |(1 - P_b Q_b(U_{i+1}))^-1 (1 - P_b Q_b(U_i)) xi|^2 - |xi|^2
    against dense Schur complements of the outer blocks (the inverse through
    a dense solve, not through Eq. (inverseschur))."""
    dims, outer, inner = (8, 4, 4, 4), (4, 2, 2, 2), (2, 1, 1, 1)
    nest = recursive.Nested(dims, outer, inner)
    U = gauge.generate_links(dims, 0.3, 75)
    Up = _perturbed(U, 0.3, 76)
    blocks = [0, 9, 15]
    d = recursive.sub_level(U, Up, nest, K, N, seed=5, counter=9, mode=mode, blocks=blocks)
    P = recursive.sub_projector(nest)
    black = nest.sub.black_sites()
    bl = np.repeat(black.reshape(-1), 12)
    Pm = _proj_dense(P, black)
    I = np.eye(len(Pm))

    def one_minus_PQ(Fb):
        Dm = _dense(lambda v: dirac.apply_D_open(Fb, v, K), outer + (4, 3))
        Dbb, Dbw = Dm[np.ix_(bl, bl)], Dm[np.ix_(bl, ~bl)]
        Dwb, Dww = Dm[np.ix_(~bl, bl)], Dm[np.ix_(~bl, ~bl)]
        return I - Pm @ np.linalg.solve(Dbb, Dbw @ np.linalg.solve(Dww, Dwb))

    for i in range(N):
        Ua, Ub = estimator.pair(U, Up, i, N, mode)
        xi_all = estimator.noise(nest.outer, 5, 9, recursive.LEVEL_SUB, i)
        for b in range(nest.outer.n_blocks):
            if b not in blocks:
                assert np.isnan(d[b, i])
                continue
            xi = estimator.project(P, dirac.extract_block(xi_all, nest.outer, b)).reshape(-1)[bl]
            A = one_minus_PQ(dirac.extract_block(Ua, nest.outer, b))
            Bm = one_minus_PQ(dirac.extract_block(Ub, nest.outer, b))
            y = np.linalg.solve(Bm, A @ xi)
            ref = np.vdot(y, y).real - np.vdot(xi, xi).real
            assert abs(d[b, i] - ref) < 1e-9 * max(1.0, abs(ref)), (b, i, d[b, i], ref)


def test_sub_estimator_closed_form():
    """Sec. 4.1 for the outer-block Schur level: over many noise draws
    E[Delta] = Tr(M^dag M - 1) and E[e^-Delta] = det(M^dag M)^-1 =
    |det D-hat_b(U') / det D-hat_b(U)|^-2 (from dense LU of D_b and D_b')."""
    dims, outer, inner = (4, 4, 2, 2), (2, 2, 1, 1), (2, 1, 1, 1)
    nest = recursive.Nested(dims, outer, inner)
    U = gauge.generate_links(dims, 0.3, 77)
    Up = _perturbed(U, 0.08, 78)
    b = 5
    n = 1500
    d = np.array([recursive.sub_level(U, Up, nest, K, 1, seed=11, counter=c, mode="independent", blocks=[b])[b, 0]
                  for c in range(n)])

    def logdet_schur(F):
        Fb = dirac.extract_block(F, nest.outer, b)
        full = np.linalg.slogdet(_dense(lambda v: dirac.apply_D_open(Fb, v, K), outer + (4, 3)))[1]
        parts = sum(np.linalg.slogdet(_dense(
            lambda v: dirac.apply_D_open(dirac.extract_block(Fb, nest.sub, c), v, K), inner + (4, 3)))[1]
            for c in range(nest.sub.n_blocks))
        return full - parts

    log_target = -2.0 * (logdet_schur(U) - logdet_schur(Up))   # log det(M^dag M)^-1
    ew = np.exp(-d)
    se = ew.std(ddof=1) / np.sqrt(n)
    assert abs(ew.mean() - np.exp(log_target)) < 5 * se + 1e-12, (ew.mean(), np.exp(log_target), se)
    assert abs(np.log(ew.mean()) - log_target) < 0.05


# --- the 5-step filter ---------------------------------------------------------------

def test_filter_reduces_to_one_level_without_inner_split():
    """Outer blocks made of a single inner block: P_b = 0, stage 2 accepts
    every block with Delta_b = 0, and the step equals the filter without
    recursion (same proposal, decisions, estimates and final field)."""
    dims, B = (4, 4, 4, 4), (2, 2, 2, 2)
    nest = recursive.Nested(dims, B, B)
    assert np.all(recursive.sub_projector(nest) == 0)
    U = gauge.generate_links(dims, 0.5, 79)
    prm = dict(kappa=K, beta0=5.3, n_iter=1, n_or=1, n_block=2, n_global=2, beta_block=0.3, beta_global=-0.1,
               tol=1e-12)
    for step in range(2):
        U5, r5 = recursive.filter_step(U, nest, recursive.RecursiveParams(n_sub=2, beta_sub=0.7, **prm), 9, step)
        U4, r4 = ofilter.filter_step(U, lattice.Geometry(dims, B), ofilter.FilterParams(**prm), 9, step)
        assert np.array_equal(r5["accept_block"], r4["accept_block"])
        assert np.abs(r5["delta_block"] - r4["delta_block"]).max() < 1e-12
        assert np.all(r5["accept_sub"])
        assert r5["accept_global"] == r4["accept_global"]
        assert abs(r5["delta_global"] - r4["delta_global"]) < 1e-12
        assert r5["shift"] == r4["shift"]
        assert np.array_equal(U5, U4)
        U = U5


def test_filter_step_bookkeeping():
    """External proposal on the active links, per-block decisions at both
    block stages (inner blocks 3^4): the links that survive stage 2 are those
    of inner blocks accepted at stage 1 whose outer block was accepted at
    stage 2; unchanged outer blocks carry Delta_b = 0; the stage-2 estimate
    is the one between U and the field after stage 1, plus beta_sub times
    the action change of the accepted inner blocks.  (The global level and
    the final merge are covered by the reduction to the filter without
    recursion; they are switched off here to keep the test short.)"""
    dims, outer, inner = (12, 6, 6, 6), (6, 3, 3, 3), (3, 3, 3, 3)
    nest = recursive.Nested(dims, outer, inner)
    U = gauge.generate_links(dims, 0.4, 80)
    act = nest.inner.active_links()
    Up = np.where(act[..., None, None], _perturbed(U, 0.25, 81), U)
    prm = recursive.RecursiveParams(kappa=K, beta0=5.3, n_block=2, n_sub=2, tol=1e-10, beta_block=1.5,
                                    beta_sub=0.5, global_level=False)
    ds = ofilter.per_block_action_change(U, Up, nest.inner)
    for step in range(2):
        Unew, rec = recursive.filter_step(U, nest, prm, 3, step, proposal=Up, translate=False)
        acc_in, acc_out, acc2 = rec["accept_block"], rec["accept_sub"], rec["accept_after_sub"]
        assert 0 < acc_in.sum() < len(acc_in)
        assert np.array_equal(acc2, acc_in & acc_out[nest.outer_of_inner])
        changed = np.bincount(nest.outer_of_inner, weights=acc_in, minlength=nest.outer.n_blocks) > 0
        assert np.array_equal(rec["changed_sub"], changed)
        assert np.all(rec["delta_sub"][~changed] == 0) and np.all(acc_out[~changed])
        U1 = np.where((acc_in[nest.inner.block_index][..., None] & act)[..., None, None], Up, U)
        check = np.nonzero(changed)[0][:2]
        est = recursive.sub_level(U, U1, nest, K, 2, 3, step, tol=1e-10, blocks=check).sum(axis=1)
        ref = est[check] + 0.5 * np.bincount(nest.outer_of_inner, weights=ds * acc_in,
                                             minlength=nest.outer.n_blocks)[check]
        assert np.abs(rec["delta_sub"][check] - ref).max() < 1e-8
        keep = acc2[nest.inner.block_index][..., None] & act
        assert np.array_equal(Unew, np.where(keep[..., None, None], Up, U))


def test_filter_with_learned_level_and_gauge_fixing_reduces_to_one_level():
    """The same reduction with the learned level and relative gauge fixing
    switched on (3^4 blocks: per-block decisions and one interior point per
    block): decisions, h, estimates and the final field equal those of the
    filter without recursion."""
    from oracle import mlp
    dims, B = (6, 6, 6, 6), (3, 3, 3, 3)
    nest = recursive.Nested(dims, B, B)
    U = gauge.generate_links(dims, 0.5, 83)
    p = mlp.init_params(5)
    p["ys"] = 3.0
    gf = dict(max_iter=50)
    prm = dict(kappa=K, beta0=5.3, n_iter=1, n_or=1, n_block=2, n_global=2, tol=1e-12, learned=p, gauge_fix=gf)
    seen_h = False
    for step in range(2):
        U5, r5 = recursive.filter_step(U, nest, recursive.RecursiveParams(n_sub=2, **prm), 9, step)
        U4, r4 = ofilter.filter_step(U, lattice.Geometry(dims, B), ofilter.FilterParams(**prm), 9, step)
        assert np.array_equal(r5["passed_learned"], r4["passed_learned"])
        assert np.abs(r5["h"] - r4["h"]).max() < 1e-12
        seen_h |= bool(np.any(r5["h"] != 0))
        assert np.array_equal(r5["accept_block"], r4["accept_block"])
        assert np.abs(r5["delta_block"] - r4["delta_block"]).max() < 1e-12
        assert r5["accept_global"] == r4["accept_global"]
        assert abs(r5["delta_global"] - r4["delta_global"]) < 1e-12
        assert np.array_equal(U5, U4)
        U = U5
    assert seen_h
