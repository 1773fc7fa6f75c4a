"""Pins of the HYP-smeared links and the block HYP plaquette action (App. C,
Sec. 5): the projection against a direct maximisation, the first smearing
step against the pinned staple sum, gauge, translation, axis-permutation
and reflection covariance, the hypercube locality of the construction by
enumeration, and the block factorisation of the action."""
import itertools

import numpy as np
from scipy.optimize import minimize

from oracle import gauge, hyp, lattice
from oracle.gauge import dag
from tests import seeded


def _field(dims, seed, eps=0.6):
    return gauge.generate_links(dims, eps, seed)


def _su3_exp(omega):
    return gauge.expm_i_hermitian(gauge.hermitian_generators(omega), 1.0)


# --- projection -----------------------------------------------------------------

def test_projection_properties():
    """SU(3) output, SU(3) and positive multiples of it fixed, gauge
    covariance Proj[G M H^dag] = G Proj[M] H^dag."""
    M = np.stack([seeded.complex_matrix(3, s) for s in range(20)])
    W = hyp.project_su3(M)
    assert np.abs(W @ dag(W) - np.eye(3)).max() < 1e-14
    assert np.abs(np.linalg.det(W) - 1).max() < 1e-14
    S = seeded.haar_su3((20,), 3)
    assert np.abs(hyp.project_su3(S) - S).max() < 1e-14
    assert np.abs(hyp.project_su3(2.5 * S) - S).max() < 1e-14
    G, H = seeded.haar_su3((20,), 4), seeded.haar_su3((20,), 5)
    assert np.abs(hyp.project_su3(G @ M @ dag(H)) - G @ W @ dag(H)).max() < 1e-13


def test_projection_maximises_overlap_when_det_is_positive():
    """For det M > 0 the projection is the SU(3) matrix maximising
    Re Tr(X^dag M) (polar decomposition): no SU(3) direction improves it."""
    for s in range(5):
        M = seeded.complex_matrix(3, 10 + s)
        M = M * np.exp(-1j * np.angle(np.linalg.det(M)) / 3)
        W = hyp.project_su3(M)
        best = np.real(np.trace(dag(W) @ M))
        f = lambda om: -np.real(np.trace(dag(W @ _su3_exp(om)) @ M))
        r = minimize(f, 0.3 * np.random.default_rng(s).standard_normal(8), method="BFGS")
        assert -r.fun <= best + 1e-10
        X = seeded.haar_su3((200,), 20 + s)
        assert np.all(np.real(np.trace(dag(X) @ M, axis1=-2, axis2=-1)) <= best + 1e-12)


# --- smearing ---------------------------------------------------------------------

def test_cold_field_and_su3():
    dims = (4, 4, 4, 4)
    one = np.broadcast_to(np.eye(3, dtype=np.complex128), dims + (4, 3, 3)).copy()
    assert np.abs(hyp.smear(one) - one).max() < 1e-15
    V = hyp.smear(_field(dims, 7))
    assert np.abs(V @ dag(V) - np.eye(3)).max() < 1e-14
    assert np.abs(np.linalg.det(V) - 1).max() < 1e-14
    U = _field(dims, 7)
    assert np.abs(hyp.smear(U, (0.0, 0.0, 0.0)) - U).max() < 1e-14


def test_first_step_alone_is_staple_smearing():
    """alpha = (a1, 0, 0): V = Proj[(1 - a1) U + a1/6 (sum of the six
    staples)], the staple sum from the heatbath's staple routine."""
    dims = (4, 4, 4, 4)
    U = _field(dims, 8)
    V = hyp.smear(U, (0.75, 0.0, 0.0))
    for mu in range(4):
        ref = hyp.project_su3(0.25 * U[..., mu, :, :] + (0.75 / 6) * dag(gauge.staples(U, mu)))
        assert np.abs(V[..., mu, :, :] - ref).max() < 1e-13


def test_gauge_covariance():
    dims = (4, 4, 4, 4)
    U = _field(dims, 9)
    g = seeded.haar_su3(dims, 10)
    Ug = np.empty_like(U)
    for mu in range(4):
        Ug[..., mu, :, :] = g @ U[..., mu, :, :] @ dag(lattice.gauge_shift(g, mu, +1))
    V, Vg = hyp.smear(U), hyp.smear(Ug)
    for mu in range(4):
        assert np.abs(Vg[..., mu, :, :] - g @ V[..., mu, :, :] @ dag(lattice.gauge_shift(g, mu, +1))).max() < 1e-12


def test_translation_and_axis_permutation():
    dims = (4, 4, 4, 4)
    U = _field(dims, 11)
    V = hyp.smear(U)
    s = (1, 3, 0, 2)
    assert np.abs(hyp.smear(np.roll(U, s, axis=(0, 1, 2, 3))) - np.roll(V, s, axis=(0, 1, 2, 3))).max() < 1e-13
    for perm in ((1, 0, 2, 3), (3, 1, 0, 2), (2, 3, 1, 0)):
        # U'(x', perm[m]) with x'_{perm[m]} = x_m: move axis m to position perm[m]
        inv = np.argsort(perm)
        Up = np.transpose(U, list(inv) + [4, 5, 6])[..., inv, :, :]
        Vp = np.transpose(V, list(inv) + [4, 5, 6])[..., inv, :, :]
        assert np.abs(hyp.smear(Up) - Vp).max() < 1e-13


def test_reflection():
    """x0 -> -x0: U'(Rx, mu) = U(x, mu) for mu != 0 and
    U'(Rx - 0, 0) = U(x, 0)^dag; the fat links transform the same way."""
    dims = (4, 4, 4, 4)
    U = _field(dims, 12)

    def reflect(F):
        G = np.empty_like(F)
        idx = (-np.arange(dims[0])) % dims[0]
        G[idx] = F                                       # G(Rx) = F(x)
        out = G.copy()
        out[..., 0, :, :] = dag(np.roll(G[..., 0, :, :], -1, axis=0))   # out(y,0) = G(y+0,0)^dag
        return out

    assert np.abs(hyp.smear(reflect(U)) - reflect(hyp.smear(U))).max() < 1e-13


def test_hypercube_locality():
    """Changing one thin link changes exactly the fat links that share a
    hypercube with it (enumerated from the definition of the hypercubes
    attached to a link)."""
    dims = (6, 6, 6, 6)
    U = _field(dims, 13)
    V = hyp.smear(U)
    y, nu = (2, 3, 1, 4), 2
    U2 = U.copy()
    U2[y + (nu,)] = U2[y + (nu,)] @ _su3_exp(np.full(8, 0.3))
    changed = np.any(np.abs(hyp.smear(U2) - V) > 1e-12, axis=(-1, -2))
    L = np.array(dims)
    a = np.array(y) % L
    b = (np.array(y) + np.eye(4, dtype=int)[nu]) % L
    expect = np.zeros(dims + (4,), dtype=bool)
    for x in itertools.product(*[range(d) for d in dims]):
        for mu in range(4):
            base = np.array(x)
            trans = [r for r in range(4) if r != mu]
            for signs in itertools.product((1, -1), repeat=3):
                def inside(p):
                    d = (p - base) % L
                    d = np.where(d > L // 2, d - L, d)
                    if d[mu] not in (0, 1):
                        return False
                    return all(d[r] in (0, s) for r, s in zip(trans, signs))
                if inside(a) and inside(b):
                    expect[x + (mu,)] = True
                    break
    assert np.array_equal(changed, expect), (changed.sum(), expect.sum())


# --- block action -------------------------------------------------------------------

def test_block_action_is_intra_block_plaquettes():
    """alpha = 0: S_HYP,b sums (3 - ReTr U_p)/3 over the plaquettes with all
    four corners in b, checked site by site with explicit neighbour indices."""
    geom = lattice.Geometry((6, 6, 6, 6), (3, 3, 3, 3))
    U = _field(geom.dims, 14)
    S = hyp.block_hyp_action(U, geom, (0.0, 0.0, 0.0))
    ref = np.zeros(geom.n_blocks)
    L = geom.dims
    for x in itertools.product(*[range(d) for d in L]):
        for mu, nu in itertools.combinations(range(4), 2):
            xm = list(x); xm[mu] += 1
            xn = list(x); xn[nu] += 1
            xmn = list(xm); xmn[nu] += 1
            corners = [x, xm, xn, xmn]
            bl = {tuple(c[m] // 3 for m in range(4)) for c in corners}
            if len(bl) != 1 or any(c[m] >= L[m] for c in corners for m in range(4)):
                continue
            P = U[x + (mu,)] @ U[tuple(xm) + (nu,)] @ dag(U[tuple(xn) + (mu,)]) @ dag(U[x + (nu,)])
            ref[geom.block_index[x]] += (3 - np.real(np.trace(P))) / 3
    assert np.abs(S - ref).max() < 1e-12


def test_block_action_factorises_over_blocks():
    """With 3^4 blocks, changing the active links of one block changes S_HYP
    of that block only, so the changes of two blocks add; the HYP action on
    all plaquettes of the lattice does not split that way."""
    geom = lattice.Geometry((6, 6, 6, 6), (3, 3, 3, 3))
    U = _field(geom.dims, 15)
    act = geom.active_links()
    R = _su3_exp(0.4 * np.random.default_rng(16).standard_normal(geom.dims + (4, 8)))

    def change(blocks):
        sel = np.isin(geom.block_index, blocks)[..., None] & act
        return np.where(sel[..., None, None], U @ R, U)

    b1, b2 = 0, 1                                    # neighbours along x3
    S0 = hyp.block_hyp_action(U, geom)
    d1 = hyp.block_hyp_action(change([b1]), geom) - S0
    d2 = hyp.block_hyp_action(change([b2]), geom) - S0
    d12 = hyp.block_hyp_action(change([b1, b2]), geom) - S0
    assert np.all(d1[np.arange(geom.n_blocks) != b1] == 0) and d1[b1] != 0
    assert np.all(d2[np.arange(geom.n_blocks) != b2] == 0) and d2[b2] != 0
    assert np.abs(d12 - d1 - d2).max() < 1e-12
    full = lambda F: gauge.wilson_action(hyp.smear(F))
    f0 = full(U)
    cross = (full(change([b1, b2])) - f0) - (full(change([b1])) - f0) - (full(change([b2])) - f0)
    assert abs(cross) > 1e-6


# --- the HYP filter level ------------------------------------------------------------

def test_filter_hyp_level_with_zero_coefficients_changes_nothing():
    """hyp_level = (0, 0): Delta = 0 on every block, all pass, and the step
    equals the step without the level."""
    from oracle import filter as ofilter
    geom = lattice.Geometry((4, 4, 4, 4), (2, 2, 2, 2))
    U = _field(geom.dims, 17, 0.5)
    prm = dict(kappa=0.156, beta0=5.3, n_iter=1, n_or=1, n_block=2, n_global=2, tol=1e-12)
    Ua, ra = ofilter.filter_step(U, geom, ofilter.FilterParams(**prm), 9, 0)
    Ub, rb = ofilter.filter_step(U, geom, ofilter.FilterParams(hyp_level=(0.0, 0.0), **prm), 9, 0)
    assert np.all(rb["accept_hyp"]) and np.all(rb["delta_hyp"] == 0)
    assert np.array_equal(ra["accept_block"], rb["accept_block"]) and ra["accept_global"] == rb["accept_global"]
    assert np.array_equal(Ua, Ub)


def test_filter_hyp_level_bookkeeping_and_antisymmetry():
    """3^4 blocks, external proposal on the active links: the HYP level's
    Delta_b = b0 dS_w,b + b1 dS_HYP,b, its decisions follow the draw map
    (counter (step, 5, b)), blocks it rejects keep their links, and
    swapping U and U' negates every Delta_b (the action is a function of
    the field, which the level's detailed balance needs)."""
    from oracle import filter as ofilter, philox
    geom = lattice.Geometry((6, 6, 6, 6), (3, 3, 3, 3))
    U = _field(geom.dims, 18, 0.4)
    act = geom.active_links()
    R = _su3_exp(0.3 * np.random.default_rng(19).standard_normal(geom.dims + (4, 8)))
    Up = np.where(act[..., None, None], U @ R, U)
    b0, b1 = 0.5, 4.0
    prm = ofilter.FilterParams(kappa=0.156, beta0=5.3, n_block=2, tol=1e-10, global_level=False,
                               hyp_level=(b0, b1), beta_block_hyp=-0.5)
    Unew, rec = ofilter.filter_step(U, geom, prm, 21, 4, proposal=Up, translate=False)
    dsw = ofilter.per_block_action_change(U, Up, geom)
    dsh = hyp.block_hyp_change(U, Up, geom)
    assert np.abs(rec["delta_hyp"] - (b0 * dsw + b1 * dsh)).max() < 1e-12
    u = np.array([philox.accept_uniform(21, 4, 5, b) for b in range(geom.n_blocks)])
    assert np.array_equal(rec["accept_hyp"], (rec["delta_hyp"] <= 0) | (u < np.exp(-rec["delta_hyp"])))
    assert 0 < rec["accept_hyp"].sum() < geom.n_blocks
    assert not np.any(rec["accept_block"] & ~rec["accept_hyp"])
    keep = rec["accept_block"][geom.block_index][..., None] & act
    assert np.array_equal(Unew, np.where(keep[..., None, None], Up, U))
    back = b0 * ofilter.per_block_action_change(Up, U, geom) + b1 * hyp.block_hyp_change(Up, U, geom)
    assert np.abs(back + rec["delta_hyp"]).max() < 1e-12
