"""Pins of the oracle's solver, stochastic estimators and acceptance rules.

Deterministic estimator values are compared with dense linear algebra
(numpy solve / LU); the statistical statements of Sec. 4.1 and App. A.2 are
checked through their closed forms."""
import json
import os

import numpy as np
import pytest

from oracle import dirac, estimator, filter as ofilter, gauge, lattice, linalg, philox
from tests import seeded

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
K = 0.156


def _dense(apply, n_sites, shape):
    return dirac.dense_matrix(apply, n_sites, shape)


def _perturbed(U, eps, seed):
    """U' = U exp(i eps H): a nearby SU(3) field (seeded input)."""
    g = np.random.default_rng(seed)
    om = g.standard_normal(U.shape[:-2] + (8,))
    return U @ gauge.expm_i_hermitian(gauge.hermitian_generators(om), eps)


# --- solver --------------------------------------------------------------------

def test_cgnr_matches_dense_solve():
    dims = (4, 2, 2, 4)
    U = seeded.gauge_field(dims, 1)
    b = seeded.spinor(dims, 2)
    x, it, rel = linalg.cgnr(lambda v: dirac.apply_D(U, v, K), lambda v: dirac.apply_D(U, v, K, dagger=True), b, tol=1e-13)
    D = _dense(lambda v: dirac.apply_D(U, v, K), 64, dims + (4, 3))
    xd = np.linalg.solve(D, b.reshape(-1)).reshape(b.shape)
    assert rel <= 1e-13
    assert np.abs(x - xd).max() < 1e-11
    assert it > 0


def test_lu_logabsdet():
    for n, seed in ((5, 1), (40, 2), (120, 3)):
        A = seeded.complex_matrix(n, seed)
        assert abs(linalg.lu_logabsdet(A) - np.linalg.slogdet(A)[1]) < 1e-10 * n
    geom = lattice.Geometry((4, 4, 4, 4), (2, 2, 2, 2))
    U = gauge.generate_links(geom.dims, 0.3, 0x50534D53)
    Ub = dirac.extract_block(U, geom, 5)
    Db = _dense(lambda v: dirac.apply_D_open(Ub, v, 0.15), 16, (2, 2, 2, 2, 4, 3))
    assert abs(linalg.lu_logabsdet(Db) - np.linalg.slogdet(Db)[1]) < 1e-10


# --- block-level estimator -----------------------------------------------------

@pytest.mark.parametrize("mode,N", [("independent", 3), ("interp", 4)])
def test_block_estimator_equals_dense(mode, N):
    """Delta_{b,i} = |D_b(U_{i+1})^-1 D_b(U_i) xi|^2 - |xi|^2 against dense solves."""
    dims = (4, 4, 4, 4)
    geom = lattice.Geometry(dims, (2, 2, 2, 2))
    U = gauge.generate_links(dims, 0.3, 11)
    Up = _perturbed(U, 0.3, 12)
    blocks = [0, 7, 15]
    d = estimator.block_level(U, Up, geom, 0.15, N, seed=5, counter=9, mode=mode, blocks=blocks)
    for i in range(N):
        Ua, Ub = estimator.pair(U, Up, i, N, mode)
        xi = estimator.noise(geom, 5, 9, estimator.LEVEL_BLOCK, i)
        for b in blocks:
            A = _dense(lambda v: dirac.apply_D_open(dirac.extract_block(Ua, geom, b), v, 0.15), 16, (2, 2, 2, 2, 4, 3))
            B = _dense(lambda v: dirac.apply_D_open(dirac.extract_block(Ub, geom, b), v, 0.15), 16, (2, 2, 2, 2, 4, 3))
            x = dirac.extract_block(xi, geom, b).reshape(-1)
            y = np.linalg.solve(B, A @ x)
            ref = np.vdot(y, y).real - np.vdot(x, x).real
            assert abs(d[b, i] - ref) < 1e-9 * max(1.0, abs(ref))


def test_interpolation_telescopes():
    """Eq. (param): prod_i det(M_i^dag M_i) = det(M^dag M) on a Dirichlet block."""
    geom = lattice.Geometry((4, 4, 4, 4), (2, 2, 2, 2))
    U = gauge.generate_links(geom.dims, 0.3, 21)
    Up = _perturbed(U, 0.4, 22)
    N = 5
    tot = 0.0
    Dblk = lambda F: _dense(lambda v: dirac.apply_D_open(dirac.extract_block(F, geom, 3), v, 0.15), 16, (2, 2, 2, 2, 4, 3))
    for i in range(N):
        A = Dblk(estimator.interpolate(U, Up, i, N))
        B = Dblk(estimator.interpolate(U, Up, i + 1, N))
        M = np.linalg.solve(B, A)
        tot += np.linalg.slogdet(M.conj().T @ M)[1]
    M = np.linalg.solve(Dblk(Up), Dblk(U))
    assert abs(tot - np.linalg.slogdet(M.conj().T @ M)[1]) < 1e-9


def test_estimator_closed_forms():
    """Sec. 4.1: at fixed (U, U'), E[e^-Delta] = det(M^dag M)^-1, E[Delta] =
    Tr(M^dag M - 1), Var[Delta] = sum_k (lambda_k - 1)^2 (Eq. (varstoch2)),
    E[e^-2 Delta] = det(2 M^dag M - 1)^-1,
    with the oracle's Philox noise on one 2^4 Dirichlet block (192 dims)."""
    geom = lattice.Geometry((4, 4, 4, 4), (2, 2, 2, 2))
    U = gauge.generate_links(geom.dims, 0.3, 31)
    Up = _perturbed(U, 0.12, 32)
    Dblk = lambda F: _dense(lambda v: dirac.apply_D_open(dirac.extract_block(F, geom, 0), v, 0.15), 16, (2, 2, 2, 2, 4, 3))
    M = np.linalg.solve(Dblk(Up), Dblk(U))
    lam = np.linalg.eigvalsh(M.conj().T @ M)
    assert lam.min() > 0.5          # the variance of e^-Delta exists (Sec. 4.1)
    n = 6000
    xi = np.stack([philox.noise_field(77, 0, j, 16).reshape(-1) for j in range(n)])
    y = xi @ M.T
    delta = np.sum(np.abs(y) ** 2, axis=1) - np.sum(np.abs(xi) ** 2, axis=1)
    var_exact = np.sum((lam - 1.0) ** 2)
    assert abs(delta.mean() - np.sum(lam - 1.0)) < 5 * np.sqrt(var_exact / n)
    assert abs(delta.var() / var_exact - 1.0) < 0.15
    ew = np.exp(-delta)
    target = np.exp(-np.sum(np.log(lam)))
    sd = np.sqrt(np.exp(-np.sum(np.log(2 * lam - 1))) - target ** 2)
    assert abs(ew.mean() - target) < 5 * sd / np.sqrt(n)
    # second moment (Sec. 4.1): E[e^-2Delta] = det(2 M^dag M - 1)^-1, with
    # finite variance when lambda_min > 3/4 (E[e^-4Delta] = det(4 M^dag M - 3)^-1)
    assert lam.min() > 0.75
    ew2 = np.exp(-2 * delta)
    target2 = np.exp(-np.sum(np.log(2 * lam - 1)))
    sd2 = np.sqrt(np.exp(-np.sum(np.log(4 * lam - 3))) - target2 ** 2)
    assert abs(ew2.mean() - target2) < 5 * sd2 / np.sqrt(n)


# --- global (Schur) estimator --------------------------------------------------

def test_schur_estimator_equals_dense():
    """Delta = |(1-Q(U'))^-1 (1-Q(U)) xi|^2 - |xi|^2 for P = 1 on black sites
    (blocks of extent <= 2), against dense Schur complements."""
    dims = (4, 4, 2, 2)
    geom = lattice.Geometry(dims, (2, 2, 1, 1))
    U = gauge.generate_links(dims, 0.3, 41)
    Up = _perturbed(U, 0.2, 42)
    d = estimator.global_level(U, Up, geom, K, 2, seed=3, counter=4, mode="independent")
    black = np.repeat(geom.black_sites().reshape(-1), 12)

    def one_minus_Q(F):
        D = _dense(lambda v: dirac.apply_D(F, v, K), geom.V, dims + (4, 3))
        Dbb, Dbw = D[np.ix_(black, black)], D[np.ix_(black, ~black)]
        Dwb, Dww = D[np.ix_(~black, black)], D[np.ix_(~black, ~black)]
        return np.eye(black.sum()) - np.linalg.solve(Dbb, Dbw @ np.linalg.solve(Dww, Dwb))

    M = np.linalg.solve(one_minus_Q(Up), one_minus_Q(U))
    for i in range(2):
        xi = estimator.noise(geom, 3, 4, estimator.LEVEL_GLOBAL, i).reshape(-1)[black]
        y = M @ xi
        ref = np.vdot(y, y).real - np.vdot(xi, xi).real
        assert abs(d[i] - ref) < 1e-9 * max(1.0, abs(ref))


def test_inverse_schur_identity_with_projector():
    """Eq. (inverseschur): (1 - PQ)(1 - P D^-1 D_wb) = 1 on range(P), 8^4 lattice
    with 4^4 blocks (rank-2 spin projectors on one-face sites)."""
    dims = (8, 8, 8, 8)
    geom = lattice.Geometry(dims, (4, 4, 4, 4))
    U = gauge.generate_links(dims, 0.5, 51)
    P = geom.projector()
    s = estimator.project(P, seeded.spinor(dims, 52))
    w = estimator.inv_one_minus_PQ(U, s, geom, K, P, 1e-13)
    back = estimator.one_minus_PQ(U, w, geom, K, P, 1e-13)
    assert np.abs(back - s).max() < 1e-10


# --- acceptance ----------------------------------------------------------------

@pytest.mark.parametrize("case", GOLDEN["gaussian_acceptance"]["cases"])
def test_gaussian_acceptance_golden(case):
    """Eq. (acceptance) reproduces the acceptances printed in Sec. 6."""
    assert abs(ofilter.gaussian_acceptance(case["sigma2"]) - case["acceptance"]) <= case["err"]


def test_gaussian_acceptance_monte_carlo():
    """Metropolis with Gaussian Delta ~ N(S/2, S) accepts erfc(sqrt(S/8)) of the time."""
    S = 1.0
    n = 20000
    g = np.random.default_rng(5)
    delta = S / 2 + np.sqrt(S) * g.standard_normal(n)
    u = philox.uniforms(9, philox.TAG_ACCEPT, philox.make_ctr(0, 1, np.arange(n)))[:, 0]
    acc = np.array([ofilter.accept(d, x) for d, x in zip(delta, u)])
    assert abs(acc.mean() - ofilter.gaussian_acceptance(S)) < 5 * np.sqrt(0.25 / n)


def test_stochastic_acceptance_formula():
    """App. A.2: P_acc from the eigenvalues of M^dag M against the Monte Carlo
    frequency of the oracle's decision rule; the detailed-balance ratio
    P(U->U')/P(U'->U) = |det M|^-2 and the bound P <= min(1, |det M|^-2)."""
    n = 12
    M = np.eye(n) + seeded.complex_matrix(n, 61, scale=0.25)
    lam = np.linalg.eigvalsh(M.conj().T @ M)
    p_fwd = ofilter.stochastic_acceptance(lam)
    p_rev = ofilter.stochastic_acceptance(1.0 / lam)
    det2 = np.prod(lam)
    assert abs(p_fwd / p_rev - 1.0 / det2) < 1e-8 / det2
    assert p_fwd <= min(1.0, 1.0 / det2) + 1e-12
    ns = 20000
    xi = philox.noise_field(13, 2, 0, ns)
    delta = np.sum(np.abs(xi @ M.T) ** 2, axis=1) - np.sum(np.abs(xi) ** 2, axis=1)
    u = philox.uniforms(13, philox.TAG_ACCEPT, philox.make_ctr(2, 3, np.arange(ns)))[:, 0]
    acc = np.mean([ofilter.accept(d, x) for d, x in zip(delta, u)])
    assert abs(acc - p_fwd) < 5 * np.sqrt(p_fwd * (1 - p_fwd) / ns)


# --- exact block level ------------------------------------------------------------

def test_exact_block_change_is_the_estimator_target():
    """dS_b = 2 (ln|det D_b(U)| - ln|det D_b(U')|) equals -ln det(M^dag M)^-1
    with M = D_b(U')^-1 D_b(U) (the target of E[e^-Delta], Sec. 4.1), and
    summing it over blocks with the exact Schur factor gives the change of
    ln|det D|^2 (Eq. (ddfactor))."""
    geom = lattice.Geometry((4, 4, 2, 2), (2, 2, 1, 1))
    U = gauge.generate_links(geom.dims, 0.4, 81)
    Up = _perturbed(U, 0.2, 82)
    ds = ofilter.exact_block_change(U, Up, geom, K)
    for b in (0, 5):
        shape = geom.block + (4, 3)
        A = _dense(lambda v: dirac.apply_D_open(dirac.extract_block(U, geom, b), v, K), geom.Vb, shape)
        B = _dense(lambda v: dirac.apply_D_open(dirac.extract_block(Up, geom, b), v, K), geom.Vb, shape)
        M = np.linalg.solve(B, A)
        assert abs(ds[b] - np.linalg.slogdet(M.conj().T @ M)[1]) < 1e-10
    black = np.repeat(geom.black_sites().reshape(-1), 12)

    def logdets(F):
        D = _dense(lambda v: dirac.apply_D(F, v, K), geom.V, geom.dims + (4, 3))
        Dbb, Dbw = D[np.ix_(black, black)], D[np.ix_(black, ~black)]
        Dwb, Dww = D[np.ix_(~black, black)], D[np.ix_(~black, ~black)]
        schur = np.eye(black.sum()) - np.linalg.solve(Dbb, Dbw @ np.linalg.solve(Dww, Dwb))
        return np.linalg.slogdet(D)[1], np.linalg.slogdet(schur)[1]

    (f0, s0), (f1, s1) = logdets(U), logdets(Up)
    assert abs(ds.sum() + 2 * (s0 - s1) - 2 * (f0 - f1)) < 1e-9


def test_filter_with_exact_block_level():
    """The block level's Delta_b is the exact dS_b (plus the beta terms), and
    the global level adds beta_global_blockdet times dS_b of the accepted
    blocks."""
    geom = lattice.Geometry((4, 4, 4, 4), (2, 2, 2, 2))
    U = gauge.generate_links(geom.dims, 0.5, 83)
    prm = dict(kappa=K, beta0=5.3, n_iter=1, n_or=1, n_global=2, tol=1e-12, exact_block=True, beta_block=0.2)
    U2, rec = ofilter.filter_step(U, geom, ofilter.FilterParams(**prm), 17, 1)
    Unew, _, _ = gauge.domain_sweep(U, geom, 5.3, 1, 1, 17, 1 * ofilter.SWEEP_STRIDE)
    ds = ofilter.exact_block_change(U, Unew, geom, K)
    ref = ds + 0.2 * ofilter.per_block_action_change(U, Unew, geom)
    assert np.abs(rec["delta_block"] - ref).max() < 1e-10
    U3, rec3 = ofilter.filter_step(U, geom, ofilter.FilterParams(beta_global_blockdet=-0.07, **prm), 17, 1)
    assert np.array_equal(rec3["accept_block"], rec["accept_block"])
    assert rec["accept_block"].any()
    extra = -0.07 * ds[rec["accept_block"]].sum()
    assert abs(rec3["delta_global"] - rec["delta_global"] - extra) < 1e-9
