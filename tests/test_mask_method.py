"""The link-mask construction of the device's recursive decomposition,
checked with the oracle's operators: with the links that cross outer-block
faces set to zero, the whole-lattice operator is the outer blocks'
Dirichlet operator and the inter-block hop stays inside the outer blocks;
the links on those edges alone give the hops between outer blocks.  The
device's sequence of operations for the outer-block Schur estimate and for
the global level of the outer decomposition, restated here with these
operators, reproduces the oracle's estimates (Eqs. (ddrec), (staccN),
(inverseschur))."""
import numpy as np

from oracle import dirac, estimator, gauge, linalg, recursive
from tests import seeded

K = 0.156
DIMS, OUTER, INNER = (8, 4, 4, 4), (4, 2, 2, 2), (2, 1, 1, 1)


def _masks(nest):
    """bool [dims, 4]: the link (x, mu) crosses an outer face."""
    return np.stack([~nest.outer.fwd_intra(mu) for mu in range(4)], axis=-1)


def _perturbed(U, eps, seed):
    g = np.random.default_rng(seed)
    om = g.standard_normal(U.shape[:-2] + (8,))
    return U @ gauge.expm_i_hermitian(gauge.hermitian_generators(om), eps)


def _hops(U, psi, geom=None, mode="full"):
    """-1/2 H psi (the hopping part of Eq. (Dw) alone)."""
    if mode == "inter":
        return dirac.apply_D(U, psi, K, geom, mode="inter")
    return dirac.apply_D(U, psi, K) - (4.0 + dirac.mass_from_kappa(K)) * psi


def test_masked_links_give_the_outer_operators():
    nest = recursive.Nested(DIMS, OUTER, INNER)
    U = gauge.generate_links(DIMS, 0.5, 90)
    cr = _masks(nest)[..., None, None]
    Um, Uc = np.where(cr, 0, U), np.where(cr, U, 0)
    psi = seeded.spinor(DIMS, 91)
    # D(U_masked) = diag over outer blocks of the Dirichlet operator
    ref = np.zeros_like(psi)
    for b in range(nest.outer.n_blocks):
        dirac.insert_block(ref, nest.outer, b, dirac.apply_D_open(dirac.extract_block(U, nest.outer, b),
                                                                 dirac.extract_block(psi, nest.outer, b), K))
    assert np.abs(dirac.apply_D(Um, psi, K) - ref).max() < 1e-14
    # inter-block hops with U_masked = hops between inner blocks of one outer block
    ref = np.zeros_like(psi)
    for b in range(nest.outer.n_blocks):
        dirac.insert_block(ref, nest.outer, b, recursive.apply_D_outer(dirac.extract_block(U, nest.outer, b),
                                                                      dirac.extract_block(psi, nest.outer, b), K,
                                                                      nest.sub, "inter"))
    assert np.abs(_hops(Um, psi, nest.inner, "inter") - ref).max() < 1e-14
    # hops with the crossing links alone = the hops between outer blocks
    assert np.abs(_hops(Uc, psi) - dirac.apply_D(U, psi, K, nest.outer, mode="inter")).max() < 1e-14


def _solve(U, rhs):
    x, _, _ = linalg.cgnr(lambda v: dirac.apply_D(U, v, K), lambda v: dirac.apply_D(U, v, K, dagger=True), rhs,
                          tol=1e-13)
    return x


def test_device_sequence_reproduces_the_sub_level():
    """The device's stage 2: xi = P_b noise; t2 = D_ww^-1 D_wb xi (inner
    block solves, masked links); v = xi - P_b D_bb^-1 D_bw t2;
    w = v - P_b [D(U_masked)^-1 (0, D_wb v)]; Delta_b = |w|_b^2 - |xi|_b^2."""
    nest = recursive.Nested(DIMS, OUTER, INNER)
    U = gauge.generate_links(DIMS, 0.4, 92)
    Up = _perturbed(U, 0.3, 93)
    cr = _masks(nest)[..., None, None]
    N, seed, counter = 2, 5, 7
    Pb = recursive.sub_projector(nest)
    P = np.zeros(DIMS + (4, 4), dtype=np.complex128)
    for b in range(nest.outer.n_blocks):
        dirac.insert_block(P, nest.outer, b, Pb)
    black = (nest.inner.colour == 0)[..., None, None]
    col = nest.inner.block_colours()
    blacks = [b for b in range(nest.inner.n_blocks) if col[b] == 0]
    whites = [b for b in range(nest.inner.n_blocks) if col[b] == 1]
    got = np.zeros((nest.outer.n_blocks, N))
    for i in range(N):
        Ua, Ub = (np.where(cr, 0, F) for F in estimator.pair(U, Up, i, N, "interp"))
        xi = estimator.project(P, estimator.noise(nest.outer, seed, counter, recursive.LEVEL_SUB, i))
        t1 = _hops(Ua, xi, nest.inner, "inter") * ~black
        t2 = estimator.solve_blocks(Ua, t1, nest.inner, K, whites, 1e-13)
        t1 = _hops(Ua, t2, nest.inner, "inter") * black
        t2 = estimator.solve_blocks(Ua, t1, nest.inner, K, blacks, 1e-13)
        v = xi - estimator.project(P, t2)
        y = _hops(Ub, v * black, nest.inner, "inter") * ~black
        z = _solve(Ub, y)
        w = v - estimator.project(P, z * black)
        n2 = lambda f: np.bincount(nest.outer.block_index.reshape(-1),
                                   weights=np.sum(np.abs(f) ** 2, axis=(-1, -2)).reshape(-1),
                                   minlength=nest.outer.n_blocks)
        got[:, i] = n2(w) - n2(xi)
    ref = recursive.sub_level(U, Up, nest, K, N, seed, counter, tol=1e-13)
    assert np.abs(got - ref).max() < 1e-9


def test_device_sequence_reproduces_the_outer_global_level():
    """The device's global level of the outer decomposition: D_wb from the
    crossing links, D_ww^-1 and D_bb^-1 by whole-lattice solves with the
    masked links, (1 - PQ)^-1 with the full operator."""
    nest = recursive.Nested(DIMS, OUTER, INNER)
    U = gauge.generate_links(DIMS, 0.4, 94)
    Up = _perturbed(U, 0.3, 95)
    cr = _masks(nest)[..., None, None]
    N, seed, counter = 2, 3, 4
    P = nest.outer.projector()
    black = (nest.outer.colour == 0)[..., None, None]
    got = np.zeros(N)
    for i in range(N):
        Ua, Ub = estimator.pair(U, Up, i, N, "interp")
        xi = estimator.project(P, estimator.noise(nest.outer, seed, counter, estimator.LEVEL_GLOBAL, i))
        t1 = _hops(np.where(cr, Ua, 0), xi) * ~black
        t2 = _solve(np.where(cr, 0, Ua), t1)
        t1 = _hops(np.where(cr, Ua, 0), t2) * black
        t2 = _solve(np.where(cr, 0, Ua), t1)
        v = xi - estimator.project(P, t2)
        y = _hops(np.where(cr, Ub, 0), v) * ~black
        z = _solve(Ub, y)
        w = v - estimator.project(P, z)
        got[i] = linalg.norm2(w) - linalg.norm2(xi)
    ref = estimator.global_level(U, Up, nest.outer, K, N, seed, counter, tol=1e-13)
    assert np.abs(got - ref).max() < 1e-9
