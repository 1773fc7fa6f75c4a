"""Pins of the oracle's Wilson-Dirac operator and block pieces against the
paper's fixed points: free-field spectrum, gamma5-hermiticity, gauge
covariance, the Dirichlet block restriction, and P's defining properties."""
import itertools
import json
import os

import numpy as np
import pytest
import scipy.linalg

from oracle import dirac, estimator, gamma, gauge, lattice
from tests import seeded

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def test_gamma_clifford_algebra():
    G = gamma.GAMMA
    for m in range(4):
        assert np.allclose(G[m], G[m].conj().T)
        for n in range(4):
            assert np.allclose(G[m] @ G[n] + G[n] @ G[m], 2.0 * (m == n) * np.eye(4))
    assert np.allclose(gamma.GAMMA5, np.diag([1, 1, -1, -1]))


def _sorted(z):
    return z[np.lexsort((np.round(z.imag, 8), np.round(z.real, 8)))]


@pytest.mark.parametrize("dims,kappa", [((4, 2, 2, 2), 0.15), ((2, 4, 2, 4), 0.125), ((6, 2, 2, 2), 0.1)])
def test_free_field_spectrum(dims, kappa):
    """U = 1: eigenvalues m0 + sum(1-cos p) +- i sqrt(sum sin^2 p), 6-fold,
    antiperiodic p_0 (golden: free_field_spectrum)."""
    U = np.zeros(tuple(dims) + (4, 3, 3), dtype=complex)
    U[...] = np.eye(3)
    V = int(np.prod(dims))
    D = dirac.dense_matrix(lambda v: dirac.apply_D(U, v, kappa), V, tuple(dims) + (4, 3))
    ev = np.linalg.eigvals(D)
    m0 = dirac.mass_from_kappa(kappa)
    exp = []
    for n in itertools.product(*[range(L) for L in dims]):
        p = [(2 * n[0] + 1) * np.pi / dims[0]] + [2 * np.pi * n[k] / dims[k] for k in (1, 2, 3)]
        re = m0 + sum(1 - np.cos(q) for q in p)
        im = np.sqrt(sum(np.sin(q) ** 2 for q in p))
        exp += [re + 1j * im] * 6 + [re - 1j * im] * 6
    assert np.abs(_sorted(ev) - _sorted(np.array(exp))).max() < 1e-10


def test_plane_wave_any_size():
    """D on a plane wave e^{ipx} u equals D(p) u (free field), at 8^4."""
    dims = (8, 4, 4, 8)
    kappa = 0.13
    U = np.zeros(dims + (4, 3, 3), dtype=complex)
    U[...] = np.eye(3)
    n = (3, 1, 2, 5)
    p = [(2 * n[0] + 1) * np.pi / dims[0]] + [2 * np.pi * n[k] / dims[k] for k in (1, 2, 3)]
    x = np.indices(dims)
    phase = np.exp(1j * sum(p[m] * x[m] for m in range(4)))
    u = seeded.spinor((1,), 5)[0]
    psi = phase[..., None, None] * u
    out = dirac.apply_D(U, psi, kappa)
    m0 = dirac.mass_from_kappa(kappa)
    Dp = (m0 + sum(1 - np.cos(q) for q in p)) * np.eye(4) + 1j * sum(gamma.GAMMA[m] * np.sin(p[m]) for m in range(4))
    exp = phase[..., None, None] * (Dp @ u)
    assert np.abs(out - exp).max() < 1e-12


@pytest.mark.parametrize("interp", [False, True])
def test_gamma5_hermiticity_and_adjoint(interp):
    """<phi, D psi> = <gamma5 D gamma5 phi, psi> (also for interpolated,
    non-unitary links, Sec. 4.3), and apply_D(dagger=True) is the adjoint."""
    dims = (4, 4, 2, 4)
    U = seeded.gauge_field(dims, 1)
    if interp:
        U = estimator.interpolate(U, seeded.gauge_field(dims, 2), 1, 3)
    phi = seeded.spinor(dims, 3)
    psi = seeded.spinor(dims, 4)
    k = 0.156
    Dpsi = dirac.apply_D(U, psi, k)
    lhs = np.vdot(phi, Dpsi)
    g5Dg5phi = dirac.gamma5(dirac.apply_D(U, dirac.gamma5(phi), k))
    assert abs(lhs - np.vdot(g5Dg5phi, psi)) < 1e-10 * abs(lhs)
    assert abs(lhs - np.vdot(dirac.apply_D(U, phi, k, dagger=True), psi)) < 1e-10 * abs(lhs)


def test_gauge_covariance():
    """D(U^g)(g psi) = g (D(U) psi) with U^g(x,mu) = g(x) U(x,mu) g(x+mu)^-1 (Sec. 4.2)."""
    dims = (4, 2, 4, 2)
    U = seeded.gauge_field(dims, 11)
    g = seeded.haar_su3(dims, 12)
    Ug = np.empty_like(U)
    for mu in range(4):
        Ug[..., mu, :, :] = g @ U[..., mu, :, :] @ gauge.dag(lattice.gauge_shift(g, mu, +1))
    psi = seeded.spinor(dims, 13)
    gpsi = np.einsum("...ab,...sb->...sa", g, psi)
    lhs = dirac.apply_D(Ug, gpsi, 0.15)
    rhs = np.einsum("...ab,...sb->...sa", g, dirac.apply_D(U, psi, 0.15))
    assert np.abs(lhs - rhs).max() < 1e-12


def test_block_operator_is_dirichlet_restriction():
    """Eq. (domdec): D_b is the diagonal block of D on block b's sites."""
    dims = (4, 4, 4, 2)
    geom = lattice.Geometry(dims, (2, 2, 2, 1))
    U = seeded.gauge_field(dims, 21)
    k = 0.15
    D = dirac.dense_matrix(lambda v: dirac.apply_D(U, v, k), geom.V, dims + (4, 3))
    for b in (0, 3):
        sites = geom.site_index[geom.block_index == b]
        idx = (sites[:, None] * 12 + np.arange(12)[None, :]).reshape(-1)
        Ub = dirac.extract_block(U, geom, b)
        Db = dirac.dense_matrix(lambda v: dirac.apply_D_open(Ub, v, k), geom.Vb, geom.block + (4, 3))
        # block-local site order equals global order restricted to the block
        assert np.abs(D[np.ix_(idx, idx)] - Db).max() < 1e-14
    # the block-diagonal mode holds exactly these blocks
    Dblk = dirac.dense_matrix(lambda v: dirac.apply_D(U, v, k, geom, mode="block"), geom.V, dims + (4, 3))
    same = (geom.block_index.reshape(-1)[:, None] == geom.block_index.reshape(-1)[None, :])
    mask = np.kron(same, np.ones((12, 12), dtype=bool))
    assert np.abs(Dblk - D * mask).max() < 1e-14
    Dint = dirac.dense_matrix(lambda v: dirac.apply_D(U, v, k, geom, mode="inter"), geom.V, dims + (4, 3))
    assert np.abs(Dint + Dblk - D).max() < 1e-14


def test_dd_determinant_factorisation():
    """Eq. (ddfactor): log|det D| = sum_b log|det D_b| + log|det(1 - Q)|."""
    dims = (4, 4, 2, 2)
    geom = lattice.Geometry(dims, (2, 2, 1, 1))
    U = seeded.gauge_field(dims, 31)
    k = 0.156
    D = dirac.dense_matrix(lambda v: dirac.apply_D(U, v, k), geom.V, dims + (4, 3))
    black = np.repeat(geom.black_sites().reshape(-1), 12)
    Dbb, Dbw = D[np.ix_(black, black)], D[np.ix_(black, ~black)]
    Dwb, Dww = D[np.ix_(~black, black)], D[np.ix_(~black, ~black)]
    Q = np.linalg.solve(Dbb, Dbw @ np.linalg.solve(Dww, Dwb))
    lhs = np.linalg.slogdet(D)[1]
    blocks = 0.0
    for b in range(geom.n_blocks):
        Ub = dirac.extract_block(U, geom, b)
        Db = dirac.dense_matrix(lambda v: dirac.apply_D_open(Ub, v, k), geom.Vb, geom.block + (4, 3))
        blocks += np.linalg.slogdet(Db)[1]
    schur = np.linalg.slogdet(np.eye(Q.shape[0]) - Q)[1]
    assert abs(lhs - blocks - schur) < 1e-9 * abs(lhs)


@pytest.mark.parametrize("case", GOLDEN["dim_projector_formula"]["cases"])
def test_dim_projector_formula(case):
    """Eq. (dimproj) against the rank of the projector built site by site."""
    L, l = case["dims"], case["block"]
    geom = lattice.Geometry(L, l)
    nblk = np.prod([L[m] // l[m] for m in range(4)])
    vb = np.prod(l)
    formula = 6 * nblk * (sum(vb // l[n] for n in range(4)) - 4 * sum(l[n] - 1 for n in range(4)))
    assert geom.dim_projector() == formula


def test_projector_properties():
    """P^2 = P = P^dagger and D_wb P = D_wb (Sec. 4.4) on 8^4 with 4^4 blocks,
    where one-face sites carry rank-2 spin projectors."""
    dims = (8, 8, 8, 8)
    geom = lattice.Geometry(dims, (4, 4, 4, 4))
    P = geom.projector()
    assert np.abs(P @ P - P).max() < 1e-15
    assert np.abs(P - np.conj(np.swapaxes(P, -1, -2))).max() < 1e-15
    U = seeded.gauge_field(dims, 41)
    black = geom.black_sites()[..., None, None]
    psi = seeded.spinor(dims, 42) * black
    a = dirac.apply_D(U, psi, 0.15, geom, mode="inter") * ~black
    b = dirac.apply_D(U, estimator.project(P, psi), 0.15, geom, mode="inter") * ~black
    assert np.abs(a - b).max() < 1e-14
    # a wrong face sign must break the property (sensitivity of this pin)
    Pbad = P.copy()
    one = (np.real(np.trace(P, axis1=-2, axis2=-1)) > 1.5) & (np.real(np.trace(P, axis1=-2, axis2=-1)) < 2.5)
    Pbad[one] = np.eye(4) - P[one]
    c = dirac.apply_D(U, estimator.project(Pbad, psi), 0.15, geom, mode="inter") * ~black
    assert np.abs(a - c).max() > 1e-3


def test_active_link_fraction():
    """Sec. 5: about 9.4% of all links are active with 4^4 blocks (golden)."""
    g = GOLDEN["active_link_fraction_4x4x4x4_blocks"]
    geom = lattice.Geometry((8, 8, 8, 8), (4, 4, 4, 4))
    frac = geom.active_links().mean()
    assert frac == 96 / 1024
    assert abs(frac - g["value"]) <= g["printed_precision"]


def test_active_links_decouple_blocks():
    """No plaquette holds active links of two different blocks (l >= 3), the
    property the paper's active-link rule is built for (Sec. 3)."""
    geom = lattice.Geometry((8, 8, 8, 8), (4, 4, 4, 4))
    act = geom.active_links()
    bidx = geom.block_index
    for mu in range(4):
        for nu in range(4):
            if mu == nu:
                continue
            links = [(act[..., mu], bidx), (lattice.gauge_shift(act[..., nu], mu, +1), lattice.gauge_shift(bidx, mu, +1)),
                     (lattice.gauge_shift(act[..., mu], nu, +1), lattice.gauge_shift(bidx, nu, +1)), (act[..., nu], bidx)]
            for (a1, b1), (a2, b2) in itertools.combinations(links, 2):
                both = a1 & a2
                assert np.all(b1[both] == b2[both])


def test_link_generator():
    """U = exp(i eps H): unitary, det 1, equal to scipy's expm."""
    dims = (2, 2, 2, 2)
    U = gauge.generate_links(dims, 0.5, 7)
    I3 = np.eye(3)
    assert np.abs(U @ gauge.dag(U) - I3).max() < 1e-14
    assert np.abs(np.linalg.det(U) - 1).max() < 1e-14
    from oracle import philox
    om = philox.link_omegas(7, 16)
    H = gauge.hermitian_generators(om)
    assert np.abs(np.trace(H, axis1=-2, axis2=-1)).max() < 1e-15
    for k in (0, 5, 63):
        ref = scipy.linalg.expm(1j * 0.5 * H[k])
        assert np.abs(U.reshape(-1, 3, 3)[k] - ref).max() < 1e-13
