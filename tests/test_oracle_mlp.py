"""Pins of the oracle's learned-level pieces: domain features (closed forms,
gauge invariance, brute force) and the FP64 MLP gradients (finite
differences), antisymmetry of the surrogate."""
import numpy as np
import scipy.linalg

from oracle import gauge, lattice, mlp
from tests import seeded


def test_features_unit_field():
    geom = lattice.Geometry((8, 8, 8, 8), (4, 4, 4, 4))
    U = np.zeros(geom.dims + (4, 3, 3), dtype=complex)
    U[...] = np.eye(3)
    f = mlp.domain_features(U, geom)
    assert np.allclose(f[:, :6], 1.0) and np.allclose(f[:, 6:], 0.0)


def test_features_constant_abelian_field():
    """U(x,1) = exp(i theta x0 T), T = diag(1,-1,0), other links 1: inside a
    block every (0,1) plaquette and clover leaf is exp(i theta T), so the
    plaquette mean is (2 cos theta + 1)/3 and Tr F_01^2 = 2 sin^2 theta."""
    geom = lattice.Geometry((8, 4, 4, 4), (4, 4, 4, 4))
    theta = 0.3
    T = np.diag([1.0, -1.0, 0.0])
    U = np.zeros(geom.dims + (4, 3, 3), dtype=complex)
    U[...] = np.eye(3)
    for t in range(geom.dims[0]):
        U[t, :, :, :, 1] = scipy.linalg.expm(1j * theta * t * T)
    f = mlp.domain_features(U, geom)
    assert np.allclose(f[:, 0], (2 * np.cos(theta) + 1) / 3)
    assert np.allclose(f[:, 1:6], 1.0)
    assert np.allclose(f[:, 6:12], 0.0, atol=1e-15)
    assert np.allclose(f[:, 12], 2 * np.sin(theta) ** 2)
    assert np.allclose(f[:, 13:18], 0.0, atol=1e-15)


def test_features_gauge_invariant():
    geom = lattice.Geometry((8, 4, 4, 8), (4, 4, 4, 4))
    U = gauge.generate_links(geom.dims, 0.5, 3)
    g = seeded.haar_su3(geom.dims, 4)
    Ug = np.empty_like(U)
    for mu in range(4):
        Ug[..., mu, :, :] = g @ U[..., mu, :, :] @ gauge.dag(lattice.gauge_shift(g, mu, +1))
    assert np.abs(mlp.domain_features(U, geom) - mlp.domain_features(Ug, geom)).max() < 1e-12


def test_features_brute_force_plaquettes():
    """Per-block plaquette mean and variance by explicit loops."""
    geom = lattice.Geometry((4, 4, 4, 8), (2, 2, 2, 4))
    U = gauge.generate_links(geom.dims, 0.5, 5)
    f = mlp.domain_features(U, geom)
    b = 3
    B = np.unravel_index(b, geom.nb)
    for k, (mu, nu) in enumerate(mlp.PLANES):
        vals = []
        P = gauge.plaquette_field(U, mu, nu)
        for y in np.ndindex(*geom.block):
            if y[mu] < geom.block[mu] - 1 and y[nu] < geom.block[nu] - 1:
                x = tuple(B[m] * geom.block[m] + y[m] for m in range(4))
                vals.append(np.real(np.trace(P[x])) / 3)
        assert abs(f[b, k] - np.mean(vals)) < 1e-14
        assert abs(f[b, 6 + k] - np.var(vals)) < 1e-14


def test_mlp_gradient_finite_differences():
    g = np.random.default_rng(7)
    p = mlp.init_params(11)
    p["mu"] = g.standard_normal(64) * 0.1
    p["sigma"] = 1.0 + g.random(64)
    p["b1"] = g.standard_normal(256) * 0.1
    p["b2"] = g.standard_normal(256) * 0.1
    z = g.standard_normal((9, 64))
    y = g.standard_normal(9)
    loss, grads = mlp.loss_and_grad(p, z, y)
    eps = 1e-6
    for key, idx in (("W1", (3, 5)), ("W1", (200, 63)), ("b1", (17,)), ("W2", (10, 250)), ("b2", (3,)),
                     ("w3", (100,)), ("b3", None)):
        q = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in p.items()}
        if idx is None:
            q[key] = p[key] + eps
            lp, _ = mlp.loss_and_grad(q, z, y)
            q[key] = p[key] - eps
            lm, _ = mlp.loss_and_grad(q, z, y)
            num = (lp - lm) / (2 * eps)
            ana = grads[key]
        else:
            q[key][idx] += eps
            lp, _ = mlp.loss_and_grad(q, z, y)
            q[key][idx] -= 2 * eps
            lm, _ = mlp.loss_and_grad(q, z, y)
            num = (lp - lm) / (2 * eps)
            ana = grads[key][idx]
        assert abs(num - ana) < 1e-6 * max(1.0, abs(ana)), (key, idx, num, ana)


def test_surrogate_antisymmetric():
    p = mlp.init_params(3)
    z = np.random.default_rng(1).standard_normal((5, 64))
    assert np.allclose(mlp.antisym(p, z), -mlp.antisym(p, mlp.swap(z)))


def test_bf16_rounding_model():
    """bf16(): round to nearest even on the 16 dropped bits."""
    assert mlp.bf16(1.0) == 1.0
    assert mlp.bf16(1.0 + 2 ** -8) == 1.0 + 2 ** -7 or mlp.bf16(1.0 + 2 ** -8) == 1.0
    assert mlp.bf16(1.0 + 2 ** -8) == 1.0           # tie -> even
    assert mlp.bf16(1.0 + 3 * 2 ** -8) == 1.0 + 2 ** -6  # tie -> even (up)
    assert mlp.bf16(1.0 + 2 ** -7) == 1.0 + 2 ** -7
    x = np.random.default_rng(0).standard_normal(1000)
    assert np.all(np.abs(mlp.bf16(x) - x) <= 2 ** -8 * np.abs(x))
    p = mlp.init_params(2)
    z = np.random.default_rng(3).standard_normal((20, 64))
    a, b = mlp.antisym(p, z), mlp.antisym_rounded(p, z)
    assert np.linalg.norm(a - b) <= 0.25 * np.linalg.norm(a)


def test_pair_features_distance():
    """Slot 18 (both halves) is the block distance of Eq. (sprodgf): zero for
    identical fields, (3 - ReTr R)/12 per link for U' = U R with R fixed, and
    symmetric in (U, U')."""
    geom = lattice.Geometry((8, 4, 4, 4), (4, 4, 4, 4))
    U = gauge.generate_links(geom.dims, 0.5, 9)
    z0 = mlp.pair_features(U, U, geom)
    assert np.allclose(z0[:, 18], 0.0) and np.allclose(z0[:, 50], 0.0)
    R = gauge.expm_i_hermitian(gauge.hermitian_generators(np.arange(8) * 0.1), 0.7)
    Up = U @ R
    z = mlp.pair_features(U, Up, geom)
    assert np.allclose(z[:, 18], (3.0 - np.real(np.trace(R))) / 12.0)
    zr = mlp.pair_features(Up, U, geom)
    assert np.allclose(zr[:, 18], z[:, 18])
    assert np.allclose(zr[:, :18], z[:, 32:50]) and np.allclose(zr[:, 32:50], z[:, :18])
