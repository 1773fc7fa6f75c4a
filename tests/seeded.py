"""Seeded synthetic inputs shared by the oracle tests and the GPU parity tests.

Holds none of the method's arithmetic: plain numpy ``default_rng`` draws in the
canonical layout (spinors [x0, x1, x2, x3, spin, colour], links
[x0, x1, x2, x3, mu, 3, 3], complex128).
"""
import numpy as np


def rng(seed):
    return np.random.default_rng(seed)


def spinor(dims, seed):
    g = rng(seed)
    shape = tuple(dims) + (4, 3)
    return (g.standard_normal(shape) + 1j * g.standard_normal(shape)) / np.sqrt(2.0)


def haar_su3(shape, seed):
    """Random SU(3) matrices (QR of complex Gaussian, phases fixed, det -> 1)."""
    g = rng(seed)
    Z = (g.standard_normal(tuple(shape) + (3, 3)) + 1j * g.standard_normal(tuple(shape) + (3, 3))) / np.sqrt(2.0)
    Q, R = np.linalg.qr(Z)
    d = np.diagonal(R, axis1=-2, axis2=-1)
    Q = Q * (d / np.abs(d))[..., None, :]
    det = np.linalg.det(Q)
    return Q / (det ** (1.0 / 3.0))[..., None, None]


def gauge_field(dims, seed):
    return haar_su3(tuple(dims) + (4,), seed)


def complex_matrix(n, seed, scale=1.0):
    g = rng(seed)
    return scale * (g.standard_normal((n, n)) + 1j * g.standard_normal((n, n))) / np.sqrt(2.0)
