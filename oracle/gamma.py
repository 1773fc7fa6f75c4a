"""Euclidean Dirac matrices used by Eq. (Dw).  TEST INFRASTRUCTURE ONLY.

The paper does not fix a basis.  Chiral basis, written in 2x2 blocks:

    gamma_mu = [[0, e_mu], [e_mu^dagger, 0]],  e_0 = -1,  e_k = -i sigma_k,

so that gamma_mu are Hermitian, {gamma_mu, gamma_nu} = 2 delta_{mu nu}, and
gamma_5 = gamma_0 gamma_1 gamma_2 gamma_3 = diag(1, 1, -1, -1).  Every physical
pin (spectrum, determinants, gamma_5-hermiticity) is basis independent.
"""
import numpy as np

SIGMA = [
    np.array([[0, 1], [1, 0]], dtype=np.complex128),
    np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
    np.array([[1, 0], [0, -1]], dtype=np.complex128),
]


def _gamma(e):
    g = np.zeros((4, 4), dtype=np.complex128)
    g[0:2, 2:4] = e
    g[2:4, 0:2] = e.conj().T
    return g


GAMMA = np.stack([_gamma(-np.eye(2, dtype=np.complex128))] + [_gamma(-1j * s) for s in SIGMA])
GAMMA5 = GAMMA[0] @ GAMMA[1] @ GAMMA[2] @ GAMMA[3]
ONE4 = np.eye(4, dtype=np.complex128)
