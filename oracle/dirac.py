"""Wilson-Dirac operator and its domain-decomposition pieces.
TEST INFRASTRUCTURE ONLY.

Eq. (Dw):
    (D_w + m0) psi(x) = (4 + m0) psi(x)
        - 1/2 sum_mu { U(x,mu) (1 - gamma_mu) psi(x + mu)
                       + U(x - mu, mu)^dagger (1 + gamma_mu) psi(x - mu) },
    kappa = 1 / (2 m0 + 8),
with antiperiodic boundary conditions in time for the quark field.  D below
always means D_w + m0.  Links enter through U and U^dagger only (never
U^{-1}), as Sec. 4.3 requires for interpolated, non-unitary links.

Eq. (domdec): with the block checkerboard, D = [[D_bb, D_bw], [D_wb, D_ww]];
D_bb and D_ww are block diagonal with the Dirichlet block operators D_b
(hops that leave a block dropped), and D_bw, D_wb hold the hops between
blocks.

The adjoint is written out directly: D^dagger is Eq. (Dw) with gamma_mu ->
-gamma_mu.
"""
import numpy as np

from .gamma import GAMMA, ONE4
from .lattice import fermion_shift, gauge_shift


def mass_from_kappa(kappa):
    return 1.0 / (2.0 * kappa) - 4.0


def _spin(M, psi):
    """Apply a 4x4 spin matrix to psi[..., 4, 3]."""
    return np.einsum("st,...tc->...sc", M, psi)


def _colour(U, psi):
    """Apply 3x3 colour matrices U[..., 3, 3] to psi[..., 4, 3]."""
    return np.einsum("...ab,...sb->...sa", U, psi)


def _colour_dag(U, psi):
    return np.einsum("...ba,...sb->...sa", np.conj(U), psi)


def apply_D(U, psi, kappa, geom=None, mode="full", dagger=False):
    """D psi (or D^dagger psi) on the whole lattice.

    mode: 'full'  -- Eq. (Dw) on the torus;
          'block' -- block-diagonal part D_bb + D_ww (Dirichlet blocks);
          'inter' -- hops between different blocks only (D_bw + D_wb),
                     without the diagonal term.
    """
    m0 = mass_from_kappa(kappa)
    s = -1.0 if dagger else 1.0
    out = np.zeros_like(psi) if mode == "inter" else (4.0 + m0) * psi
    for mu in range(4):
        Pm = ONE4 - s * GAMMA[mu]
        Pp = ONE4 + s * GAMMA[mu]
        Umu = U[..., mu, :, :]
        fwd = _colour(Umu, _spin(Pm, fermion_shift(psi, mu, +1)))
        bwd = _colour_dag(gauge_shift(Umu, mu, -1), _spin(Pp, fermion_shift(psi, mu, -1)))
        if mode != "full":
            keep_f = geom.fwd_intra(mu)
            keep_b = geom.bwd_intra(mu)
            if mode == "inter":
                keep_f, keep_b = ~keep_f, ~keep_b
            fwd = fwd * keep_f[..., None, None]
            bwd = bwd * keep_b[..., None, None]
        out = out - 0.5 * (fwd + bwd)
    return out


def apply_D_open(Ub, psi, kappa, dagger=False):
    """D_b on one block given as a small array [l0..l3, ...] with Dirichlet
    (open) boundaries in every direction: hops leaving the array are dropped."""
    m0 = mass_from_kappa(kappa)
    s = -1.0 if dagger else 1.0
    out = (4.0 + m0) * psi
    for mu in range(4):
        Pm = ONE4 - s * GAMMA[mu]
        Pp = ONE4 + s * GAMMA[mu]
        Umu = Ub[..., mu, :, :]
        n = psi.shape[mu]
        fwd = np.zeros_like(psi)
        bwd = np.zeros_like(psi)
        sl_lo = [slice(None)] * 4
        sl_hi = [slice(None)] * 4
        sl_lo[mu] = slice(0, n - 1)
        sl_hi[mu] = slice(1, n)
        sl_lo, sl_hi = tuple(sl_lo), tuple(sl_hi)
        # x in [0, n-2]: U(x,mu)(1-gamma)psi(x+mu)
        fwd[sl_lo] = _colour(Umu[sl_lo], _spin(Pm, psi[sl_hi]))
        # x in [1, n-1]: U(x-mu,mu)^dag (1+gamma) psi(x-mu)
        bwd[sl_hi] = _colour_dag(Umu[sl_lo], _spin(Pp, psi[sl_lo]))
        out = out - 0.5 * (fwd + bwd)
    return out


def extract_block(field, geom, b):
    """Sub-array of a site field belonging to block b (block index order)."""
    nb = geom.nb
    B = np.unravel_index(b, nb)
    sl = tuple(slice(B[m] * geom.block[m], (B[m] + 1) * geom.block[m]) for m in range(4))
    return field[sl]


def insert_block(field, geom, b, sub):
    nb = geom.nb
    B = np.unravel_index(b, nb)
    sl = tuple(slice(B[m] * geom.block[m], (B[m] + 1) * geom.block[m]) for m in range(4))
    field[sl] = sub


def gamma5(psi):
    g5 = np.array([1.0, 1.0, -1.0, -1.0])
    return psi * g5[:, None]


def dense_matrix(apply, n_sites, shape):
    """Dense matrix of a linear map on spinor fields of the given shape,
    column by column (small lattices only)."""
    n = n_sites * 12
    M = np.empty((n, n), dtype=np.complex128)
    e = np.zeros(n, dtype=np.complex128)
    for k in range(n):
        e[:] = 0
        e[k] = 1.0
        M[:, k] = apply(e.reshape(shape)).reshape(n)
    return M
