"""Stochastic determinant-ratio estimates.  TEST INFRASTRUCTURE ONLY.

Eq. (stacc): min{1, det(M^dagger M)^-1} -> min{1, exp(-|M eta|^2 + |eta|^2)}.
Eq. (gfparam): U_i = ((N-i)/N) U + (i/N) U',  i = 0..N.
Eq. (Mparam), (staccN): M_i = D(U_{i+1})^-1 D(U_i), one noise xi_i per
factor, Delta = sum_i (|M_i xi_i|^2 - |xi_i|^2).
(Relative gauge fixing, Sec. 4.2, is not applied: g = 1.)

Block level: D -> D_b, one Delta_b per block b (Eq. (4step) step 1 with the
block determinants estimated stochastically).

Global level, Sec. 4.4: D-hat = 1 - Q, Q = D_bb^-1 D_bw D_ww^-1 D_wb,
det(1 - Q) = det(1 - PQ) (Eq. (detschur)), noise on range(P), and
(1 - PQ)^-1 = 1 - P D^-1 D_wb (Eq. (inverseschur), D_wb padded with zeros).

Noise: draw map TAG_NOISE with stream = (level << 32) | i, level 1 for the
block level and 2 for the global level.  For the global level the full
12-component noise xi' is drawn on every site and xi = P xi' (an orthogonal
projection of an isotropic complex Gaussian is an isotropic complex Gaussian
on range(P)).

Mode 'independent' (diagnostic, not for accept/reject): every factor uses the
un-interpolated pair, M = D(U')^-1 D(U), with an independent noise each.
"""
import numpy as np

from . import philox
from .dirac import apply_D, apply_D_open, extract_block, insert_block
from .linalg import cgnr, norm2

LEVEL_BLOCK = 1
LEVEL_GLOBAL = 2


def interpolate(U, Up, i, N):
    """Eq. (gfparam)."""
    return ((N - i) / N) * U + (i / N) * Up


def pair(U, Up, i, N, mode):
    if mode == "independent":
        return U, Up
    return interpolate(U, Up, i, N), interpolate(U, Up, i + 1, N)


def noise(geom, seed, counter, level, i):
    z = philox.noise_field(seed, counter, (level << 32) | i, geom.V)
    return z.reshape(geom.dims + (4, 3))


def solve_blocks(U, rhs, geom, kappa, blocks, tol):
    """Solve D_b y_b = rhs_b for the listed blocks (Dirichlet block operator on
    the block-local array).  Other sites of the result are zero."""
    y = np.zeros_like(rhs)
    for b in blocks:
        Ub = extract_block(U, geom, b)
        rb = extract_block(rhs, geom, b)
        xb, _, _ = cgnr(lambda v: apply_D_open(Ub, v, kappa),
                        lambda v: apply_D_open(Ub, v, kappa, dagger=True), rb, tol=tol)
        insert_block(y, geom, b, xb)
    return y


def solve_full(U, rhs, geom, kappa, tol):
    x, it, rel = cgnr(lambda v: apply_D(U, v, kappa),
                      lambda v: apply_D(U, v, kappa, dagger=True), rhs, tol=tol)
    return x


def block_sq_norms(f, geom):
    """|f_b|^2 for every block b."""
    n2 = np.sum(np.abs(f) ** 2, axis=(-1, -2))
    return np.bincount(geom.block_index.reshape(-1), weights=n2.reshape(-1), minlength=geom.n_blocks)


def block_level(U, Up, geom, kappa, N, seed, counter, tol=1e-13, mode="interp", blocks=None):
    """Delta contributions [n_blocks, N]: entry (b, i) = |M_{b,i} xi_i|_b^2 - |xi_i|_b^2
    with M_{b,i} = D_b(U_{i+1})^-1 D_b(U_i).  Blocks not listed are NaN."""
    if blocks is None:
        blocks = range(geom.n_blocks)
    blocks = list(blocks)
    out = np.full((geom.n_blocks, N), np.nan)
    for i in range(N):
        Ua, Ub = pair(U, Up, i, N, mode)
        xi = noise(geom, seed, counter, LEVEL_BLOCK, i)
        eta = apply_D(Ua, xi, kappa, geom, mode="block")
        y = solve_blocks(Ub, eta, geom, kappa, blocks, tol)
        ny = block_sq_norms(y, geom)
        nx = block_sq_norms(xi, geom)
        for b in blocks:
            out[b, i] = ny[b] - nx[b]
    return out


def project(P, psi):
    return np.einsum("...st,...tc->...sc", P, psi)


def one_minus_PQ(U, xi, geom, kappa, P, tol):
    """(1 - PQ) xi for xi supported on black sites."""
    black = geom.black_sites()[..., None, None]
    white = ~black
    col = geom.block_colours()
    blacks = [b for b in range(geom.n_blocks) if col[b] == 0]
    whites = [b for b in range(geom.n_blocks) if col[b] == 1]
    t1 = apply_D(U, xi * black, kappa, geom, mode="inter") * white      # D_wb xi
    t2 = solve_blocks(U, t1, geom, kappa, whites, tol)                  # D_ww^-1
    t3 = apply_D(U, t2, kappa, geom, mode="inter") * black              # D_bw
    t4 = solve_blocks(U, t3, geom, kappa, blacks, tol)                  # D_bb^-1
    return xi - project(P, t4)


def inv_one_minus_PQ(U, s, geom, kappa, P, tol):
    """(1 - PQ)^-1 s = s - P [D^-1 (0, D_wb s)]_black (Eq. (inverseschur))."""
    black = geom.black_sites()[..., None, None]
    white = ~black
    y = apply_D(U, s * black, kappa, geom, mode="inter") * white
    z = solve_full(U, y, geom, kappa, tol)
    return s - project(P, z * black)


def global_level(U, Up, geom, kappa, N, seed, counter, tol=1e-13, mode="interp"):
    """Delta contributions [N] of the Schur-complement step:
    |(1-PQ(U_{i+1}))^-1 (1-PQ(U_i)) xi_i|^2 - |xi_i|^2."""
    P = geom.projector()
    out = np.empty(N)
    for i in range(N):
        Ua, Ub = pair(U, Up, i, N, mode)
        xi = project(P, noise(geom, seed, counter, LEVEL_GLOBAL, i))
        v = one_minus_PQ(Ua, xi, geom, kappa, P, tol)
        w = inv_one_minus_PQ(Ub, v, geom, kappa, P, tol)
        out[i] = norm2(w) - norm2(xi)
    return out
