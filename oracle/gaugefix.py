"""Relative gauge fixing of a pair of gauge fields (Sec. 4.2 and App. B).
TEST INFRASTRUCTURE ONLY: imported by tests, the package's smoke check and
the benchmark's CPU baseline, never by the product path.

The pair (U, U') is brought close in the sense of the scalar product of
Eq. (sprodgf),
    (U, U') = 1/(12 V) sum_{x,mu} Re Tr{1 - U(x,mu)^dag U'(x,mu)},
by the transformation of Eq. (relgf) with the choice g_1 = g_2^{-1} = g of
Eq. (choiceg), U -> U^g, U' -> U'^{g^{-1}}, where
U^g(x,mu) = g(x) U(x,mu) g(x+mu)^{-1}.  The transformation is defined only on
the interior ("black") points of the blocks, the sites whose eight
neighbours all lie in the same block (Sec. 4.2), so every block is an
independent problem and g = 1 on every block boundary.

App. B solves the local condition min_g Re Tr{1 - (g^dag)^2 Delta} with
Delta = W_f + W_b by the steepest-descent scheme of Davies et al.  Readings
taken here:
  * each step is a transformation h(x) of the current pair, applied as
    U^h and U'^{h^{-1}} (Eq. (choiceg) imposed on every step); Delta(x) is
    then W_f + W_b evaluated on the current pair with g = 1, i.e.
        Delta(x) = sum_mu [U'(x,mu) U(x,mu)^dag + U'(x-mu,mu)^dag U(x-mu,mu)];
  * Eq. (ming) is the step of the relative transformation g^2, which is
    what enters Eq. (eq:GF:fminendform) through (g^dag)^2: the pair's
    relative rotation per step is h(x)^2 = exp(+alpha/2 Y(x)), so each field
    takes h(x) = exp(+alpha/4 Y(x)), Y = Delta - Delta^dag - Tr(Delta -
    Delta^dag)/3.  Under this reading the single-site optimum is
    alpha = 1/|Delta|, about 1/8 near convergence, inside the paper's range
    0.10 - 0.15.  The sign is the one that lowers the functional for the
    convention U^g above (the printed minus sign belongs to the opposite
    convention);
  * theta(x) = Re Tr{Y Y^dag} = -Tr{Y^2} >= 0, and a block has converged
    when the mean of theta over its interior points is below theta_tol
    (1e-3 in App. B);
  * "no convergence" = theta_tol not reached within max_iter steps; the
    block then restarts from the unfixed pair with alpha lowered by 0.01,
    down to alpha_min = 0.10; after the last alpha its final state is kept;
  * every block orders its pair canonically before iterating (the field
    whose first differing real number, in the order (local site, mu, entry),
    is smaller comes first) and hands the two transformations back in the
    caller's order.  Swapping U and U' therefore swaps the outputs exactly,
    in any arithmetic, which is the symmetry detailed balance needs
    (Sec. 4.2: the reverse move uses g~_1 = g_2, g~_2 = g_1).
The endpoints of the interpolation of Eq. (gfparam) are U_0 = U^{g_1} and
U_N = U'^{g_2}; g_1 and g_2 are SU(3) fields (g_2 = g_1^{-1} up to the
non-commutativity of successive steps)."""
import numpy as np

from .gauge import dag, reunitarise
from .lattice import gauge_shift


def interior_mask(geom):
    """True on sites whose eight neighbours lie in the same block."""
    m = np.ones(geom.dims, dtype=bool)
    for mu in range(4):
        m &= (geom.local[mu] >= 1) & (geom.local[mu] <= geom.block[mu] - 2)
    return m


def sprod(U, Up):
    """(U, U') of Eq. (sprodgf)."""
    V = int(np.prod(U.shape[:4]))
    return float(np.sum(np.real(3.0 - np.einsum("...ji,...ji->...", np.conj(U), Up)))) / (12.0 * V)


def block_sprod(U, Up, geom):
    """Eq. (sprodgf) summed over the links (x, mu) with x in each block,
    normalised by 12 Vb."""
    d = np.sum(np.real(3.0 - np.einsum("...ji,...ji->...", np.conj(U), Up)), axis=-1)
    return np.bincount(geom.block_index.ravel(), weights=d.ravel(), minlength=geom.n_blocks) / (12.0 * geom.Vb)


def transform(U, g):
    """U^g(x, mu) = g(x) U(x, mu) g(x + mu)^{-1} for SU(3) g[dims, 3, 3]."""
    out = np.empty_like(U)
    for mu in range(4):
        out[..., mu, :, :] = g @ U[..., mu, :, :] @ dag(gauge_shift(g, mu, +1))
    return out


def _expm_antihermitian(Y):
    """exp(Y) for antihermitian Y[..., 3, 3], from the eigendecomposition of
    the Hermitian matrix -iY."""
    w, V = np.linalg.eigh(-1j * Y)
    return np.einsum("...ij,...j,...kj->...ik", V, np.exp(1j * w), np.conj(V))


def delta(Uh, Uph):
    """Delta(x) = W_f(x) + W_b(x) of App. B on the current pair (g = 1)."""
    D = np.zeros(Uh.shape[:4] + (3, 3), dtype=np.complex128)
    for mu in range(4):
        D += Uph[..., mu, :, :] @ dag(Uh[..., mu, :, :])
        D += gauge_shift(dag(Uph[..., mu, :, :]) @ Uh[..., mu, :, :], mu, -1)
    return D


def generator(D):
    """Y = Delta - Delta^dag - Tr(Delta - Delta^dag)/3 and theta = Re Tr(Y Y^dag)."""
    Y = D - dag(D)
    tr = np.trace(Y, axis1=-2, axis2=-1)
    Y = Y - (tr / 3.0)[..., None, None] * np.eye(3)
    theta = np.real(np.einsum("...ij,...ij->...", Y, np.conj(Y)))
    return Y, theta


def canonical_swap(U, Up, geom):
    """Per block: True when U' comes first in the canonical order (its first
    differing real number, over (local site lexicographic, mu, row, column,
    re/im), is the smaller one).  Blocks where U == U' are not swapped."""
    out = np.zeros(geom.n_blocks, dtype=bool)
    loc = geom.local
    lx = ((loc[0] * geom.block[1] + loc[1]) * geom.block[2] + loc[2]) * geom.block[3] + loc[3]
    a = U.view(np.float64).reshape(geom.dims + (4, 18))
    b = Up.view(np.float64).reshape(geom.dims + (4, 18))
    bi = geom.block_index
    for blk in range(geom.n_blocks):
        m = bi == blk
        order = np.argsort(lx[m], kind="stable")
        ab = a[m][order].reshape(-1)
        bb = b[m][order].reshape(-1)
        diff = np.nonzero(ab != bb)[0]
        if len(diff):
            out[blk] = bb[diff[0]] < ab[diff[0]]
    return out


def relative_gauge_fix(U, Up, geom, alpha0=0.15, alpha_min=0.10, dalpha=0.01, theta_tol=1e-3, max_iter=1000):
    """Transformations (g_1, g_2) with U^{g_1}, U'^{g_2} relatively gauge
    fixed, and per-block (alpha used, steps at that alpha, final mean theta,
    swapped) as a dict of arrays."""
    interior = interior_mask(geom)
    nb = geom.n_blocks
    bi = geom.block_index
    n_int = np.bincount(bi[interior], minlength=nb)
    swap = canonical_swap(U, Up, geom)
    sw_site = swap[bi]
    # canonical pair (A, B): per link, the block of x decides (links that
    # touch an interior point lie inside that point's block)
    sel = sw_site[..., None, None, None]
    A0 = np.where(sel, Up, U)
    B0 = np.where(sel, U, Up)
    eye = np.broadcast_to(np.eye(3, dtype=np.complex128), geom.dims + (3, 3))
    alpha = np.full(nb, float(alpha0))
    steps = np.zeros(nb, dtype=np.int64)
    theta_b = np.zeros(nb)
    done = n_int == 0
    A, B = A0.copy(), B0.copy()
    gA, gB = eye.copy(), eye.copy()
    while not np.all(done):
        Y, theta = generator(delta(A, B))
        theta = np.where(interior, theta, 0.0)
        tb = np.bincount(bi.ravel(), weights=theta.ravel(), minlength=nb) / np.maximum(n_int, 1)
        live = ~done
        theta_b[live] = tb[live]
        conv = live & (tb < theta_tol)
        done |= conv
        live = ~done
        # blocks out of steps at this alpha: restart with a smaller alpha, or stop
        out = live & (steps >= max_iter)
        lower = out & (alpha - dalpha >= alpha_min - 1e-12)
        stop = out & ~lower
        done |= stop
        if np.any(lower):
            alpha[lower] -= dalpha
            steps[lower] = 0
            rs = lower[bi]
            A = np.where(rs[..., None, None, None], A0, A)
            B = np.where(rs[..., None, None, None], B0, B)
            gA = np.where(rs[..., None, None], eye, gA)
            gB = np.where(rs[..., None, None], eye, gB)
            continue
        live = ~done
        if not np.any(live):
            break
        step_site = interior & live[bi]
        h = _expm_antihermitian(0.25 * alpha[bi][..., None, None] * Y)
        h = np.where(step_site[..., None, None], h, eye)
        hd = dag(h)
        for mu in range(4):
            hf = gauge_shift(h, mu, +1)
            A[..., mu, :, :] = h @ A[..., mu, :, :] @ dag(hf)
            B[..., mu, :, :] = hd @ B[..., mu, :, :] @ hf
        gA = h @ gA
        gB = hd @ gB
        steps[live] += 1
    gA, gB = reunitarise(gA), reunitarise(gB)
    s2 = sw_site[..., None, None]
    g1 = np.where(s2, gB, gA)
    g2 = np.where(s2, gA, gB)
    info = {"alpha": alpha, "steps": steps, "theta": theta_b, "swapped": swap, "n_interior": n_int}
    return g1, g2, info


def fixed_pair(U, Up, geom, **kw):
    """(U^{g_1}, U'^{g_2}, info): the endpoints of the interpolation."""
    g1, g2, info = relative_gauge_fix(U, Up, geom, **kw)
    return transform(U, g1), transform(Up, g2), info
