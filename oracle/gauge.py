"""Gauge-field routines.  TEST INFRASTRUCTURE ONLY.

* Link generator U = exp(i eps H), H = sum_a omega_a lambda_a / 2 with
  Gell-Mann lambda_a and omega_a ~ N(0,1) (draw map TAG_LINK); the Hermitian
  exponential is taken through numpy's eigendecomposition, then the matrix is
  reunitarised.
* Reunitarisation: Gram-Schmidt on rows 0 and 1, row 2 = conj(row0 x row1).
* Wilson plaquette action, Eq. (Sw): S_w = (1/6) sum over oriented plaquettes
  of ReTr(1 - U_p) = (1/3) sum over x, mu<nu of ReTr(1 - U_{mu nu}(x)).
* Pure-gauge proposal (Sec. 6): Cabibbo-Marinari updates in the SU(2)
  subgroups (0,1), (0,2), (1,2), taken per link in forward or reversed order
  with probability 1/2.  Heatbath in each subgroup samples a0 with density
  sqrt(1-a0^2) exp(alpha a0), alpha = 2 beta k / 3, by Kennedy-Pendleton
  (Phys. Lett. B156 (1985) 393) for alpha >= 2 and by Creutz's method
  (Phys. Rev. D21 (1980) 2308) for alpha < 2; overrelaxation is the SU(2)
  reflection R = (v^dagger)^2 (Adler; Petronzio-Vicari).  One iteration is
  HB + n_or OR sweeps in forward subset order, then n_or OR + HB in reversed
  order (symmetrised, App. A.1).  Subsets are the checkerboard (mu, site
  parity) of active links, with the block colour as outermost loop when the
  blocks have an extent <= 2.
"""
import numpy as np

from . import philox
from .lattice import gauge_shift

GELL_MANN = np.zeros((8, 3, 3), dtype=np.complex128)
GELL_MANN[0][0, 1] = GELL_MANN[0][1, 0] = 1
GELL_MANN[1][0, 1] = -1j
GELL_MANN[1][1, 0] = 1j
GELL_MANN[2][0, 0] = 1
GELL_MANN[2][1, 1] = -1
GELL_MANN[3][0, 2] = GELL_MANN[3][2, 0] = 1
GELL_MANN[4][0, 2] = -1j
GELL_MANN[4][2, 0] = 1j
GELL_MANN[5][1, 2] = GELL_MANN[5][2, 1] = 1
GELL_MANN[6][1, 2] = -1j
GELL_MANN[6][2, 1] = 1j
GELL_MANN[7] = np.diag([1, 1, -2]) / np.sqrt(3)

SUBGROUPS = ((0, 1), (0, 2), (1, 2))
KP_THRESHOLD = 2.0
MAX_ATTEMPTS = 1000


def dag(M):
    return np.conj(np.swapaxes(M, -1, -2))


def reunitarise(U):
    """Project 3x3 matrices (any leading shape) onto SU(3) by Gram-Schmidt."""
    U = np.array(U, dtype=np.complex128, copy=True)
    r0 = U[..., 0, :]
    r0 = r0 / np.sqrt(np.sum(np.abs(r0) ** 2, axis=-1, keepdims=True))
    r1 = U[..., 1, :]
    r1 = r1 - np.sum(np.conj(r0) * r1, axis=-1, keepdims=True) * r0
    r1 = r1 / np.sqrt(np.sum(np.abs(r1) ** 2, axis=-1, keepdims=True))
    r2 = np.conj(np.cross(r0, r1))
    return np.stack([r0, r1, r2], axis=-2)


def hermitian_generators(omega):
    """H = sum_a omega_a lambda_a / 2 for omega[..., 8]."""
    return 0.5 * np.einsum("...a,aij->...ij", omega, GELL_MANN)


def expm_i_hermitian(H, eps):
    """exp(i eps H) for Hermitian H[..., 3, 3] via eigendecomposition."""
    w, V = np.linalg.eigh(H)
    return np.einsum("...ij,...j,...kj->...ik", V, np.exp(1j * eps * w), np.conj(V))


def generate_links(dims, eps, seed):
    """Synthetic gauge field U = reunitarise(exp(i eps H)), shape [dims, 4, 3, 3]."""
    V = int(np.prod(dims))
    om = philox.link_omegas(seed, V)
    U = expm_i_hermitian(hermitian_generators(om), eps)
    return reunitarise(U).reshape(tuple(dims) + (4, 3, 3))


def plaquette_field(U, mu, nu):
    """U_{mu nu}(x) = U(x,mu) U(x+mu,nu) U(x+nu,mu)^dag U(x,nu)^dag."""
    Umu = U[..., mu, :, :]
    Unu = U[..., nu, :, :]
    return Umu @ gauge_shift(Unu, mu, +1) @ dag(gauge_shift(Umu, nu, +1)) @ dag(Unu)


def wilson_action(U):
    """S_w of Eq. (Sw) without the factor beta."""
    s = 0.0
    for mu in range(4):
        for nu in range(mu + 1, 4):
            P = plaquette_field(U, mu, nu)
            s += np.sum(3.0 - np.real(np.trace(P, axis1=-2, axis2=-1)))
    return s / 3.0


def mean_plaquette(U):
    """<ReTr U_p>/3 averaged over x and the 6 planes."""
    tot = 0.0
    for mu in range(4):
        for nu in range(mu + 1, 4):
            tot += np.mean(np.real(np.trace(plaquette_field(U, mu, nu), axis1=-2, axis2=-1)))
    return tot / 18.0


def staples(U, mu):
    """A(x) = sum_{nu != mu} [U(x+mu,nu) U(x+nu,mu)^dag U(x,nu)^dag
    + U(x+mu-nu,nu)^dag U(x-nu,mu)^dag U(x-nu,nu)], so that the plaquettes
    containing U(x,mu) sum to ReTr(U(x,mu) A(x))."""
    A = np.zeros(U.shape[:4] + (3, 3), dtype=np.complex128)
    Umu = U[..., mu, :, :]
    for nu in range(4):
        if nu == mu:
            continue
        Unu = U[..., nu, :, :]
        up = gauge_shift(Unu, mu, +1) @ dag(gauge_shift(Umu, nu, +1)) @ dag(Unu)
        Unu_m = gauge_shift(Unu, nu, -1)
        Umu_m = gauge_shift(Umu, nu, -1)
        Unu_pm = gauge_shift(Unu_m, mu, +1)
        dn = dag(Unu_pm) @ dag(Umu_m) @ Unu_m
        A += up + dn
    return A


# --- SU(2) subgroup algebra (2x2 complex matrices) ---------------------------

def quat_to_mat(q):
    """(q0, q1, q2, q3) -> q0 + i q.sigma as 2x2 complex."""
    m = np.empty(q.shape[:-1] + (2, 2), dtype=np.complex128)
    m[..., 0, 0] = q[..., 0] + 1j * q[..., 3]
    m[..., 0, 1] = q[..., 2] + 1j * q[..., 1]
    m[..., 1, 0] = -q[..., 2] + 1j * q[..., 1]
    m[..., 1, 1] = q[..., 0] - 1j * q[..., 3]
    return m


def su2_part(w):
    """Quaternion components of the SU(2)-proportional part of 2x2 w."""
    r0 = 0.5 * np.real(w[..., 0, 0] + w[..., 1, 1])
    r1 = 0.5 * np.imag(w[..., 0, 1] + w[..., 1, 0])
    r2 = 0.5 * np.real(w[..., 0, 1] - w[..., 1, 0])
    r3 = 0.5 * np.imag(w[..., 0, 0] - w[..., 1, 1])
    return np.stack([r0, r1, r2, r3], axis=-1)


def sample_a0(alpha, seed, sweep, link, code):
    """a0 with density sqrt(1-a0^2) exp(alpha a0) on [-1, 1], one per link.
    Returns (a0, failed) where failed marks links that hit MAX_ATTEMPTS."""
    n = alpha.shape[0]
    a0 = np.ones(n)
    pending = np.ones(n, dtype=bool)
    kp = alpha >= KP_THRESHOLD
    attempt = 0
    while pending.any() and attempt < MAX_ATTEMPTS:
        idx = np.nonzero(pending)[0]
        u = philox.uniforms(seed, philox.TAG_HB, philox.make_ctr(sweep, link[idx], code, attempt))
        al = alpha[idx]
        # Kennedy-Pendleton: x = 1 - a0 ~ Gamma(3/2)/alpha, accept w.p. sqrt(1 - x/2)
        x = -(np.log(u[:, 0]) + np.cos(2.0 * np.pi * u[:, 1]) ** 2 * np.log(u[:, 2])) / al
        acc_kp = u[:, 3] ** 2 <= 1.0 - 0.5 * x
        # Creutz: a0 ~ exp(alpha a0) on [-1,1] by inversion, accept w.p. sqrt(1 - a0^2)
        c = 1.0 + np.log(u[:, 0] + (1.0 - u[:, 0]) * np.exp(-2.0 * al)) / al
        acc_cr = u[:, 1] ** 2 <= 1.0 - c * c
        cand = np.where(kp[idx], 1.0 - x, c)
        acc = np.where(kp[idx], acc_kp, acc_cr)
        a0[idx[acc]] = cand[acc]
        pending[idx[acc]] = False
        attempt += 1
    return a0, pending


def su2_heatbath_element(a0, seed, sweep, link, code):
    """x = a0 + i a.sigma with a uniform on the sphere of radius sqrt(1-a0^2)."""
    u = philox.uniforms(seed, philox.TAG_HB, philox.make_ctr(sweep, link, code, 0))
    cth = 2.0 * u[:, 0] - 1.0
    sth = np.sqrt(np.maximum(0.0, 1.0 - cth * cth))
    phi = 2.0 * np.pi * u[:, 1]
    rad = np.sqrt(np.maximum(0.0, 1.0 - a0 * a0))
    q = np.stack([a0, rad * sth * np.cos(phi), rad * sth * np.sin(phi), rad * cth], axis=-1)
    return quat_to_mat(q)


def update_links(Ul, A, beta, kind, seed, sweep, link):
    """Cabibbo-Marinari update of the links Ul[n,3,3] with staples A[n,3,3].
    kind: 'hb' or 'or'.  Returns (new links, number of failed a0 draws)."""
    Ul = Ul.copy()
    n = Ul.shape[0]
    u_ord = philox.uniforms(seed, philox.TAG_HB, philox.make_ctr(sweep, link, 0, 0))[:, 0]
    forward = u_ord < 0.5
    failed = 0
    for k in range(3):
        sg = np.where(forward, k, 2 - k)
        i = np.array([SUBGROUPS[s][0] for s in sg])
        j = np.array([SUBGROUPS[s][1] for s in sg])
        W = Ul @ A
        ar = np.arange(n)
        w = np.empty((n, 2, 2), dtype=np.complex128)
        w[:, 0, 0] = W[ar, i, i]
        w[:, 0, 1] = W[ar, i, j]
        w[:, 1, 0] = W[ar, j, i]
        w[:, 1, 1] = W[ar, j, j]
        r = su2_part(w)
        kn = np.sqrt(np.sum(r * r, axis=-1))
        ok = kn > 0.0
        v = np.where(ok[:, None], r / np.where(ok, kn, 1.0)[:, None], np.array([1.0, 0, 0, 0]))
        vdag = quat_to_mat(v * np.array([1.0, -1.0, -1.0, -1.0]))
        if kind == "hb":
            alpha = 2.0 * beta * kn / 3.0
            alpha = np.where(ok, alpha, 1.0)
            a0, fail = sample_a0(alpha, seed, sweep, link, 1 + 2 * k)
            failed += int(fail.sum())
            x = su2_heatbath_element(a0, seed, sweep, link, 2 + 2 * k)
            R = x @ vdag
            R = np.where((ok & ~fail)[:, None, None], R, np.eye(2))
        else:
            R = vdag @ vdag
            R = np.where(ok[:, None, None], R, np.eye(2))
        rows_i = Ul[ar, i, :]
        rows_j = Ul[ar, j, :]
        Ul[ar, i, :] = R[:, 0, 0, None] * rows_i + R[:, 0, 1, None] * rows_j
        Ul[ar, j, :] = R[:, 1, 0, None] * rows_i + R[:, 1, 1, None] * rows_j
    return Ul, failed


def sweep_subsets(geom, active):
    """Ordered checkerboard subsets [(mu, mask)] of active links."""
    subsets = []
    colours = (0, 1) if min(geom.block) <= 2 else (None,)
    for c in colours:
        for mu in range(4):
            for p in (0, 1):
                m = active[..., mu] & (geom.parity == p)
                if c is not None:
                    m = m & (geom.colour == c)
                subsets.append((mu, m))
    return subsets


def one_sweep(U, geom, subsets, beta, kind, seed, sweep):
    failed = 0
    for mu, mask in subsets:
        if not mask.any():
            continue
        A = staples(U, mu)[mask]
        link = (geom.site_index[mask] * 4 + mu).astype(np.uint64)
        Unew, f = update_links(U[..., mu, :, :][mask], A, beta, kind, seed, sweep, link)
        failed += f
        Umu = U[..., mu, :, :]
        Umu[mask] = Unew
        U[..., mu, :, :] = Umu
    return failed


def domain_sweep(U, geom, beta, n_iter, n_or, seed, sweep0):
    """Proposal T_0 on the active links: n_iter symmetrised iterations.
    Returns (new field, next sweep id, failed draws).  Active links are
    reunitarised at the end."""
    U = np.array(U, copy=True)
    active = geom.active_links()
    subsets = sweep_subsets(geom, active)
    rev = subsets[::-1]
    s = int(sweep0)
    failed = 0
    for _ in range(n_iter):
        failed += one_sweep(U, geom, subsets, beta, "hb", seed, s)
        s += 1
        for _ in range(n_or):
            one_sweep(U, geom, subsets, beta, "or", seed, s)
            s += 1
        for _ in range(n_or):
            one_sweep(U, geom, rev, beta, "or", seed, s)
            s += 1
        failed += one_sweep(U, geom, rev, beta, "hb", seed, s)
        s += 1
    U[active] = reunitarise(U[active])
    return U, s, failed
