"""HYP-smeared links and the HYP plaquette action of the parametrised filter
levels (App. C; Sec. 5: "one level of smearing" with the parameters of the
HYP construction of Hasenfratz and Knechtli, Phys. Rev. D 64 (2001) 034504).
TEST INFRASTRUCTURE ONLY: imported by tests, the package's smoke check and
the benchmark's CPU baseline, never by the product path.

One level of HYP smearing builds the fat link V(x,mu) in three steps, each
a weighted sum of the link and its staples followed by a projection onto
SU(3), and all of them confined to the hypercubes that contain the link:

  Vbar(x,mu;nu,rho) = Proj[(1 - a3) U(x,mu)
        + a3/2 sum_{+-eta} staple_eta(U, U)(x,mu)],
      eta the one direction different from mu, nu and rho;
  Vtil(x,mu;nu) = Proj[(1 - a2) U(x,mu)
        + a2/4 sum_{rho != mu,nu} sum_{+-} staple_rho(Vbar(.,rho;nu,mu), Vbar(.,mu;rho,nu))(x,mu)];
  V(x,mu) = Proj[(1 - a1) U(x,mu)
        + a1/6 sum_{nu != mu} sum_{+-} staple_nu(Vtil(.,nu;mu), Vtil(.,mu;nu))(x,mu)];

with staple_nu(T, W)(x,mu) = T(x,nu) W(x+nu,mu) T(x+mu,nu)^dag in the
positive direction and T(x-nu,nu)^dag W(x-nu,mu) T(x-nu+mu,nu) in the
negative one, and (a1, a2, a3) = (0.75, 0.6, 0.3).

Projection (the paper does not state one; reading recorded in the design
notes): the unitary polar factor W = M (M^dag M)^{-1/2}, then the phase of
det W removed with the principal cube root,
Proj[M] = W exp(-i arg(det W) / 3), arg in (-pi, pi].  It is gauge
covariant, Proj[g M h^dag] = g Proj[M] h^dag for g, h in SU(3), and leaves
SU(3) matrices unchanged.

Block HYP action S^(1) = sum_b S_HYP,b (reading): S_HYP,b is Eq. (Sw) on the
fat links, restricted to the plaquettes whose four corners lie in block b.
A fat link inside a block depends only on links inside that block and on
links that are never active (on a neighbour block's face, or crossing a
face), so with blocks of extent >= 3 S_HYP,b changes only with the active
links of b and the HYP filter level factorises over blocks.  A plaquette
across a face would combine fat links changed by two blocks.
"""
import numpy as np

from .gauge import dag
from .lattice import gauge_shift

ALPHA = (0.75, 0.6, 0.3)


def project_su3(M):
    """Proj[M] for 3x3 matrices of any leading shape (see the module text)."""
    H = dag(M) @ M
    w, Q = np.linalg.eigh(H)
    inv_sqrt = np.einsum("...ij,...j,...kj->...ik", Q, 1.0 / np.sqrt(w), np.conj(Q))
    W = M @ inv_sqrt
    phase = np.angle(np.linalg.det(W))
    return W * np.exp(-1j * phase / 3.0)[..., None, None]


def staple(T, W, mu, nu, sign):
    """staple_nu(T, W)(x, mu) for fields T (links in direction nu) and W
    (links in direction mu), each [L0..L3, 3, 3]."""
    if sign > 0:
        return T @ gauge_shift(W, nu, +1) @ dag(gauge_shift(T, mu, +1))
    Tm = gauge_shift(T, nu, -1)
    return dag(Tm) @ gauge_shift(W, nu, -1) @ gauge_shift(Tm, mu, +1)


def _others(*dirs):
    return [d for d in range(4) if d not in dirs]


def smear(U, alpha=ALPHA):
    """Fat links V[..., mu, 3, 3] of one level of HYP smearing."""
    a1, a2, a3 = alpha
    Ul = [U[..., mu, :, :] for mu in range(4)]
    # level 3: Vbar[(mu, frozenset{nu, rho})]
    vbar = {}
    for mu in range(4):
        for nu in range(4):
            for rho in range(nu + 1, 4):
                if mu in (nu, rho):
                    continue
                (eta,) = _others(mu, nu, rho)
                S = staple(Ul[eta], Ul[mu], mu, eta, +1) + staple(Ul[eta], Ul[mu], mu, eta, -1)
                vbar[(mu, frozenset((nu, rho)))] = project_su3((1 - a3) * Ul[mu] + (a3 / 2) * S)
    # level 2: Vtil[(mu, nu)]
    vtil = {}
    for mu in range(4):
        for nu in range(4):
            if nu == mu:
                continue
            S = np.zeros_like(Ul[mu])
            for rho in _others(mu, nu):
                T = vbar[(rho, frozenset((nu, mu)))]
                W = vbar[(mu, frozenset((rho, nu)))]
                S = S + staple(T, W, mu, rho, +1) + staple(T, W, mu, rho, -1)
            vtil[(mu, nu)] = project_su3((1 - a2) * Ul[mu] + (a2 / 4) * S)
    # level 1: V[mu]
    V = np.empty_like(U)
    for mu in range(4):
        S = np.zeros_like(Ul[mu])
        for nu in _others(mu):
            T = vtil[(nu, mu)]
            W = vtil[(mu, nu)]
            S = S + staple(T, W, mu, nu, +1) + staple(T, W, mu, nu, -1)
        V[..., mu, :, :] = project_su3((1 - a1) * Ul[mu] + (a1 / 6) * S)
    return V


def block_plaquette_action(V, geom):
    """Eq. (Sw) (without beta) on the links V, per block, restricted to the
    plaquettes whose four corners lie in the block."""
    out = np.zeros(geom.n_blocks)
    for mu in range(4):
        for nu in range(mu + 1, 4):
            Vm, Vn = V[..., mu, :, :], V[..., nu, :, :]
            P = Vm @ gauge_shift(Vn, mu, +1) @ dag(gauge_shift(Vm, nu, +1)) @ dag(Vn)
            s = (3.0 - np.real(np.trace(P, axis1=-2, axis2=-1))) / 3.0
            inside = (geom.local[mu] <= geom.block[mu] - 2) & (geom.local[nu] <= geom.block[nu] - 2)
            out += np.bincount(geom.block_index[inside], weights=s[inside], minlength=geom.n_blocks)
    return out


def block_hyp_action(U, geom, alpha=ALPHA):
    """S_HYP,b for every block."""
    return block_plaquette_action(smear(U, alpha), geom)


def block_hyp_change(U, Up, geom, alpha=ALPHA):
    """Delta S_HYP,b = S_HYP,b(U') - S_HYP,b(U) for every block."""
    return block_hyp_action(Up, geom, alpha) - block_hyp_action(U, geom, alpha)
