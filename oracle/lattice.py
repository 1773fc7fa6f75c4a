"""Lattice geometry of the method.  TEST INFRASTRUCTURE ONLY.

Canonical layout: arrays indexed [x0, x1, x2, x3, ...] with x3 fastest and
mu = 0 the time direction.  Links U[x, mu] connect x to x + mu-hat.

Domain decomposition (Sec. 3, Fig. 1): blocks of extent l_mu tile the
lattice; block coordinates B_mu = x_mu // l_mu, block index lexicographic in
(B0, B1, B2, B3) with B3 fastest, colour = (B0+B1+B2+B3) mod 2 with colour 0
"black".  A black/white checkerboard needs an even number of blocks in every
direction.

Active links (Sec. 3): links with both endpoints in one block and at most one
endpoint on the block boundary.  For blocks with an extent <= 2 no link
satisfies this; there every intra-block link is taken as active (reading of
the paper recorded in the design notes).

Projector P (Sec. 4.4, Eq. (detschur)): on each site of a black block, the
orthogonal projector onto the span of range((1 + gamma_mu)/2) for every +mu
face of the block the site lies on and range((1 - gamma_mu)/2) for every -mu
face.  A hop x -> x + mu-hat into another block carries (1 + gamma_mu) psi(x)
in the backward term of Eq. (Dw), so D_wb only sees that range; two or more
faces span the whole spin space.  Zero on interior and white sites.
"""
import numpy as np

from .gamma import GAMMA, ONE4


def fermion_shift(f, mu, sign):
    """g(x) = f(x + sign*mu-hat) with antiperiodic wrap in time (mu = 0) and
    periodic wrap in space (Eq. (Dw) boundary conditions)."""
    g = np.roll(f, -sign, axis=mu)
    if mu == 0:
        idx = [slice(None)] * g.ndim
        idx[0] = -1 if sign > 0 else 0
        g[tuple(idx)] *= -1.0
    return g


def gauge_shift(f, mu, sign):
    """g(x) = f(x + sign*mu-hat), periodic."""
    return np.roll(f, -sign, axis=mu)


class Geometry:
    def __init__(self, dims, block=None):
        self.dims = tuple(int(d) for d in dims)
        self.block = tuple(int(b) for b in (block if block is not None else dims))
        for L, l in zip(self.dims, self.block):
            if L % l:
                raise ValueError("block extent must divide lattice extent")
        self.V = int(np.prod(self.dims))
        self.Vb = int(np.prod(self.block))
        self.nb = tuple(L // l for L, l in zip(self.dims, self.block))
        self.n_blocks = int(np.prod(self.nb))
        x = np.indices(self.dims)
        self.x = x
        self.parity = x.sum(axis=0) % 2
        self.local = np.stack([x[m] % self.block[m] for m in range(4)])
        self.bcoord = np.stack([x[m] // self.block[m] for m in range(4)])
        b = self.bcoord
        self.block_index = ((b[0] * self.nb[1] + b[1]) * self.nb[2] + b[2]) * self.nb[3] + b[3]
        self.colour = b.sum(axis=0) % 2
        self.colouring_ok = all(n % 2 == 0 for n in self.nb)
        self.site_index = np.arange(self.V).reshape(self.dims)

    # --- block structure -------------------------------------------------
    def fwd_intra(self, mu):
        """True where the hop x -> x + mu-hat stays inside x's block."""
        return self.local[mu] != self.block[mu] - 1

    def bwd_intra(self, mu):
        """True where the hop x -> x - mu-hat stays inside x's block."""
        return self.local[mu] != 0

    def on_block_boundary(self, loc):
        """loc: local coordinates [4, ...]; True where any coordinate sits on a
        block face."""
        out = np.zeros(loc.shape[1:], dtype=bool)
        for m in range(4):
            out |= (loc[m] == 0) | (loc[m] == self.block[m] - 1)
        return out

    def active_links(self):
        """bool [L0, L1, L2, L3, 4]: links updated by the domain sweep."""
        act = np.zeros(self.dims + (4,), dtype=bool)
        small = min(self.block) <= 2
        b0 = self.on_block_boundary(self.local)
        for mu in range(4):
            intra = self.fwd_intra(mu)
            if small:
                act[..., mu] = intra
                continue
            loc1 = self.local.copy()
            loc1[mu] = loc1[mu] + 1
            b1 = self.on_block_boundary(loc1)
            act[..., mu] = intra & ((b0.astype(int) + b1.astype(int)) <= 1)
        return act

    def block_colours(self):
        """colour (0 black, 1 white) of every block, in block index order."""
        B = np.indices(self.nb).reshape(4, -1)
        return B.sum(axis=0) % 2

    def black_sites(self):
        return self.colour == 0

    def projector(self):
        """P as a per-site 4x4 spin matrix, shape [L0, L1, L2, L3, 4, 4]."""
        if not self.colouring_ok:
            raise ValueError("Schur complement needs an even number of blocks per direction")
        P = np.zeros(self.dims + (4, 4), dtype=np.complex128)
        nface = np.zeros(self.dims, dtype=int)
        single = np.zeros(self.dims + (4, 4), dtype=np.complex128)
        for mu in range(4):
            plus = self.local[mu] == self.block[mu] - 1
            minus = self.local[mu] == 0
            for mask, sgn in ((plus, +1.0), (minus, -1.0)):
                nface += mask
                single[mask] = 0.5 * (ONE4 + sgn * GAMMA[mu])
        black = self.black_sites()
        one = black & (nface == 1)
        many = black & (nface >= 2)
        P[one] = single[one]
        P[many] = ONE4
        return P

    def dim_projector(self):
        """Rank of P (complex dimension of the noise space of the Schur step)."""
        P = self.projector()
        spin_rank = np.real(np.trace(P, axis1=-2, axis2=-1)).round().astype(int)
        return int(3 * spin_rank.sum())

    def translate(self, U, s):
        """Random translation (Sec. 3): U'(x) = U(x - s), periodic."""
        return np.roll(U, shift=tuple(s), axis=(0, 1, 2, 3))
