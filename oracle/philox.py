"""Philox-4x64-10 and the random-number draw map of the method.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Generator
---------
Philox-4x64 with 10 rounds, from its published definition (J. K. Salmon,
M. A. Moraes, R. O. Dror, D. E. Shaw, "Parallel random numbers: as easy as
1, 2, 3", SC'11): a 256-bit counter (four 64-bit words) and a 128-bit key
(two words); one round maps

    (hi0, lo0) = M0 * c0,  (hi1, lo1) = M1 * c2      (128-bit products)
    c' = (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0)

and the key is bumped by the Weyl constants (W0, W1) between rounds.
Pinned against ``numpy.random.Philox`` (an independent implementation of the
same generator) in ``tests/test_oracle_rng.py``.

Draw map (shared convention with the CUDA path, written out independently
there).  ``site`` is the canonical lexicographic site index (x3 fastest),
``link = 4*site + mu``.

* uniform from a 64-bit word w:  u = ((w >> 12) + 1/2) * 2^-52, exact in
  double precision and inside [2^-53, 1 - 2^-53].
* TAG_LINK  (1): ctr = (link, j, 0, 0), j = 0, 1 -> 8 uniforms -> 4
  Box-Muller pairs -> omega_0..omega_7 ~ N(0,1).
* TAG_NOISE (2): ctr = (counter, stream, site, j), j = 0..5; call j gives the
  complex components 2j (from u0,u1) and 2j+1 (from u2,u3) of the 12-vector
  (spin*3 + colour); z = sqrt(-ln u_a) * exp(2 pi i u_b), so Re z and Im z are
  N(0, 1/2) and E|z|^2 = 1, the measure of Eq. (pfmeasure).
* TAG_HB    (3): ctr = (sweep, link, code, attempt); code 0: subgroup order
  (u0 < 1/2 -> forward); code 1+2k: attempts of the SU(2) a0 draw at subgroup
  position k; code 2+2k: the direction on the 2-sphere at position k.
* TAG_ACCEPT(4): ctr = (counter, level, block, 0) -> u0 for accept/reject.
* TAG_SHIFT (5): ctr = (counter, 0, 0, 0) -> u_mu -> random translation.
"""
import numpy as np

M0 = 0xD2E7470EE14C6C93
M1 = 0xCA5A826395121157
W0 = 0x9E3779B97F4A7C15
W1 = 0xBB67AE8584CAA73B

TAG_LINK = 1
TAG_NOISE = 2
TAG_HB = 3
TAG_ACCEPT = 4
TAG_SHIFT = 5

_M32 = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)


def _mulhilo(m, b):
    """128-bit product of the constant ``m`` and the uint64 array ``b``,
    returned as (hi, lo) 64-bit words (schoolbook on 32-bit halves)."""
    m = int(m)
    a0 = np.uint64(m & 0xFFFFFFFF)
    a1 = np.uint64(m >> 32)
    b0 = b & _M32
    b1 = b >> _S32
    p00 = a0 * b0
    p01 = a0 * b1
    p10 = a1 * b0
    p11 = a1 * b1
    mid = (p00 >> _S32) + (p01 & _M32) + (p10 & _M32)
    hi = p11 + (p01 >> _S32) + (p10 >> _S32) + (mid >> _S32)
    lo = np.uint64(m) * b
    return hi, lo


def philox4x64(ctr, key):
    """Philox-4x64-10 block function.

    ctr: uint64 array [..., 4]; key: pair of ints/uint64 (or arrays broadcastable
    against ctr[..., 0]).  Returns uint64 array [..., 4].
    """
    with np.errstate(over="ignore"):
        c = np.asarray(ctr, dtype=np.uint64)
        c0, c1, c2, c3 = (c[..., i].copy() for i in range(4))
        k0 = np.asarray(key[0], dtype=np.uint64) + np.zeros_like(c0)
        k1 = np.asarray(key[1], dtype=np.uint64) + np.zeros_like(c0)
        w0 = np.uint64(W0)
        w1 = np.uint64(W1)
        for r in range(10):
            if r > 0:
                k0 = k0 + w0
                k1 = k1 + w1
            hi0, lo0 = _mulhilo(M0, c0)
            hi1, lo1 = _mulhilo(M1, c2)
            c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
        return np.stack([c0, c1, c2, c3], axis=-1)


def to_uniform(w):
    """64-bit words -> doubles in the open interval (0, 1)."""
    return ((np.asarray(w, dtype=np.uint64) >> np.uint64(12)).astype(np.float64) + 0.5) * (2.0 ** -52)


def uniforms(seed, tag, ctr):
    """Four uniforms per counter: array [..., 4]."""
    return to_uniform(philox4x64(ctr, (np.uint64(seed), np.uint64(tag))))


def make_ctr(*words, shape=None):
    """Stack counter words (scalars or arrays, broadcast) into [..., 4] uint64."""
    ws = [np.asarray(w, dtype=np.uint64) for w in words]
    while len(ws) < 4:
        ws.append(np.uint64(0))
    b = np.broadcast_arrays(*ws)
    return np.stack(b, axis=-1)


def link_omegas(seed, n_sites):
    """omega[link, a], a = 0..7, standard normal, for links 0..4*n_sites-1
    (draw map TAG_LINK)."""
    link = np.arange(4 * n_sites, dtype=np.uint64)
    out = np.empty((4 * n_sites, 8))
    for j in range(2):
        u = uniforms(seed, TAG_LINK, make_ctr(link, j))
        for k in range(2):
            r = np.sqrt(-2.0 * np.log(u[:, 2 * k]))
            th = 2.0 * np.pi * u[:, 2 * k + 1]
            out[:, 4 * j + 2 * k] = r * np.cos(th)
            out[:, 4 * j + 2 * k + 1] = r * np.sin(th)
    return out


def noise_field(seed, counter, stream, n_sites):
    """Complex Gaussian 12-vectors per site, shape [n_sites, 12]
    (draw map TAG_NOISE); E|z|^2 = 1 per component."""
    site = np.arange(n_sites, dtype=np.uint64)
    z = np.empty((n_sites, 12), dtype=np.complex128)
    for j in range(6):
        u = uniforms(seed, TAG_NOISE, make_ctr(counter, stream, site, j))
        for m in range(2):
            r = np.sqrt(-np.log(u[:, 2 * m]))
            th = 2.0 * np.pi * u[:, 2 * m + 1]
            z[:, 2 * j + m] = r * (np.cos(th) + 1j * np.sin(th))
    return z


def accept_uniform(seed, counter, level, block):
    """u0 for the accept/reject decision of (counter, level, block)."""
    return float(uniforms(seed, TAG_ACCEPT, make_ctr(counter, level, block))[0])


def shift_vector(seed, counter, dims):
    """Random translation vector s_mu in [0, L_mu) (draw map TAG_SHIFT)."""
    u = uniforms(seed, TAG_SHIFT, make_ctr(counter))
    return tuple(min(int(np.floor(u[m] * dims[m])), dims[m] - 1) for m in range(4))
