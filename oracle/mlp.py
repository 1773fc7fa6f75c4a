"""Learned delayed-acceptance level: domain features and an FP64 MLP.
TEST INFRASTRUCTURE ONLY.

The paper has no learned level; this follows the mechanism of App. C
("auxiliary action" whose coefficients sum to zero over the later levels):
a deterministic antisymmetric surrogate h(U, U') = -h(U', U) of the block
log det ratio is accepted with min{1, exp(-h_b)} per block, and the next
(stochastic block) level uses Delta_b - h_b, so the chain stays exact.

Features of a domain (block) b, 32 numbers per gauge field:
  f[k]      mean of ReTr U_{mu nu}(x)/3 over plaquettes inside the block,
  f[6 + k]  their population variance,
  f[12 + k] mean over sites with all four clover leaves inside the block of
            Tr(F_{mu nu}^2), F = traceless part of (Q - Q^dagger)/(8i), Q the
            sum of the four leaves,
  f[18..31] = 0,
for the planes k = (0,1), (0,2), (0,3), (1,2), (1,3), (2,3).

Network input z = [f(U_b), f(U'_b)] (64), standardised with a mean / scale
vector; h1 = relu(W1 z + b1), h2 = relu(W2 h1 + b2), n = w3 . h2 + b3;
h = ys (n(f, f') - n(f', f)) / 2 with an output scale ys.  Loss: mean
squared error to Delta_b.
"""
import numpy as np

from .gauge import dag, plaquette_field
from .lattice import gauge_shift

PLANES = ((0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3))
N_FEAT = 32
HIDDEN = 256


def _sh(U, mu, s):
    return gauge_shift(U, mu, s)


def clover_leaves(U, mu, nu):
    """Sum Q of the four plaquette leaves at x in the (mu, nu) plane."""
    Um, Un = U[..., mu, :, :], U[..., nu, :, :]
    L1 = Um @ _sh(Un, mu, +1) @ dag(_sh(Um, nu, +1)) @ dag(Un)
    Um_m = _sh(Um, mu, -1)
    Un_m = _sh(Un, mu, -1)
    L2 = Un @ dag(_sh(Um_m, nu, +1)) @ dag(Un_m) @ Um_m
    Um_mn = _sh(Um_m, nu, -1)
    Un_mn = _sh(Un_m, nu, -1)
    Un_n = _sh(Un, nu, -1)
    L3 = dag(Um_m) @ dag(Un_mn) @ Um_mn @ Un_n
    Um_n = _sh(Um, nu, -1)
    L4 = dag(Un_n) @ Um_n @ _sh(Un_n, mu, +1) @ dag(Um)
    return L1 + L2 + L3 + L4


def domain_features(U, geom):
    """f[b, 32] for every block b (block index order)."""
    nb = geom.n_blocks
    f = np.zeros((nb, N_FEAT))
    bidx = geom.block_index
    loc = geom.local
    l = geom.block
    for k, (mu, nu) in enumerate(PLANES):
        P = np.real(np.trace(plaquette_field(U, mu, nu), axis1=-2, axis2=-1)) / 3.0
        inside = (loc[mu] < l[mu] - 1) & (loc[nu] < l[nu] - 1)
        cnt = np.bincount(bidx[inside], minlength=nb)
        s1 = np.bincount(bidx[inside], weights=P[inside], minlength=nb)
        mean = s1 / np.maximum(cnt, 1)
        dev = (P - mean[bidx]) ** 2
        s2 = np.bincount(bidx[inside], weights=dev[inside], minlength=nb)
        f[:, k] = mean
        f[:, 6 + k] = s2 / np.maximum(cnt, 1)
        Q = clover_leaves(U, mu, nu)
        F = (Q - dag(Q)) / 8j
        tr = np.trace(F, axis1=-2, axis2=-1) / 3.0
        F = F - tr[..., None, None] * np.eye(3)
        trF2 = np.real(np.trace(F @ F, axis1=-2, axis2=-1))
        inner = (loc[mu] >= 1) & (loc[mu] <= l[mu] - 2) & (loc[nu] >= 1) & (loc[nu] <= l[nu] - 2)
        c2 = np.bincount(bidx[inner], minlength=nb)
        s3 = np.bincount(bidx[inner], weights=trF2[inner], minlength=nb)
        f[:, 12 + k] = s3 / np.maximum(c2, 1)
    return f


def pair_features(U, Up, geom):
    """Rows [f(U_b), f(U'_b)] with the block distance of Eq. (sprodgf),
    d_b = sum over the links starting in b of ReTr(1 - U^dagger U') / (12 * n_links),
    in slot 18 of both halves."""
    z = np.concatenate([domain_features(U, geom), domain_features(Up, geom)], axis=1)
    tr = np.real(np.einsum("...ab,...ab->...", np.conj(U), Up))       # ReTr(U^dagger U') per link
    per_site = np.sum(3.0 - tr, axis=-1)
    d = np.bincount(geom.block_index.reshape(-1), weights=per_site.reshape(-1), minlength=geom.n_blocks)
    d = d / (12.0 * 4 * geom.Vb)
    z[:, 18] = d
    z[:, N_FEAT + 18] = d
    return z


def init_params(seed, n_in=2 * N_FEAT, hidden=HIDDEN):
    """He-normal weights, zero biases (the GPU path draws its own; parity
    tests pass parameters explicitly)."""
    g = np.random.default_rng(seed)
    return {
        "W1": g.standard_normal((hidden, n_in)) * np.sqrt(2.0 / n_in), "b1": np.zeros(hidden),
        "W2": g.standard_normal((hidden, hidden)) * np.sqrt(2.0 / hidden), "b2": np.zeros(hidden),
        "w3": g.standard_normal(hidden) * np.sqrt(1.0 / hidden), "b3": 0.0,
        "mu": np.zeros(n_in), "sigma": np.ones(n_in), "ys": 1.0,
    }


def forward(p, z):
    """n(z) for a batch z[B, 64]; returns (n, cache)."""
    x = (z - p["mu"]) / p["sigma"]
    a1 = x @ p["W1"].T + p["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(a2, 0.0)
    n = h2 @ p["w3"] + p["b3"]
    return n, (x, a1, h1, a2, h2)


def backward(p, cache, dn):
    """Gradients of sum(dn * n) with respect to the parameters."""
    x, a1, h1, a2, h2 = cache
    g = {"w3": h2.T @ dn, "b3": float(np.sum(dn))}
    d2 = np.outer(dn, p["w3"]) * (a2 > 0)
    g["W2"] = d2.T @ h1
    g["b2"] = d2.sum(axis=0)
    d1 = (d2 @ p["W2"]) * (a1 > 0)
    g["W1"] = d1.T @ x
    g["b1"] = d1.sum(axis=0)
    return g


def swap(z):
    n = z.shape[1] // 2
    return np.concatenate([z[:, n:], z[:, :n]], axis=1)


def antisym(p, z):
    """h(z) = ys (n(f, f') - n(f', f)) / 2."""
    a, _ = forward(p, z)
    b, _ = forward(p, swap(z))
    return p.get("ys", 1.0) * 0.5 * (a - b)


def loss_and_grad(p, z, y):
    """Mean squared error of h against labels y and its gradient."""
    ys = p.get("ys", 1.0)
    a, ca = forward(p, z)
    b, cb = forward(p, swap(z))
    h = ys * 0.5 * (a - b)
    r = h - y
    loss = float(np.mean(r * r))
    dh = 2.0 * r / len(y)
    ga = backward(p, ca, 0.5 * ys * dh)
    gb = backward(p, cb, -0.5 * ys * dh)
    grads = {k: ga[k] + gb[k] for k in ga}
    return loss, grads


# flat parameter block of the CUDA path: W1[256][64], b1, W2[256][256], b2,
# w3, b3, mu[64], sigma[64], ys
def unflatten(v):
    v = np.asarray(v, dtype=np.float64)
    o = 0

    def take(n, shape=None):
        nonlocal o
        a = v[o:o + n]
        o += n
        return a.reshape(shape) if shape else a
    p = {"W1": take(HIDDEN * 64, (HIDDEN, 64)), "b1": take(HIDDEN), "W2": take(HIDDEN * HIDDEN, (HIDDEN, HIDDEN)),
         "b2": take(HIDDEN), "w3": take(HIDDEN), "b3": float(take(1)[0]), "mu": take(64), "sigma": take(64),
         "ys": float(take(1)[0])}
    return p


def flatten_grads(g):
    return np.concatenate([g["W1"].ravel(), g["b1"], g["W2"].ravel(), g["b2"], g["w3"], [g["b3"]]])


# --- the device's precision --------------------------------------------------
# The CUDA path rounds the standardised input, the weights W1, W2 and the
# first hidden activation to BF16 (round to nearest even) and accumulates in
# FP32; in the backward pass the GEMM operands D2, D1 and X are rounded to
# BF16 as well.  These functions apply the same roundings (accumulating in
# FP64), so that the device's arithmetic can be checked at its own precision;
# the FP64 functions above remain the definition.

def bf16(x):
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    b = f.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def _f32(x):
    return np.asarray(x, dtype=np.float32).astype(np.float64)


def forward_rounded(p, z):
    x = _f32((_f32(z) - _f32(p["mu"])) / _f32(p["sigma"]))
    h1 = np.maximum(bf16(x) @ bf16(p["W1"]).T + _f32(p["b1"]), 0.0)
    h2 = np.maximum(bf16(h1) @ bf16(p["W2"]).T + _f32(p["b2"]), 0.0)
    n = h2 @ _f32(p["w3"]) + float(np.float32(p["b3"]))
    return n, (x, h1, h2)


def antisym_rounded(p, z):
    a, _ = forward_rounded(p, z)
    b, _ = forward_rounded(p, swap(z))
    return float(np.float32(p.get("ys", 1.0))) * 0.5 * (a - b)


def loss_and_grad_rounded(p, z, y):
    ys = float(np.float32(p.get("ys", 1.0)))
    a, (xa, h1a, h2a) = forward_rounded(p, z)
    b, (xb, h1b, h2b) = forward_rounded(p, swap(z))
    h = ys * 0.5 * (a - b)
    r = h - y
    loss = float(np.mean(r * r))
    d = ys * r / len(y)
    dn = np.concatenate([d, -d])
    X = np.concatenate([xa, xb])
    H1 = np.concatenate([h1a, h1b])
    H2 = np.concatenate([h2a, h2b])
    g = {"w3": H2.T @ dn, "b3": float(dn.sum())}
    D2 = np.outer(dn, _f32(p["w3"])) * (H2 > 0)
    g["W2"] = bf16(D2).T @ bf16(H1)
    g["b2"] = D2.sum(axis=0)
    D1 = (bf16(D2) @ bf16(p["W2"])) * (H1 > 0)
    g["W1"] = bf16(D1).T @ bf16(X)
    g["b1"] = D1.sum(axis=0)
    return loss, g
