// Device-side building blocks shared by the kernels of the library:
// complex arithmetic, Philox-4x64-10, the even-odd block-major lattice
// layout, precision-generic field access and the Wilson hop of Eq. (Dw).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace psms {

// ---------------------------------------------------------------------------
// complex numbers
// ---------------------------------------------------------------------------
template <class R>
struct cpx {
    R re, im;
};

template <class R>
__host__ __device__ __forceinline__ cpx<R> mk(R a, R b) { return cpx<R>{a, b}; }
template <class R>
__device__ __forceinline__ cpx<R> operator+(cpx<R> a, cpx<R> b) { return {a.re + b.re, a.im + b.im}; }
template <class R>
__device__ __forceinline__ cpx<R> operator-(cpx<R> a, cpx<R> b) { return {a.re - b.re, a.im - b.im}; }
template <class R>
__device__ __forceinline__ cpx<R> operator*(R s, cpx<R> a) { return {s * a.re, s * a.im}; }
template <class R>
__device__ __forceinline__ cpx<R> cmul(cpx<R> a, cpx<R> b) {
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
// conj(a) * b
template <class R>
__device__ __forceinline__ cpx<R> cjmul(cpx<R> a, cpx<R> b) {
    return {a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re};
}
// a + b*c
template <class R>
__device__ __forceinline__ cpx<R> cfma(cpx<R> b, cpx<R> c, cpx<R> a) {
    return {fma(b.re, c.re, fma(-b.im, c.im, a.re)), fma(b.re, c.im, fma(b.im, c.re, a.im))};
}
// a + conj(b)*c
template <class R>
__device__ __forceinline__ cpx<R> cjfma(cpx<R> b, cpx<R> c, cpx<R> a) {
    return {fma(b.re, c.re, fma(b.im, c.im, a.re)), fma(b.re, c.im, fma(-b.im, c.re, a.im))};
}
template <class R>
__device__ __forceinline__ cpx<R> times_i(cpx<R> a) { return {-a.im, a.re}; }
template <class R>
__device__ __forceinline__ cpx<R> conj(cpx<R> a) { return {a.re, -a.im}; }
template <class R>
__device__ __forceinline__ R norm2(cpx<R> a) { return a.re * a.re + a.im * a.im; }

// ---------------------------------------------------------------------------
// Philox-4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11)
// ---------------------------------------------------------------------------
struct u64x4 {
    uint64_t w[4];
};

__host__ __device__ __forceinline__ void mulhilo64(uint64_t a, uint64_t b, uint64_t &hi, uint64_t &lo) {
#ifdef __CUDA_ARCH__
    lo = a * b;
    hi = __umul64hi(a, b);
#else
    unsigned __int128 p = (unsigned __int128)a * b;
    lo = (uint64_t)p;
    hi = (uint64_t)(p >> 64);
#endif
}

__host__ __device__ __forceinline__ u64x4 philox(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3,
                                                 uint64_t k0, uint64_t k1) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += W0;
            k1 += W1;
        }
        uint64_t hi0, lo0, hi1, lo1;
        mulhilo64(M0, c0, hi0, lo0);
        mulhilo64(M1, c2, hi1, lo1);
        uint64_t n0 = hi1 ^ c1 ^ k0;
        uint64_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    return u64x4{{c0, c1, c2, c3}};
}

// uniform in [2^-53, 1 - 2^-53], exact in double precision
__host__ __device__ __forceinline__ double to_uniform(uint64_t w) {
    return ((double)(w >> 12) + 0.5) * 0x1.0p-52;
}

enum : uint64_t { TAG_LINK = 1, TAG_NOISE = 2, TAG_HB = 3, TAG_ACCEPT = 4, TAG_SHIFT = 5 };

struct uni4 {
    double u[4];
};

__host__ __device__ __forceinline__ uni4 uniforms(uint64_t seed, uint64_t tag, uint64_t c0, uint64_t c1,
                                                  uint64_t c2, uint64_t c3) {
    u64x4 w = philox(c0, c1, c2, c3, seed, tag);
    uni4 r;
    for (int i = 0; i < 4; ++i) r.u[i] = to_uniform(w.w[i]);
    return r;
}

// ---------------------------------------------------------------------------
// lattice geometry: even-odd, block-major layout
//
// A site x (global coordinates, mu = 0 time) lies in block B_mu = x_mu / l_mu
// with local coordinates y_mu = x_mu mod l_mu.  Blocks carry a rank: with a
// black/white checkerboard (even block count in every direction) black blocks
// (sum B even) come first, rank = colour * nb/2 + (b >> 1) with b the
// lexicographic block index; otherwise rank = b.  Within a block the sites
// of one parity are numbered j = (lexicographic local index) >> 1 (l_3 is
// even).  The internal site index is
//     s = parity * V/2 + rank * Vb/2 + j,
// so every parity half and every block's part of it is contiguous.
// ---------------------------------------------------------------------------
struct Geom {
    int L[4];
    int l[4];
    int lsh[4];      // log2 l
    int nb[4];
    int lstride[4];  // local lexicographic strides (l1 l2 l3, l2 l3, l3, 1)
    int bstride[4];  // block lexicographic strides
    int nblocks;
    int nbh;         // nblocks / 2 when coloured, else 0
    int coloured;
    int Vh;          // V / 2
    int Vbh;         // Vb / 2
    int vbh_sh;      // log2 Vbh
    long long V;
};

// per-rank table entry: block coordinates and the ranks of the 8 neighbours
struct BlockInfo {
    int B[4];
    int lex;
    int nbr[8];      // 2*mu + 0: +mu neighbour, 2*mu + 1: -mu neighbour
};

__host__ __device__ __forceinline__ int rank_of_lex(const Geom &g, int b, const int B[4]) {
    if (!g.coloured) return b;
    int c = (B[0] + B[1] + B[2] + B[3]) & 1;
    return c * g.nbh + (b >> 1);
}

// local coordinates of the j-th site of parity p in a block
__device__ __forceinline__ int local_lex(const Geom &g, int p, int j, int y[4]) {
    int ll = 2 * j;
    y[3] = ll & (g.l[3] - 1);
    y[2] = (ll >> g.lsh[3]) & (g.l[2] - 1);
    y[1] = (ll >> (g.lsh[3] + g.lsh[2])) & (g.l[1] - 1);
    y[0] = ll >> (g.lsh[3] + g.lsh[2] + g.lsh[1]);
    if (((y[0] + y[1] + y[2] + y[3]) & 1) != p) {
        ll += 1;
        y[3] += 1;
    }
    return ll;
}

// internal index of the site at global coordinates x (host and device)
__host__ __device__ __forceinline__ long long site_index(const Geom &g, const int x[4]) {
    int B[4], y[4];
    for (int m = 0; m < 4; ++m) {
        B[m] = x[m] >> g.lsh[m];
        y[m] = x[m] & (g.l[m] - 1);
    }
    int b = ((B[0] * g.nb[1] + B[1]) * g.nb[2] + B[2]) * g.nb[3] + B[3];
    int r = rank_of_lex(g, b, B);
    int p = (x[0] + x[1] + x[2] + x[3]) & 1;
    int ll = ((y[0] * g.l[1] + y[1]) * g.l[2] + y[2]) * g.l[3] + y[3];
    return (long long)p * g.Vh + (long long)r * g.Vbh + (ll >> 1);
}

// canonical lexicographic index of global coordinates
__host__ __device__ __forceinline__ long long lex_index(const Geom &g, const int x[4]) {
    return (((long long)x[0] * g.L[1] + x[1]) * g.L[2] + x[2]) * g.L[3] + x[3];
}

// decode internal index s into parity, rank, j, local and global coordinates
__device__ __forceinline__ void decode(const Geom &g, const BlockInfo *__restrict__ binfo, long long s, int &p,
                                       int &r, int &j, int y[4], int x[4]) {
    p = s >= g.Vh;
    int sp = (int)(s - (long long)p * g.Vh);
    r = sp >> g.vbh_sh;
    j = sp & (g.Vbh - 1);
    local_lex(g, p, j, y);
    const BlockInfo &bi = binfo[r];
    for (int m = 0; m < 4; ++m) x[m] = bi.B[m] * g.l[m] + y[m];
}

// is the link (x, mu) active (Sec. 3)?  y: local coordinates of x.
__host__ __device__ __forceinline__ bool link_active(const Geom &g, const int y[4], int mu, int all) {
    if (all) return true;
    if (y[mu] == g.l[mu] - 1) return false;  // leaves the block
    bool small = false;
    for (int m = 0; m < 4; ++m) small |= (g.l[m] <= 2);
    if (small) return true;
    int y1[4] = {y[0], y[1], y[2], y[3]};
    y1[mu] += 1;
    int nb0 = 0, nb1 = 0;
    for (int m = 0; m < 4; ++m) {
        nb0 |= (y[m] == 0) | (y[m] == g.l[m] - 1);
        nb1 |= (y1[m] == 0) | (y1[m] == g.l[m] - 1);
    }
    return nb0 + nb1 <= 1;
}

// ---------------------------------------------------------------------------
// precision-generic field access.  A field of `cs` sites stores component c
// (c = 3 spin + colour) of site s at element idx(c, cs, s): components are
// grouped in 16-byte units of 2^VSH complex numbers (FP64: 1, FP32: 2,
// BF16: 4), unit u of site s at unit index u * cs + s, so that a thread
// loads a whole spinor with 12, 6 or 3 vector loads and a warp's loads of
// one unit are contiguous.  FP64 links: U[mu][e][s]; FP32 links: per mu four
// 16-byte units (e = 0..7) then one 8-byte element (e = 8).
// ---------------------------------------------------------------------------
template <class T>
struct Store;

template <>
struct Store<double> {
    using elem = double2;
    using R = double;
    static constexpr int VSH = 0;
    static __host__ __device__ __forceinline__ long long idx(int c, long long cs, long long s) { return c * cs + s; }
    static __device__ __forceinline__ cpx<double> ldi(const elem *p, long long i) {
        double2 v = p[i];
        return {v.x, v.y};
    }
    // read-only path: only for data no thread writes during the launch
    static __device__ __forceinline__ cpx<double> ldro(const elem *p, long long i) {
        double2 v = __ldg(p + i);
        return {v.x, v.y};
    }
    static __device__ __forceinline__ void sti(elem *p, long long i, cpx<double> v) { p[i] = make_double2(v.re, v.im); }
    static __device__ __forceinline__ cpx<double> ld(const elem *p, int c, long long cs, long long s) {
        return ldi(p, idx(c, cs, s));
    }
    static __device__ __forceinline__ void st(elem *p, int c, long long cs, long long s, cpx<double> v) {
        sti(p, idx(c, cs, s), v);
    }
};

template <>
struct Store<float> {
    using elem = float2;
    using R = float;
    static constexpr int VSH = 1;
    static __host__ __device__ __forceinline__ long long idx(int c, long long cs, long long s) {
        return (((long long)(c >> 1)) * cs + s) * 2 + (c & 1);
    }
    static __device__ __forceinline__ cpx<float> ldi(const elem *p, long long i) {
        float2 v = p[i];
        return {v.x, v.y};
    }
    static __device__ __forceinline__ cpx<float> ldro(const elem *p, long long i) {
        float2 v = __ldg(p + i);
        return {v.x, v.y};
    }
    static __device__ __forceinline__ void sti(elem *p, long long i, cpx<float> v) { p[i] = make_float2(v.re, v.im); }
    static __device__ __forceinline__ cpx<float> ld(const elem *p, int c, long long cs, long long s) {
        return ldi(p, idx(c, cs, s));
    }
    static __device__ __forceinline__ void st(elem *p, int c, long long cs, long long s, cpx<float> v) {
        sti(p, idx(c, cs, s), v);
    }
};

template <>
struct Store<__nv_bfloat16> {
    using elem = __nv_bfloat162;
    using R = float;
    static constexpr int VSH = 2;
    static __host__ __device__ __forceinline__ long long idx(int c, long long cs, long long s) {
        return (((long long)(c >> 2)) * cs + s) * 4 + (c & 3);
    }
    static __device__ __forceinline__ cpx<float> ldi(const elem *p, long long i) {
        float2 v = __bfloat1622float2(p[i]);
        return {v.x, v.y};
    }
    static __device__ __forceinline__ cpx<float> ldro(const elem *p, long long i) {
        float2 v = __bfloat1622float2(__ldg(p + i));
        return {v.x, v.y};
    }
    static __device__ __forceinline__ void sti(elem *p, long long i, cpx<float> v) {
        p[i] = __floats2bfloat162_rn(v.re, v.im);
    }
    static __device__ __forceinline__ cpx<float> ld(const elem *p, int c, long long cs, long long s) {
        return ldi(p, idx(c, cs, s));
    }
    static __device__ __forceinline__ void st(elem *p, int c, long long cs, long long s, cpx<float> v) {
        sti(p, idx(c, cs, s), v);
    }
};

// element index of link entry e of direction mu at site s
template <class S>
__host__ __device__ __forceinline__ long long link_idx(long long V, int mu, int e, long long s) {
    if constexpr (S::VSH == 0) {
        return ((long long)mu * 9 + e) * V + s;
    } else {
        const long long base = (long long)mu * 9 * V;
        return e < 8 ? base + 2 * ((long long)(e >> 1) * V + s) + (e & 1) : base + 8 * V + s;
    }
}

template <class R>
struct Spinor {
    cpx<R> c[4][3];
};
template <class R>
struct Half {
    cpx<R> c[2][3];
};
template <class R>
struct SU3 {
    cpx<R> e[3][3];
};

__device__ __forceinline__ cpx<float> bf_lo(uint32_t w) {
    return {__uint_as_float(w << 16), __uint_as_float(w & 0xFFFF0000u)};
}

// whole spinor of site s with 16-byte vector loads (RO: read-only cache path)
template <class S, bool RO>
__device__ __forceinline__ Spinor<typename S::R> load_spinor_v(const typename S::elem *p, long long cs, long long s) {
    Spinor<typename S::R> v;
    if constexpr (S::VSH == 0) {
#pragma unroll
        for (int c = 0; c < 12; ++c) v.c[c / 3][c % 3] = RO ? S::ldro(p, c * cs + s) : S::ldi(p, c * cs + s);
    } else if constexpr (S::VSH == 1) {
        const float4 *q = reinterpret_cast<const float4 *>(p);
#pragma unroll
        for (int u = 0; u < 6; ++u) {
            const float4 w = RO ? __ldg(q + u * cs + s) : q[u * cs + s];
            v.c[(2 * u) / 3][(2 * u) % 3] = {w.x, w.y};
            v.c[(2 * u + 1) / 3][(2 * u + 1) % 3] = {w.z, w.w};
        }
    } else {
        const uint4 *q = reinterpret_cast<const uint4 *>(p);
#pragma unroll
        for (int u = 0; u < 3; ++u) {
            const uint4 w = RO ? __ldg(q + u * cs + s) : q[u * cs + s];
            const uint32_t ww[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
            for (int m = 0; m < 4; ++m) v.c[(4 * u + m) / 3][(4 * u + m) % 3] = bf_lo(ww[m]);
        }
    }
    return v;
}

template <class S>
__device__ __forceinline__ Spinor<typename S::R> load_spinor(const typename S::elem *p, long long cs, long long s) {
    return load_spinor_v<S, false>(p, cs, s);
}

template <class S>
__device__ __forceinline__ Spinor<typename S::R> load_spinor_ro(const typename S::elem *p, long long cs, long long s) {
    return load_spinor_v<S, true>(p, cs, s);
}

template <class S>
__device__ __forceinline__ void store_spinor(typename S::elem *p, long long cs, long long s,
                                             const Spinor<typename S::R> &v) {
    if constexpr (S::VSH == 0) {
#pragma unroll
        for (int c = 0; c < 12; ++c) S::sti(p, c * cs + s, v.c[c / 3][c % 3]);
    } else if constexpr (S::VSH == 1) {
        float4 *q = reinterpret_cast<float4 *>(p);
#pragma unroll
        for (int u = 0; u < 6; ++u) {
            const cpx<float> a = v.c[(2 * u) / 3][(2 * u) % 3], b = v.c[(2 * u + 1) / 3][(2 * u + 1) % 3];
            q[u * cs + s] = make_float4(a.re, a.im, b.re, b.im);
        }
    } else {
        uint4 *q = reinterpret_cast<uint4 *>(p);
#pragma unroll
        for (int u = 0; u < 3; ++u) {
            uint32_t ww[4];
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const cpx<float> a = v.c[(4 * u + m) / 3][(4 * u + m) % 3];
                __nv_bfloat162 h = __floats2bfloat162_rn(a.re, a.im);
                ww[m] = *reinterpret_cast<uint32_t *>(&h);
            }
            q[u * cs + s] = make_uint4(ww[0], ww[1], ww[2], ww[3]);
        }
    }
}

template <class S>
__device__ __forceinline__ SU3<typename S::R> load_link(const typename S::elem *U, long long V, int mu, long long s) {
    SU3<typename S::R> u;
    if constexpr (S::VSH == 0) {
        const typename S::elem *q = U + (long long)mu * 9 * V + s;
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) u.e[a][b] = S::ldro(q, (3 * a + b) * V);
    } else {
        const float2 *base = reinterpret_cast<const float2 *>(U) + (long long)mu * 9 * V;
        const float4 *q = reinterpret_cast<const float4 *>(base);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float4 w = __ldg(q + k * V + s);
            u.e[(2 * k) / 3][(2 * k) % 3] = {w.x, w.y};
            u.e[(2 * k + 1) / 3][(2 * k + 1) % 3] = {w.z, w.w};
        }
        const float2 w = __ldg(base + 8 * V + s);
        u.e[2][2] = {w.x, w.y};
    }
    return u;
}

// ---------------------------------------------------------------------------
// Wilson hop, Eq. (Dw).  With the chiral basis gamma_mu = [[0, e],[e^+, 0]]
// the projectors 1 -/+ s*gamma_mu (s = +1 for D, -1 for D^dagger) have rank 2:
//   (1 + t gamma_mu) psi = (h, t e^+ h),  h = psi_up + t e psi_dn,
// with t = -s for the forward and t = +s for the backward term.
//   e_0 = -1, e_1 = -i sigma_1, e_2 = -i sigma_2, e_3 = -i sigma_3.
// ---------------------------------------------------------------------------
template <class R>
__device__ __forceinline__ Half<R> project(int mu, R t, const Spinor<R> &p) {
    Half<R> h;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        cpx<R> u0 = p.c[0][c], u1 = p.c[1][c], d0 = p.c[2][c], d1 = p.c[3][c];
        switch (mu) {
            case 0:  // e psi_d = (-d0, -d1)
                h.c[0][c] = u0 - t * d0;
                h.c[1][c] = u1 - t * d1;
                break;
            case 1:  // e psi_d = (-i d1, -i d0)
                h.c[0][c] = u0 - t * times_i(d1);
                h.c[1][c] = u1 - t * times_i(d0);
                break;
            case 2:  // e psi_d = (-d1, d0)
                h.c[0][c] = u0 - t * d1;
                h.c[1][c] = u1 + t * d0;
                break;
            default:  // e psi_d = (-i d0, i d1)
                h.c[0][c] = u0 - t * times_i(d0);
                h.c[1][c] = u1 + t * times_i(d1);
                break;
        }
    }
    return h;
}

// acc += (w, t e^+ w)
template <class R>
__device__ __forceinline__ void reconstruct_add(int mu, R t, const Half<R> &w, Spinor<R> &acc) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        cpx<R> w0 = w.c[0][c], w1 = w.c[1][c];
        acc.c[0][c] = acc.c[0][c] + w0;
        acc.c[1][c] = acc.c[1][c] + w1;
        switch (mu) {
            case 0:  // e^+ = -1
                acc.c[2][c] = acc.c[2][c] - t * w0;
                acc.c[3][c] = acc.c[3][c] - t * w1;
                break;
            case 1:  // e^+ = i sigma_1: (i w1, i w0)
                acc.c[2][c] = acc.c[2][c] + t * times_i(w1);
                acc.c[3][c] = acc.c[3][c] + t * times_i(w0);
                break;
            case 2:  // e^+ = [[0,1],[-1,0]]: (w1, -w0)
                acc.c[2][c] = acc.c[2][c] + t * w1;
                acc.c[3][c] = acc.c[3][c] - t * w0;
                break;
            default:  // e^+ = i sigma_3: (i w0, -i w1)
                acc.c[2][c] = acc.c[2][c] + t * times_i(w0);
                acc.c[3][c] = acc.c[3][c] - t * times_i(w1);
                break;
        }
    }
}

template <class R>
__device__ __forceinline__ Half<R> su3_mul(const SU3<R> &u, const Half<R> &h) {
    Half<R> w;
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            cpx<R> z = cmul(u.e[a][0], h.c[s][0]);
            z = cfma(u.e[a][1], h.c[s][1], z);
            z = cfma(u.e[a][2], h.c[s][2], z);
            w.c[s][a] = z;
        }
    return w;
}

template <class R>
__device__ __forceinline__ Half<R> su3_dag_mul(const SU3<R> &u, const Half<R> &h) {
    Half<R> w;
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            cpx<R> z = cjmul(u.e[0][a], h.c[s][0]);
            z = cjfma(u.e[1][a], h.c[s][1], z);
            z = cjfma(u.e[2][a], h.c[s][2], z);
            w.c[s][a] = z;
        }
    return w;
}

template <class R>
__device__ __forceinline__ void zero(Spinor<R> &v) {
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) v.c[a][b] = mk<R>(0, 0);
}

// hop modes: which hops of Eq. (Dw) are kept
enum HopMode : int { HOP_ALL = 0, HOP_INTRA = 1, HOP_INTER = 2 };

// Neighbour of the site (rank r, parity p, local coords y, local lex ll) in
// direction mu, sign sg.  Returns false if `mode` drops the hop; otherwise
// sets the internal index of the neighbour (opposite parity) and the
// boundary sign (-1 for a hop across the antiperiodic time boundary).
__device__ __forceinline__ bool neighbour(const Geom &g, const BlockInfo &bi, int r, int p, const int y[4], int ll,
                                          int mu, int sg, int mode, long long &sn, int &bsign) {
    int yn = y[mu] + sg;
    bool inside = (unsigned)yn < (unsigned)g.l[mu];
    if (mode == HOP_INTRA && !inside) return false;
    if (mode == HOP_INTER && inside) return false;
    int rn = r;
    int lln = ll + sg * g.lstride[mu];
    bsign = 1;
    if (!inside) {
        rn = bi.nbr[2 * mu + (sg > 0 ? 0 : 1)];
        lln = ll - sg * (g.l[mu] - 1) * g.lstride[mu];
        if (mu == 0 && ((sg > 0 && bi.B[0] == g.nb[0] - 1) || (sg < 0 && bi.B[0] == 0))) bsign = -1;
    }
    sn = (long long)(1 - p) * g.Vh + (long long)rn * g.Vbh + (lln >> 1);
    return true;
}

}  // namespace psms
