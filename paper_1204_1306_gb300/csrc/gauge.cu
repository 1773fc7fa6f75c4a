// Gauge-field kernels (FP64): synthetic link generator, reunitarisation,
// plaquette action (Eq. (Sw)), the pure-gauge proposal of Sec. 6
// (checkerboard Cabibbo-Marinari heatbath and overrelaxation on the active
// links of Sec. 3), random translation, the interpolation of Eq. (gfparam)
// and the merge of accepted blocks.
#include "gauge.hpp"

#include <cmath>
#include <vector>

namespace psms {

using C = cpx<double>;

struct M3 {
    C e[3][3];
};

__host__ __device__ __forceinline__ C cm(C a, C b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__host__ __device__ __forceinline__ C ca(C a, C b) { return {a.re + b.re, a.im + b.im}; }
__host__ __device__ __forceinline__ C cs(C a, C b) { return {a.re - b.re, a.im - b.im}; }
__host__ __device__ __forceinline__ C cc(C a) { return {a.re, -a.im}; }

__device__ __forceinline__ M3 mul(const M3 &a, const M3 &b) {
    M3 r;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            C z = cm(a.e[i][0], b.e[0][j]);
            z = ca(z, cm(a.e[i][1], b.e[1][j]));
            z = ca(z, cm(a.e[i][2], b.e[2][j]));
            r.e[i][j] = z;
        }
    return r;
}

__device__ __forceinline__ M3 dagm(const M3 &a) {
    M3 r;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) r.e[i][j] = cc(a.e[j][i]);
    return r;
}

__device__ __forceinline__ M3 ldU(const double2 *U, long long V, int mu, long long s) {
    M3 m;
    const double2 *q = U + (long long)mu * 9 * V + s;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double2 v = q[(3 * a + b) * V];
            m.e[a][b] = {v.x, v.y};
        }
    return m;
}

__device__ __forceinline__ void stU(double2 *U, long long V, int mu, long long s, const M3 &m) {
    double2 *q = U + (long long)mu * 9 * V + s;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) q[(3 * a + b) * V] = make_double2(m.e[a][b].re, m.e[a][b].im);
}

// Gram-Schmidt on rows 0, 1; row 2 = conj(row0 x row1)
__device__ __forceinline__ M3 reunit(M3 u) {
    double n0 = 0;
    for (int j = 0; j < 3; ++j) n0 += norm2(u.e[0][j]);
    n0 = 1.0 / sqrt(n0);
    for (int j = 0; j < 3; ++j) u.e[0][j] = n0 * u.e[0][j];
    C d = {0, 0};
    for (int j = 0; j < 3; ++j) d = ca(d, cm(cc(u.e[0][j]), u.e[1][j]));
    for (int j = 0; j < 3; ++j) u.e[1][j] = cs(u.e[1][j], cm(d, u.e[0][j]));
    double n1 = 0;
    for (int j = 0; j < 3; ++j) n1 += norm2(u.e[1][j]);
    n1 = 1.0 / sqrt(n1);
    for (int j = 0; j < 3; ++j) u.e[1][j] = n1 * u.e[1][j];
    u.e[2][0] = cc(cs(cm(u.e[0][1], u.e[1][2]), cm(u.e[0][2], u.e[1][1])));
    u.e[2][1] = cc(cs(cm(u.e[0][2], u.e[1][0]), cm(u.e[0][0], u.e[1][2])));
    u.e[2][2] = cc(cs(cm(u.e[0][0], u.e[1][1]), cm(u.e[0][1], u.e[1][0])));
    return u;
}

// exp(X) of a 3x3 complex matrix by scaling and squaring with a degree-18
// Taylor polynomial (Horner form) after scaling ||X||_F below 1/2.
__device__ M3 expm3(M3 X) {
    double nf = 0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) nf += norm2(X.e[i][j]);
    nf = sqrt(nf);
    int sq = 0;
    while (nf > 0.5 && sq < 60) {
        nf *= 0.5;
        ++sq;
    }
    const double sc = ldexp(1.0, -sq);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) X.e[i][j] = sc * X.e[i][j];
    M3 E;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) E.e[i][j] = {i == j ? 1.0 : 0.0, 0.0};
    for (int n = 18; n >= 1; --n) {
        // E = I + X E / n
        M3 T = mul(X, E);
        const double inv = 1.0 / n;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) E.e[i][j] = {(i == j ? 1.0 : 0.0) + inv * T.e[i][j].re, inv * T.e[i][j].im};
    }
    for (int k = 0; k < sq; ++k) E = mul(E, E);
    return E;
}

// ---------------------------------------------------------------------------
// link generator: U = reunitarise(exp(i eps H)), H = sum_a omega_a lambda_a/2
// ---------------------------------------------------------------------------
__global__ void link_init_kernel(Geom g, double2 *U, double eps, uint64_t seed) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 4 * g.V) return;
    const long long lex = t >> 2;
    const int mu = (int)(t & 3);
    int x[4];
    long long rem = lex;
    x[3] = (int)(rem % g.L[3]);
    rem /= g.L[3];
    x[2] = (int)(rem % g.L[2]);
    rem /= g.L[2];
    x[1] = (int)(rem % g.L[1]);
    x[0] = (int)(rem / g.L[1]);
    double om[8];
    for (int j = 0; j < 2; ++j) {
        uni4 u = uniforms(seed, TAG_LINK, (uint64_t)t, (uint64_t)j, 0, 0);
        for (int k = 0; k < 2; ++k) {
            const double r = sqrt(-2.0 * log(u.u[2 * k]));
            const double th = 2.0 * M_PI * u.u[2 * k + 1];
            om[4 * j + 2 * k] = r * cos(th);
            om[4 * j + 2 * k + 1] = r * sin(th);
        }
    }
    // H = sum_a omega_a lambda_a / 2 (Gell-Mann matrices)
    const double is3 = 1.0 / sqrt(3.0);
    M3 H;
    H.e[0][0] = {0.5 * (om[2] + is3 * om[7]), 0};
    H.e[1][1] = {0.5 * (-om[2] + is3 * om[7]), 0};
    H.e[2][2] = {0.5 * (-2.0 * is3 * om[7]), 0};
    H.e[0][1] = {0.5 * om[0], -0.5 * om[1]};
    H.e[1][0] = {0.5 * om[0], 0.5 * om[1]};
    H.e[0][2] = {0.5 * om[3], -0.5 * om[4]};
    H.e[2][0] = {0.5 * om[3], 0.5 * om[4]};
    H.e[1][2] = {0.5 * om[5], -0.5 * om[6]};
    H.e[2][1] = {0.5 * om[5], 0.5 * om[6]};
    M3 X;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) X.e[i][j] = {-eps * H.e[i][j].im, eps * H.e[i][j].re};  // i eps H
    M3 Uu = reunit(expm3(X));
    stU(U, g.V, mu, site_index(g, x), Uu);
}

void link_init(psms_ctx *c, double2 *U, double eps, uint64_t seed) {
    const long long n = 4 * c->g.V;
    link_init_kernel<<<(unsigned)((n + 127) / 128), 128, 0, c->stream>>>(c->g, U, eps, seed);
    PSMS_LAUNCH_CHECK("link_init");
}

// ---------------------------------------------------------------------------
// neighbours with periodic wrap in global coordinates
// ---------------------------------------------------------------------------
__device__ __forceinline__ long long shifted(const Geom &g, const int x[4], int mu, int dm, int nu, int dn) {
    int y[4] = {x[0], x[1], x[2], x[3]};
    y[mu] += dm;
    y[nu] += dn;
    for (int m = 0; m < 4; ++m) {
        if (y[m] < 0) y[m] += g.L[m];
        if (y[m] >= g.L[m]) y[m] -= g.L[m];
    }
    return site_index(g, y);
}

// sum of the 6 staples: ReTr(U(x,mu) A) = sum of the plaquettes holding U(x,mu)
__device__ M3 staple(const Geom &g, const double2 *U, const int x[4], int mu) {
    M3 A;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) A.e[i][j] = {0, 0};
    const long long s = site_index(g, x);
    for (int nu = 0; nu < 4; ++nu) {
        if (nu == mu) continue;
        const long long sp_mu = shifted(g, x, mu, 1, nu, 0);
        const long long sp_nu = shifted(g, x, nu, 1, mu, 0);
        const long long sm_nu = shifted(g, x, nu, -1, mu, 0);
        const long long spm = shifted(g, x, mu, 1, nu, -1);
        M3 up = mul(mul(ldU(U, g.V, nu, sp_mu), dagm(ldU(U, g.V, mu, sp_nu))), dagm(ldU(U, g.V, nu, s)));
        M3 dn = mul(mul(dagm(ldU(U, g.V, nu, spm)), dagm(ldU(U, g.V, mu, sm_nu))), ldU(U, g.V, nu, sm_nu));
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) A.e[i][j] = ca(A.e[i][j], ca(up.e[i][j], dn.e[i][j]));
    }
    return A;
}

// ---------------------------------------------------------------------------
// Cabibbo-Marinari update of one subset (mu, parity[, block colour])
// ---------------------------------------------------------------------------
struct C2 {
    C e[2][2];
};

__device__ __forceinline__ C2 q2m(double q0, double q1, double q2, double q3) {
    C2 m;
    m.e[0][0] = {q0, q3};
    m.e[0][1] = {q2, q1};
    m.e[1][0] = {-q2, q1};
    m.e[1][1] = {q0, -q3};
    return m;
}

__device__ __forceinline__ C2 mul2(const C2 &a, const C2 &b) {
    C2 r;
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) r.e[i][j] = ca(cm(a.e[i][0], b.e[0][j]), cm(a.e[i][1], b.e[1][j]));
    return r;
}

constexpr int MAX_ATTEMPTS = 1000;
constexpr double KP_THRESHOLD = 2.0;

__global__ void cm_update_kernel(Geom g, const BlockInfo *binfo, double2 *U, int mu, int parity, int colour, int all,
                                 double beta, int kind, uint64_t seed, uint64_t sweep, int *failed) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= g.Vh) return;
    const long long s = (long long)parity * g.Vh + t;
    int p, r, j, y[4], x[4];
    decode(g, binfo, s, p, r, j, y, x);
    if (colour >= 0) {
        const BlockInfo &bi = binfo[r];
        if (((bi.B[0] + bi.B[1] + bi.B[2] + bi.B[3]) & 1) != colour) return;
    }
    if (!link_active(g, y, mu, all)) return;
    const M3 A = staple(g, U, x, mu);
    M3 Ul = ldU(U, g.V, mu, s);
    const uint64_t link = (uint64_t)(4 * lex_index(g, x) + mu);
    const bool forward = uniforms(seed, TAG_HB, sweep, link, 0, 0).u[0] < 0.5;
    int nfail = 0;
    for (int k = 0; k < 3; ++k) {
        const int sgi = forward ? k : 2 - k;
        const int i0 = (sgi == 2) ? 1 : 0;
        const int j0 = (sgi == 0) ? 1 : 2;
        // W = Ul A, 2x2 sub-block (i0, j0)
        M3 W = mul(Ul, A);
        C w00 = W.e[i0][i0], w01 = W.e[i0][j0], w10 = W.e[j0][i0], w11 = W.e[j0][j0];
        double r0 = 0.5 * (w00.re + w11.re);
        double r1 = 0.5 * (w01.im + w10.im);
        double r2 = 0.5 * (w01.re - w10.re);
        double r3 = 0.5 * (w00.im - w11.im);
        const double kn = sqrt(r0 * r0 + r1 * r1 + r2 * r2 + r3 * r3);
        if (!(kn > 0.0)) continue;
        const double ik = 1.0 / kn;
        C2 vdag = q2m(r0 * ik, -r1 * ik, -r2 * ik, -r3 * ik);
        C2 R;
        if (kind == 0) {
            const double alpha = 2.0 * beta * kn / 3.0;
            double a0 = 1.0;
            bool ok = false;
            for (int att = 0; att < MAX_ATTEMPTS; ++att) {
                uni4 u = uniforms(seed, TAG_HB, sweep, link, (uint64_t)(1 + 2 * k), (uint64_t)att);
                if (alpha >= KP_THRESHOLD) {
                    const double cth = cos(2.0 * M_PI * u.u[1]);
                    const double xx = -(log(u.u[0]) + cth * cth * log(u.u[2])) / alpha;
                    if (u.u[3] * u.u[3] <= 1.0 - 0.5 * xx) {
                        a0 = 1.0 - xx;
                        ok = true;
                        break;
                    }
                } else {
                    const double cr = 1.0 + log(u.u[0] + (1.0 - u.u[0]) * exp(-2.0 * alpha)) / alpha;
                    if (u.u[1] * u.u[1] <= 1.0 - cr * cr) {
                        a0 = cr;
                        ok = true;
                        break;
                    }
                }
            }
            if (!ok) {
                ++nfail;
                continue;
            }
            uni4 d = uniforms(seed, TAG_HB, sweep, link, (uint64_t)(2 + 2 * k), 0);
            const double cth = 2.0 * d.u[0] - 1.0;
            const double sth = sqrt(fmax(0.0, 1.0 - cth * cth));
            const double phi = 2.0 * M_PI * d.u[1];
            const double rad = sqrt(fmax(0.0, 1.0 - a0 * a0));
            C2 X = q2m(a0, rad * sth * cos(phi), rad * sth * sin(phi), rad * cth);
            R = mul2(X, vdag);
        } else {
            R = mul2(vdag, vdag);
        }
        for (int c = 0; c < 3; ++c) {
            C ri = Ul.e[i0][c], rj = Ul.e[j0][c];
            Ul.e[i0][c] = ca(cm(R.e[0][0], ri), cm(R.e[0][1], rj));
            Ul.e[j0][c] = ca(cm(R.e[1][0], ri), cm(R.e[1][1], rj));
        }
    }
    stU(U, g.V, mu, s, Ul);
    if (nfail && failed) atomicAdd(failed, nfail);
}

__global__ void reunit_active_kernel(Geom g, const BlockInfo *binfo, double2 *U, int all) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 4 * g.V) return;
    const long long s = t >> 2;
    const int mu = (int)(t & 3);
    int p, r, j, y[4], x[4];
    decode(g, binfo, s, p, r, j, y, x);
    if (!link_active(g, y, mu, all)) return;
    stU(U, g.V, mu, s, reunit(ldU(U, g.V, mu, s)));
}

int gauge_sweep(psms_ctx *c, double2 *U, int active_set, int n_iter, int n_or, double beta, uint64_t seed,
                uint64_t sweep0) {
    const Geom &g = c->g;
    const int all = active_set == PSMS_ACTIVE_ALL;
    bool small = false;
    for (int m = 0; m < 4; ++m) small |= g.l[m] <= 2;
    struct Sub {
        int mu, p, colour;
    };
    std::vector<Sub> subs;
    const int ncol = (small && !all) ? 2 : 1;
    for (int col = 0; col < ncol; ++col)
        for (int mu = 0; mu < 4; ++mu)
            for (int p = 0; p < 2; ++p) subs.push_back({mu, p, ncol == 2 ? col : -1});
    int *failed = (int *)scratch(c, "hb_failed", sizeof(int));
    cuda_check(cudaMemsetAsync(failed, 0, sizeof(int), c->stream), "hb memset");
    const int NT = 128;
    const unsigned nb = (unsigned)((g.Vh + NT - 1) / NT);
    auto sweep = [&](int kind, bool rev, uint64_t sid) {
        for (size_t i = 0; i < subs.size(); ++i) {
            const Sub &q = subs[rev ? subs.size() - 1 - i : i];
            cm_update_kernel<<<nb, NT, 0, c->stream>>>(g, c->d_binfo, U, q.mu, q.p, q.colour, all, beta, kind, seed,
                                                       sid, failed);
            PSMS_LAUNCH_CHECK("cm_update_kernel");
        }
    };
    uint64_t s = sweep0;
    for (int it = 0; it < n_iter; ++it) {
        sweep(0, false, s++);
        for (int k = 0; k < n_or; ++k) sweep(1, false, s++);
        for (int k = 0; k < n_or; ++k) sweep(1, true, s++);
        sweep(0, true, s++);
    }
    const long long n = 4 * g.V;
    reunit_active_kernel<<<(unsigned)((n + 127) / 128), 128, 0, c->stream>>>(g, c->d_binfo, U, all);
    PSMS_LAUNCH_CHECK("reunit");
    int h = 0;
    cuda_check(cudaMemcpyAsync(&h, failed, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "hb failed");
    cuda_check(cudaStreamSynchronize(c->stream), "hb sync");
    return h;
}

// ---------------------------------------------------------------------------
// plaquette: per-CTA partial sums of sum_{mu<nu} ReTr U_{mu nu}(x)
// ---------------------------------------------------------------------------
__global__ void plaquette_kernel(Geom g, const BlockInfo *binfo, const double2 *U, double *partial) {
    __shared__ double sh[4];
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double acc = 0;
    if (s < g.V) {
        int p, r, j, y[4], x[4];
        decode(g, binfo, s, p, r, j, y, x);
        for (int mu = 0; mu < 4; ++mu)
            for (int nu = mu + 1; nu < 4; ++nu) {
                const long long a = shifted(g, x, mu, 1, nu, 0);
                const long long b = shifted(g, x, nu, 1, mu, 0);
                M3 P = mul(mul(mul(ldU(U, g.V, mu, s), ldU(U, g.V, nu, a)), dagm(ldU(U, g.V, mu, b))),
                           dagm(ldU(U, g.V, nu, s)));
                acc += P.e[0][0].re + P.e[1][1].re + P.e[2][2].re;
            }
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) partial[blockIdx.x] = sh[0] + sh[1] + sh[2] + sh[3];
}

void plaquette_sum(psms_ctx *c, const double2 *U, double *d_out) {
    const int NT = 128;
    const int nb = (int)((c->g.V + NT - 1) / NT);
    double *partial = (double *)scratch(c, "plaq_partial", sizeof(double) * nb);
    plaquette_kernel<<<nb, NT, 0, c->stream>>>(c->g, c->d_binfo, U, partial);
    PSMS_LAUNCH_CHECK("plaquette");
    reduce_partials(c, partial, nb, 1, d_out);
}

// ---------------------------------------------------------------------------
// translation U'(x) = U(x - s), interpolation, merge
// ---------------------------------------------------------------------------
__global__ void translate_kernel(Geom g, const BlockInfo *binfo, const double2 *src, double2 *dst, int s0, int s1,
                                 int s2, int s3) {
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.V) return;
    int p, r, j, y[4], x[4];
    decode(g, binfo, s, p, r, j, y, x);
    int sh[4] = {s0, s1, s2, s3};
    int z[4];
    for (int m = 0; m < 4; ++m) z[m] = ((x[m] - sh[m]) % g.L[m] + g.L[m]) % g.L[m];
    const long long sz = site_index(g, z);
    for (int mu = 0; mu < 4; ++mu)
        for (int e = 0; e < 9; ++e) dst[((long long)mu * 9 + e) * g.V + s] = src[((long long)mu * 9 + e) * g.V + sz];
}

void translate(psms_ctx *c, const double2 *src, double2 *dst, const int sh[4]) {
    const int NT = 128;
    translate_kernel<<<(unsigned)((c->g.V + NT - 1) / NT), NT, 0, c->stream>>>(c->g, c->d_binfo, src, dst, sh[0], sh[1],
                                                                               sh[2], sh[3]);
    PSMS_LAUNCH_CHECK("translate");
}

// out_i = ((N - i)/N) U + (i/N) U', i = i0 .. i0 + n - 1, FP64 and optional FP32
// FP32 link element index of the FP64 element t = (mu * 9 + e) * V + s
// U_i = ((N - i)/N) U + (i/N) U' for i = i0 .. i0 + n - 1, one thread per
// link: the link of both endpoints is read once, every system's FP64 copy
// ([mu][e][s]) and FP32 copy (four 16-byte units of element pairs, then
// element 8) are written with full coalesced stores
__global__ void interp_kernel(const double2 *U, const double2 *Up, double2 *out64, float2 *out32, int N, int i0,
                              int n, long long V) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 4 * V) return;
    const int mu = (int)(t / V);
    const long long s = t - (long long)mu * V;
    double2 u[9], v[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) {
        u[e] = U[((long long)mu * 9 + e) * V + s];
        v[e] = Up[((long long)mu * 9 + e) * V + s];
    }
    const long long n_el = 36 * V;
    for (int k = 0; k < n; ++k) {
        const int i = i0 + k;
        const double a = (double)(N - i) / N, b = (double)i / N;
        double2 w[9];
#pragma unroll
        for (int e = 0; e < 9; ++e) w[e] = make_double2(a * u[e].x + b * v[e].x, a * u[e].y + b * v[e].y);
        if (out64) {
#pragma unroll
            for (int e = 0; e < 9; ++e) out64[(long long)k * n_el + ((long long)mu * 9 + e) * V + s] = w[e];
        }
        if (out32) {
            float2 *o = out32 + (long long)k * n_el + (long long)mu * 9 * V;
            float4 *o4 = reinterpret_cast<float4 *>(o);
#pragma unroll
            for (int q = 0; q < 4; ++q)
                o4[(long long)q * V + s] = make_float4((float)w[2 * q].x, (float)w[2 * q].y, (float)w[2 * q + 1].x,
                                                       (float)w[2 * q + 1].y);
            o[8 * V + s] = make_float2((float)w[8].x, (float)w[8].y);
        }
    }
}

void interpolate(psms_ctx *c, const double2 *U, const double2 *Up, double2 *out64, float2 *out32, int N, int i0,
                 int n) {
    const long long nl = 4 * c->g.V;
    interp_kernel<<<(unsigned)((nl + 255) / 256), 256, 0, c->stream>>>(U, Up, out64, out32, N, i0, n, c->g.V);
    PSMS_LAUNCH_CHECK("interpolate");
}

// FP32 copy of an FP64 link field (n_el = 36 V elements), one thread per
// link, full 16-byte stores of the element pairs
__global__ void to_f32_kernel(const double2 *a, float2 *b, long long V) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 4 * V) return;
    const int mu = (int)(t / V);
    const long long s = t - (long long)mu * V;
    const double2 *q = a + (long long)mu * 9 * V + s;
    float2 *o = b + (long long)mu * 9 * V;
    float4 *o4 = reinterpret_cast<float4 *>(o);
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const double2 x = q[(2 * p) * V], y = q[(2 * p + 1) * V];
        o4[(long long)p * V + s] = make_float4((float)x.x, (float)x.y, (float)y.x, (float)y.y);
    }
    const double2 z = q[8 * V];
    o[8 * V + s] = make_float2((float)z.x, (float)z.y);
}

void links_to_f32(psms_ctx *c, const double2 *a, float2 *b, long long n_el) {
    const long long V = n_el / 36;
    to_f32_kernel<<<(unsigned)((4 * V + 255) / 256), 256, 0, c->stream>>>(a, b, V);
    PSMS_LAUNCH_CHECK("links_to_f32");
}

// dst = old, except active links of blocks with accept[lex] != 0 taken from prop
__global__ void merge_kernel(Geom g, const BlockInfo *binfo, const double2 *old, const double2 *prop, double2 *dst,
                             const int *accept) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 4 * g.V) return;
    const long long s = t >> 2;
    const int mu = (int)(t & 3);
    int p, r, j, y[4], x[4];
    decode(g, binfo, s, p, r, j, y, x);
    const bool take = link_active(g, y, mu, 0) && accept[binfo[r].lex];
    const double2 *src = take ? prop : old;
    for (int e = 0; e < 9; ++e) dst[((long long)mu * 9 + e) * g.V + s] = src[((long long)mu * 9 + e) * g.V + s];
}

void merge_blocks(psms_ctx *c, const double2 *old, const double2 *prop, double2 *dst, const int *d_accept) {
    const long long n = 4 * c->g.V;
    merge_kernel<<<(unsigned)((n + 127) / 128), 128, 0, c->stream>>>(c->g, c->d_binfo, old, prop, dst, d_accept);
    PSMS_LAUNCH_CHECK("merge");
}

// ---------------------------------------------------------------------------
// canonical <-> internal layouts
// ---------------------------------------------------------------------------
__global__ void gauge_canon_kernel(Geom g, const double2 *canon, double2 *U, int to_internal) {
    const long long lex = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (lex >= g.V) return;
    int x[4];
    long long rem = lex;
    x[3] = (int)(rem % g.L[3]);
    rem /= g.L[3];
    x[2] = (int)(rem % g.L[2]);
    rem /= g.L[2];
    x[1] = (int)(rem % g.L[1]);
    x[0] = (int)(rem / g.L[1]);
    const long long s = site_index(g, x);
    for (int mu = 0; mu < 4; ++mu)
        for (int e = 0; e < 9; ++e) {
            const long long ic = (lex * 4 + mu) * 9 + e;
            const long long ii = ((long long)mu * 9 + e) * g.V + s;
            if (to_internal)
                U[ii] = canon[ic];
            else
                ((double2 *)canon)[ic] = U[ii];
        }
}

void gauge_canonical(psms_ctx *c, const double2 *canon, double2 *U, int to_internal) {
    const int NT = 128;
    gauge_canon_kernel<<<(unsigned)((c->g.V + NT - 1) / NT), NT, 0, c->stream>>>(c->g, canon, U, to_internal);
    PSMS_LAUNCH_CHECK("gauge_canonical");
}

template <class S>
__global__ void spinor_canon_kernel(Geom g, const double2 *canon, typename S::elem *nat, int to_native) {
    const long long lex = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (lex >= g.V) return;
    int x[4];
    long long rem = lex;
    x[3] = (int)(rem % g.L[3]);
    rem /= g.L[3];
    x[2] = (int)(rem % g.L[2]);
    rem /= g.L[2];
    x[1] = (int)(rem % g.L[1]);
    x[0] = (int)(rem / g.L[1]);
    const long long s = site_index(g, x);
    using R = typename S::R;
    for (int c = 0; c < 12; ++c) {
        if (to_native) {
            double2 v = canon[lex * 12 + c];
            S::st(nat, c, g.V, s, mk<R>((R)v.x, (R)v.y));
        } else {
            cpx<R> v = S::ld(nat, c, g.V, s);
            ((double2 *)canon)[lex * 12 + c] = make_double2((double)v.re, (double)v.im);
        }
    }
}

void spinor_canonical(psms_ctx *c, const double2 *canon, void *nat, int prec, int to_native) {
    const int NT = 128;
    const unsigned nb = (unsigned)((c->g.V + NT - 1) / NT);
    switch (prec) {
        case P64: spinor_canon_kernel<Store<double>><<<nb, NT, 0, c->stream>>>(c->g, canon, (double2 *)nat, to_native); break;
        case P32: spinor_canon_kernel<Store<float>><<<nb, NT, 0, c->stream>>>(c->g, canon, (float2 *)nat, to_native); break;
        default:
            spinor_canon_kernel<Store<__nv_bfloat16>><<<nb, NT, 0, c->stream>>>(c->g, canon, (__nv_bfloat162 *)nat,
                                                                              to_native);
            break;
    }
    PSMS_LAUNCH_CHECK("spinor_canonical");
}

}  // namespace psms
