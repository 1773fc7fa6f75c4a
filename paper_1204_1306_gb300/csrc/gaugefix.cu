// Relative gauge fixing of a pair of gauge fields (Sec. 4.2, App. B).
//
// The transformation lives on the interior points of the blocks (sites whose
// eight neighbours are in the same block), so every block is an independent
// problem: one CTA per block runs the whole steepest-descent iteration on
// its own links, with no inter-CTA communication.  Each step computes, at
// every interior point,
//     Delta(x) = sum_mu [B(x,mu) A(x,mu)^dag + B(x-mu,mu)^dag A(x-mu,mu)]
// (W_f + W_b of App. B on the current pair A, B), Y = Delta - Delta^dag -
// Tr(Delta - Delta^dag)/3 and theta(x) = sum |Y_ij|^2, and, unless the mean
// of theta over the block's interior is below theta_tol, applies
// h(x) = exp(alpha/4 Y(x)) as A -> A^h, B -> B^{h^{-1}}: the relative
// rotation h^2 = exp(alpha/2 Y) is the step of Eq. (ming).  A block that has
// not converged after max_iter steps restarts from the unfixed pair with
// alpha lowered by dalpha, down to alpha_min.
//
// Exactness of the method needs the map (U, U') -> (g_1, g_2) to satisfy
// (U', U) -> (g_2, g_1) (Sec. 4.2).  Every block therefore iterates on its
// pair in a canonical order (the field whose first differing real number,
// in the order (local site, mu, entry, re/im), is smaller comes first), so
// the swapped call runs the identical arithmetic and hands back the
// swapped result bit for bit, whatever the precision of the iteration.  The
// accumulated transformations are reunitarised and applied in FP64, so the
// endpoints U^{g_1}, U'^{g_2} are gauge transforms of U, U' to FP64
// rounding and the determinants the estimators target are unchanged.
#include "gaugefix.hpp"

#include <vector>

namespace psms {

namespace {

template <class R>
struct Mat {
    cpx<R> e[3][3];
};

template <class R>
__device__ __forceinline__ Mat<R> ident() {
    Mat<R> m;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) m.e[i][j] = {R(i == j), R(0)};
    return m;
}

template <class R>
__device__ __forceinline__ Mat<R> mmul(const Mat<R> &a, const Mat<R> &b) {
    Mat<R> r;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            cpx<R> z = cmul(a.e[i][0], b.e[0][j]);
            z = z + cmul(a.e[i][1], b.e[1][j]);
            z = z + cmul(a.e[i][2], b.e[2][j]);
            r.e[i][j] = z;
        }
    return r;
}

// a b^dag
template <class R>
__device__ __forceinline__ Mat<R> mmul_nd(const Mat<R> &a, const Mat<R> &b) {
    Mat<R> r;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            cpx<R> z = cjmul(b.e[j][0], a.e[i][0]);
            z = z + cjmul(b.e[j][1], a.e[i][1]);
            z = z + cjmul(b.e[j][2], a.e[i][2]);
            r.e[i][j] = z;
        }
    return r;
}

// a^dag b
template <class R>
__device__ __forceinline__ Mat<R> mmul_dn(const Mat<R> &a, const Mat<R> &b) {
    Mat<R> r;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            cpx<R> z = cjmul(a.e[0][i], b.e[0][j]);
            z = z + cjmul(a.e[1][i], b.e[1][j]);
            z = z + cjmul(a.e[2][i], b.e[2][j]);
            r.e[i][j] = z;
        }
    return r;
}

// exp(X) by scaling and squaring: Taylor polynomial of degree K (Horner
// form) after halving X until ||X||_F <= 1/2 (truncation error below
// 2^-(K+1)/(K+1)!: K = 18 for FP64, 9 for FP32).
template <class R>
__device__ Mat<R> mexp(Mat<R> X) {
    constexpr int K = sizeof(R) == 8 ? 18 : 9;
    R nf = 0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) nf += X.e[i][j].re * X.e[i][j].re + X.e[i][j].im * X.e[i][j].im;
    nf = sqrt(nf);
    int sq = 0;
    while (nf > R(0.5) && sq < 40) {
        nf *= R(0.5);
        ++sq;
    }
    const R sc = ldexp(R(1), -sq);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) X.e[i][j] = sc * X.e[i][j];
    Mat<R> E = ident<R>();
    for (int n = K; n >= 1; --n) {
        Mat<R> T = mmul(X, E);
        const R inv = R(1) / R(n);
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) E.e[i][j] = {R(i == j) + inv * T.e[i][j].re, inv * T.e[i][j].im};
    }
    for (int k = 0; k < sq; ++k) E = mmul(E, E);
    return E;
}

// Gram-Schmidt on rows 0, 1; row 2 = conj(row0 x row1) (FP64)
__device__ Mat<double> reunit64(Mat<double> u) {
    double n0 = 0;
    for (int j = 0; j < 3; ++j) n0 += u.e[0][j].re * u.e[0][j].re + u.e[0][j].im * u.e[0][j].im;
    n0 = 1.0 / sqrt(n0);
    for (int j = 0; j < 3; ++j) u.e[0][j] = n0 * u.e[0][j];
    cpx<double> d = {0, 0};
    for (int j = 0; j < 3; ++j) d = d + cjmul(u.e[0][j], u.e[1][j]);
    for (int j = 0; j < 3; ++j) u.e[1][j] = u.e[1][j] - cmul(d, u.e[0][j]);
    double n1 = 0;
    for (int j = 0; j < 3; ++j) n1 += u.e[1][j].re * u.e[1][j].re + u.e[1][j].im * u.e[1][j].im;
    n1 = 1.0 / sqrt(n1);
    for (int j = 0; j < 3; ++j) u.e[1][j] = n1 * u.e[1][j];
    auto cc = [](cpx<double> a) { return cpx<double>{a.re, -a.im}; };
    u.e[2][0] = cc(cmul(u.e[0][1], u.e[1][2]) - cmul(u.e[0][2], u.e[1][1]));
    u.e[2][1] = cc(cmul(u.e[0][2], u.e[1][0]) - cmul(u.e[0][0], u.e[1][2]));
    u.e[2][2] = cc(cmul(u.e[0][0], u.e[1][1]) - cmul(u.e[0][1], u.e[1][0]));
    return u;
}

// fields of 3x3 matrices at element (k * 9 + e) * V + s (k = mu for links)
template <class R>
__device__ __forceinline__ Mat<R> ldm(const cpx<R> *p, long long V, int k, long long s) {
    Mat<R> m;
    const cpx<R> *q = p + (long long)k * 9 * V + s;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) m.e[a][b] = q[(3 * a + b) * V];
    return m;
}

template <class R>
__device__ __forceinline__ void stm(cpx<R> *p, long long V, int k, long long s, const Mat<R> &m) {
    cpx<R> *q = p + (long long)k * 9 * V + s;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) q[(3 * a + b) * V] = m.e[a][b];
}

__device__ __forceinline__ Mat<double> ld64(const double2 *p, long long V, int k, long long s) {
    Mat<double> m;
    const double2 *q = p + (long long)k * 9 * V + s;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            const double2 v = q[(3 * a + b) * V];
            m.e[a][b] = {v.x, v.y};
        }
    return m;
}

__device__ __forceinline__ void st64(double2 *p, long long V, int k, long long s, const Mat<double> &m) {
    double2 *q = p + (long long)k * 9 * V + s;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) q[(3 * a + b) * V] = make_double2(m.e[a][b].re, m.e[a][b].im);
}

__device__ __forceinline__ bool interior(const Geom &g, const int y[4]) {
    bool in = true;
    for (int m = 0; m < 4; ++m) in &= (y[m] >= 1) & (y[m] <= g.l[m] - 2);
    return in;
}

// internal index of the site with local coordinates y in the block of rank r
__device__ __forceinline__ long long block_site(const Geom &g, int r, const int y[4]) {
    const int ll = ((y[0] * g.l[1] + y[1]) * g.l[2] + y[2]) * g.l[3] + y[3];
    const int p = (y[0] + y[1] + y[2] + y[3]) & 1;
    return (long long)p * g.Vh + (long long)r * g.Vbh + (ll >> 1);
}

// i in [0, Vb): parity i / Vbh, j = i % Vbh
__device__ __forceinline__ long long site_of(const Geom &g, int r, int i, int y[4]) {
    const int p = i >= g.Vbh;
    const int j = i - p * g.Vbh;
    local_lex(g, p, j, y);
    return (long long)p * g.Vh + (long long)r * g.Vbh + j;
}

constexpr int NT = 256;

// per block: canonical order of the pair.  swap[lex] = 1 when U' comes first.
__global__ void __launch_bounds__(NT) orient_kernel(Geom g, const BlockInfo *binfo, const double2 *U,
                                                    const double2 *Up, int *swap) {
    __shared__ long long kmin[NT];
    const int r = blockIdx.x;
    const long long V = g.V;
    const int Vb = 2 * g.Vbh;
    long long best = 0x7fffffffffffffffLL;
    for (int i = threadIdx.x; i < Vb; i += NT) {
        int y[4];
        const long long s = site_of(g, r, i, y);
        const long long ll = ((y[0] * g.l[1] + y[1]) * g.l[2] + y[2]) * g.l[3] + y[3];
        for (int mu = 0; mu < 4; ++mu)
            for (int e = 0; e < 9; ++e) {
                const double2 a = U[((long long)mu * 9 + e) * V + s];
                const double2 b = Up[((long long)mu * 9 + e) * V + s];
                const long long k0 = ((ll * 4 + mu) * 9 + e) * 2;
                if (a.x != b.x) {
                    best = min(best, k0);
                } else if (a.y != b.y) {
                    best = min(best, k0 + 1);
                }
            }
    }
    kmin[threadIdx.x] = best;
    __syncthreads();
    for (int w = NT / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) kmin[threadIdx.x] = min(kmin[threadIdx.x], kmin[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        int sw = 0;
        const long long k = kmin[0];
        if (k != 0x7fffffffffffffffLL) {
            const int c = (int)(k & 1);
            const int e = (int)((k >> 1) % 9);
            const int mu = (int)(((k >> 1) / 9) & 3);
            const int ll = (int)(((k >> 1) / 9) >> 2);
            int y[4];
            y[3] = ll % g.l[3];
            y[2] = (ll / g.l[3]) % g.l[2];
            y[1] = (ll / (g.l[3] * g.l[2])) % g.l[1];
            y[0] = ll / (g.l[3] * g.l[2] * g.l[1]);
            const long long s = block_site(g, r, y);
            const double2 a = U[((long long)mu * 9 + e) * V + s];
            const double2 b = Up[((long long)mu * 9 + e) * V + s];
            sw = c ? (b.y < a.y) : (b.x < a.x);
        }
        swap[binfo[r].lex] = sw;
    }
}

template <class R>
struct IterArgs {
    Geom g;
    const BlockInfo *binfo;
    const double2 *U, *Up;
    cpx<R> *A, *B;     // current pair [mu][e][s]
    cpx<R> *gA, *gB;   // accumulated transformations [e][s]
    cpx<R> *H;         // step transformation [e][s]
    const int *swap;   // per lex block
    double alpha0, alpha_min, dalpha, theta_tol;
    int max_iter;
    int *steps_out;      // per lex block
    double *alpha_out;   // per lex block
    double *theta_out;   // per lex block
};

template <class R>
__device__ void load_pair(const IterArgs<R> &a, int r, int sw) {
    const Geom &g = a.g;
    const long long V = g.V;
    const int Vb = 2 * g.Vbh;
    const double2 *src0 = sw ? a.Up : a.U;
    const double2 *src1 = sw ? a.U : a.Up;
    for (int i = threadIdx.x; i < Vb; i += NT) {
        int y[4];
        const long long s = site_of(g, r, i, y);
        for (int mu = 0; mu < 4; ++mu)
            for (int e = 0; e < 9; ++e) {
                const long long k = ((long long)mu * 9 + e) * V + s;
                a.A[k] = {R(src0[k].x), R(src0[k].y)};
                a.B[k] = {R(src1[k].x), R(src1[k].y)};
            }
        if (interior(g, y)) {
            stm(a.gA, V, 0, s, ident<R>());
            stm(a.gB, V, 0, s, ident<R>());
        }
    }
}

// one CTA per block (rank r = blockIdx.x): the whole iteration
template <class R>
__global__ void __launch_bounds__(NT) iterate_kernel(const IterArgs<R> a) {
    __shared__ double red[NT];
    __shared__ int s_act, s_steps;
    __shared__ double s_alpha, s_theta;
    const Geom &g = a.g;
    const int r = blockIdx.x;
    const int lex = a.binfo[r].lex;
    const long long V = g.V;
    const int Vb = 2 * g.Vbh;
    int nint = 1;
    for (int m = 0; m < 4; ++m) nint *= (g.l[m] >= 3 ? g.l[m] - 2 : 0);
    const int sw = a.swap[lex];
    if (threadIdx.x == 0) {
        s_alpha = a.alpha0;
        s_steps = 0;
        s_theta = 0;
    }
    if (nint == 0) {
        if (threadIdx.x == 0) {
            a.steps_out[lex] = 0;
            a.alpha_out[lex] = a.alpha0;
            a.theta_out[lex] = 0;
        }
        return;
    }
    load_pair(a, r, sw);
    __syncthreads();
    for (;;) {
        // phase A: Delta, Y, theta and the step h at every interior point
        const R q = R(0.25 * s_alpha);
        double th = 0;
        for (int i = threadIdx.x; i < Vb; i += NT) {
            int y[4];
            const long long s = site_of(g, r, i, y);
            if (!interior(g, y)) continue;
            Mat<R> D;
            for (int ii = 0; ii < 3; ++ii)
                for (int jj = 0; jj < 3; ++jj) D.e[ii][jj] = {R(0), R(0)};
            for (int mu = 0; mu < 4; ++mu) {
                const Mat<R> f = mmul_nd(ldm(a.B, V, mu, s), ldm(a.A, V, mu, s));
                int ym[4] = {y[0], y[1], y[2], y[3]};
                ym[mu] -= 1;
                const long long sm = block_site(g, r, ym);
                const Mat<R> b = mmul_dn(ldm(a.B, V, mu, sm), ldm(a.A, V, mu, sm));
                for (int ii = 0; ii < 3; ++ii)
                    for (int jj = 0; jj < 3; ++jj) D.e[ii][jj] = D.e[ii][jj] + f.e[ii][jj] + b.e[ii][jj];
            }
            Mat<R> Y;
            for (int ii = 0; ii < 3; ++ii)
                for (int jj = 0; jj < 3; ++jj)
                    Y.e[ii][jj] = {D.e[ii][jj].re - D.e[jj][ii].re, D.e[ii][jj].im + D.e[jj][ii].im};
            const R tr3 = (Y.e[0][0].im + Y.e[1][1].im + Y.e[2][2].im) / R(3);
            for (int ii = 0; ii < 3; ++ii) Y.e[ii][ii].im -= tr3;
            R t = 0;
            for (int ii = 0; ii < 3; ++ii)
                for (int jj = 0; jj < 3; ++jj) t += Y.e[ii][jj].re * Y.e[ii][jj].re + Y.e[ii][jj].im * Y.e[ii][jj].im;
            th += (double)t;
            for (int ii = 0; ii < 3; ++ii)
                for (int jj = 0; jj < 3; ++jj) Y.e[ii][jj] = q * Y.e[ii][jj];
            stm(a.H, V, 0, s, mexp(Y));
        }
        red[threadIdx.x] = th;
        __syncthreads();
        for (int w = NT / 2; w > 0; w >>= 1) {
            if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            const double tb = red[0] / nint;
            s_theta = tb;
            int act;
            if (tb < a.theta_tol) {
                act = 2;
            } else if (s_steps >= a.max_iter) {
                if (s_alpha - a.dalpha >= a.alpha_min - 1e-12) {
                    s_alpha -= a.dalpha;
                    s_steps = 0;
                    act = 1;
                } else {
                    act = 2;
                }
            } else {
                act = 0;
                s_steps += 1;
            }
            s_act = act;
        }
        __syncthreads();
        const int act = s_act;
        if (act == 2) break;
        if (act == 1) {
            load_pair(a, r, sw);
            __syncthreads();
            continue;
        }
        // phase B: A -> h(x) A h(x+mu)^dag, B -> h(x)^dag B h(x+mu) on every
        // link that touches an interior point; g_A -> h g_A, g_B -> h^dag g_B
        for (int i = threadIdx.x; i < Vb; i += NT) {
            int y[4];
            const long long s = site_of(g, r, i, y);
            const bool ix = interior(g, y);
            Mat<R> hx = ix ? ldm(a.H, V, 0, s) : ident<R>();
            for (int mu = 0; mu < 4; ++mu) {
                if (y[mu] == g.l[mu] - 1) continue;  // leaves the block: x is on a face
                int yp[4] = {y[0], y[1], y[2], y[3]};
                yp[mu] += 1;
                const bool iy = interior(g, yp);
                if (!ix && !iy) continue;
                const Mat<R> hy = iy ? ldm(a.H, V, 0, block_site(g, r, yp)) : ident<R>();
                stm(a.A, V, mu, s, mmul_nd(mmul(hx, ldm(a.A, V, mu, s)), hy));
                stm(a.B, V, mu, s, mmul(mmul_dn(hx, ldm(a.B, V, mu, s)), hy));
            }
            if (ix) {
                stm(a.gA, V, 0, s, mmul(hx, ldm(a.gA, V, 0, s)));
                stm(a.gB, V, 0, s, mmul_dn(hx, ldm(a.gB, V, 0, s)));
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        a.steps_out[lex] = s_steps;
        a.alpha_out[lex] = s_alpha;
        a.theta_out[lex] = s_theta;
    }
}

// G1, G2 (FP64, [e][s]): reunitarised transformations in the caller's order,
// the identity off the interiors
template <class R>
__global__ void final_g_kernel(Geom g, const BlockInfo *binfo, const cpx<R> *gA, const cpx<R> *gB, const int *swap,
                               double2 *G1, double2 *G2) {
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.V) return;
    int p, r, j, y[4], x[4];
    decode(g, binfo, s, p, r, j, y, x);
    Mat<double> a = ident<double>(), b = ident<double>();
    if (interior(g, y)) {
        const Mat<R> ma = ldm(gA, g.V, 0, s), mb = ldm(gB, g.V, 0, s);
        for (int ii = 0; ii < 3; ++ii)
            for (int jj = 0; jj < 3; ++jj) {
                a.e[ii][jj] = {double(ma.e[ii][jj].re), double(ma.e[ii][jj].im)};
                b.e[ii][jj] = {double(mb.e[ii][jj].re), double(mb.e[ii][jj].im)};
            }
        a = reunit64(a);
        b = reunit64(b);
    }
    const int sw = swap[binfo[r].lex];
    st64(G1, g.V, 0, s, sw ? b : a);
    st64(G2, g.V, 0, s, sw ? a : b);
}

// out(x, mu) = G(x) U(x, mu) G(x + mu)^dag (out may alias U)
__global__ void apply_kernel(Geom g, const BlockInfo *binfo, const double2 *G, const double2 *U, double2 *out) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 4 * g.V) return;
    const long long s = t >> 2;
    const int mu = (int)(t & 3);
    int p, r, j, y[4], x[4];
    decode(g, binfo, s, p, r, j, y, x);
    x[mu] = (x[mu] + 1) % g.L[mu];
    const long long sn = site_index(g, x);
    const Mat<double> gx = ld64(G, g.V, 0, s), gy = ld64(G, g.V, 0, sn);
    st64(out, g.V, mu, s, mmul_nd(mmul(gx, ld64(U, g.V, mu, s)), gy));
}

template <class R>
void run_iteration(psms_ctx *c, const double2 *U, const double2 *Up, const int *d_swap, const GaugeFixParams &prm,
                   int *d_steps, double *d_alpha, double *d_theta, double2 *G1, double2 *G2) {
    const Geom &g = c->g;
    const size_t mb = sizeof(cpx<R>) * 9 * (size_t)g.V;
    IterArgs<R> a;
    a.g = g;
    a.binfo = c->d_binfo;
    a.U = U;
    a.Up = Up;
    a.A = (cpx<R> *)scratch(c, "gf_A", 4 * mb);
    a.B = (cpx<R> *)scratch(c, "gf_B", 4 * mb);
    a.gA = (cpx<R> *)scratch(c, "gf_gA", mb);
    a.gB = (cpx<R> *)scratch(c, "gf_gB", mb);
    a.H = (cpx<R> *)scratch(c, "gf_H", mb);
    a.swap = d_swap;
    a.alpha0 = prm.alpha0;
    a.alpha_min = prm.alpha_min;
    a.dalpha = prm.dalpha;
    a.theta_tol = prm.theta_tol;
    a.max_iter = prm.max_iter;
    a.steps_out = d_steps;
    a.alpha_out = d_alpha;
    a.theta_out = d_theta;
    iterate_kernel<R><<<g.nblocks, NT, 0, c->stream>>>(a);
    PSMS_LAUNCH_CHECK("gf_iterate");
    final_g_kernel<R><<<(unsigned)((g.V + 127) / 128), 128, 0, c->stream>>>(g, c->d_binfo, a.gA, a.gB, d_swap, G1,
                                                                             G2);
    PSMS_LAUNCH_CHECK("gf_final_g");
}

}  // namespace

void gauge_fix_pair(psms_ctx *c, const double2 *U, const double2 *Up, double2 *out0, double2 *outN,
                    const GaugeFixParams &prm, GaugeFixInfo *info) {
    const Geom &g = c->g;
    const int nb = g.nblocks;
    int *d_swap = (int *)scratch(c, "gf_swap", sizeof(int) * nb);
    int *d_steps = (int *)scratch(c, "gf_steps", sizeof(int) * nb);
    double *d_alpha = (double *)scratch(c, "gf_alpha", sizeof(double) * nb);
    double *d_theta = (double *)scratch(c, "gf_theta", sizeof(double) * nb);
    double2 *G1 = (double2 *)scratch(c, "gf_G1", sizeof(double2) * 9 * (size_t)g.V);
    double2 *G2 = (double2 *)scratch(c, "gf_G2", sizeof(double2) * 9 * (size_t)g.V);
    orient_kernel<<<nb, NT, 0, c->stream>>>(g, c->d_binfo, U, Up, d_swap);
    PSMS_LAUNCH_CHECK("gf_orient");
    if (prm.prec == P64)
        run_iteration<double>(c, U, Up, d_swap, prm, d_steps, d_alpha, d_theta, G1, G2);
    else
        run_iteration<float>(c, U, Up, d_swap, prm, d_steps, d_alpha, d_theta, G1, G2);
    const long long n = 4 * g.V;
    apply_kernel<<<(unsigned)((n + 127) / 128), 128, 0, c->stream>>>(g, c->d_binfo, G1, U, out0);
    PSMS_LAUNCH_CHECK("gf_apply");
    apply_kernel<<<(unsigned)((n + 127) / 128), 128, 0, c->stream>>>(g, c->d_binfo, G2, Up, outN);
    PSMS_LAUNCH_CHECK("gf_apply");
    if (info) {
        info->G1 = G1;
        info->G2 = G2;
        info->d_steps = d_steps;
        info->d_alpha = d_alpha;
        info->d_theta = d_theta;
        info->d_swap = d_swap;
    }
}

}  // namespace psms

namespace psms {

namespace {
__global__ void export_kernel(Geom g, const double2 *G, double2 *canon) {
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
    for (int e = 0; e < 9; ++e) canon[lex * 9 + e] = G[(long long)e * g.V + s];
}
}  // namespace

void gauge_fix_export(psms_ctx *c, const double2 *G, double2 *canon) {
    export_kernel<<<(unsigned)((c->g.V + 127) / 128), 128, 0, c->stream>>>(c->g, G, canon);
    PSMS_LAUNCH_CHECK("gf_export");
}

}  // namespace psms
