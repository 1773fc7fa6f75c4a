// Stochastic determinant-ratio estimates and the hierarchical filter step.
//
//  Eq. (stacc):   min{1, det(M^dag M)^-1} -> min{1, exp(-|M xi|^2 + |xi|^2)}
//  Eq. (gfparam): U_i = ((N-i)/N) U + (i/N) U'   (relative gauge fixing off)
//  Eq. (staccN):  Delta = sum_i |M_i xi_i|^2 - |xi_i|^2,  M_i = op(U_{i+1})^-1 op(U_i)
//  Block level:   op = D_b on every Dirichlet block (Sec. 3).
//  Global level:  op = 1 - PQ, Q = D_bb^-1 D_bw D_ww^-1 D_wb (Eq. (ddfactor)),
//                 (1 - PQ)^-1 = 1 - P D^-1 D_wb (Eq. (inverseschur)), noise
//                 on range(P) (Eq. (detschur)).
//  Filter:        Eq. (hierarchy) with the levels of Eq. (4step) (one DD
//                 level), random translation after the global step (Sec. 3).
//
// All interpolation steps i are batched into every launch (system index =
// i), and all blocks of a level are solved by one persistent launch.
#include "estimator.hpp"
#include "interp_plan.hpp"
#include "gauge.hpp"
#include "solver.hpp"

#include <algorithm>
#include <cmath>
#include <vector>

namespace psms {

// ---------------------------------------------------------------------------
// noise: TAG_NOISE, counter (counter, (level << 32) | i, lex site, j)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void apply_P(const Geom &g, int r, const int y[4], Spinor<double> &v) {
    const bool black = g.coloured && r < g.nbh;
    int nf = 0, fmu = 0;
    double ft = 0;
    for (int m = 0; m < 4; ++m) {
        if (y[m] == g.l[m] - 1) {
            ++nf;
            fmu = m;
            ft = 1.0;
        } else if (y[m] == 0) {
            ++nf;
            fmu = m;
            ft = -1.0;
        }
    }
    if (!black || nf == 0) {
        zero(v);
        return;
    }
    if (nf >= 2) return;
    // P = (1 + t gamma_mu)/2  -> (h, t e^+ h)/2 with h = psi_u + t e psi_d
    Half<double> h = project(fmu, ft, v);
    zero(v);
    reconstruct_add(fmu, ft, h, v);
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 3; ++b) v.c[a][b] = 0.5 * v.c[a][b];
}

__global__ void noise_kernel(Geom g, const BlockInfo *binfo, double2 *out, long long bs, uint64_t seed,
                             uint64_t counter, uint64_t level, int proj, int i0) {
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.V) return;
    const uint64_t i = blockIdx.y;
    int p, r, j, y[4], x[4];
    decode(g, binfo, s, p, r, j, y, x);
    const uint64_t lex = (uint64_t)lex_index(g, x);
    const uint64_t stream = (level << 32) | (uint64_t)(i0 + i);
    Spinor<double> v;
    for (int jj = 0; jj < 6; ++jj) {
        uni4 u = uniforms(seed, TAG_NOISE, counter, stream, lex, (uint64_t)jj);
        for (int m = 0; m < 2; ++m) {
            const double rad = sqrt(-log(u.u[2 * m]));
            // e^{2 pi i u_b}: one sincospi call (exact argument reduction)
            double sn, cs;
            sincospi(2.0 * u.u[2 * m + 1], &sn, &cs);
            const int comp = 2 * jj + m;
            v.c[comp / 3][comp % 3] = {rad * cs, rad * sn};
        }
    }
    if (proj) apply_P(g, r, y, v);
    store_spinor<Store<double>>(out + i * bs, g.V, s, v);
}

void noise(psms_ctx *c, double2 *out, int n, uint64_t seed, uint64_t counter, int level, int proj, int i0) {
    const int NT = 128;
    dim3 grid((unsigned)((c->g.V + NT - 1) / NT), n);
    noise_kernel<<<grid, NT, 0, c->stream>>>(c->g, c->d_binfo, out, 12 * c->g.V, seed, counter, (uint64_t)level, proj,
                                             i0);
    PSMS_LAUNCH_CHECK("noise");
}

// out = y - P z  (all sites; P = 0 off the black block boundaries)
__global__ void sub_proj_kernel(Geom g, const BlockInfo *binfo, double2 *out, const double2 *y, const double2 *z,
                                long long bs) {
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.V) return;
    const long long k = blockIdx.y;
    int p, r, j, yy[4], x[4];
    decode(g, binfo, s, p, r, j, yy, x);
    Spinor<double> zv = load_spinor<Store<double>>(z + k * bs, g.V, s);
    Spinor<double> yv = load_spinor<Store<double>>(y + k * bs, g.V, s);
    apply_P(g, r, yy, zv);
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 3; ++b) yv.c[a][b] = yv.c[a][b] - zv.c[a][b];
    store_spinor<Store<double>>(out + k * bs, g.V, s, yv);
}

static void sub_proj(psms_ctx *c, double2 *out, const double2 *y, const double2 *z, int n) {
    const int NT = 128;
    dim3 grid((unsigned)((c->g.V + NT - 1) / NT), n);
    sub_proj_kernel<<<grid, NT, 0, c->stream>>>(c->g, c->d_binfo, out, y, z, 12 * c->g.V);
    PSMS_LAUNCH_CHECK("sub_proj");
}

// per (system, block) |v|^2 over the block's sites, out[k * n_ranks + rl]
template <int NT>
__global__ void __launch_bounds__(NT) block_norm_kernel(Geom g, const double2 *v, long long bs, int rank_lo,
                                                        int n_ranks, double *out) {
    __shared__ double sh[NT / 32];
    const int rl = blockIdx.x, k = blockIdx.y, r = rank_lo + rl;
    double acc = 0;
    for (int p = 0; p < 2; ++p)
        for (int j = threadIdx.x; j < g.Vbh; j += NT) {
            const long long s = (long long)p * g.Vh + (long long)r * g.Vbh + j;
            for (int q = 0; q < 12; ++q) {
                double2 w = v[k * bs + q * g.V + s];
                acc += w.x * w.x + w.y * w.y;
            }
        }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0;
        for (int i = 0; i < NT / 32; ++i) t += sh[i];
        out[(long long)k * n_ranks + rl] = t;
    }
}

// delta[lex(r) * N + i0 + i] = a[i * nr + r] - b[i * nr + r], i < n; 0 for
// blocks the mask (an earlier level) turned away, whose solves were skipped
__global__ void block_delta_kernel(const BlockInfo *binfo, const double *a, const double *b, int nr, int n, int N,
                                   int i0, const int *mask, double *delta) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nr * n) return;
    const int i = t / nr, r = t % nr;
    const int lex = binfo[r].lex;
    delta[(long long)lex * N + i0 + i] = (mask && !mask[lex]) ? 0.0 : a[t] - b[t];
}

int chunk_size(psms_ctx *c, int N, double bytes_per_site) {
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    double budget = std::min(64e9, 0.45 * (double)tot);
    int k = (int)(budget / (bytes_per_site * (double)c->g.V));
    if (c->max_chunk > 0) k = std::min(k, c->max_chunk);
    // chunks of equal size (N = 12 with room for 11 runs as 6 + 6, not
    // 11 + 1, so that no chunk runs a lone system through a level's fixed
    // per-chunk work)
    return balanced_chunk(std::max(N, 1), k);
}

static void check_status(psms_ctx *c, const int *d_status, int n, const char *what) {
    std::vector<int> h(n);
    cuda_check(cudaMemcpyAsync(h.data(), d_status, sizeof(int) * n, cudaMemcpyDeviceToHost, c->stream), what);
    cuda_check(cudaStreamSynchronize(c->stream), what);
    for (int v : h)
        if (v) fail(PSMS_ENOCONV, std::string(what) + ": a block solve missed its tolerance");
}

// interpolated link fields U_0..U_N (FP64, FP32 when needed) in scratch
struct Interp {
    double2 *u64;
    float2 *u32;
    long long bs;  // complex elements per field
};

// fields U_{i0} .. U_{i0+n} of Eq. (gfparam) (or U, U' in the independent mode)
static Interp make_interp(psms_ctx *c, const double2 *U, const double2 *Up, int N, int mode, bool need32,
                          const char *tag, int i0, int n) {
    const long long nel = 36 * c->g.V;
    Interp it;
    it.bs = nel;
    const int nf = (mode == PSMS_EST_INDEPENDENT) ? 2 : n + 1;
    it.u64 = (double2 *)scratch(c, std::string("interp64_") + tag, sizeof(double2) * nel * nf);
    it.u32 = need32 ? (float2 *)scratch(c, std::string("interp32_") + tag, sizeof(float2) * nel * nf) : nullptr;
    if (mode == PSMS_EST_INDEPENDENT) {
        interpolate(c, U, Up, it.u64, it.u32, 1, 0, 2);  // field 0 = U, field 1 = U'
    } else {
        interpolate(c, U, Up, it.u64, it.u32, N, i0, n + 1);
    }
    return it;
}

// link pointers for op(U_i) (first) and op(U_{i+1}) (second) of system i
struct Pair {
    const double2 *a64, *b64;
    const float2 *a32, *b32;
    long long bs;
};
static Pair pair_of(const Interp &it, int mode) {
    Pair p;
    if (mode == PSMS_EST_INDEPENDENT) {
        p.a64 = it.u64;
        p.b64 = it.u64 + it.bs;
        p.a32 = it.u32;
        p.b32 = it.u32 ? it.u32 + it.bs : nullptr;
        p.bs = 0;
    } else {
        p.a64 = it.u64;
        p.b64 = it.u64 + it.bs;
        p.a32 = it.u32;
        p.b32 = it.u32 ? it.u32 + it.bs : nullptr;
        p.bs = it.bs;
    }
    return p;
}

static long long block_level_chunk(psms_ctx *c, const double2 *U, const double2 *Up, int N, int i0, int n, int mode,
                                   uint64_t seed, uint64_t counter, double tol, int inner, double *d_delta,
                                   const int *d_mask) {
    const Geom &g = c->g;
    const long long V = g.V;
    const long long fs = 12 * V;
    const int nr = g.nblocks;
    Interp it = make_interp(c, U, Up, N, mode, inner != P64, "blk", i0, n);
    Pair pr = pair_of(it, mode);
    double2 *xi = (double2 *)scratch(c, "bl_xi", sizeof(double2) * fs * n);
    double2 *eta = (double2 *)scratch(c, "bl_eta", sizeof(double2) * fs * n);
    double2 *ysol = (double2 *)scratch(c, "bl_y", sizeof(double2) * fs * n);
    noise(c, xi, n, seed, counter, PSMS_LEVEL_BLOCK, 0, i0);
    // eta_i = D_blk(U_i) xi_i = A xi - H_intra(xi)/2
    HopCall h;
    h.prec = P64;
    h.U = pr.a64;
    h.U_bs = pr.bs;
    h.n_sys = n;
    h.p = -1;
    h.mode = HOP_INTRA;
    h.in = View<void>{xi, V, 0, fs};
    h.out = View<void>{eta, V, 0, fs};
    h.y = h.in;
    h.a = c->A;
    h.b = -0.5;
    hop_launch(c, h);
    int *iters = (int *)scratch(c, "bl_iters", sizeof(int) * nr * n);
    double *resid = (double *)scratch(c, "bl_resid", sizeof(double) * nr * n);
    double *xn = (double *)scratch(c, "bl_xn", sizeof(double) * nr * n);
    double *xin = (double *)scratch(c, "bl_xin", sizeof(double) * nr * n);
    int *status = (int *)scratch(c, "bl_status", sizeof(int) * nr * n);
    BlockSolveReq q;
    q.rank_lo = 0;
    q.n_ranks = nr;
    q.n_sys = n;
    q.b = View<double2>{eta, V, 0, fs};
    q.x = View<double2>{ysol, V, 0, fs};
    q.U64 = pr.b64;
    q.U32 = pr.b32;
    q.U64_bs = pr.bs;
    q.tol = tol;
    q.inner_prec = inner;
    q.iters = iters;
    q.resid = resid;
    q.xnorm2 = xn;
    q.status = status;
    q.block_active = d_mask;
    block_solve(c, q);
    block_norm_kernel<128><<<dim3(nr, n), 128, 0, c->stream>>>(g, xi, fs, 0, nr, xin);
    PSMS_LAUNCH_CHECK("block_norm_kernel");
    block_delta_kernel<<<(nr * n + 127) / 128, 128, 0, c->stream>>>(c->d_binfo, xn, xin, nr, n, N, i0, d_mask,
                                                                   d_delta);
    PSMS_LAUNCH_CHECK("block_delta_kernel");
    check_status(c, status, nr * n, "block level");
    std::vector<int> hit(nr * n);
    cuda_check(cudaMemcpyAsync(hit.data(), iters, sizeof(int) * nr * n, cudaMemcpyDeviceToHost, c->stream), "iters");
    cuda_check(cudaStreamSynchronize(c->stream), "iters");
    long long tot = 0;
    for (int v : hit) tot += v;
    prof_block_bytes(c, tot, inner);
    return tot / nr;  // whole-lattice-equivalent iterations
}

long long block_level(psms_ctx *c, const double2 *U, const double2 *Up, int N, int mode, uint64_t seed,
                      uint64_t counter, double tol, int inner, double *d_delta, const int *d_mask) {
    const int ch = chunk_size(c, N, inner == P64 ? 2600.0 : 2100.0);
    long long tot = 0;
    for (int i0 = 0; i0 < N; i0 += ch)
        tot += block_level_chunk(c, U, Up, N, i0, std::min(ch, N - i0), mode, seed, counter, tol, inner, d_delta,
                                 d_mask);
    return tot;
}

// v = (1 - P Q(U_i)) xi for all systems; links per system via Pair (first = U_i)
static long long one_minus_PQ(psms_ctx *c, const double2 *U64, const float2 *U32, long long Ubs, int N,
                              const double2 *xi, double2 *v, double tol, int inner) {
    const Geom &g = c->g;
    const long long V = g.V, fs = 12 * V;
    const int nbh = g.nbh;
    double2 *t1 = (double2 *)scratch(c, "pq_t1", sizeof(double2) * fs * N);
    double2 *t2 = (double2 *)scratch(c, "pq_t2", sizeof(double2) * fs * N);
    int *iters = (int *)scratch(c, "pq_iters", sizeof(int) * nbh * N);
    double *resid = (double *)scratch(c, "pq_resid", sizeof(double) * nbh * N);
    int *status = (int *)scratch(c, "pq_status", sizeof(int) * nbh * N);
    long long tot = 0;
    std::vector<int> hit(nbh * N);
    auto solve_ranks = [&](int lo, double2 *b, double2 *x) {
        BlockSolveReq q;
        q.rank_lo = lo;
        q.n_ranks = nbh;
        q.n_sys = N;
        q.b = View<double2>{b, V, 0, fs};
        q.x = View<double2>{x, V, 0, fs};
        q.U64 = U64;
        q.U32 = U32;
        q.U64_bs = Ubs;
        q.tol = tol;
        q.inner_prec = inner;
        q.iters = iters;
        q.resid = resid;
        q.status = status;
        block_solve(c, q);
        check_status(c, status, nbh * N, "Schur block solve");
        cuda_check(cudaMemcpyAsync(hit.data(), iters, sizeof(int) * nbh * N, cudaMemcpyDeviceToHost, c->stream), "it");
        cuda_check(cudaStreamSynchronize(c->stream), "it");
        long long here = 0;
        for (int w : hit) here += w;
        prof_block_bytes(c, here, inner);
        tot += here;
    };
    // block iterations are returned in whole-lattice-equivalent units below
    HopCall h;
    h.prec = P64;
    h.U = U64;
    h.U_bs = Ubs;
    h.n_sys = N;
    h.p = -1;
    h.mode = HOP_INTER;
    h.b = -0.5;
    // t1 = D_wb xi   (white output blocks)
    h.rank_lo = nbh;
    h.n_ranks = nbh;
    h.in = View<void>{(void *)xi, V, 0, fs};
    h.out = View<void>{t1, V, 0, fs};
    hop_launch(c, h);
    // t2 = D_ww^-1 t1
    solve_ranks(nbh, t1, t2);
    // t1 = D_bw t2   (black output blocks)
    h.rank_lo = 0;
    h.in = View<void>{t2, V, 0, fs};
    h.out = View<void>{t1, V, 0, fs};
    hop_launch(c, h);
    // t2 = D_bb^-1 t1
    solve_ranks(0, t1, t2);
    // v = xi - P t2 (t2 holds stale white-block values; P = 0 there)
    sub_proj(c, v, xi, t2, N);
    return tot / g.nblocks;
}

// w = (1 - P Q(U_{i+1}))^-1 v = v - P [D^-1 (0, D_wb v)]_black
static long long inv_one_minus_PQ(psms_ctx *c, const double2 *U64, const float2 *U32, const LinkInterp &li,
                                  long long Ubs, int N,
                                  const double2 *v, double2 *w, double tol, int inner) {
    const Geom &g = c->g;
    const long long V = g.V, fs = 12 * V;
    double2 *y = (double2 *)scratch(c, "ipq_y", sizeof(double2) * fs * N);
    double2 *z = (double2 *)scratch(c, "ipq_z", sizeof(double2) * fs * N);
    cuda_check(cudaMemsetAsync(y, 0, sizeof(double2) * fs * N, c->stream), "ipq memset");
    HopCall h;
    h.prec = P64;
    h.U = U64;
    h.U_bs = Ubs;
    h.n_sys = N;
    h.p = -1;
    h.mode = HOP_INTER;
    h.b = -0.5;
    h.rank_lo = g.nbh;
    h.n_ranks = g.nbh;
    h.in = View<void>{(void *)v, V, 0, fs};
    h.out = View<void>{y, V, 0, fs};
    hop_launch(c, h);
    FullSolveReq q;
    q.n_sys = N;
    q.b = View<double2>{y, V, 0, fs};
    q.x = View<double2>{z, V, 0, fs};
    q.U64 = U64;
    q.U32 = U32;
    q.li32 = li;
    q.U64_bs = Ubs;
    q.tol = tol;
    q.inner_prec = inner;
    psms_solve_info info;
    solve_full_batch(c, q, &info);
    // z holds values on white sites too; P vanishes there
    sub_proj(c, w, v, z, N);
    return info.inner_iters;
}

__global__ void link_diff_kernel(const float2 *u0, const float2 *u1, long long V, unsigned char *flag) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 4 * V) return;
    const int mu = (int)(t / V);
    const long long s = t - (long long)mu * V;
    const SU3<float> a = load_link<Store<float>>(u0, V, mu, s), b = load_link<Store<float>>(u1, V, mu, s);
    bool d = false;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) d = d || a.e[i][j].re != b.e[i][j].re || a.e[i][j].im != b.e[i][j].im;
    flag[t] = d ? 1 : 0;
}

SharedEnds shared_ends(psms_ctx *c, const double2 *ends64, const char *tag) {
    const long long V = c->g.V, nel = 36 * V;
    SharedEnds e;
    e.u0 = (float2 *)scratch(c, std::string("ends32_") + tag, sizeof(float2) * 2 * nel);
    e.u1 = e.u0 + nel;
    e.flag = (unsigned char *)scratch(c, std::string("endsflag_") + tag, (size_t)(4 * V));
    links_to_f32(c, ends64, e.u0, nel);
    links_to_f32(c, ends64 + nel, e.u1, nel);
    link_diff_kernel<<<(unsigned)((4 * V + 255) / 256), 256, 0, c->stream>>>(e.u0, e.u1, V, e.flag);
    PSMS_LAUNCH_CHECK("link_diff_kernel");
    return e;
}

LinkInterp link_interp(psms_ctx *c, const SharedEnds &e, int N, int i0, int n, int shift, int mode,
                       const char *tag) {
    std::vector<float2> h(n);
    interp_coefs(N, i0, n, shift, mode == PSMS_EST_INDEPENDENT, reinterpret_cast<float *>(h.data()));
    float2 *d = (float2 *)scratch(c, std::string("li_ab_") + tag, sizeof(float2) * n);
    cuda_check(cudaMemcpyAsync(d, h.data(), sizeof(float2) * n, cudaMemcpyHostToDevice, c->stream), "link coefs");
    cuda_check(cudaStreamSynchronize(c->stream), "link coefs");
    LinkInterp li;
    li.U0 = e.u0;
    li.U1 = e.u1;
    li.ab = d;
    li.flag = e.flag;
    return li;
}

static long long global_level_chunk(psms_ctx *c, const double2 *U, const double2 *Up, int N, int i0, int n,
                                    int mode, uint64_t seed, uint64_t counter, double tol, int inner,
                                    double *h_delta) {
    const Geom &g = c->g;
    const long long V = g.V, fs = 12 * V;
    Interp it = make_interp(c, U, Up, N, mode, inner != P64, "glb", i0, n);
    Pair pr = pair_of(it, mode);
    double2 *xi = (double2 *)scratch(c, "gl_xi", sizeof(double2) * fs * n);
    double2 *v = (double2 *)scratch(c, "gl_v", sizeof(double2) * fs * n);
    double2 *w = (double2 *)scratch(c, "gl_w", sizeof(double2) * fs * n);
    noise(c, xi, n, seed, counter, PSMS_LEVEL_GLOBAL, 1, i0);
    long long tot = one_minus_PQ(c, pr.a64, pr.a32, pr.bs, n, xi, v, tol, inner);
    // the whole-lattice FP32 solves read shared endpoint links (op(U_{i+1}))
    LinkInterp li;
    if (inner != P64 && c->shared_links) {
        double2 *e64 = (double2 *)scratch(c, "ends64_glb", sizeof(double2) * 2 * it.bs);
        interpolate(c, U, Up, e64, nullptr, 1, 0, 2);
        li = link_interp(c, shared_ends(c, e64, "glb"), N, i0, n, 1, mode, "glb");
    }
    tot += inv_one_minus_PQ(c, pr.b64, pr.b32, li, pr.bs, n, v, w, tol, inner);
    double *nw = (double *)scratch(c, "gl_nw", sizeof(double) * n);
    double *nx = (double *)scratch(c, "gl_nx", sizeof(double) * n);
    norm2_batch(c, P64, View<void>{w, V, 0, fs}, 0, V, n, nw);
    norm2_batch(c, P64, View<void>{xi, V, 0, fs}, 0, V, n, nx);
    std::vector<double> a(n), b(n);
    cuda_check(cudaMemcpyAsync(a.data(), nw, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream), "gl");
    cuda_check(cudaMemcpyAsync(b.data(), nx, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream), "gl");
    cuda_check(cudaStreamSynchronize(c->stream), "gl");
    for (int i = 0; i < n; ++i) h_delta[i0 + i] = a[i] - b[i];
    return tot;
}

long long global_level(psms_ctx *c, const double2 *U, const double2 *Up, int N, int mode, uint64_t seed,
                       uint64_t counter, double tol, int inner, double *d_delta) {
    if (!c->g.coloured) fail(PSMS_EINVAL, "the Schur complement needs an even number of blocks in every direction");
    const int ch = chunk_size(c, N, inner == P64 ? 4600.0 : 3700.0);
    std::vector<double> h(N);
    long long tot = 0;
    for (int i0 = 0; i0 < N; i0 += ch)
        tot += global_level_chunk(c, U, Up, N, i0, std::min(ch, N - i0), mode, seed, counter, tol, inner, h.data());
    cuda_check(cudaMemcpyAsync(d_delta, h.data(), sizeof(double) * N, cudaMemcpyHostToDevice, c->stream), "gl");
    cuda_check(cudaStreamSynchronize(c->stream), "gl");
    return tot;
}

// ---------------------------------------------------------------------------
// accept / reject (Eq. (hierarchy)): accept iff Delta <= 0 or u < exp(-Delta),
// u from TAG_ACCEPT, counter (step, level, block, 0)
// ---------------------------------------------------------------------------
__global__ void accept_kernel(const double *delta, int nb, int N, int per_block, uint64_t seed, uint64_t step,
                              uint64_t level, double extra_sum, const double *extra_per_block, double coef,
                              double *dsum_out, int *acc, const int *mask) {
    if (per_block) {
        const int b = blockIdx.x * blockDim.x + threadIdx.x;
        if (b >= nb) return;
        double d = 0;
        for (int i = 0; i < N; ++i) d += delta[(long long)b * N + i];
        if (extra_per_block) d += coef * extra_per_block[b];
        const double u = uniforms(seed, TAG_ACCEPT, step, level, (uint64_t)b, 0).u[0];
        acc[b] = (d <= 0.0 || u < exp(-d)) ? 1 : 0;
        if (mask && !mask[b]) acc[b] = 0;
        dsum_out[b] = d;
    } else {
        if (blockIdx.x != 0 || threadIdx.x != 0) return;
        double tot = 0;
        for (int b = 0; b < nb; ++b) {
            double d = 0;
            for (int i = 0; i < N; ++i) d += delta[(long long)b * N + i];
            if (extra_per_block) d += coef * extra_per_block[b];
            dsum_out[b] = d;
            tot += d;
        }
        tot += extra_sum;
        const double u = uniforms(seed, TAG_ACCEPT, step, level, 0, 0).u[0];
        const int a = (tot <= 0.0 || u < exp(-tot)) ? 1 : 0;
        for (int b = 0; b < nb; ++b) acc[b] = a;
        dsum_out[nb] = tot;
    }
}

void decide(psms_ctx *c, const double *d_delta, int nb, int N, int per_block, uint64_t seed, uint64_t step, int level,
            double extra_sum, const double *d_extra_pb, double coef, double *d_dsum, int *d_acc, const int *d_mask) {
    accept_kernel<<<(nb + 127) / 128, 128, 0, c->stream>>>(d_delta, nb, N, per_block, seed, step, (uint64_t)level,
                                                           extra_sum, d_extra_pb, coef, d_dsum, d_acc, d_mask);
    PSMS_LAUNCH_CHECK("accept");
}

__global__ void f2d_kernel(const float *a, double *b, int n) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) b[t] = (double)a[t];
}

void float_to_double(psms_ctx *c, const float *a, double *b, int n) {
    f2d_kernel<<<(n + 127) / 128, 128, 0, c->stream>>>(a, b, n);
    PSMS_LAUNCH_CHECK("f2d");
}

}  // namespace psms
