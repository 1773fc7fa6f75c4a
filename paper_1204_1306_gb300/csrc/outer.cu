// Recursive domain decomposition (Eq. (ddrec); the 5-step filter of Sec. 5):
// outer blocks of extent B tiled by the context's blocks (the inner blocks).
//
// The outer decomposition is expressed through link masks, so that every
// operator runs on the library's existing kernels:
//   * links on the edges that cross an outer-block face set to zero give the
//     Dirichlet operator of the outer blocks, D_O = diag(D_b), as the
//     whole-lattice operator of those links (the hop kernel multiplies every
//     hop by its link; the antiperiodic time boundary is an outer face);
//     the whole-lattice solver then inverts all outer blocks at once;
//   * the same masked links leave the inner blocks' Dirichlet operators
//     unchanged (their links never cross an outer face), and their
//     inter-block hops are the hops between inner blocks of one outer block;
//   * links kept on the crossing edges only give the hops between outer
//     blocks.
// Stage 2 (SUB) estimates det D-hat_b for every outer block b (the Schur
// complement of b's inner blocks), Stage 3 (OUTER) the global Schur
// complement of the outer blocks, each by Eq. (staccN) with Eq.
// (inverseschur), as the oracle's recursive module does.
#include <string>
#include <vector>

#include "estimator.hpp"
#include "gauge.hpp"
#include "outer.cuh"
#include "outer.hpp"
#include "solver.hpp"

namespace psms {
namespace {

struct OG {
    int l[4], B[4];
};

OG og_of(const psms_ctx *c) {
    OG o;
    for (int m = 0; m < 4; ++m) {
        o.l[m] = c->g.l[m];
        o.B[m] = c->outer[m];
    }
    return o;
}

// kind 1: zero the links that cross an outer face; kind 2: zero all others
__global__ void mask_links_kernel(Geom g, const BlockInfo *binfo, OG o, double2 *U, long long bs, int kind) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 4 * g.V) return;
    const int mu = (int)(t / g.V);
    const long long s = t - (long long)mu * g.V;
    int p, r, j, y[4], x[4];
    decode(g, binfo, s, p, r, j, y, x);
    const bool cr = outer::crossing(x, mu, o.B);
    if ((kind == 1 && !cr) || (kind == 2 && cr)) return;
    double2 *q = U + (long long)blockIdx.y * bs + (long long)mu * 9 * g.V + s;
    for (int e = 0; e < 9; ++e) q[(long long)e * g.V] = make_double2(0.0, 0.0);
}

// v <- P v in place (P of the SUB or OUTER decomposition)
__global__ void proj_kernel(Geom g, const BlockInfo *binfo, OG o, int mode, double2 *v, long long bs) {
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.V) return;
    double2 *vk = v + (long long)blockIdx.y * bs;
    int p, r, j, y[4], x[4];
    decode(g, binfo, s, p, r, j, y, x);
    Spinor<double> w = load_spinor<Store<double>>(vk, g.V, s);
    int fmu, ft;
    const int nf = outer::faces(mode, x, o.l, o.B, fmu, ft);
    if (outer::colour(mode, x, o.l, o.B) != 0 || nf == 0) {
        zero(w);
    } else if (nf == 1) {
        const Half<double> h = project(fmu, (double)ft, w);
        zero(w);
        reconstruct_add(fmu, (double)ft, h, w);
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 3; ++b) w.c[a][b] = 0.5 * w.c[a][b];
    }
    store_spinor<Store<double>>(vk, g.V, s, w);
}

// zero the sites whose outer block does not have colour `keep`
__global__ void colour_kernel(Geom g, const BlockInfo *binfo, OG o, double2 *v, long long bs, int keep) {
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.V) return;
    int p, r, j, y[4], x[4];
    decode(g, binfo, s, p, r, j, y, x);
    if (outer::colour(outer::OUTER, x, o.l, o.B) == keep) return;
    double2 *vk = v + (long long)blockIdx.y * bs;
    for (int q = 0; q < 12; ++q) vk[(long long)q * g.V + s] = make_double2(0.0, 0.0);
}

// out = y - z elementwise
__global__ void sub_kernel(double2 *out, const double2 *y, const double2 *z, long long n) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    out[t] = make_double2(y[t].x - z[t].x, y[t].y - z[t].y);
}

// per (system, rank) |v|^2 over the inner block's sites, out[k * nr + r]
constexpr int kNormNT = 128;
__global__ void __launch_bounds__(kNormNT) rank_norm_kernel(Geom g, const double2 *v, long long bs, double *out) {
    __shared__ double sh[kNormNT / 32];
    const int r = blockIdx.x, k = blockIdx.y;
    double acc = 0;
    for (int p = 0; p < 2; ++p)
        for (int j = threadIdx.x; j < g.Vbh; j += kNormNT) {
            const long long s = (long long)p * g.Vh + (long long)r * g.Vbh + j;
            for (int q = 0; q < 12; ++q) {
                const double2 w = v[(long long)k * bs + (long long)q * g.V + s];
                acc += w.x * w.x + w.y * w.y;
            }
        }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0;
        for (int i = 0; i < kNormNT / 32; ++i) t += sh[i];
        out[(long long)k * gridDim.x + r] = t;
    }
}

// flag[lex(r)] = 1 when any link starting in block r differs between U and Up
constexpr int kChgNT = 128;
__global__ void __launch_bounds__(kChgNT) block_changed_kernel(Geom g, const BlockInfo *binfo, const double2 *U,
                                                               const double2 *Up, int *flag) {
    const int r = blockIdx.x;
    int diff = 0;
    for (int t = threadIdx.x; t < 2 * g.Vbh && !diff; t += kChgNT) {
        const int p = t >= g.Vbh ? 1 : 0;
        const long long s = (long long)p * g.Vh + (long long)r * g.Vbh + (t - p * g.Vbh);
        for (int e = 0; e < 36 && !diff; ++e) {
            const double2 a = U[(long long)e * g.V + s], b = Up[(long long)e * g.V + s];
            diff = (a.x != b.x) || (a.y != b.y);
        }
    }
    diff = __syncthreads_or(diff);
    if (threadIdx.x == 0) flag[binfo[r].lex] = diff ? 1 : 0;
}

constexpr int NT = 128;

void mask_links(psms_ctx *c, double2 *U, long long bs, int n_fields, int kind) {
    dim3 grid((unsigned)((4 * c->g.V + NT - 1) / NT), n_fields);
    mask_links_kernel<<<grid, NT, 0, c->stream>>>(c->g, c->d_binfo, og_of(c), U, bs, kind);
    PSMS_LAUNCH_CHECK("mask_links");
}

void project_sites(psms_ctx *c, int mode, double2 *v, int n) {
    dim3 grid((unsigned)((c->g.V + NT - 1) / NT), n);
    proj_kernel<<<grid, NT, 0, c->stream>>>(c->g, c->d_binfo, og_of(c), mode, v, 12 * c->g.V);
    PSMS_LAUNCH_CHECK("outer_proj");
}

void keep_colour(psms_ctx *c, double2 *v, int n, int keep) {
    dim3 grid((unsigned)((c->g.V + NT - 1) / NT), n);
    colour_kernel<<<grid, NT, 0, c->stream>>>(c->g, c->d_binfo, og_of(c), v, 12 * c->g.V, keep);
    PSMS_LAUNCH_CHECK("outer_colour");
}

// out = y - P z (z is overwritten by P z)
void sub_projected(psms_ctx *c, int mode, double2 *out, const double2 *y, double2 *z, int n) {
    project_sites(c, mode, z, n);
    const long long m = 12 * c->g.V * n;
    sub_kernel<<<(unsigned)((m + 255) / 256), 256, 0, c->stream>>>(out, y, z, m);
    PSMS_LAUNCH_CHECK("outer_sub");
}

// interpolated link fields U_{i0} .. U_{i0+n} (or U, U' when independent),
// masked by `kind` (0 none, 1 crossing links zeroed, 2 only crossing kept),
// FP64 and, when asked, their FP32 copies
struct LinkSet {
    double2 *u64 = nullptr;
    float2 *u32 = nullptr;
    long long nel = 0;
    int nf = 0;
};

LinkSet make_links(psms_ctx *c, const double2 *U, const double2 *Up, int N, int mode, int i0, int n, int kind,
                   bool need32, const char *tag) {
    LinkSet ls;
    ls.nel = 36 * c->g.V;
    ls.nf = mode == PSMS_EST_INDEPENDENT ? 2 : n + 1;
    ls.u64 = (double2 *)scratch(c, std::string("ol64_") + tag, sizeof(double2) * ls.nel * ls.nf);
    if (mode == PSMS_EST_INDEPENDENT)
        interpolate(c, U, Up, ls.u64, nullptr, 1, 0, 2);
    else
        interpolate(c, U, Up, ls.u64, nullptr, N, i0, n + 1);
    if (kind) mask_links(c, ls.u64, ls.nel, ls.nf, kind);
    if (need32) {
        ls.u32 = (float2 *)scratch(c, std::string("ol32_") + tag, sizeof(float2) * ls.nel * ls.nf);
        for (int f = 0; f < ls.nf; ++f) links_to_f32(c, ls.u64 + f * ls.nel, ls.u32 + f * ls.nel, ls.nel);
    }
    return ls;
}

// links of op(U_i) (a) and op(U_{i+1}) (b) for system 0, and the stride
// between systems
struct LP {
    const double2 *a64, *b64;
    const float2 *a32, *b32;
    long long bs;
};

LP pair_of(const LinkSet &ls, int mode) {
    LP p;
    p.a64 = ls.u64;
    p.b64 = ls.u64 + ls.nel;
    p.a32 = ls.u32;
    p.b32 = ls.u32 ? ls.u32 + ls.nel : nullptr;
    p.bs = mode == PSMS_EST_INDEPENDENT ? 0 : ls.nel;
    return p;
}

void check_status(psms_ctx *c, const int *d_status, int n, const char *what) {
    std::vector<int> h(n);
    cuda_check(cudaMemcpyAsync(h.data(), d_status, sizeof(int) * n, cudaMemcpyDeviceToHost, c->stream), what);
    cuda_check(cudaStreamSynchronize(c->stream), what);
    for (int v : h)
        if (v) fail(PSMS_ENOCONV, std::string(what) + ": a block solve missed its tolerance");
}

// per inner-block rank: 1 when its outer block has colour `keep` (device)
const int *outer_colour_ranks(psms_ctx *c, int keep) {
    const Geom &g = c->g;
    std::vector<int> h(g.nblocks);
    for (int r = 0; r < g.nblocks; ++r) {
        int col = 0;
        for (int m = 0; m < 4; ++m) col += c->h_binfo[r].B[m] * g.l[m] / c->outer[m];
        h[r] = (col & 1) == keep ? 1 : 0;
    }
    int *d = (int *)scratch(c, keep ? "outer_ranks1" : "outer_ranks0", sizeof(int) * g.nblocks);
    cuda_check(cudaMemcpyAsync(d, h.data(), sizeof(int) * g.nblocks, cudaMemcpyHostToDevice, c->stream), "ranks");
    cuda_check(cudaStreamSynchronize(c->stream), "ranks");
    return d;
}

// whole-lattice solve of n systems with the given links; rank_active
// (optional) restricts it to the inner blocks of one outer colour when the
// links decouple the colours and b vanishes on the other
long long solve_all(psms_ctx *c, const double2 *U64, const float2 *U32, long long bs, int n, const double2 *b,
                    double2 *x, double tol, int inner, const int *rank_active = nullptr,
                    const LinkInterp &li = LinkInterp{}) {
    const long long V = c->g.V, fs = 12 * V;
    FullSolveReq q;
    q.n_sys = n;
    q.b = View<double2>{const_cast<double2 *>(b), V, 0, fs};
    q.x = View<double2>{x, V, 0, fs};
    q.U64 = U64;
    q.U32 = U32;
    q.li32 = li;
    q.U64_bs = bs;
    q.tol = tol;
    q.inner_prec = inner;
    q.rank_active = rank_active;
    psms_solve_info info;
    solve_full_batch(c, q, &info);
    return info.inner_iters;
}

// shared FP32 endpoint links (U, U' masked by `kind`) of the whole-lattice
// FP32 solves
SharedEnds outer_ends(psms_ctx *c, const double2 *U, const double2 *Up, int kind, const char *tag) {
    const long long nel = 36 * c->g.V;
    double2 *e64 = (double2 *)scratch(c, std::string("oends64_") + tag, sizeof(double2) * 2 * nel);
    interpolate(c, U, Up, e64, nullptr, 1, 0, 2);
    if (kind) mask_links(c, e64, nel, 2, kind);
    return shared_ends(c, e64, tag);
}

// out = -1/2 H(in) with the given links over the whole lattice
void hop_all(psms_ctx *c, const double2 *U64, long long bs, int n, const double2 *in, double2 *out) {
    const long long V = c->g.V, fs = 12 * V;
    HopCall h;
    h.prec = P64;
    h.U = U64;
    h.U_bs = bs;
    h.n_sys = n;
    h.p = -1;
    h.mode = HOP_ALL;
    h.b = -0.5;
    h.in = View<void>{(void *)in, V, 0, fs};
    h.out = View<void>{out, V, 0, fs};
    hop_launch(c, h);
}

// outer block (lexicographic over the outer blocks) of every inner rank
std::vector<int> outer_of_rank(const psms_ctx *c) {
    const Geom &g = c->g;
    int nbo[4];
    for (int m = 0; m < 4; ++m) nbo[m] = g.L[m] / c->outer[m];
    std::vector<int> out(g.nblocks);
    for (int r = 0; r < g.nblocks; ++r) {
        int b = 0;
        for (int m = 0; m < 4; ++m) b = b * nbo[m] + c->h_binfo[r].B[m] * g.l[m] / c->outer[m];
        out[r] = b;
    }
    return out;
}

long long sub_chunk(psms_ctx *c, const double2 *U, const double2 *Up, int N, int i0, int n, int mode, uint64_t seed,
                    uint64_t counter, double tol, int inner, std::vector<double> &h_delta) {
    const Geom &g = c->g;
    const long long V = g.V, fs = 12 * V;
    const int nbh = g.nbh, nr = g.nblocks;
    LinkSet ls = make_links(c, U, Up, N, mode, i0, n, 1, inner != P64, "sub");
    LP pr = pair_of(ls, mode);
    auto buf = [&](const char *name) { return (double2 *)scratch(c, name, sizeof(double2) * fs * n); };
    double2 *xi = buf("sub_xi"), *v = buf("sub_v"), *w = buf("sub_w"), *t1 = buf("sub_t1"), *t2 = buf("sub_t2");
    noise(c, xi, n, seed, counter, PSMS_LEVEL_SUB, 0, i0);
    project_sites(c, outer::SUB, xi, n);
    int *iters = (int *)scratch(c, "sub_iters", sizeof(int) * nbh * n);
    double *resid = (double *)scratch(c, "sub_resid", sizeof(double) * nbh * n);
    int *status = (int *)scratch(c, "sub_status", sizeof(int) * nbh * n);
    long long tot = 0;
    std::vector<int> hit(nbh * n);
    auto solve_ranks = [&](int lo, const double2 *U64, const float2 *U32, double2 *b, double2 *x) {
        BlockSolveReq q;
        q.rank_lo = lo;
        q.n_ranks = nbh;
        q.n_sys = n;
        q.b = View<double2>{b, V, 0, fs};
        q.x = View<double2>{x, V, 0, fs};
        q.U64 = U64;
        q.U32 = U32;
        q.U64_bs = pr.bs;
        q.tol = tol;
        q.inner_prec = inner;
        q.iters = iters;
        q.resid = resid;
        q.status = status;
        block_solve(c, q);
        check_status(c, status, nbh * n, "outer-block Schur: inner block solve");
        cuda_check(cudaMemcpyAsync(hit.data(), iters, sizeof(int) * nbh * n, cudaMemcpyDeviceToHost, c->stream), "it");
        cuda_check(cudaStreamSynchronize(c->stream), "it");
        long long here = 0;
        for (int k : hit) here += k;
        tot += here / nr;
    };
    // v = (1 - P_b Q_b(U_i)) xi; with the crossing links zeroed the
    // inter-block hops stay inside the outer blocks
    HopCall h;
    h.prec = P64;
    h.U = pr.a64;
    h.U_bs = pr.bs;
    h.n_sys = n;
    h.p = -1;
    h.mode = HOP_INTER;
    h.b = -0.5;
    h.rank_lo = nbh;  // D_wb xi on the white inner blocks
    h.n_ranks = nbh;
    h.in = View<void>{xi, V, 0, fs};
    h.out = View<void>{t1, V, 0, fs};
    hop_launch(c, h);
    solve_ranks(nbh, pr.a64, pr.a32, t1, t2);  // D_ww^-1
    h.rank_lo = 0;                              // D_bw on the black inner blocks
    h.in = View<void>{t2, V, 0, fs};
    h.out = View<void>{t1, V, 0, fs};
    hop_launch(c, h);
    solve_ranks(0, pr.a64, pr.a32, t1, t2);  // D_bb^-1 (t2 keeps stale white values; P_b = 0 there)
    sub_projected(c, outer::SUB, v, xi, t2, n);
    // w = (1 - P_b Q_b(U_{i+1}))^-1 v = v - P_b [D_O^-1 (0, D_wb v)]_black
    cuda_check(cudaMemsetAsync(t1, 0, sizeof(double2) * fs * n, c->stream), "sub memset");
    h.U = pr.b64;
    h.rank_lo = nbh;
    h.in = View<void>{v, V, 0, fs};
    h.out = View<void>{t1, V, 0, fs};
    hop_launch(c, h);
    LinkInterp li;
    if (inner != P64 && c->shared_links) li = link_interp(c, outer_ends(c, U, Up, 1, "sub"), N, i0, n, 1, mode, "sub");
    tot += solve_all(c, pr.b64, pr.b32, pr.bs, n, t1, t2, tol, inner, nullptr, li);
    sub_projected(c, outer::SUB, w, v, t2, n);
    // per outer block |w|^2 - |xi|^2, summed over its inner blocks in rank order
    double *nw = (double *)scratch(c, "sub_nw", sizeof(double) * nr * n);
    double *nx = (double *)scratch(c, "sub_nx", sizeof(double) * nr * n);
    rank_norm_kernel<<<dim3(nr, n), kNormNT, 0, c->stream>>>(g, w, fs, nw);
    PSMS_LAUNCH_CHECK("sub_norm");
    rank_norm_kernel<<<dim3(nr, n), kNormNT, 0, c->stream>>>(g, xi, fs, nx);
    PSMS_LAUNCH_CHECK("sub_norm");
    std::vector<double> a(nr * n), b(nr * n);
    cuda_check(cudaMemcpyAsync(a.data(), nw, sizeof(double) * nr * n, cudaMemcpyDeviceToHost, c->stream), "sub");
    cuda_check(cudaMemcpyAsync(b.data(), nx, sizeof(double) * nr * n, cudaMemcpyDeviceToHost, c->stream), "sub");
    cuda_check(cudaStreamSynchronize(c->stream), "sub");
    const std::vector<int> ob = outer_of_rank(c);
    const int no = n_outer(c);
    for (int k = 0; k < n; ++k) {
        std::vector<double> sa(no, 0.0), sb(no, 0.0);
        for (int r = 0; r < nr; ++r) {
            sa[ob[r]] += a[(long long)k * nr + r];
            sb[ob[r]] += b[(long long)k * nr + r];
        }
        for (int o = 0; o < no; ++o) h_delta[(long long)o * N + i0 + k] = sa[o] - sb[o];
    }
    return tot;
}

long long outer_global_chunk(psms_ctx *c, const double2 *U, const double2 *Up, int N, int i0, int n, int mode,
                             uint64_t seed, uint64_t counter, double tol, int inner, std::vector<double> &h_delta) {
    const long long V = c->g.V, fs = 12 * V;
    // the whole-lattice FP32 solves read shared endpoint links: no FP32
    // copies of the interpolated fields
    const bool shared = inner != P64 && c->shared_links;
    LinkSet lf = make_links(c, U, Up, N, mode, i0, n, 0, inner != P64 && !shared, "ogf");
    LinkSet lm = make_links(c, U, Up, N, mode, i0, n, 1, inner != P64 && !shared, "ogm");
    LinkInterp lim, lif;
    if (shared) {
        lim = link_interp(c, outer_ends(c, U, Up, 1, "ogm"), N, i0, n, 0, mode, "ogm");
        lif = link_interp(c, outer_ends(c, U, Up, 0, "ogf"), N, i0, n, 1, mode, "ogf");
    }
    LinkSet lc = make_links(c, U, Up, N, mode, i0, n, 2, false, "ogc");
    LP pf = pair_of(lf, mode), pm = pair_of(lm, mode), pc = pair_of(lc, mode);
    auto buf = [&](const char *name) { return (double2 *)scratch(c, name, sizeof(double2) * fs * n); };
    double2 *xi = buf("og_xi"), *v = buf("og_v"), *w = buf("og_w"), *t1 = buf("og_t1"), *t2 = buf("og_t2");
    noise(c, xi, n, seed, counter, PSMS_LEVEL_GLOBAL, 0, i0);
    project_sites(c, outer::OUTER, xi, n);
    long long tot = 0;
    // v = (1 - P Q(U_i)) xi, Q = D_bb^-1 D_bw D_ww^-1 D_wb over the outer blocks
    // the outer Dirichlet solves touch one colour of outer blocks each: the
    // masked links decouple the outer blocks and the right-hand sides vanish
    // on the other colour, so only that colour's inner blocks are iterated
    const int *white = outer_colour_ranks(c, 1), *black = outer_colour_ranks(c, 0);
    hop_all(c, pc.a64, pc.bs, n, xi, t1);  // hops between outer blocks
    keep_colour(c, t1, n, 1);               // D_wb xi
    tot += solve_all(c, pm.a64, pm.a32, pm.bs, n, t1, t2, tol, inner, white, lim);  // D_ww^-1 (outer Dirichlet)
    hop_all(c, pc.a64, pc.bs, n, t2, t1);
    keep_colour(c, t1, n, 0);  // D_bw
    tot += solve_all(c, pm.a64, pm.a32, pm.bs, n, t1, t2, tol, inner, black, lim);  // D_bb^-1
    sub_projected(c, outer::OUTER, v, xi, t2, n);
    // w = (1 - P Q(U_{i+1}))^-1 v = v - P [D^-1 (0, D_wb v)]_black
    hop_all(c, pc.b64, pc.bs, n, v, t1);
    keep_colour(c, t1, n, 1);
    tot += solve_all(c, pf.b64, pf.b32, pf.bs, n, t1, t2, tol, inner, nullptr, lif);
    sub_projected(c, outer::OUTER, w, v, t2, n);
    double *nw = (double *)scratch(c, "og_nw", sizeof(double) * n);
    double *nx = (double *)scratch(c, "og_nx", sizeof(double) * n);
    norm2_batch(c, P64, View<void>{w, V, 0, fs}, 0, V, n, nw);
    norm2_batch(c, P64, View<void>{xi, V, 0, fs}, 0, V, n, nx);
    std::vector<double> a(n), b(n);
    cuda_check(cudaMemcpyAsync(a.data(), nw, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream), "og");
    cuda_check(cudaMemcpyAsync(b.data(), nx, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream), "og");
    cuda_check(cudaStreamSynchronize(c->stream), "og");
    for (int k = 0; k < n; ++k) h_delta[i0 + k] = a[k] - b[k];
    return tot;
}

}  // namespace

void block_changed(psms_ctx *c, const double2 *U, const double2 *Up, int *d_flag) {
    block_changed_kernel<<<c->g.nblocks, kChgNT, 0, c->stream>>>(c->g, c->d_binfo, U, Up, d_flag);
    PSMS_LAUNCH_CHECK("block_changed");
}

bool has_outer(const psms_ctx *c) { return c->outer[0] > 0; }

int n_outer(const psms_ctx *c) {
    int n = 1;
    for (int m = 0; m < 4; ++m) n *= c->g.L[m] / c->outer[m];
    return n;
}

void set_outer(psms_ctx *c, const int *B) {
    if (!B || B[0] == 0) {
        for (int m = 0; m < 4; ++m) c->outer[m] = 0;
        return;
    }
    const Geom &g = c->g;
    for (int m = 0; m < 4; ++m) {
        if (B[m] <= 0 || B[m] % g.l[m] || g.L[m] % B[m])
            fail(PSMS_EINVAL, "outer blocks must be multiples of the blocks and divide the lattice");
        if ((B[m] / g.l[m]) % 2 || (g.L[m] / B[m]) % 2)
            fail(PSMS_EINVAL, "need an even number of blocks per outer block and of outer blocks per direction");
    }
    for (int m = 0; m < 4; ++m) c->outer[m] = B[m];
}

long long sub_level(psms_ctx *c, const double2 *U, const double2 *Up, int N, int mode, uint64_t seed,
                    uint64_t counter, double tol, int inner, double *h_delta) {
    if (!has_outer(c)) fail(PSMS_EINVAL, "no outer blocks set (psms_set_outer_blocks)");
    const int ch = chunk_size(c, N, 2600.0);
    std::vector<double> h((long long)n_outer(c) * N, 0.0);
    long long tot = 0;
    for (int i0 = 0; i0 < N; i0 += ch)
        tot += sub_chunk(c, U, Up, N, i0, std::min(ch, N - i0), mode, seed, counter, tol, inner, h);
    for (size_t k = 0; k < h.size(); ++k) h_delta[k] = h[k];
    return tot;
}

long long outer_global_level(psms_ctx *c, const double2 *U, const double2 *Up, int N, int mode, uint64_t seed,
                             uint64_t counter, double tol, int inner, double *h_delta) {
    if (!has_outer(c)) fail(PSMS_EINVAL, "no outer blocks set (psms_set_outer_blocks)");
    const int ch = chunk_size(c, N, 4800.0);
    std::vector<double> h(N, 0.0);
    long long tot = 0;
    for (int i0 = 0; i0 < N; i0 += ch)
        tot += outer_global_chunk(c, U, Up, N, i0, std::min(ch, N - i0), mode, seed, counter, tol, inner, h);
    for (int i = 0; i < N; ++i) h_delta[i] = h[i];
    return tot;
}

}  // namespace psms
