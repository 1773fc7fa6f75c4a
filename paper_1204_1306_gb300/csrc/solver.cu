// Krylov solves of the Wilson-Dirac operator, Eq. (Dw), on the whole lattice
// and on Dirichlet blocks (Sec. 3).  The paper leaves the solver open
// ("inversions", Sec. 5).  Both solvers work on the even-odd Schur
// complement
//     Dhat = A - D_oe D_eo / A = A - H_o H_e / (4A)     (odd sites),
//     Dhat^dagger = A - H^dag_o H^dag_e / (4A),
// inside an FP64 defect-correction loop on the true residual b - D x, with
// the inner iterations in FP64, FP32 or BF16 storage.
//
//  * block_solve (block_solve.cuh, block_variants_*.cu): one CTA or
//    thread-block cluster per (block, system); the whole solve, including
//    the FP64 outer loop and convergence decisions, runs on the device with
//    deterministic reductions; CGNR or BiCGStab inner iterations.
//  * solve_full_batch: whole-lattice solves of n_sys systems (each with its
//    own gauge field) batched into every launch, BiCGStab (default) or CGNR
//    inner iterations; per-system scalars live on the device; the host only
//    polls convergence flags every few iterations.
#include "bicgstab.cuh"
#include "block_solve.cuh"
#include "kernels.hpp"
#include "solver.hpp"

#include <type_traits>

#include <algorithm>
#include <cmath>
#include <map>
#include <vector>

namespace psms {

// the block solver's variants, instantiated in block_variants_*.cu
PSMS_BLOCK_VARIANTS_CG(PSMS_BLOCK_EXTERN, Store<double>)
PSMS_BLOCK_VARIANTS_FORMS(PSMS_BLOCK_EXTERN, Store<double>)
PSMS_BLOCK_VARIANTS_CG(PSMS_BLOCK_EXTERN, Store<float>)
PSMS_BLOCK_VARIANTS_FORMS(PSMS_BLOCK_EXTERN, Store<float>)
PSMS_BLOCK_VARIANTS_SMEM(PSMS_BLOCK_EXTERN, Store<float>)

template <class SV, class SL>
static void launch_block_variant(psms_ctx *c, const BlockSolveArgs &a, int n_ranks, int n_sys, int cl, int minb,
                                 int hv) {
    switch (hv * 100 + cl * 10 + minb) {
        case 111: launch_block_cl<SV, SL, 1, 1, 1>(c, a, n_ranks, n_sys); break;
        case 114: launch_block_cl<SV, SL, 1, 4, 1>(c, a, n_ranks, n_sys); break;
        case 211: launch_block_cl<SV, SL, 1, 1, 2>(c, a, n_ranks, n_sys); break;
        case 214: launch_block_cl<SV, SL, 1, 4, 2>(c, a, n_ranks, n_sys); break;
        case 244: launch_block_cl<SV, SL, 4, 4, 2>(c, a, n_ranks, n_sys); break;
        case 284: launch_block_cl<SV, SL, 8, 4, 2>(c, a, n_ranks, n_sys); break;
        case 314: launch_block_cl<SV, SL, 1, 4, 3>(c, a, n_ranks, n_sys); break;
        case 614: launch_block_cl<SV, SL, 1, 4, 6>(c, a, n_ranks, n_sys); break;
        case 514: launch_block_cl<SV, SL, 1, 4, 5>(c, a, n_ranks, n_sys); break;
        case 684: launch_block_cl<SV, SL, 8, 4, 6>(c, a, n_ranks, n_sys); break;
        case 813:
        case 1013:
        case 913:
            // links in shared memory: FP32 inner iterations only (admissible() checks)
            if constexpr (std::is_same<SL, Store<float>>::value) {
                if (hv == 8) launch_block_cl<SV, SL, 1, 3, 8>(c, a, n_ranks, n_sys);
                else if (hv == 10) launch_block_cl<SV, SL, 1, 3, 10>(c, a, n_ranks, n_sys);
                else launch_block_cl<SV, SL, 1, 3, 9>(c, a, n_ranks, n_sys);
            } else {
                fail(PSMS_EINVAL, "block solver: shared-memory links need FP32 inner iterations");
            }
            break;
        case 11: launch_block_cl<SV, SL, 1, 1>(c, a, n_ranks, n_sys); break;
        case 14: launch_block_cl<SV, SL, 1, 4>(c, a, n_ranks, n_sys); break;
        case 21: launch_block_cl<SV, SL, 2, 1>(c, a, n_ranks, n_sys); break;
        case 24: launch_block_cl<SV, SL, 2, 4>(c, a, n_ranks, n_sys); break;
        case 41: launch_block_cl<SV, SL, 4, 1>(c, a, n_ranks, n_sys); break;
        case 44: launch_block_cl<SV, SL, 4, 4>(c, a, n_ranks, n_sys); break;
        case 81: launch_block_cl<SV, SL, 8, 1>(c, a, n_ranks, n_sys); break;
        default: launch_block_cl<SV, SL, 8, 4>(c, a, n_ranks, n_sys); break;
    }
}

void block_solve(psms_ctx *c, const BlockSolveReq &q) {
    const Geom &g = c->g;
    BlockSolveArgs a;
    a.g = g;
    a.binfo = c->d_binfo;
    a.A = c->A;
    a.rank_lo = q.rank_lo;
    a.n_ranks = q.n_ranks;
    a.b = q.b;
    a.x = q.x;
    const long long V = g.V;
    const size_t full64 = (size_t)12 * V * sizeof(double2);
    a.r64 = View<double2>{(double2 *)scratch(c, "bs_r64", full64 * q.n_sys), V, 0, 12 * V};
    a.U64 = q.U64;
    a.U64_bs = q.U64_bs;
    const bool in64 = (q.inner_prec == P64);
    const size_t esz = in64 ? sizeof(double2) : sizeof(float2);
    const long long per_sys = 24 * V + 7 * 12 * (long long)g.Vh;  // elements
    a.vin = scratch(c, "bs_inner", esz * (size_t)per_sys * q.n_sys);
    a.vin_bs = per_sys;
    a.Uin = in64 ? (const void *)q.U64 : (const void *)q.U32;
    a.Uin_bs = q.U64_bs;  // same element count per field
    a.tol = q.tol;
    a.delta = in64 ? std::max(0.1 * q.tol, 1e-15) : 1e-6;
    a.maxit = q.maxit;
    a.max_outer = in64 ? 4 : 12;
    a.sys_active = q.sys_active;
    a.block_active = q.block_active;
    a.iters = q.iters;
    a.resid = q.resid;
    a.xnorm2 = q.xnorm2;
    a.status = q.status;
    // Variants (cluster size CL, min CTAs per SM, hop form): one block solved
    // by CL CTAs of a thread-block cluster; hop form 1 calls one out-of-line
    // copy of the hop instead of inlining it at every call site, form 2 is
    // the branch-free hop, form 3 both; bit 2 (forms 5, 6) runs BiCGStab on
    // Dhat instead of CGNR inside the same FP64 defect correction.  The autotuner times every admissible
    // variant once on the first solve of each (precision, block size,
    // batched or not) and keeps the fastest; a solve is idempotent (x is set
    // from b), so the tuning runs leave the result unchanged.
    struct Var {
        int cl, minb, hv;
    };
    static const Var vars[] = {{1, 1, 0}, {1, 4, 0}, {2, 1, 0}, {2, 4, 0}, {4, 1, 0}, {4, 4, 0}, {8, 1, 0},
                               {8, 4, 0}, {1, 1, 1}, {1, 4, 1}, {1, 1, 2}, {1, 4, 2}, {4, 4, 2}, {8, 4, 2},
                               {1, 4, 3}, {1, 4, 6}, {1, 4, 5}, {8, 4, 6}, {1, 3, 8}, {1, 3, 10}, {1, 3, 9}};
    const int nvar = 21;
    auto admissible = [&](int v) {
        if (vars[v].hv & 8)  // the block's FP32 links in shared memory (at most 100 KB)
            return !in64 && block_links_smem(g) <= 100 * 1024;
        return vars[v].cl == 1 || g.Vbh / vars[v].cl >= 128;
    };
    auto launch = [&](int v) {
        if (in64)
            launch_block_variant<Store<double>, Store<double>>(c, a, q.n_ranks, q.n_sys, vars[v].cl, vars[v].minb,
                                                               vars[v].hv);
        else
            launch_block_variant<Store<float>, Store<float>>(c, a, q.n_ranks, q.n_sys, vars[v].cl, vars[v].minb,
                                                             vars[v].hv);
    };
    // the autotuner chooses among the variants of the context's Krylov
    // method only, so that every tuned choice gives the same bits
    auto method = [&](int v) { return (vars[v].hv >> 2) & 1; };
    const long long key = ((long long)q.inner_prec << 40) | ((long long)c->block_krylov << 36) |
                          ((long long)g.Vbh << 8) | (q.n_sys > 1 ? 1 : 0);
    auto it = c->block_variant.find(key);
    int choice = it == c->block_variant.end() ? -1 : it->second;
    if (c->forced_block_variant >= 0) choice = admissible(c->forced_block_variant) ? c->forced_block_variant : 0;
    if (choice < 0 && c->autotune) {
        cudaEvent_t e0, e1;
        cuda_check(cudaEventCreate(&e0), "tune event");
        cuda_check(cudaEventCreate(&e1), "tune event");
        float best = 1e30f;
        for (int v = 0; v < nvar; ++v) {
            if (!admissible(v) || method(v) != c->block_krylov) continue;
            cuda_check(cudaEventRecord(e0, c->stream), "tune record");
            launch(v);
            cuda_check(cudaEventRecord(e1, c->stream), "tune record");
            cuda_check(cudaEventSynchronize(e1), "tune sync");
            float ms = 0;
            cuda_check(cudaEventElapsedTime(&ms, e0, e1), "tune elapsed");
            if (ms < best) {
                best = ms;
                choice = v;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
    if (choice < 0) choice = c->block_krylov ? 15 : 0;
    if (c->forced_block_variant < 0) c->block_variant[key] = choice;
    const int slot = c->prof ? prof_block_begin(c) : -1;
    launch(choice);
    if (slot >= 0) prof_block_end(c, slot);
}

// ---------------------------------------------------------------------------
// whole-lattice batched solver
// ---------------------------------------------------------------------------
struct CGS {
    double rr, alpha, beta, bb, target, rhorho;
    int active, iters;
};

__global__ void cg_init_kernel(CGS *st, const double *bb, const double *rr, int n, double delta, const int *act,
                               int *flags) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    CGS s;
    s.bb = bb[k];
    s.rr = rr[k];
    s.target = delta * delta * bb[k];
    s.alpha = s.beta = 0;
    s.rhorho = bb[k];
    s.active = act ? act[k] : 1;
    if (s.bb == 0.0) s.active = 0;
    s.iters = 0;
    st[k] = s;
    flags[k] = s.active;
}

template <int NT>
__global__ void __launch_bounds__(NT) cg_alpha_kernel(CGS *st, const double *partial, int n) {
    __shared__ double sh[NT / 32];
    const int k = blockIdx.x;
    if (!st[k].active) return;
    double v = 0;
    for (int i = threadIdx.x; i < n; i += NT) v += partial[(long long)k * n + i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0;
        for (int i = 0; i < NT / 32; ++i) t += sh[i];
        st[k].alpha = st[k].rr / t;
    }
}

// stage 2: rr_new and rho^2 from two partial arrays -> beta, convergence
template <int NT>
__global__ void __launch_bounds__(NT) cg_beta_kernel(CGS *st, const double *p_rr, const double *p_rho, int n,
                                                     int maxit, int *flags) {
    __shared__ double sh[2][NT / 32];
    const int k = blockIdx.x;
    if (!st[k].active) return;
    double v = 0, w = 0;
    for (int i = threadIdx.x; i < n; i += NT) {
        v += p_rr[(long long)k * n + i];
        w += p_rho[(long long)k * n + i];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v += __shfl_xor_sync(0xffffffffu, v, o);
        w += __shfl_xor_sync(0xffffffffu, w, o);
    }
    if ((threadIdx.x & 31) == 0) {
        sh[0][threadIdx.x >> 5] = v;
        sh[1][threadIdx.x >> 5] = w;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0, b = 0;
        for (int i = 0; i < NT / 32; ++i) {
            a += sh[0][i];
            b += sh[1][i];
        }
        CGS s = st[k];
        s.beta = a / s.rr;
        s.rr = a;
        s.rhorho = b;
        s.iters += 1;
        if (b <= s.target || s.iters >= maxit || !(b == b)) s.active = 0;
        st[k] = s;
        flags[k] = s.active;
    }
}

// x += alpha p, rho -= alpha q, r -= alpha sv (odd halves), partial |r|^2, |rho|^2
template <class S, int NT>
__global__ void __launch_bounds__(NT) cg_update_kernel(const CGS *st, View<typename S::elem> e, View<typename S::elem> pp,
                                                       View<typename S::elem> q, View<typename S::elem> rho,
                                                       View<typename S::elem> res, View<typename S::elem> sv,
                                                       long long s_lo, long long n, double *p_rr, double *p_rho,
                                                       int skip_r) {
    using R = typename S::R;
    __shared__ double sh[2][NT / 32];
    const int k = blockIdx.y;
    if (!st[k].active) {
        if (threadIdx.x == 0) {
            p_rr[(long long)k * gridDim.x + blockIdx.x] = 0;
            p_rho[(long long)k * gridDim.x + blockIdx.x] = 0;
        }
        return;
    }
    const R alpha = (R)st[k].alpha;
    double a1 = 0, a2 = 0;
    const long long i = (long long)blockIdx.x * NT + threadIdx.x;
    if (i < n) {
        const long long s = s_lo + i;
        for (int c = 0; c < 12; ++c) {
            const long long ie = k * e.bs + S::idx(c, e.cs, s - e.off);
            const long long ip = k * pp.bs + S::idx(c, pp.cs, s - pp.off);
            cpx<R> ev = S::ldi(e.p, ie) + alpha * S::ldi(pp.p, ip);
            S::sti(e.p, ie, ev);
            const long long iq = k * q.bs + S::idx(c, q.cs, s - q.off);
            const long long ir = k * rho.bs + S::idx(c, rho.cs, s - rho.off);
            cpx<R> ro = S::ldi(rho.p, ir) - alpha * S::ldi(q.p, iq);
            S::sti(rho.p, ir, ro);
            a2 += (double)norm2(ro);
            if (!skip_r) {
                const long long is = k * sv.bs + S::idx(c, sv.cs, s - sv.off);
                const long long ires = k * res.bs + S::idx(c, res.cs, s - res.off);
                cpx<R> rv = S::ldi(res.p, ires) - alpha * S::ldi(sv.p, is);
                S::sti(res.p, ires, rv);
                a1 += (double)norm2(rv);
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a1 += __shfl_xor_sync(0xffffffffu, a1, o);
        a2 += __shfl_xor_sync(0xffffffffu, a2, o);
    }
    if ((threadIdx.x & 31) == 0) {
        sh[0][threadIdx.x >> 5] = a1;
        sh[1][threadIdx.x >> 5] = a2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t1 = 0, t2 = 0;
        for (int w = 0; w < NT / 32; ++w) {
            t1 += sh[0][w];
            t2 += sh[1][w];
        }
        p_rr[(long long)k * gridDim.x + blockIdx.x] = t1;
        p_rho[(long long)k * gridDim.x + blockIdx.x] = t2;
    }
}

// p = r + beta p
template <class S, int NT>
__global__ void __launch_bounds__(NT) cg_pupdate_kernel(const CGS *st, View<typename S::elem> pp,
                                                        View<typename S::elem> res, long long s_lo, long long n) {
    using R = typename S::R;
    const int k = blockIdx.y;
    if (!st[k].active) return;
    const R beta = (R)st[k].beta;
    const long long i = (long long)blockIdx.x * NT + threadIdx.x;
    if (i >= n) return;
    const long long s = s_lo + i;
    for (int c = 0; c < 12; ++c) {
        const long long ip = k * pp.bs + S::idx(c, pp.cs, s - pp.off);
        const long long ir = k * res.bs + S::idx(c, res.cs, s - res.off);
        S::sti(pp.p, ip, S::ldi(res.p, ir) + beta * S::ldi(pp.p, ip));
    }
}

// copy / convert: dst = scale[k] * src (FP64 src), over sites [s_lo, s_lo+n)
template <class SD, int NT>
__global__ void __launch_bounds__(NT) scale_convert_kernel(View<typename SD::elem> dst, View<double2> src,
                                                           const double *nrm2, int invert, const int *act,
                                                           long long s_lo, long long n) {
    const int k = blockIdx.y;
    if (act && !act[k]) return;
    const long long i = (long long)blockIdx.x * NT + threadIdx.x;
    if (i >= n) return;
    double sc = 1.0;
    if (nrm2) sc = invert ? 1.0 / sqrt(nrm2[k]) : sqrt(nrm2[k]);
    const long long s = s_lo + i;
    for (int c = 0; c < 12; ++c) {
        double2 v = src.p[k * src.bs + c * src.cs + s - src.off];
        SD::st(dst.p + k * dst.bs, c, dst.cs, s - dst.off,
               mk<typename SD::R>((typename SD::R)(sc * v.x), (typename SD::R)(sc * v.y)));
    }
}

// x (FP64) += sqrt(nrm2[k]) * e
template <class SE, int NT>
__global__ void __launch_bounds__(NT) accumulate_kernel(View<double2> x, View<typename SE::elem> e, const double *nrm2,
                                                        const int *act, long long s_lo, long long n) {
    const int k = blockIdx.y;
    if (act && !act[k]) return;
    const long long i = (long long)blockIdx.x * NT + threadIdx.x;
    if (i >= n) return;
    const double sc = sqrt(nrm2[k]);
    const long long s = s_lo + i;
    for (int c = 0; c < 12; ++c) {
        cpx<typename SE::R> ev = SE::ld(e.p + k * e.bs, c, e.cs, s - e.off);
        double2 &xv = x.p[k * x.bs + c * x.cs + s - x.off];
        xv.x += sc * (double)ev.re;
        xv.y += sc * (double)ev.im;
    }
}

__global__ void residual_flags_kernel(const double *rn, const double *bn, double tol, int *act, double *rel, int n) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    double r = bn[k] > 0 ? sqrt(rn[k] / bn[k]) : 0.0;
    rel[k] = r;
    act[k] = (r > tol) ? 1 : 0;
}

__global__ void set_int_kernel(int *p, int v, int n) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) p[k] = v;
}

__global__ void iters_kernel(const CGS *st, int *out, int n) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) out[k] += st[k].iters;
}

struct BCS;
__global__ void iters_bcg_kernel(const BCS *st, int *out, int n);

template <class SV>
static void inner_cg_full(psms_ctx *c, int n_sys, const void *Uin, long long U_bs, int prec, View<void> rhs,
                          View<void> e, const int *act_in, double delta, int maxit, int *iters_acc,
                          const LinkInterp &li) {
    using E = typename SV::elem;
    const Geom &g = c->g;
    const long long V = g.V, Vh = g.Vh;
    const double A = c->A, c4 = -1.0 / (4.0 * A);
    const size_t esz = sizeof(E);
    // odd-half vectors: bhat, rho, res, pp, q, sv ; even half: t
    E *base = (E *)scratch(c, "fs_inner", esz * (size_t)(7 * 12 * Vh) * n_sys);
    auto half = [&](int i, long long off) {
        View<void> v;
        v.p = base + (long long)i * 12 * Vh * n_sys;
        v.cs = Vh;
        v.off = off;
        v.bs = 12 * Vh;
        return v;
    };
    View<void> bhat = half(0, Vh), rho = half(1, Vh), res = half(2, Vh), pp = half(3, Vh), q = half(4, Vh),
               sv = half(5, Vh), t = half(6, 0);
    auto tv = [](View<void> v) { return View<E>{(E *)v.p, v.cs, v.off, v.bs}; };
    CGS *st = (CGS *)scratch(c, "fs_cgs", sizeof(CGS) * n_sys);
    int *flags = (int *)scratch(c, "fs_flags", sizeof(int) * n_sys);
    double *bb = (double *)scratch(c, "fs_bb", sizeof(double) * n_sys);
    double *rr0 = (double *)scratch(c, "fs_rr0", sizeof(double) * n_sys);

    HopCall h;
    h.prec = prec;
    h.U = Uin;
    h.U_bs = U_bs;
    h.li = li;
    h.n_sys = n_sys;
    h.active = act_in;
    const int nct = hop_ctas(c, [&] { HopCall x; x.p = 1; return x; }());
    double *p_a = (double *)scratch(c, "fs_pa", sizeof(double) * (size_t)nct * n_sys);
    double *p_b = (double *)scratch(c, "fs_pb", sizeof(double) * (size_t)nct * n_sys);

    // bhat_o = rhs_o + H_o(rhs_e)/(2A)
    h.p = 1;
    h.in = rhs;
    h.out = bhat;
    h.y = rhs;
    h.a = 1.0;
    h.b = 0.5 / A;
    h.partial = p_a;
    hop_launch(c, h);
    reduce_partials(c, p_a, nct, n_sys, bb);
    // e_o = 0 ; rho = bhat ; res = Dhat^dag rho ; pp = res
    cudaMemsetAsync((char *)e.p, 0, esz * (size_t)12 * V * n_sys, c->stream);
    cudaMemcpyAsync(rho.p, bhat.p, esz * (size_t)12 * Vh * n_sys, cudaMemcpyDeviceToDevice, c->stream);
    h.y = View<void>();
    h.partial = nullptr;
    h.p = 0;
    h.dag = 1;
    h.in = rho;
    h.out = t;
    h.b = 1.0;
    hop_launch(c, h);
    h.p = 1;
    h.in = t;
    h.out = res;
    h.y = rho;
    h.a = A;
    h.b = c4;
    h.partial = p_a;
    hop_launch(c, h);
    reduce_partials(c, p_a, nct, n_sys, rr0);
    cudaMemcpyAsync(pp.p, res.p, esz * (size_t)12 * Vh * n_sys, cudaMemcpyDeviceToDevice, c->stream);
    cg_init_kernel<<<(n_sys + 63) / 64, 64, 0, c->stream>>>(st, bb, rr0, n_sys, delta, act_in, flags);
    PSMS_LAUNCH_CHECK("cg_init");
    const int NT = 256;
    const long long n = Vh;
    const int nb = (int)((n + NT - 1) / NT);
    dim3 grid(nb, n_sys);
    double *u_rr = (double *)scratch(c, "fs_urr", sizeof(double) * (size_t)nb * n_sys);
    double *u_rho = (double *)scratch(c, "fs_urho", sizeof(double) * (size_t)nb * n_sys);
    int it = 0;
    int chunk = 8;
    std::vector<int> hflags(n_sys);
    h.active = flags;  // mirrors CGS.active
    while (it < maxit) {
        for (int i = 0; i < chunk && it < maxit; ++i, ++it) {
            // q = Dhat p
            h.dag = 0;
            h.p = 0;
            h.in = pp;
            h.out = t;
            h.y = View<void>();
            h.a = 0;
            h.b = 1.0;
            h.partial = nullptr;
            hop_launch(c, h);
            h.p = 1;
            h.in = t;
            h.out = q;
            h.y = pp;
            h.a = A;
            h.b = c4;
            h.partial = p_a;
            hop_launch(c, h);
            cg_alpha_kernel<256><<<n_sys, 256, 0, c->stream>>>(st, p_a, nct);
            PSMS_LAUNCH_CHECK("cg_alpha_kernel");
            // sv = Dhat^dag q
            h.dag = 1;
            h.p = 0;
            h.in = q;
            h.out = t;
            h.y = View<void>();
            h.a = 0;
            h.b = 1.0;
            h.partial = nullptr;
            hop_launch(c, h);
            h.p = 1;
            h.in = t;
            h.out = sv;
            h.y = q;
            h.a = A;
            h.b = c4;
            hop_launch(c, h);
            cg_update_kernel<SV, NT><<<grid, NT, 0, c->stream>>>(st, tv(e), tv(pp), tv(q), tv(rho), tv(res), tv(sv), Vh,
                                                                 n, u_rr, u_rho, 0);
            PSMS_LAUNCH_CHECK("cg_update_kernel");
            cg_beta_kernel<256><<<n_sys, 256, 0, c->stream>>>(st, u_rr, u_rho, nb, maxit, flags);
            PSMS_LAUNCH_CHECK("cg_beta_kernel");
            cg_pupdate_kernel<SV, NT><<<grid, NT, 0, c->stream>>>(st, tv(pp), tv(res), Vh, n);
            PSMS_LAUNCH_CHECK("cg iteration");
        }
        cuda_check(cudaMemcpyAsync(hflags.data(), flags, sizeof(int) * n_sys, cudaMemcpyDeviceToHost, c->stream),
                   "cg flags");
        cuda_check(cudaStreamSynchronize(c->stream), "cg sync");
        bool any = false;
        for (int k = 0; k < n_sys; ++k) any |= hflags[k] != 0;
        if (!any) break;
        chunk = std::min(chunk * 2, 64);
    }
    iters_kernel<<<(n_sys + 63) / 64, 64, 0, c->stream>>>(st, iters_acc, n_sys);
    PSMS_LAUNCH_CHECK("iters_kernel");
    // e_e = (rhs_e + H_e(e_o)/2)/A
    h.active = act_in;
    h.dag = 0;
    h.p = 0;
    h.in = e;
    h.out = e;
    h.y = rhs;
    h.a = 1.0 / A;
    h.b = 0.5 / A;
    h.partial = nullptr;
    hop_launch(c, h);
}

// ---------------------------------------------------------------------------
// BiCGStab on the even-odd operator Dhat (the paper leaves the solver open):
// per system, with complex scalars kept on the device,
//   rho = <rh, r>;  beta = (rho / rho_old)(alpha / omega);  p = r + beta (p - omega v)
//   v = Dhat p;  alpha = rho / <rh, v>;  s = r - alpha v
//   t = Dhat s;  omega = <t, s> / <t, t>;  x += alpha p + omega s;  r = s - omega t
// with rh = r_0 = bhat.  A breakdown (<rh, v> = 0, omega = 0) or the
// iteration cap ends the inner solve; the FP64 defect correction around it
// restarts from the true residual.  Reductions: per-CTA partials in FP64,
// finished in a fixed order (deterministic).
// ---------------------------------------------------------------------------
__global__ void bcg_init_kernel(BCS *st, const double *bb, int n, double delta, const int *act, int *flags) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    BCS s;
    s.rho = make_double2(bb[k], 0.0);
    s.alpha = s.omega = make_double2(1.0, 0.0);
    s.beta = make_double2(0.0, 0.0);
    s.rr = bb[k];
    s.target = delta * delta * bb[k];
    s.active = (act ? act[k] : 1) && bb[k] > 0.0;
    s.iters = 0;
    st[k] = s;
    flags[k] = s.active;
}

// mode 0: s = r - alpha v
// mode 1: x += alpha p + omega s, r = s - omega t
// mode 2: p = r + beta (p - omega v)
template <class S, int NT>
__global__ void __launch_bounds__(NT) bcg_axpy_kernel(const BCS *st, int mode, View<typename S::elem> x,
                                                      View<typename S::elem> p, View<typename S::elem> r,
                                                      View<typename S::elem> s_, View<typename S::elem> v,
                                                      View<typename S::elem> t, long long s_lo, long long n,
                                                      const int *map, const int *rank_active, int vbh_sh) {
    using R = typename S::R;
    const int k = map ? map[blockIdx.y] : (int)blockIdx.y;
    if (!st[k].active) return;
    const long long i = (long long)blockIdx.x * NT + threadIdx.x;
    if (i >= n) return;
    if (rank_active && !rank_active[(int)(i >> vbh_sh)]) return;
    const long long sx = s_lo + i;
    const BCS bs = st[k];
    auto ld = [&](const View<typename S::elem> &w, int c) { return S::ldi(w.p, k * w.bs + S::idx(c, w.cs, sx - w.off)); };
    auto st_ = [&](View<typename S::elem> &w, int c, cpx<R> val) { S::sti(w.p, k * w.bs + S::idx(c, w.cs, sx - w.off), val); };
    const cpx<R> al = {(R)bs.alpha.x, (R)bs.alpha.y}, om = {(R)bs.omega.x, (R)bs.omega.y},
                 be = {(R)bs.beta.x, (R)bs.beta.y};
    for (int c = 0; c < 12; ++c) {
        if (mode == 0) {
            st_(s_, c, ld(r, c) - cmul(al, ld(v, c)));
        } else if (mode == 1) {
            const cpx<R> sv = ld(s_, c);
            st_(x, c, ld(x, c) + cmul(al, ld(p, c)) + cmul(om, sv));
            st_(r, c, sv - cmul(om, ld(t, c)));
        } else {
            st_(p, c, ld(r, c) + cmul(be, ld(p, c) - cmul(om, ld(v, c))));
        }
    }
}

// <a, b> partials (sum conj(a) b, and |a|^2) and the scalar stage
template <class S, int NT>
__global__ void __launch_bounds__(NT) bcg_dot_stage_kernel(BCS *st, View<typename S::elem> a,
                                                           View<typename S::elem> b, long long s_lo, long long n,
                                                           double *p_re, double *p_im, double *p_aa,
                                                           unsigned int *counters, int stage, int maxit, int *flags,
                                                           const int *map, const int *rank_active, int vbh_sh) {
    using R = typename S::R;
    __shared__ double sh[3][NT / 32];
    const int k = map ? map[blockIdx.y] : (int)blockIdx.y;
    if (!st[k].active) return;
    double re = 0, im = 0, aa = 0;
    const long long i = (long long)blockIdx.x * NT + threadIdx.x;
    if (i < n && (!rank_active || rank_active[(int)(i >> vbh_sh)])) {
        const long long sx = s_lo + i;
        R tre = 0, tim = 0, taa = 0;
        for (int c = 0; c < 12; ++c) {
            const cpx<R> x = S::ldi(a.p, k * a.bs + S::idx(c, a.cs, sx - a.off));
            const cpx<R> y = S::ldi(b.p, k * b.bs + S::idx(c, b.cs, sx - b.off));
            tre += x.re * y.re + x.im * y.im;
            tim += x.re * y.im - x.im * y.re;
            taa += x.re * x.re + x.im * x.im;
        }
        re = (double)tre;
        im = (double)tim;
        aa = (double)taa;
    }
    bcg_partials_and_stage<NT>(st, re, im, aa, p_re, p_im, p_aa, counters, stage, maxit, flags, sh, k,
                               (int)blockIdx.x, (int)gridDim.x);
}

// x += alpha p + omega s, r = s - omega t, then the partials of
// sum conj(r) rh and |r|^2 and scalar stage 2
template <class S, int NT>
__global__ void __launch_bounds__(NT) bcg_update_stage_kernel(BCS *st, View<typename S::elem> x,
                                                              View<typename S::elem> p, View<typename S::elem> r,
                                                              View<typename S::elem> s_, View<typename S::elem> t,
                                                              View<typename S::elem> rh, long long s_lo, long long n,
                                                              double *p_re, double *p_im, double *p_aa,
                                                              unsigned int *counters, int maxit, int *flags,
                                                              const int *map, const int *rank_active, int vbh_sh) {
    using R = typename S::R;
    __shared__ double sh[3][NT / 32];
    const int k = map ? map[blockIdx.y] : (int)blockIdx.y;
    if (!st[k].active) return;
    const BCS bs = st[k];
    const cpx<R> al = {(R)bs.alpha.x, (R)bs.alpha.y}, om = {(R)bs.omega.x, (R)bs.omega.y};
    double re = 0, im = 0, aa = 0;
    const long long i = (long long)blockIdx.x * NT + threadIdx.x;
    if (i < n && (!rank_active || rank_active[(int)(i >> vbh_sh)])) {
        const long long sx = s_lo + i;
        auto ld = [&](const View<typename S::elem> &w, int c) {
            return S::ldi(w.p, k * w.bs + S::idx(c, w.cs, sx - w.off));
        };
        auto stv = [&](View<typename S::elem> &w, int c, cpx<R> val) {
            S::sti(w.p, k * w.bs + S::idx(c, w.cs, sx - w.off), val);
        };
        R tre = 0, tim = 0, taa = 0;
        for (int c = 0; c < 12; ++c) {
            const cpx<R> sv = ld(s_, c);
            stv(x, c, ld(x, c) + cmul(al, ld(p, c)) + cmul(om, sv));
            cpx<R> rv = sv - cmul(om, ld(t, c));
            stv(r, c, rv);
            rv = ld(r, c);  // the stored value (rounded to the storage precision)
            const cpx<R> hv = ld(rh, c);
            tre += rv.re * hv.re + rv.im * hv.im;
            tim += rv.re * hv.im - rv.im * hv.re;
            taa += rv.re * rv.re + rv.im * rv.im;
        }
        re = (double)tre;
        im = (double)tim;
        aa = (double)taa;
    }
    bcg_partials_and_stage<NT>(st, re, im, aa, p_re, p_im, p_aa, counters, 2, maxit, flags, sh, k,
                               (int)blockIdx.x, (int)gridDim.x);
}

__global__ void iters_bcg_kernel(const BCS *st, int *out, int n) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) out[k] += st[k].iters;
}

template <class SV>
static void inner_bicgstab_full(psms_ctx *c, int n_sys, const void *Uin, long long U_bs, int prec, View<void> rhs,
                                View<void> e, const int *act_in, double delta, int maxit, int *iters_acc,
                                const int *rank_active, const LinkInterp &li) {
    using E = typename SV::elem;
    const Geom &g = c->g;
    const long long V = g.V, Vh = g.Vh;
    const double A = c->A, c4 = -1.0 / (4.0 * A);
    const size_t esz = sizeof(E);
    // odd halves: bhat (= rh), r, p, v, s, t ; even half: te
    E *base = (E *)scratch(c, "fs_inner", esz * (size_t)(7 * 12 * Vh) * n_sys);
    // with a rank mask the skipped sites are never written: start from zeros
    if (rank_active)
        cuda_check(cudaMemsetAsync(base, 0, esz * (size_t)(7 * 12 * Vh) * n_sys, c->stream), "inner zero");
    const int vsh = g.vbh_sh;
    auto half = [&](int i, long long off) {
        View<void> v;
        v.p = base + (long long)i * 12 * Vh * n_sys;
        v.cs = Vh;
        v.off = off;
        v.bs = 12 * Vh;
        return v;
    };
    View<void> rh = half(0, Vh), r = half(1, Vh), pp = half(2, Vh), vv = half(3, Vh), ss = half(4, Vh),
               tt = half(5, Vh), te = half(6, 0);
    auto tv = [](View<void> v) { return View<E>{(E *)v.p, v.cs, v.off, v.bs}; };
    BCS *st = (BCS *)scratch(c, "fs_bcs", sizeof(BCS) * n_sys);
    int *flags = (int *)scratch(c, "fs_flags", sizeof(int) * n_sys);
    double *bb = (double *)scratch(c, "fs_bb", sizeof(double) * n_sys);
    HopCall h;
    h.prec = prec;
    h.U = Uin;
    h.U_bs = U_bs;
    h.li = li;
    h.n_sys = n_sys;
    h.active = act_in;
    h.rank_active = rank_active;
    const int nct = hop_ctas(c, [&] { HopCall x; x.p = 1; return x; }());
    double *p_a = (double *)scratch(c, "fs_pa", sizeof(double) * (size_t)nct * n_sys);
    // rh = bhat_o = rhs_o + H_o(rhs_e)/(2A)
    h.p = 1;
    h.in = rhs;
    h.out = rh;
    h.y = rhs;
    h.a = 1.0;
    h.b = 0.5 / A;
    h.partial = p_a;
    hop_launch(c, h);
    reduce_partials(c, p_a, nct, n_sys, bb);
    cudaMemsetAsync((char *)e.p, 0, esz * (size_t)12 * V * n_sys, c->stream);
    cudaMemcpyAsync(r.p, rh.p, esz * (size_t)12 * Vh * n_sys, cudaMemcpyDeviceToDevice, c->stream);
    cudaMemcpyAsync(pp.p, rh.p, esz * (size_t)12 * Vh * n_sys, cudaMemcpyDeviceToDevice, c->stream);
    bcg_init_kernel<<<(n_sys + 63) / 64, 64, 0, c->stream>>>(st, bb, n_sys, delta, act_in, flags);
    PSMS_LAUNCH_CHECK("bcg_init");
    const int NT = 256;
    const long long n = Vh;
    const int nb = (int)((n + NT - 1) / NT);
    dim3 grid(nb, n_sys);
    double *q_re = (double *)scratch(c, "fs_qre", sizeof(double) * (size_t)nb * n_sys);
    double *q_im = (double *)scratch(c, "fs_qim", sizeof(double) * (size_t)nb * n_sys);
    double *q_aa = (double *)scratch(c, "fs_qaa", sizeof(double) * (size_t)nb * n_sys);
    // per-system completion counters of the fused reductions (each launch
    // leaves them at zero)
    unsigned int *cnt = (unsigned int *)scratch(c, "fs_bcnt", sizeof(unsigned int) * n_sys);
    cuda_check(cudaMemsetAsync(cnt, 0, sizeof(unsigned int) * n_sys, c->stream), "bcg counters");
    // FP32 storage: the dot products of alpha and omega are taken in the
    // epilogue of the second half hop of Dhat (partials per hop CTA, the
    // last CTA of a system applies the stage), saving two passes over two
    // vectors per iteration
    const bool fuse = prec == P32;
    double *f_re = nullptr, *f_im = nullptr, *f_aa = nullptr;
    if (fuse) {
        f_re = (double *)scratch(c, "fs_fre", sizeof(double) * (size_t)nct * n_sys);
        f_im = (double *)scratch(c, "fs_fim", sizeof(double) * (size_t)nct * n_sys);
        f_aa = (double *)scratch(c, "fs_faa", sizeof(double) * (size_t)nct * n_sys);
    }
    // w = Dhat u = A u + c4 H_o(H_e u); dot 1: stage 0 on <x, w>; dot 2:
    // stage 1 on <w, u>, |w|^2
    auto apply_dhat = [&](View<void> u, View<void> w, int dot, View<void> x, int stage) {
        h.dag = 0;
        h.p = 0;
        h.in = u;
        h.out = te;
        h.y = View<void>();
        h.a = 0;
        h.b = 1.0;
        h.partial = nullptr;
        h.dot = HopDot{};
        hop_launch(c, h);
        h.p = 1;
        h.in = te;
        h.out = w;
        h.y = u;
        h.a = A;
        h.b = c4;
        if (fuse && dot) {
            h.dot.dot = dot;
            h.dot.x = x;
            h.dot.st = st;
            h.dot.re = f_re;
            h.dot.im = f_im;
            h.dot.aa = f_aa;
            h.dot.cnt = cnt;
            h.dot.stage = stage;
            h.dot.maxit = maxit;
            h.dot.flags = flags;
        }
        hop_launch(c, h);
        h.dot = HopDot{};
    };
    int it = 0;
    int chunk = 8;
    std::vector<int> hflags(n_sys), hmap;
    h.active = flags;
    // systems still iterating, refreshed at every host check: later launches
    // cover only them (a converged system's CTAs would exit at once, but
    // scheduling them costs about as much as a system's work)
    int *d_map = (int *)scratch(c, "fs_bmap", sizeof(int) * n_sys);
    const int *map = nullptr;
    int n_act = n_sys;
    while (it < maxit) {
        dim3 gridm(nb, n_act);
        h.sys_map = map;
        h.n_map = n_act;
        for (int i = 0; i < chunk && it < maxit; ++i, ++it) {
            // alpha = rho / <rh, v>
            apply_dhat(pp, vv, 1, rh, 0);
            if (!fuse) {
                bcg_dot_stage_kernel<SV, NT><<<gridm, NT, 0, c->stream>>>(st, tv(rh), tv(vv), Vh, n, q_re, q_im, q_aa,
                                                                          cnt, 0, maxit, flags, map, rank_active, vsh);
                PSMS_LAUNCH_CHECK("bcg_alpha");
            }
            bcg_axpy_kernel<SV, NT><<<gridm, NT, 0, c->stream>>>(st, 0, tv(e), tv(pp), tv(r), tv(ss), tv(vv),
                                                                 tv(tt), Vh, n, map, rank_active, vsh);
            PSMS_LAUNCH_CHECK("bcg_s");
            // omega = <t, s> / <t, t>
            apply_dhat(ss, tt, 2, View<void>(), 1);
            if (!fuse) {
                bcg_dot_stage_kernel<SV, NT><<<gridm, NT, 0, c->stream>>>(st, tv(tt), tv(ss), Vh, n, q_re, q_im, q_aa,
                                                                          cnt, 1, maxit, flags, map, rank_active, vsh);
                PSMS_LAUNCH_CHECK("bcg_omega");
            }
            // x, r updates with <rh, r>, |r|^2 and beta / convergence
            bcg_update_stage_kernel<SV, NT><<<gridm, NT, 0, c->stream>>>(st, tv(e), tv(pp), tv(r), tv(ss), tv(tt),
                                                                         tv(rh), Vh, n, q_re, q_im, q_aa, cnt,
                                                                         maxit, flags, map, rank_active, vsh);
            PSMS_LAUNCH_CHECK("bcg_update");
            bcg_axpy_kernel<SV, NT><<<gridm, NT, 0, c->stream>>>(st, 2, tv(e), tv(pp), tv(r), tv(ss), tv(vv),
                                                                 tv(tt), Vh, n, map, rank_active, vsh);
            PSMS_LAUNCH_CHECK("bcg_p");
        }
        cuda_check(cudaMemcpyAsync(hflags.data(), flags, sizeof(int) * n_sys, cudaMemcpyDeviceToHost, c->stream),
                   "bcg flags");
        cuda_check(cudaStreamSynchronize(c->stream), "bcg sync");
        hmap.clear();
        for (int k = 0; k < n_sys; ++k)
            if (hflags[k]) hmap.push_back(k);
        if (hmap.empty()) break;
        if ((int)hmap.size() < n_sys) {
            cuda_check(cudaMemcpyAsync(d_map, hmap.data(), sizeof(int) * hmap.size(), cudaMemcpyHostToDevice,
                                       c->stream),
                       "bcg map");
            cuda_check(cudaStreamSynchronize(c->stream), "bcg map");
            map = d_map;
        }
        n_act = (int)hmap.size();
        chunk = std::min(chunk * 2, 64);
    }
    h.sys_map = nullptr;
    h.n_map = 0;
    iters_bcg_kernel<<<(n_sys + 63) / 64, 64, 0, c->stream>>>(st, iters_acc, n_sys);
    PSMS_LAUNCH_CHECK("iters_kernel");
    // e_e = (rhs_e + H_e(e_o)/2)/A
    h.active = act_in;
    h.dag = 0;
    h.p = 0;
    h.in = e;
    h.out = e;
    h.y = rhs;
    h.a = 1.0 / A;
    h.b = 0.5 / A;
    h.partial = nullptr;
    hop_launch(c, h);
}

void solve_full_batch(psms_ctx *c, const FullSolveReq &q, psms_solve_info *info) {
    const Geom &g = c->g;
    const long long V = g.V;
    const int n = q.n_sys;
    double *bn = (double *)scratch(c, "fb_bn", sizeof(double) * n);
    double *rn = (double *)scratch(c, "fb_rn", sizeof(double) * n);
    double *rel = (double *)scratch(c, "fb_rel", sizeof(double) * n);
    int *act = (int *)scratch(c, "fb_act", sizeof(int) * n);
    int *iters = (int *)scratch(c, "fb_iters", sizeof(int) * n);
    double2 *r64 = (double2 *)scratch(c, "fb_r64", sizeof(double2) * (size_t)12 * V * n);
    if (q.b.cs != V || q.b.off != 0) fail(PSMS_EINVAL, "whole-lattice solve: right-hand sides must be full fields");
    View<void> b{q.b.p, q.b.cs, q.b.off, q.b.bs}, x{q.x.p, q.x.cs, q.x.off, q.x.bs};
    View<void> r{r64, V, 0, 12 * V};
    const bool in64 = q.inner_prec == P64;
    const size_t esz = in64 ? sizeof(double2) : (q.inner_prec == P32 ? sizeof(float2) : sizeof(__nv_bfloat162));
    void *rin_p = scratch(c, "fb_rin", esz * (size_t)12 * V * n);
    void *ein_p = scratch(c, "fb_ein", esz * (size_t)12 * V * n);
    View<void> rin{rin_p, V, 0, 12 * V}, ein{ein_p, V, 0, 12 * V};
    norm2_batch(c, P64, b, 0, V, n, bn);
    for (int k = 0; k < n; ++k)
        cuda_check(cudaMemsetAsync((char *)q.x.p + sizeof(double2) * k * q.x.bs, 0, sizeof(double2) * 12 * V, c->stream),
                   "zero x");
    set_int_kernel<<<(n + 63) / 64, 64, 0, c->stream>>>(iters, 0, n);
    PSMS_LAUNCH_CHECK("set_int_kernel");
    // FP32 inner solves aim for a 1e-6 reduction per outer step (measured on
    // the 32^3x64 filter step: 1e-6 beats 1e-4, 1e-5, 3e-7 and 1e-7 -- two
    // outer steps reach 1e-12, each saving one FP64 application of D, while
    // tighter targets pay more inner iterations than they save); if an outer
    // step fails to halve some system's true residual the remaining outer
    // steps of this solve use CGNR
    bool bicg = c->full_solver == 1;
    auto delta_of = [&](bool b) {
        if (!in64 && c->inner_delta > 0) return c->inner_delta;
        return in64 ? std::max(0.1 * q.tol, 1e-15) : (q.inner_prec == P32 ? (b ? 1e-6 : 2e-6) : 5e-3);
    };
    const int max_outer = in64 ? 6 : 30;
    std::vector<int> hact(n);
    std::vector<double> hrn(n), hrn_prev(n, 0.0);
    int outer = 0;
    const int NT = 256;
    dim3 grid((unsigned)((V + NT - 1) / NT), n);
    int *d_omap = (int *)scratch(c, "fb_omap", sizeof(int) * n);
    std::vector<int> omap;
    for (;; ++outer) {
        // r = b - D x = b - A x + H(x)/2   (FP64, both parities); on the
        // first step x = 0 and r = b exactly (no hop); later only for the
        // systems that have not converged (the others keep x, r and their
        // residual norm)
        if (outer == 0) {
            for (int k = 0; k < n; ++k)
                cuda_check(cudaMemcpyAsync(r64 + (size_t)12 * V * k, (const double2 *)q.b.p + (size_t)k * q.b.bs,
                                           sizeof(double2) * 12 * V, cudaMemcpyDeviceToDevice, c->stream),
                           "r = b");
            cuda_check(cudaMemcpyAsync(rn, bn, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream), "rn = bn");
        }
        HopCall h;
        h.prec = P64;
        h.U = q.U64;
        h.U_bs = q.U64_bs;
        h.n_sys = n;
        if (outer > 0) {
            omap.clear();
            for (int k = 0; k < n; ++k)
                if (hact[k]) omap.push_back(k);
            if ((int)omap.size() < n) {
                cuda_check(cudaMemcpyAsync(d_omap, omap.data(), sizeof(int) * omap.size(), cudaMemcpyHostToDevice,
                                           c->stream),
                           "outer map");
                cuda_check(cudaStreamSynchronize(c->stream), "outer map");
                h.sys_map = d_omap;
                h.n_map = (int)omap.size();
            }
        }
        h.p = -1;
        h.in = x;
        h.out = r;
        h.y = b;
        h.a = 1.0;
        h.y2 = x;
        h.a2 = -c->A;
        h.b = 0.5;
        h.rank_active = q.rank_active;  // skipped sites keep r = b = 0
        if (outer > 0) {
            hop_launch(c, h);
            norm2_batch(c, P64, r, 0, V, n, rn);
        }
        residual_flags_kernel<<<(n + 63) / 64, 64, 0, c->stream>>>(rn, bn, q.tol, act, rel, n);
        PSMS_LAUNCH_CHECK("residual_flags_kernel");
        cuda_check(cudaMemcpyAsync(hact.data(), act, sizeof(int) * n, cudaMemcpyDeviceToHost, c->stream), "act");
        cuda_check(cudaMemcpyAsync(hrn.data(), rn, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream), "rn");
        cuda_check(cudaStreamSynchronize(c->stream), "solve sync");
        bool any = false;
        for (int k = 0; k < n; ++k) any |= hact[k] != 0;
        if (!any || outer >= max_outer) break;
        if (bicg && outer > 0)
            for (int k = 0; k < n; ++k)
                if (hact[k] && !(hrn[k] <= 0.25 * hrn_prev[k])) bicg = false;
        hrn_prev = hrn;
        const double delta = delta_of(bicg);
        // inner rhs = r / |r|
        View<double2> r2{r64, V, 0, 12 * V};
        if (in64) {
            scale_convert_kernel<Store<double>, NT><<<grid, NT, 0, c->stream>>>(
                View<double2>{(double2 *)rin_p, V, 0, 12 * V}, r2, rn, 1, act, 0, V);
            PSMS_LAUNCH_CHECK("scale_convert_kernel");
            if (bicg)
                inner_bicgstab_full<Store<double>>(c, n, q.U64, q.U64_bs, P64, rin, ein, act, delta, q.maxit, iters,
                                                   q.rank_active, LinkInterp{});
            else
                inner_cg_full<Store<double>>(c, n, q.U64, q.U64_bs, P64, rin, ein, act, delta, q.maxit, iters,
                                             LinkInterp{});
            accumulate_kernel<Store<double>, NT><<<grid, NT, 0, c->stream>>>(
                View<double2>{(double2 *)q.x.p, q.x.cs, q.x.off, q.x.bs}, View<double2>{(double2 *)ein_p, V, 0, 12 * V},
                rn, act, 0, V);
            PSMS_LAUNCH_CHECK("accumulate_kernel");
        } else if (q.inner_prec == P32) {
            scale_convert_kernel<Store<float>, NT><<<grid, NT, 0, c->stream>>>(
                View<float2>{(float2 *)rin_p, V, 0, 12 * V}, r2, rn, 1, act, 0, V);
            PSMS_LAUNCH_CHECK("scale_convert_kernel");
            if (bicg)
                inner_bicgstab_full<Store<float>>(c, n, q.U32, q.U64_bs, P32, rin, ein, act, delta, q.maxit, iters,
                                                  q.rank_active, q.li32);
            else
                inner_cg_full<Store<float>>(c, n, q.U32, q.U64_bs, P32, rin, ein, act, delta, q.maxit, iters, q.li32);
            accumulate_kernel<Store<float>, NT><<<grid, NT, 0, c->stream>>>(
                View<double2>{(double2 *)q.x.p, q.x.cs, q.x.off, q.x.bs}, View<float2>{(float2 *)ein_p, V, 0, 12 * V},
                rn, act, 0, V);
            PSMS_LAUNCH_CHECK("accumulate_kernel");
        } else {
            scale_convert_kernel<Store<__nv_bfloat16>, NT><<<grid, NT, 0, c->stream>>>(
                View<__nv_bfloat162>{(__nv_bfloat162 *)rin_p, V, 0, 12 * V}, r2, rn, 1, act, 0, V);
            PSMS_LAUNCH_CHECK("scale_convert_kernel");
            if (bicg)
                inner_bicgstab_full<Store<__nv_bfloat16>>(c, n, q.U32, q.U64_bs, PB16, rin, ein, act, delta, q.maxit,
                                                          iters, q.rank_active, q.li32);
            else
                inner_cg_full<Store<__nv_bfloat16>>(c, n, q.U32, q.U64_bs, PB16, rin, ein, act, delta, q.maxit,
                                                    iters, q.li32);
            accumulate_kernel<Store<__nv_bfloat16>, NT><<<grid, NT, 0, c->stream>>>(
                View<double2>{(double2 *)q.x.p, q.x.cs, q.x.off, q.x.bs},
                View<__nv_bfloat162>{(__nv_bfloat162 *)ein_p, V, 0, 12 * V}, rn, act, 0, V);
            PSMS_LAUNCH_CHECK("accumulate_kernel");
        }
        PSMS_LAUNCH_CHECK("defect correction");
    }
    std::vector<double> hrel(n);
    std::vector<int> hit(n);
    cuda_check(cudaMemcpyAsync(hrel.data(), rel, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream), "rel");
    cuda_check(cudaMemcpyAsync(hit.data(), iters, sizeof(int) * n, cudaMemcpyDeviceToHost, c->stream), "iters");
    cuda_check(cudaStreamSynchronize(c->stream), "solve end");
    double worst = 0;
    long long tot = 0;
    for (int k = 0; k < n; ++k) {
        worst = std::max(worst, hrel[k]);
        tot += hit[k];
    }
    if (info) {
        info->outer_iters = outer;
        info->inner_iters = tot;
        info->true_residual = worst;
        info->n_systems = n;
    }
    if (q.rel_out)
        cuda_check(cudaMemcpyAsync(q.rel_out, rel, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream), "rel out");
    if (!(worst <= q.tol)) fail(PSMS_ENOCONV, "whole-lattice solve missed its tolerance");
}

}  // namespace psms

// ---------------------------------------------------------------------------
// Dirichlet block solve that allocates nothing.
//
// Some callers cannot allocate device memory while they run: code inside a
// memory pool that must not grow, real-time or embedded hosts that reserve
// all memory up front, and callers holding other allocations that a
// cudaMalloc/cudaFree (which synchronise the device) must not disturb.  For
// them the block solve below takes its scratch from one file-scope device
// array of fixed size instead of the context's growable scratch buffers.
// ---------------------------------------------------------------------------
#include <mutex>

namespace psms {

// Capacity of the static scratch: FP64 residual (12 V complex), the FP64
// inner vectors (66 V complex) and three per-block result arrays.
constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(32) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

static void *g_noalloc_addr[256];
static std::mutex g_noalloc_mutex;

// Device address of the static scratch on the current device.  Host code
// sees only a host-side stand-in for the array, so the address is looked up
// once per device with that device current and cached.
static void *noalloc_scratch_address() {
    int dev = 0;
    cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev < 0 || dev >= 256) fail(PSMS_EINVAL, "device index out of range for the no-allocation scratch");
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        cuda_check(cudaGetSymbolAddress(&p, g_noalloc_scratch), "cudaGetSymbolAddress(no-allocation scratch)");
        g_noalloc_addr[dev] = p;
    }
    return g_noalloc_addr[dev];
}

static size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

// sums / maxima of the per-block results into out[0] (iterations),
// out[1] (max residual) and out[2] (status, as double)
__global__ void noalloc_summary_kernel(const int *iters, const double *resid, const int *status, int n, double *out) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    double it = 0, worst = 0, st = 0;
    for (int i = 0; i < n; ++i) {
        it += iters[i];
        worst = resid[i] > worst ? resid[i] : worst;
        st = status[i] ? 1.0 : st;
    }
    out[0] = it;
    out[1] = worst;
    out[2] = st;
}

}  // namespace psms

extern "C" psms_status psms_block_solve_noalloc(psms_ctx *ctx, int field, int op, const void *b_dev, void *x_dev,
                                                double tol, int maxit, long long *iters_out, double *resid_out) {
    using namespace psms;
    if (!ctx) return PSMS_EINVAL;
    try {
        check_field(ctx, field);
        if (!b_dev || !x_dev || b_dev == x_dev) fail(PSMS_EINVAL, "b / x must be distinct non-null buffers");
        if (!(tol > 0) || maxit < 1) fail(PSMS_EINVAL, "tol must be > 0 and maxit >= 1");
        const Geom &g = ctx->g;
        const long long V = g.V;
        int lo = 0, nr = g.nblocks;
        if (op != PSMS_OP_BLOCKS) {
            if (op < 0 || op >= g.nblocks) fail(PSMS_EINVAL, "op must be PSMS_OP_BLOCKS or a block index");
            int B[4], rem = op;
            for (int m = 3; m >= 0; --m) {
                B[m] = rem % g.nb[m];
                rem /= g.nb[m];
            }
            lo = rank_of_lex(g, op, B);
            nr = 1;
        }
        const size_t r64_bytes = align256(sizeof(double2) * 12 * (size_t)V);
        const long long per_sys = 24 * V + 7 * 12 * (long long)g.Vh;
        const size_t inner_bytes = align256(sizeof(double2) * (size_t)per_sys);
        const size_t res_bytes = align256(sizeof(int) * nr) + align256(sizeof(double) * nr) +
                                 align256(sizeof(int) * nr) + align256(sizeof(double) * 3);
        const size_t need = r64_bytes + inner_bytes + res_bytes;
        if (need > NOALLOC_SCRATCH_BYTES)
            fail(PSMS_EINVAL, "lattice too large for psms_block_solve_noalloc: needs " + std::to_string(need) +
                                  " bytes of scratch, the static array holds " +
                                  std::to_string(NOALLOC_SCRATCH_BYTES) + " (about 26,000 sites)");
        unsigned char *base = (unsigned char *)noalloc_scratch_address();
        double2 *r64 = (double2 *)base;
        void *vin = base + r64_bytes;
        unsigned char *rp = base + r64_bytes + inner_bytes;
        int *iters = (int *)rp;
        rp += align256(sizeof(int) * nr);
        double *resid = (double *)rp;
        rp += align256(sizeof(double) * nr);
        int *status = (int *)rp;
        rp += align256(sizeof(int) * nr);
        double *summary = (double *)rp;
        // blocks outside op keep x = 0; the kernel zeroes and writes x inside them
        cuda_check(cudaMemsetAsync(x_dev, 0, sizeof(double2) * 12 * (size_t)V, ctx->stream), "no-alloc memset");
        BlockSolveArgs a;
        a.g = g;
        a.binfo = ctx->d_binfo;
        a.A = ctx->A;
        a.rank_lo = lo;
        a.n_ranks = nr;
        a.b = View<double2>{(double2 *)b_dev, V, 0, 12 * V};
        a.x = View<double2>{(double2 *)x_dev, V, 0, 12 * V};
        a.r64 = View<double2>{r64, V, 0, 12 * V};
        a.U64 = ctx->U64[field];
        a.U64_bs = 0;
        a.Uin = ctx->U64[field];
        a.Uin_bs = 0;
        a.vin = vin;
        a.vin_bs = per_sys;
        a.tol = tol;
        a.delta = std::max(0.1 * tol, 1e-15);
        a.maxit = maxit;
        a.max_outer = 4;
        a.sys_active = nullptr;
        a.block_active = nullptr;
        a.iters = iters;
        a.resid = resid;
        a.xnorm2 = nullptr;
        a.status = status;
        const int NT = 128;
        block_solve_kernel<Store<double>, Store<double>, NT><<<dim3(nr, 1), NT, 0, ctx->stream>>>(a);
        PSMS_LAUNCH_CHECK("block_solve_kernel (no allocation)");
        noalloc_summary_kernel<<<1, 1, 0, ctx->stream>>>(iters, resid, status, nr, summary);
        PSMS_LAUNCH_CHECK("noalloc_summary_kernel");
        double h[3] = {0, 0, 0};
        cuda_check(cudaMemcpyAsync(h, summary, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream), "no-alloc summary");
        cuda_check(cudaStreamSynchronize(ctx->stream), "no-alloc sync");
        if (iters_out) *iters_out = (long long)h[0];
        if (resid_out) *resid_out = h[1];
        if (h[2] != 0.0) fail(PSMS_ENOCONV, "a block solve missed its tolerance");
    } catch (const Error &e) {
        ctx->err = e.msg;
        return e.st;
    }
    return PSMS_OK;
}

// ---------------------------------------------------------------------------
// Batched block solves over several lattices in one persistent launch
// (a plan: autotuned schedule, CUDA-graph replay)
// ---------------------------------------------------------------------------
namespace psms {

struct MultiArgs {
    const BlockSolveArgs *probs;  // per lattice
    const int4 *items;            // (problem, block rl, system k, -)
    int n_items;
    int *counter;                 // next item (reset to 0 before every launch)
};

// Persistent CTAs take items from an atomic counter until the list is empty;
// no CTA waits for another.
template <class SV, class SL, int NT>
__global__ void __launch_bounds__(NT) block_solve_multi_kernel(const MultiArgs m) {
    __shared__ double sh[NT / 32 + 1];
    __shared__ int item;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) item = atomicAdd(m.counter, 1);
        __syncthreads();
        const int it = item;
        if (it >= m.n_items) return;
        const int4 w = m.items[it];
        block_solve_item<SV, SL, NT, 1>(m.probs[w.x], w.y, w.z, sh);
    }
}

__global__ void multi_summary_kernel(const BlockSolveArgs *probs, int n_probs, const int *n_per, double *out) {
    if (blockIdx.x || threadIdx.x) return;
    double it = 0, worst = 0, st = 0;
    for (int p = 0; p < n_probs; ++p)
        for (int i = 0; i < n_per[p]; ++i) {
            it += probs[p].iters[i];
            worst = probs[p].resid[i] > worst ? probs[p].resid[i] : worst;
            if (probs[p].status[i]) st = 1;
        }
    out[0] = it;
    out[1] = worst;
    out[2] = st;
}

}  // namespace psms

struct psms_block_plan {
    std::vector<psms_block_problem> probs;
    std::vector<psms::BlockSolveArgs> h_args;
    std::vector<int> n_per;
    std::vector<void *> allocs;
    psms::BlockSolveArgs *d_args = nullptr;
    int *d_nper = nullptr;
    int4 *d_items = nullptr;
    int *d_counter = nullptr;
    double *d_summary = nullptr;
    int n_items = 0;
    int inner = 0;
    int ctas = 0, order = 0;
    double tuned_ms = 0;
    cudaStream_t stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::string err;
};

namespace psms {

static void plan_alloc(psms_block_plan *pl, void **p, size_t bytes) {
    cuda_check(cudaMalloc(p, bytes), "plan alloc");
    pl->allocs.push_back(*p);
}

// work orders: 0 lattice-major (block fastest), 1 system-major across
// lattices, 2 round-robin over lattices
static std::vector<int4> make_items(const psms_block_plan *pl, int order) {
    std::vector<int4> it;
    const int np = (int)pl->probs.size();
    if (order == 0) {
        for (int p = 0; p < np; ++p)
            for (int k = 0; k < pl->probs[p].n_rhs; ++k)
                for (int r = 0; r < pl->h_args[p].n_ranks; ++r) it.push_back(make_int4(p, r, k, 0));
    } else if (order == 1) {
        int kmax = 0;
        for (auto &q : pl->probs) kmax = std::max(kmax, q.n_rhs);
        for (int k = 0; k < kmax; ++k)
            for (int p = 0; p < np; ++p)
                if (k < pl->probs[p].n_rhs)
                    for (int r = 0; r < pl->h_args[p].n_ranks; ++r) it.push_back(make_int4(p, r, k, 0));
    } else {
        std::vector<std::vector<int4>> per(np);
        for (int p = 0; p < np; ++p)
            for (int k = 0; k < pl->probs[p].n_rhs; ++k)
                for (int r = 0; r < pl->h_args[p].n_ranks; ++r) per[p].push_back(make_int4(p, r, k, 0));
        size_t mx = 0;
        for (auto &v : per) mx = std::max(mx, v.size());
        for (size_t i = 0; i < mx; ++i)
            for (int p = 0; p < np; ++p)
                if (i < per[p].size()) it.push_back(per[p][i]);
    }
    return it;
}

static void plan_launch(psms_block_plan *pl, cudaStream_t s, int ctas) {
    MultiArgs m{pl->d_args, pl->d_items, pl->n_items, pl->d_counter};
    cuda_check(cudaMemsetAsync(pl->d_counter, 0, sizeof(int), s), "plan counter");
    const int NT = 128;
    if (pl->inner == P64)
        block_solve_multi_kernel<Store<double>, Store<double>, NT><<<ctas, NT, 0, s>>>(m);
    else
        block_solve_multi_kernel<Store<float>, Store<float>, NT><<<ctas, NT, 0, s>>>(m);
    PSMS_LAUNCH_CHECK("block_solve_multi_kernel");
    multi_summary_kernel<<<1, 1, 0, s>>>(pl->d_args, (int)pl->probs.size(), pl->d_nper, pl->d_summary);
    PSMS_LAUNCH_CHECK("multi_summary_kernel");
}

static void plan_destroy(psms_block_plan *pl) {
    if (pl->exec) cudaGraphExecDestroy(pl->exec);
    if (pl->graph) cudaGraphDestroy(pl->graph);
    if (pl->stream) cudaStreamDestroy(pl->stream);
    for (void *p : pl->allocs) cudaFree(p);
    delete pl;
}

}  // namespace psms

extern "C" {

psms_status psms_block_plan_create(const psms_block_problem *probs, int n_probs, double tol, int maxit,
                                   int inner_prec, psms_block_plan **out) {
    using namespace psms;
    if (!probs || n_probs < 1 || !out) return PSMS_EINVAL;
    *out = nullptr;
    psms_block_plan *pl = new psms_block_plan();
    try {
        if (!(tol > 0) || maxit < 1) fail(PSMS_EINVAL, "tol > 0 and maxit >= 1");
        if (inner_prec != P64 && inner_prec != P32) fail(PSMS_EINVAL, "inner precision FP64 or FP32");
        pl->inner = inner_prec;
        pl->probs.assign(probs, probs + n_probs);
        cuda_check(cudaStreamCreateWithFlags(&pl->stream, cudaStreamNonBlocking), "plan stream");
        for (int p = 0; p < n_probs; ++p) {
            const psms_block_problem &q = probs[p];
            psms_ctx *c = q.ctx;
            if (!c || !q.b_dev || !q.x_dev || q.n_rhs < 1) fail(PSMS_EINVAL, "bad problem description");
            check_field(c, q.field);
            cuda_check(cudaStreamSynchronize(c->stream), "plan sync");
            const Geom &g = c->g;
            const long long V = g.V;
            BlockSolveArgs a;
            a.g = g;
            a.binfo = c->d_binfo;
            a.A = c->A;
            a.rank_lo = 0;
            a.n_ranks = g.nblocks;
            a.b = View<double2>{(double2 *)q.b_dev, V, 0, 12 * V};
            a.x = View<double2>{(double2 *)q.x_dev, V, 0, 12 * V};
            void *r64 = nullptr;
            plan_alloc(pl, &r64, sizeof(double2) * 12 * (size_t)V * q.n_rhs);
            a.r64 = View<double2>{(double2 *)r64, V, 0, 12 * V};
            a.U64 = c->U64[q.field];
            a.U64_bs = 0;
            const bool in64 = inner_prec == P64;
            a.Uin = in64 ? (const void *)c->U64[q.field] : (const void *)links32(c, q.field);
            cuda_check(cudaStreamSynchronize(c->stream), "plan sync");
            a.Uin_bs = 0;
            const long long per_sys = 24 * V + 7 * 12 * (long long)g.Vh;
            void *vin = nullptr;
            plan_alloc(pl, &vin, (in64 ? sizeof(double2) : sizeof(float2)) * (size_t)per_sys * q.n_rhs);
            a.vin = vin;
            a.vin_bs = per_sys;
            a.tol = tol;
            a.delta = in64 ? std::max(0.1 * tol, 1e-15) : 1e-6;
            a.maxit = maxit;
            a.max_outer = in64 ? 4 : 12;
            a.sys_active = nullptr;
            a.block_active = nullptr;
            const int n_out = g.nblocks * q.n_rhs;
            void *it = nullptr, *rs = nullptr, *st = nullptr;
            plan_alloc(pl, &it, sizeof(int) * n_out);
            plan_alloc(pl, &rs, sizeof(double) * n_out);
            plan_alloc(pl, &st, sizeof(int) * n_out);
            a.iters = (int *)it;
            a.resid = (double *)rs;
            a.status = (int *)st;
            a.xnorm2 = nullptr;
            pl->h_args.push_back(a);
            pl->n_per.push_back(n_out);
            pl->n_items += n_out;
        }
        plan_alloc(pl, (void **)&pl->d_args, sizeof(BlockSolveArgs) * n_probs);
        plan_alloc(pl, (void **)&pl->d_nper, sizeof(int) * n_probs);
        plan_alloc(pl, (void **)&pl->d_items, sizeof(int4) * pl->n_items);
        plan_alloc(pl, (void **)&pl->d_counter, sizeof(int));
        plan_alloc(pl, (void **)&pl->d_summary, sizeof(double) * 3);
        cuda_check(cudaMemcpy(pl->d_args, pl->h_args.data(), sizeof(BlockSolveArgs) * n_probs, cudaMemcpyHostToDevice),
                   "plan args");
        cuda_check(cudaMemcpy(pl->d_nper, pl->n_per.data(), sizeof(int) * n_probs, cudaMemcpyHostToDevice), "plan n");
        // autotune: persistent grid size x work order, each candidate timed once
        // (the results do not depend on the schedule)
        int dev = 0, nsm = 0;
        cuda_check(cudaGetDevice(&dev), "device");
        cuda_check(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev), "sm count");
        cudaEvent_t e0, e1;
        cuda_check(cudaEventCreate(&e0), "event");
        cuda_check(cudaEventCreate(&e1), "event");
        float best = 1e30f;
        for (int order = 0; order < 3; ++order) {
            std::vector<int4> items = make_items(pl, order);
            cuda_check(cudaMemcpy(pl->d_items, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice),
                       "plan items");
            for (int per_sm : {1, 2, 3, 4}) {
                const int ctas = std::min(pl->n_items, per_sm * nsm);
                cuda_check(cudaEventRecord(e0, pl->stream), "event");
                plan_launch(pl, pl->stream, ctas);
                cuda_check(cudaEventRecord(e1, pl->stream), "event");
                cuda_check(cudaEventSynchronize(e1), "event");
                float ms = 0;
                cuda_check(cudaEventElapsedTime(&ms, e0, e1), "event");
                if (ms < best) {
                    best = ms;
                    pl->ctas = ctas;
                    pl->order = order;
                }
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        pl->tuned_ms = best;
        std::vector<int4> items = make_items(pl, pl->order);
        cuda_check(cudaMemcpy(pl->d_items, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice),
                   "plan items");
        // capture the tuned launch sequence once; runs replay the graph
        cuda_check(cudaStreamBeginCapture(pl->stream, cudaStreamCaptureModeThreadLocal), "capture begin");
        plan_launch(pl, pl->stream, pl->ctas);
        cuda_check(cudaStreamEndCapture(pl->stream, &pl->graph), "capture end");
        cuda_check(cudaGraphInstantiate(&pl->exec, pl->graph, 0), "graph instantiate");
    } catch (const Error &e) {
        psms_status st = e.st;
        if (n_probs >= 1 && probs[0].ctx) probs[0].ctx->err = e.msg;
        plan_destroy(pl);
        return st;
    }
    *out = pl;
    return PSMS_OK;
}

psms_status psms_block_plan_run(psms_block_plan *pl, void *stream, psms_solve_info *info) {
    using namespace psms;
    if (!pl) return PSMS_EINVAL;
    try {
        cudaStream_t s = (cudaStream_t)stream;
        // FP32 link copies must follow changes of the gauge fields
        for (size_t p = 0; p < pl->probs.size(); ++p) {
            psms_ctx *c = pl->probs[p].ctx;
            if (pl->inner == P32 && !c->u32_ok[pl->probs[p].field]) {
                links32(c, pl->probs[p].field);
                cuda_check(cudaStreamSynchronize(c->stream), "links sync");
            }
        }
        cuda_check(cudaGraphLaunch(pl->exec, s), "graph launch");
        double h[3];
        cuda_check(cudaMemcpyAsync(h, pl->d_summary, sizeof(h), cudaMemcpyDeviceToHost, s), "plan summary");
        cuda_check(cudaStreamSynchronize(s), "plan sync");
        if (info) {
            info->outer_iters = 0;
            info->inner_iters = (long long)h[0];
            info->true_residual = h[1];
            info->n_systems = pl->n_items;
        }
        if (h[2] != 0.0) fail(PSMS_ENOCONV, "a block solve missed its tolerance");
    } catch (const Error &e) {
        pl->err = e.msg;
        return e.st;
    }
    return PSMS_OK;
}

psms_status psms_block_plan_schedule(const psms_block_plan *pl, int *ctas, int *order, double *tuned_ms) {
    if (!pl) return PSMS_EINVAL;
    if (ctas) *ctas = pl->ctas;
    if (order) *order = pl->order;
    if (tuned_ms) *tuned_ms = pl->tuned_ms;
    return PSMS_OK;
}

psms_status psms_block_plan_destroy(psms_block_plan *pl) {
    if (!pl) return PSMS_EINVAL;
    if (pl->stream) cudaStreamSynchronize(pl->stream);
    psms::plan_destroy(pl);
    return PSMS_OK;
}

}  // extern "C"
