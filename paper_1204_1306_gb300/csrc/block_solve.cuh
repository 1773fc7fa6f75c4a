// Persistent Dirichlet-block solver (Sec. 3): CTA / cluster reductions, the
// block hop in its inlined, out-of-line and branch-free forms, the whole
// solve of one (block, system) item (even-odd CGNR or BiCGStab inside an
// FP64 defect-correction loop) and the launchers of the autotuned variants.
// The variants are instantiated explicitly in block_variants_*.cu so that
// they compile in parallel; solver.cu only declares them.
#pragma once

#include "kernels.hpp"
#include "solver.hpp"

#include <cooperative_groups.h>
#include <type_traits>

namespace psms {

// ---------------------------------------------------------------------------
// CTA-level helpers for the block solver
// ---------------------------------------------------------------------------
template <int NT>
__device__ __forceinline__ double cta_sum(double v, double *sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0;
        for (int i = 0; i < NT / 32; ++i) t += sh[i];
        sh[NT / 32] = t;
    }
    __syncthreads();
    return sh[NT / 32];
}

// Sum over the CTAs of a thread-block cluster (CL CTAs share one Dirichlet
// block): each CTA reduces its part, the partials are read from every CTA's
// shared memory (distributed shared memory) in rank order, so every CTA gets
// the same deterministic total.
template <int NT, int CL>
__device__ __forceinline__ double cl_sum(double v, double *sh) {
    const double t = cta_sum<NT>(v, sh);
    if constexpr (CL == 1) {
        return t;
    } else {
        namespace cg = cooperative_groups;
        cg::cluster_group cl = cg::this_cluster();
        cl.sync();
        double tot = 0;
        for (int q = 0; q < CL; ++q) tot += *cl.map_shared_rank(&sh[NT / 32], q);
        cl.sync();
        return tot;
    }
}

// barrier between dependent phases: the CTA, or the whole cluster (release /
// acquire at cluster scope makes the global-memory writes of one CTA visible
// to the others)
template <int CL>
__device__ __forceinline__ void bar() {
    if constexpr (CL == 1) {
        __syncthreads();
    } else {
        cooperative_groups::this_cluster().sync();
    }
}

// out_p = a*y_p + b*H^intra_p(in) on the block of rank r; returns this
// thread's contribution to |out|^2.  Vectors are views (structure of arrays).
// BF = 1: branch-free form.  Every direction loads the neighbour inside the
// block under the block's own periodic wrap (always a valid, cached site) and
// a direction that leaves the block contributes an exact zero, so the eight
// hops run as one straight sequence whose loads the compiler can issue early;
// the result equals the branching form bit for bit.
// Link of direction mu at the site with internal index s of parity q, from
// global memory (LSM = 0) or from the block's copy in shared memory
// (LSM = 1: layout of the global FP32 field with V -> 2 Vbh and the site at
// q Vbh + its index in the block's parity half; plain loads).
template <class SL, int LSM>
__device__ __forceinline__ SU3<typename SL::R> blk_link(const Geom &g, const typename SL::elem *U, int r, int q,
                                                        int mu, long long s) {
    if constexpr (LSM) {
        const long long l = (long long)q * g.Vbh + (s - (long long)q * g.Vh - (long long)r * g.Vbh);
        const long long Vl = 2LL * g.Vbh;
        SU3<typename SL::R> u;
        const float2 *base = reinterpret_cast<const float2 *>(U) + (long long)mu * 9 * Vl;
        const float4 *q4 = reinterpret_cast<const float4 *>(base);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float4 w = q4[k * Vl + l];
            u.e[(2 * k) / 3][(2 * k) % 3] = {w.x, w.y};
            u.e[(2 * k + 1) / 3][(2 * k + 1) % 3] = {w.z, w.w};
        }
        const float2 w = base[8 * Vl + l];
        u.e[2][2] = {w.x, w.y};
        return u;
    } else {
        return load_link<SL>(U, g.V, mu, s);
    }
}

// Copy the FP32 links of every site of block r into shared memory (the
// layout blk_link<SL, 1> reads).
template <int NT>
__device__ __forceinline__ void stage_block_links(const Geom &g, const float2 *U, int r, float2 *sm) {
    const long long Vl = 2LL * g.Vbh;
    for (long long t = threadIdx.x; t < 4 * Vl; t += NT) {
        const int mu = (int)(t / Vl);
        const long long l = t - (long long)mu * Vl;
        const int q = l >= g.Vbh ? 1 : 0;
        const long long s = (long long)q * g.Vh + (long long)r * g.Vbh + (l - (long long)q * g.Vbh);
        const float2 *gb = U + (long long)mu * 9 * g.V;
        float2 *sb = sm + (long long)mu * 9 * Vl;
        const float4 *g4 = reinterpret_cast<const float4 *>(gb);
        float4 *s4 = reinterpret_cast<float4 *>(sb);
#pragma unroll
        for (int k = 0; k < 4; ++k) s4[k * Vl + l] = __ldg(g4 + k * g.V + s);
        sb[8 * Vl + l] = __ldg(gb + 8 * g.V + s);
    }
}

template <class S, class SL, class SY, int BF = 0, int LSM = 0>
__device__ __forceinline__ double block_hop(const Geom &g, const BlockInfo &bi, int r, int p, int dag,
                                            const typename S::elem *in, long long in_cs, long long in_off,
                                            typename S::elem *out, long long out_cs, long long out_off,
                                            const typename SY::elem *y, long long y_cs, long long y_off, double a,
                                            double b, const typename SL::elem *U, int jlo, int jhi) {
    using R = typename SL::R;
    double nrm = 0;
    const R sg = dag ? R(-1) : R(1);
    for (int j = jlo + threadIdx.x; j < jhi; j += blockDim.x) {
        int yy[4];
        const int ll = local_lex(g, p, j, yy);
        const long long s = (long long)p * g.Vh + (long long)r * g.Vbh + j;
        Spinor<R> acc;
        zero(acc);
        if constexpr (BF) {
            long long snb[8];
            R keep[8];
#pragma unroll
            for (int d = 0; d < 8; ++d) {
                const int mu = d >> 1, sgn = (d & 1) ? -1 : 1;
                int yn = yy[mu] + sgn;
                keep[d] = ((unsigned)yn < (unsigned)g.l[mu]) ? R(1) : R(0);
                yn &= g.l[mu] - 1;  // wrap inside the block (extents are powers of two)
                const int lln = ll + (yn - yy[mu]) * g.lstride[mu];
                snb[d] = (long long)(1 - p) * g.Vh + (long long)r * g.Vbh + (lln >> 1);
            }
#pragma unroll
            for (int d = 0; d < 8; ++d) {
                const int mu = d >> 1;
                const bool fwd = (d & 1) == 0;
                Spinor<R> v = load_spinor<S>(in, in_cs, snb[d] - in_off);
                const R tt = fwd ? -sg : sg;
                Half<R> h = project(mu, tt, v);
#pragma unroll
                for (int q = 0; q < 2; ++q)
#pragma unroll
                    for (int c = 0; c < 3; ++c) h.c[q][c] = keep[d] * h.c[q][c];
                SU3<R> u = blk_link<SL, LSM>(g, U, r, fwd ? p : 1 - p, mu, fwd ? s : snb[d]);
                reconstruct_add(mu, tt, fwd ? su3_mul(u, h) : su3_dag_mul(u, h), acc);
            }
        } else {
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) {
            long long sn;
            int bs;
            if (neighbour(g, bi, r, p, yy, ll, mu, +1, HOP_INTRA, sn, bs)) {
                Spinor<R> v = load_spinor<S>(in, in_cs, sn - in_off);
                const R tf = -sg;
                Half<R> h = project(mu, tf, v);
                SU3<R> u = blk_link<SL, LSM>(g, U, r, p, mu, s);
                reconstruct_add(mu, tf, su3_mul(u, h), acc);
            }
            if (neighbour(g, bi, r, p, yy, ll, mu, -1, HOP_INTRA, sn, bs)) {
                Spinor<R> v = load_spinor<S>(in, in_cs, sn - in_off);
                const R tb = sg;
                Half<R> h = project(mu, tb, v);
                SU3<R> u = blk_link<SL, LSM>(g, U, r, 1 - p, mu, sn);
                reconstruct_add(mu, tb, su3_dag_mul(u, h), acc);
            }
        }
        }
        Spinor<R> o;
        const R cb = (R)b, ca = (R)a;
        if (y) {
            Spinor<typename SY::R> v = load_spinor<SY>(y, y_cs, s - y_off);
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    o.c[q][c] = cb * acc.c[q][c] + ca * mk<R>((R)v.c[q][c].re, (R)v.c[q][c].im);
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int c = 0; c < 3; ++c) o.c[q][c] = cb * acc.c[q][c];
        }
        store_spinor<S>(out, out_cs, s - out_off, o);
        // a site's 12 components summed in the inner precision, sites in FP64
        R t = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int c = 0; c < 3; ++c) t += norm2(o.c[q][c]);
        nrm += (double)t;
    }
    return nrm;
}

// The same hop as an out-of-line function: one copy of its code serves every
// call site of the block CG (instruction-cache footprint), at the price of a
// call and of no specialisation on constant arguments.
template <class S, class SL, class SY, int BF, int LSM>
__device__ __noinline__ double block_hop_ool(const Geom &g, const BlockInfo &bi, int r, int p, int dag,
                                             const typename S::elem *in, long long in_cs, long long in_off,
                                             typename S::elem *out, long long out_cs, long long out_off,
                                             const typename SY::elem *y, long long y_cs, long long y_off, double a,
                                             double b, const typename SL::elem *U, int jlo, int jhi) {
    return block_hop<S, SL, SY, BF, LSM>(g, bi, r, p, dag, in, in_cs, in_off, out, out_cs, out_off, y, y_cs, y_off,
                                         a, b, U, jlo, jhi);
}

// HV: bit 0 = out-of-line hop, bit 1 = branch-free hop, bit 3 = links of
// the inner-precision hops in shared memory (U then points there)
template <int HV, class S, class SL, class SY>
__device__ __forceinline__ double hop_call(const Geom &g, const BlockInfo &bi, int r, int p, int dag,
                                           const typename S::elem *in, long long in_cs, long long in_off,
                                           typename S::elem *out, long long out_cs, long long out_off,
                                           const typename SY::elem *y, long long y_cs, long long y_off, double a,
                                           double b, const typename SL::elem *U, int jlo, int jhi) {
    constexpr int BF = (HV >> 1) & 1;
    // only the inner-precision links live in shared memory; the FP64
    // residual hops (S = SL = Store<double>) read global memory
    constexpr int LSM = ((HV >> 3) & 1) && std::is_same<typename SL::R, float>::value;
    if constexpr (HV & 1)
        return block_hop_ool<S, SL, SY, BF, LSM>(g, bi, r, p, dag, in, in_cs, in_off, out, out_cs, out_off, y, y_cs,
                                                 y_off, a, b, U, jlo, jhi);
    else
        return block_hop<S, SL, SY, BF, LSM>(g, bi, r, p, dag, in, in_cs, in_off, out, out_cs, out_off, y, y_cs,
                                             y_off, a, b, U, jlo, jhi);
}

template <class E>
struct BlockVecs {
    // inner-precision vectors of one system (views with the system offset applied)
    E *rhs, *e;             // full layout (cs = V, off = 0)
    E *bhat, *rho, *res, *pp, *q, *sv;  // odd halves (cs = Vh, off = Vh)
    E *t;                   // even half (cs = Vh, off = 0)
};

struct BlockSolveArgs {
    Geom g;
    const BlockInfo *binfo;
    double A;
    int rank_lo, n_ranks;
    View<double2> b, x;              // FP64 rhs / solution (full layout)
    View<double2> r64;               // FP64 residual scratch (full layout)
    const double2 *U64;
    long long U64_bs;
    const void *Uin;
    long long Uin_bs;
    void *vin;                       // inner scratch base
    long long vin_bs;                // per-system stride of the inner scratch (elements)
    double tol, delta;
    int maxit, max_outer;
    const int *sys_active;           // per system (nullable)
    const int *block_active;         // per lexicographic block (nullable)
    int *iters;                      // [k * n_ranks + r]
    double *resid;                   // [k * n_ranks + r]
    double *xnorm2;                  // [k * n_ranks + r] |x_block|^2 (nullable)
    int *status;                     // [k * n_ranks + r]
};

// The whole solve of one (block rl, system k) item by CL CTAs (a thread-block
// cluster, CL = 1: one CTA) of NT threads; CTA rank q of the cluster works on
// the sites j in [q Vbh/CL, (q+1) Vbh/CL) of each parity.
template <class SV, class SL, int NT, int CL, int HV = 0>
__device__ void block_solve_item(const BlockSolveArgs &a, const int rl, const int k, double *sh) {
    using E = typename SV::elem;
    using R = typename SL::R;
    using S64 = Store<double>;
    const Geom &g = a.g;
    const int r = a.rank_lo + rl;
    int crank = 0;
    if constexpr (CL > 1) crank = (int)cooperative_groups::this_cluster().block_rank();
    const int jlo = crank * (g.Vbh / CL), jhi = jlo + g.Vbh / CL;
    const bool lead = (threadIdx.x == 0) && (crank == 0);
    const long long out_i = (long long)k * a.n_ranks + rl;
    const BlockInfo &bi = a.binfo[r];
    if ((a.sys_active && !a.sys_active[k]) || (a.block_active && !a.block_active[bi.lex])) {
        if (lead) {
            a.iters[out_i] = 0;
            a.resid[out_i] = 0;
            a.status[out_i] = 0;
            if (a.xnorm2) a.xnorm2[out_i] = 0;
        }
        return;
    }
    const long long V = g.V, Vh = g.Vh;
    const double2 *b = a.b.p + k * a.b.bs;
    double2 *x = a.x.p + k * a.x.bs;
    double2 *r64 = a.r64.p + k * a.r64.bs;
    const double2 *U64 = a.U64 + k * a.U64_bs;
    const typename SL::elem *Uin = (const typename SL::elem *)a.Uin + k * a.Uin_bs;
    if constexpr (((HV >> 3) & 1) && std::is_same<typename SL::R, float>::value) {
        // the block's inner-precision links, read by every hop of the
        // Krylov iterations, staged once into shared memory
        extern __shared__ float4 psms_blk_smem[];
        float2 *sm = reinterpret_cast<float2 *>(psms_blk_smem);
        stage_block_links<NT>(g, reinterpret_cast<const float2 *>(Uin), r, sm);
        __syncthreads();
        Uin = reinterpret_cast<const typename SL::elem *>(sm);
    }
    E *base = (E *)a.vin + k * a.vin_bs;
    // inner scratch layout per system: rhs (V), e (V), 6 odd halves, 1 even half
    BlockVecs<E> v;
    v.rhs = base;
    v.e = base + 12 * V;
    v.bhat = base + 24 * V;
    v.rho = v.bhat + 12 * Vh;
    v.res = v.rho + 12 * Vh;
    v.pp = v.res + 12 * Vh;
    v.q = v.pp + 12 * Vh;
    v.sv = v.q + 12 * Vh;
    v.t = v.sv + 12 * Vh;
    const long long blo[2] = {(long long)r * g.Vbh, Vh + (long long)r * g.Vbh};  // block start per parity
    const double A = a.A;
    const double c4 = -1.0 / (4.0 * A);

    // x = 0, |b|^2
    double bn = 0;
    for (int p = 0; p < 2; ++p)
        for (int j = jlo + threadIdx.x; j < jhi; j += NT) {
            const long long s = blo[p] + j;
            for (int q = 0; q < 12; ++q) {
                x[q * a.x.cs + s - a.x.off] = make_double2(0, 0);
                bn += (double)norm2(S64::ld(b, q, a.b.cs, s - a.b.off));
            }
        }
    bn = cl_sum<NT, CL>(bn, sh);
    int total_it = 0, st = 0;
    double rel = 0;
    if (bn == 0.0) {
        if (lead) {
            a.iters[out_i] = 0;
            a.resid[out_i] = 0;
            a.status[out_i] = 0;
            if (a.xnorm2) a.xnorm2[out_i] = 0;
        }
        return;
    }
    for (int outer = 0;; ++outer) {
        // FP64 true residual r64 = b - D_b x  (both parities)
        // r64_p = b_p + H_p(x_{1-p})/2, then subtract A x_p; on the first
        // step x = 0, so r64 = b and |r64|^2 = |b|^2 without the FP64 hop
        // (GB300's FP64 rate makes that hop a large part of a block solve)
        double rn = 0;
        bar<CL>();
        if (outer == 0) {
            for (int p = 0; p < 2; ++p)
                for (int j = jlo + threadIdx.x; j < jhi; j += NT) {
                    const long long s = blo[p] + j;
                    for (int q = 0; q < 12; ++q)
                        S64::st(r64, q, a.r64.cs, s - a.r64.off, S64::ld(b, q, a.b.cs, s - a.b.off));
                }
            rn = bn;
        } else {
        for (int p = 0; p < 2; ++p) {
            hop_call<HV, S64, S64, S64>(g, bi, r, p, 0, x, a.x.cs, a.x.off, r64, a.r64.cs, a.r64.off, b, a.b.cs,
                                     a.b.off, 1.0, 0.5, U64, jlo, jhi);
        }
        bar<CL>();
        for (int p = 0; p < 2; ++p)
            for (int j = jlo + threadIdx.x; j < jhi; j += NT) {
                const long long s = blo[p] + j;
                for (int q = 0; q < 12; ++q) {
                    cpx<double> rv = S64::ld(r64, q, a.r64.cs, s - a.r64.off);
                    cpx<double> xv = S64::ld(x, q, a.x.cs, s - a.x.off);
                    rv = rv - A * xv;
                    S64::st(r64, q, a.r64.cs, s - a.r64.off, rv);
                    rn += norm2(rv);
                }
            }
        rn = cl_sum<NT, CL>(rn, sh);
        }
        rel = sqrt(rn / bn);
        if (rel <= a.tol) break;
        if (outer >= a.max_outer || total_it >= a.maxit) {
            st = 1;
            break;
        }
        // inner rhs = r64 / |r64| in inner precision
        const double scale = 1.0 / sqrt(rn);
        for (int p = 0; p < 2; ++p)
            for (int j = jlo + threadIdx.x; j < jhi; j += NT) {
                const long long s = blo[p] + j;
                for (int q = 0; q < 12; ++q) {
                    cpx<double> rv = S64::ld(r64, q, a.r64.cs, s - a.r64.off);
                    SV::st(v.rhs, q, V, s, mk<R>((R)(rv.re * scale), (R)(rv.im * scale)));
                }
            }
        bar<CL>();
        // bhat_o = rhs_o + H_o(rhs_e)/(2A)
        double bb = hop_call<HV, SV, SL, SV>(g, bi, r, 1, 0, v.rhs, V, 0, v.bhat, Vh, Vh, v.rhs, V, 0, 1.0,
                                          0.5 / A, Uin, jlo, jhi);
        bb = cl_sum<NT, CL>(bb, sh);
        int it = 0;
        if constexpr ((HV >> 2) & 1) {
            // BiCGStab on Dhat (hop form bit 2): rh = bhat, r = rho, p = pp,
            // v = q, s = sv, t = res; complex scalars from cluster-wide sums
            // that every thread receives alike
            for (int j = jlo + threadIdx.x; j < jhi; j += NT) {
                const long long so = blo[1] + j;
                for (int q = 0; q < 12; ++q) {
                    SV::st(v.e, q, V, so, mk<R>(0, 0));
                    const cpx<R> bv = SV::ld(v.bhat, q, Vh, so - Vh);
                    SV::st(v.rho, q, Vh, so - Vh, bv);
                    SV::st(v.pp, q, Vh, so - Vh, bv);
                }
            }
            bar<CL>();
            double rho_re = bb, rho_im = 0, al_re = 1, al_im = 0, om_re = 1, om_im = 0;
            const double target = a.delta * a.delta * bb;
            while (total_it + it < a.maxit) {
                // v = Dhat p
                hop_call<HV, SV, SL, SV>(g, bi, r, 0, 0, v.pp, Vh, Vh, v.t, Vh, 0, (const E *)nullptr, 0, 0, 0.0,
                                         1.0, Uin, jlo, jhi);
                bar<CL>();
                hop_call<HV, SV, SL, SV>(g, bi, r, 1, 0, v.t, Vh, 0, v.q, Vh, Vh, v.pp, Vh, Vh, A, c4, Uin, jlo,
                                         jhi);
                // <rh, v>
                double d_re = 0, d_im = 0;
                for (int j = jlo + threadIdx.x; j < jhi; j += NT) {
                    const long long sh_ = blo[1] + j - Vh;
                    for (int q = 0; q < 12; ++q) {
                        const cpx<R> x1 = SV::ld(v.bhat, q, Vh, sh_), y1 = SV::ld(v.q, q, Vh, sh_);
                        d_re += (double)x1.re * y1.re + (double)x1.im * y1.im;
                        d_im += (double)x1.re * y1.im - (double)x1.im * y1.re;
                    }
                }
                d_re = cl_sum<NT, CL>(d_re, sh);
                d_im = cl_sum<NT, CL>(d_im, sh);
                const double dd = d_re * d_re + d_im * d_im;
                if (!(dd > 0.0)) break;  // breakdown: the defect correction restarts
                al_re = (rho_re * d_re + rho_im * d_im) / dd;
                al_im = (rho_im * d_re - rho_re * d_im) / dd;
                const cpx<R> alc = mk<R>((R)al_re, (R)al_im);
                // s = r - alpha v
                for (int j = jlo + threadIdx.x; j < jhi; j += NT) {
                    const long long sh_ = blo[1] + j - Vh;
                    for (int q = 0; q < 12; ++q)
                        SV::st(v.sv, q, Vh, sh_, SV::ld(v.rho, q, Vh, sh_) - cmul(alc, SV::ld(v.q, q, Vh, sh_)));
                }
                bar<CL>();
                // t = Dhat s
                hop_call<HV, SV, SL, SV>(g, bi, r, 0, 0, v.sv, Vh, Vh, v.t, Vh, 0, (const E *)nullptr, 0, 0, 0.0,
                                         1.0, Uin, jlo, jhi);
                bar<CL>();
                hop_call<HV, SV, SL, SV>(g, bi, r, 1, 0, v.t, Vh, 0, v.res, Vh, Vh, v.sv, Vh, Vh, A, c4, Uin, jlo,
                                         jhi);
                // omega = <t, s> / <t, t>
                double ts_re = 0, ts_im = 0, tt = 0;
                for (int j = jlo + threadIdx.x; j < jhi; j += NT) {
                    const long long sh_ = blo[1] + j - Vh;
                    for (int q = 0; q < 12; ++q) {
                        const cpx<R> tv = SV::ld(v.res, q, Vh, sh_), sv = SV::ld(v.sv, q, Vh, sh_);
                        ts_re += (double)tv.re * sv.re + (double)tv.im * sv.im;
                        ts_im += (double)tv.re * sv.im - (double)tv.im * sv.re;
                        tt += (double)tv.re * tv.re + (double)tv.im * tv.im;
                    }
                }
                ts_re = cl_sum<NT, CL>(ts_re, sh);
                ts_im = cl_sum<NT, CL>(ts_im, sh);
                tt = cl_sum<NT, CL>(tt, sh);
                om_re = tt > 0.0 ? ts_re / tt : 0.0;
                om_im = tt > 0.0 ? ts_im / tt : 0.0;
                const cpx<R> omc = mk<R>((R)om_re, (R)om_im);
                // e += alpha p + omega s ; r = s - omega t ; <rh, r>, |r|^2
                double n_re = 0, n_im = 0, rr2 = 0;
                for (int j = jlo + threadIdx.x; j < jhi; j += NT) {
                    const long long so = blo[1] + j;
                    const long long sh_ = so - Vh;
                    for (int q = 0; q < 12; ++q) {
                        const cpx<R> sv = SV::ld(v.sv, q, Vh, sh_);
                        SV::st(v.e, q, V, so,
                               SV::ld(v.e, q, V, so) + cmul(alc, SV::ld(v.pp, q, Vh, sh_)) + cmul(omc, sv));
                        const cpx<R> rv = sv - cmul(omc, SV::ld(v.res, q, Vh, sh_));
                        SV::st(v.rho, q, Vh, sh_, rv);
                        const cpx<R> hv = SV::ld(v.bhat, q, Vh, sh_);
                        n_re += (double)hv.re * rv.re + (double)hv.im * rv.im;
                        n_im += (double)hv.re * rv.im - (double)hv.im * rv.re;
                        rr2 += (double)rv.re * rv.re + (double)rv.im * rv.im;
                    }
                }
                n_re = cl_sum<NT, CL>(n_re, sh);
                n_im = cl_sum<NT, CL>(n_im, sh);
                rr2 = cl_sum<NT, CL>(rr2, sh);
                ++it;
                if (rr2 <= target) break;
                const double oo = om_re * om_re + om_im * om_im, rr_ = rho_re * rho_re + rho_im * rho_im;
                if (!(oo > 0.0) || !(n_re * n_re + n_im * n_im > 0.0) || !(rr_ > 0.0)) break;
                // beta = (rho_new / rho)(alpha / omega)
                const double q1_re = (n_re * rho_re + n_im * rho_im) / rr_, q1_im = (n_im * rho_re - n_re * rho_im) / rr_;
                const double q2_re = (al_re * om_re + al_im * om_im) / oo, q2_im = (al_im * om_re - al_re * om_im) / oo;
                const cpx<R> bec = mk<R>((R)(q1_re * q2_re - q1_im * q2_im), (R)(q1_re * q2_im + q1_im * q2_re));
                rho_re = n_re;
                rho_im = n_im;
                // p = r + beta (p - omega v)
                for (int j = jlo + threadIdx.x; j < jhi; j += NT) {
                    const long long sh_ = blo[1] + j - Vh;
                    for (int q = 0; q < 12; ++q) {
                        const cpx<R> pv = SV::ld(v.pp, q, Vh, sh_) - cmul(omc, SV::ld(v.q, q, Vh, sh_));
                        SV::st(v.pp, q, Vh, sh_, SV::ld(v.rho, q, Vh, sh_) + cmul(bec, pv));
                    }
                }
                bar<CL>();
            }
        } else {
        // e_o = 0, rho = bhat, res = Dhat^dag rho, p = res
        for (int j = jlo + threadIdx.x; j < jhi; j += NT) {
            const long long s = blo[1] + j;
            for (int q = 0; q < 12; ++q) {
                SV::st(v.e, q, V, s, mk<R>(0, 0));
                SV::st(v.rho, q, Vh, s - Vh, SV::ld(v.bhat, q, Vh, s - Vh));
            }
        }
        bar<CL>();
        hop_call<HV, SV, SL, SV>(g, bi, r, 0, 1, v.rho, Vh, Vh, v.t, Vh, 0, (const E *)nullptr, 0, 0, 0.0, 1.0, Uin, jlo, jhi);
        bar<CL>();
        double rr = hop_call<HV, SV, SL, SV>(g, bi, r, 1, 1, v.t, Vh, 0, v.res, Vh, Vh, v.rho, Vh, Vh, A, c4, Uin, jlo, jhi);
        rr = cl_sum<NT, CL>(rr, sh);
        for (int j = jlo + threadIdx.x; j < jhi; j += NT) {
            const long long s = blo[1] + j - Vh;
            for (int q = 0; q < 12; ++q) SV::st(v.pp, q, Vh, s, SV::ld(v.res, q, Vh, s));
        }
        bar<CL>();
        const double target = a.delta * a.delta * bb;
        while (total_it + it < a.maxit) {
            // q = Dhat p
            hop_call<HV, SV, SL, SV>(g, bi, r, 0, 0, v.pp, Vh, Vh, v.t, Vh, 0, (const E *)nullptr, 0, 0, 0.0, 1.0, Uin, jlo, jhi);
            bar<CL>();
            double qq = hop_call<HV, SV, SL, SV>(g, bi, r, 1, 0, v.t, Vh, 0, v.q, Vh, Vh, v.pp, Vh, Vh, A, c4, Uin, jlo, jhi);
            qq = cl_sum<NT, CL>(qq, sh);
            const R alpha = (R)(rr / qq);
            double rhorho = 0;
            for (int j = jlo + threadIdx.x; j < jhi; j += NT) {
                const long long so = blo[1] + j;
                const long long sh_ = so - Vh;
                R tsum = 0;
                for (int q = 0; q < 12; ++q) {
                    cpx<R> e = SV::ld(v.e, q, V, so);
                    cpx<R> pv = SV::ld(v.pp, q, Vh, sh_);
                    cpx<R> qv = SV::ld(v.q, q, Vh, sh_);
                    cpx<R> ro = SV::ld(v.rho, q, Vh, sh_);
                    e = e + alpha * pv;
                    ro = ro - alpha * qv;
                    SV::st(v.e, q, V, so, e);
                    SV::st(v.rho, q, Vh, sh_, ro);
                    tsum += norm2(ro);
                }
                rhorho += (double)tsum;
            }
            rhorho = cl_sum<NT, CL>(rhorho, sh);
            ++it;
            if (rhorho <= target) break;
            // sv = Dhat^dag q
            hop_call<HV, SV, SL, SV>(g, bi, r, 0, 1, v.q, Vh, Vh, v.t, Vh, 0, (const E *)nullptr, 0, 0, 0.0, 1.0, Uin, jlo, jhi);
            bar<CL>();
            hop_call<HV, SV, SL, SV>(g, bi, r, 1, 1, v.t, Vh, 0, v.sv, Vh, Vh, v.q, Vh, Vh, A, c4, Uin, jlo, jhi);
            bar<CL>();
            double rr_new = 0;
            for (int j = jlo + threadIdx.x; j < jhi; j += NT) {
                const long long sh_ = blo[1] + j - Vh;
                R tsum = 0;
                for (int q = 0; q < 12; ++q) {
                    cpx<R> rv = SV::ld(v.res, q, Vh, sh_);
                    rv = rv - alpha * SV::ld(v.sv, q, Vh, sh_);
                    SV::st(v.res, q, Vh, sh_, rv);
                    tsum += norm2(rv);
                }
                rr_new += (double)tsum;
            }
            rr_new = cl_sum<NT, CL>(rr_new, sh);
            const R beta = (R)(rr_new / rr);
            rr = rr_new;
            for (int j = jlo + threadIdx.x; j < jhi; j += NT) {
                const long long sh_ = blo[1] + j - Vh;
                for (int q = 0; q < 12; ++q) {
                    cpx<R> pv = SV::ld(v.pp, q, Vh, sh_);
                    SV::st(v.pp, q, Vh, sh_, SV::ld(v.res, q, Vh, sh_) + beta * pv);
                }
            }
            bar<CL>();
        }
        }
        total_it += it;
        bar<CL>();
        // e_e = (rhs_e + H_e(e_o)/2) / A
        hop_call<HV, SV, SL, SV>(g, bi, r, 0, 0, v.e, V, 0, v.e, V, 0, v.rhs, V, 0, 1.0 / A, 0.5 / A, Uin, jlo, jhi);
        bar<CL>();
        // x += e / scale (FP64)
        const double unscale = sqrt(rn);
        for (int p = 0; p < 2; ++p)
            for (int j = jlo + threadIdx.x; j < jhi; j += NT) {
                const long long s = blo[p] + j;
                for (int q = 0; q < 12; ++q) {
                    cpx<R> ev = SV::ld(v.e, q, V, s);
                    cpx<double> xv = S64::ld(x, q, a.x.cs, s - a.x.off);
                    xv = xv + unscale * mk<double>((double)ev.re, (double)ev.im);
                    S64::st(x, q, a.x.cs, s - a.x.off, xv);
                }
            }
        bar<CL>();
    }
    double xn = 0;
    if (a.xnorm2) {
        for (int p = 0; p < 2; ++p)
            for (int j = jlo + threadIdx.x; j < jhi; j += NT) {
                const long long s = blo[p] + j;
                for (int q = 0; q < 12; ++q) xn += norm2(S64::ld(x, q, a.x.cs, s - a.x.off));
            }
        xn = cl_sum<NT, CL>(xn, sh);
    }
    if (lead) {
        a.iters[out_i] = total_it;
        a.resid[out_i] = rel;
        a.status[out_i] = st;
        if (a.xnorm2) a.xnorm2[out_i] = xn;
    }
}

// one CTA per (block, system): grid (n_ranks, n_sys)
template <class SV, class SL, int NT>
__global__ void __launch_bounds__(NT) block_solve_kernel(const BlockSolveArgs a) {
    __shared__ double sh[NT / 32 + 1];
    block_solve_item<SV, SL, NT, 1>(a, blockIdx.x, blockIdx.y, sh);
}

// CL CTAs (one cluster) per (block, system): grid (n_ranks * CL, n_sys),
// cluster dimension (CL, 1, 1); MINB resident CTAs per SM caps registers
template <class SV, class SL, int NT, int CL, int MINB, int HV>
__global__ void __launch_bounds__(NT, MINB) block_solve_cluster_kernel(const BlockSolveArgs a) {
    __shared__ double sh[NT / 32 + 1];
    block_solve_item<SV, SL, NT, CL, HV>(a, blockIdx.x / CL, blockIdx.y, sh);
}

// dynamic shared memory of a variant: the block's FP32 links when HV bit 3
// is set (4 directions x 9 complex x 2 Vbh sites)
inline size_t block_links_smem(const Geom &g) { return (size_t)4 * 9 * 2 * g.Vbh * sizeof(float2); }

template <class SV, class SL, int CL, int MINB, int HV = 0>
void launch_block_cl(psms_ctx *c, const BlockSolveArgs &a, int n_ranks, int n_sys) {
    constexpr int NT = 128;
    if constexpr (CL == 1) {
        size_t smem = 0;
        if constexpr ((HV >> 3) & 1) {
            smem = block_links_smem(a.g);
            cuda_check(cudaFuncSetAttribute(block_solve_cluster_kernel<SV, SL, NT, 1, MINB, HV>,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                       "block solver shared memory");
        }
        block_solve_cluster_kernel<SV, SL, NT, 1, MINB, HV><<<dim3(n_ranks, n_sys), NT, smem, c->stream>>>(a);
        PSMS_LAUNCH_CHECK("block_solve_cluster_kernel");
    } else {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(n_ranks * CL, n_sys, 1);
        cfg.blockDim = dim3(NT, 1, 1);
        cfg.dynamicSmemBytes = 0;
        cfg.stream = c->stream;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = CL;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        cuda_check(cudaLaunchKernelEx(&cfg, block_solve_cluster_kernel<SV, SL, NT, CL, MINB, HV>, a),
                   "cluster launch");
        PSMS_LAUNCH_CHECK("block_solve_cluster_kernel");
    }
}


// The autotuned variants (cluster size CL, min CTAs per SM, hop form HV) of
// one inner-precision store SV, as X(SV, CL, MINB, HV).
#define PSMS_BLOCK_VARIANTS_CG(X, SV) \
    X(SV, 1, 1, 0) X(SV, 1, 4, 0) X(SV, 2, 1, 0) X(SV, 2, 4, 0) X(SV, 4, 1, 0) X(SV, 4, 4, 0) X(SV, 8, 1, 0) X(SV, 8, 4, 0)
#define PSMS_BLOCK_VARIANTS_FORMS(X, SV) \
    X(SV, 1, 1, 1) X(SV, 1, 4, 1) X(SV, 1, 1, 2) X(SV, 1, 4, 2) X(SV, 4, 4, 2) X(SV, 8, 4, 2) X(SV, 1, 4, 3) \
    X(SV, 1, 4, 6) X(SV, 1, 4, 5) X(SV, 8, 4, 6)
#define PSMS_BLOCK_VARIANTS_SMEM(X, SV) X(SV, 1, 3, 8) X(SV, 1, 3, 10) X(SV, 1, 3, 9)
#define PSMS_BLOCK_EXTERN(SV, CL, MINB, HV) \
    extern template void launch_block_cl<SV, SV, CL, MINB, HV>(psms_ctx *, const BlockSolveArgs &, int, int);
#define PSMS_BLOCK_INSTANTIATE(SV, CL, MINB, HV) \
    template void launch_block_cl<SV, SV, CL, MINB, HV>(psms_ctx *, const BlockSolveArgs &, int, int);

}  // namespace psms
