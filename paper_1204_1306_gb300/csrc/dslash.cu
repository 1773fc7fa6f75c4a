// Wilson-Dirac hopping kernel, Eq. (Dw):
//   H(psi)(x) = sum_mu { U(x,mu)(1 - s gamma_mu) psi(x+mu)
//                      + U(x-mu,mu)^dagger (1 + s gamma_mu) psi(x-mu) },
// s = +1 for D and -1 for D^dagger, antiperiodic in time.  D = A - H/2 with
// A = 4 + m0.  One thread per output site; spin projection to half spinors
// (rank-2 projectors), SU(3) x half-spinor, reconstruction.  Fields use the
// structure-of-arrays even-odd block-major layout, so a warp reads each
// component of 32 consecutive sites in one coalesced transaction.
#include "bicgstab.cuh"
#include "kernels.hpp"

namespace psms {

template <class E>
struct HopArgs {
    Geom g;
    const BlockInfo *binfo;
    View<E> in, out, y, y2;
    double a, a2, b;
    const void *U;
    long long U_bs;
    int p, rank_lo, n_ranks, mode, dag;
    const int *active;
    double *partial;
    unsigned long long *prof_sites;  // profiling: output sites of active systems
    const int *sys_map;              // systems launched (null: all, k = blockIdx.y)
    const int *rank_active;          // per rank: 0 skips its output sites (null: none skipped)
    LinkInterp li;                   // shared-endpoint FP32 links (li.U0 null: U, U_bs)
    int nsf;                         // > 0: nsf systems fastest in blockIdx.x (gridDim.y = 1)
    int nct;                         // CTAs per system
    // fused BiCGStab reduction (dot 0: none; see HopDot)
    int dot;
    View<E> dx;
    BCS *dst;
    double *dre, *dim, *daa;
    unsigned int *dcnt;
    int dstage, dmaxit;
    int *dflags;
};

// (launched system, CTA of that system) of this CTA
__device__ __forceinline__ void hop_cta(int nsf, int &ks, int &bx) {
    if (nsf > 0) {
        ks = (int)(blockIdx.x % (unsigned)nsf);
        bx = (int)(blockIdx.x / (unsigned)nsf);
    } else {
        ks = (int)blockIdx.y;
        bx = (int)blockIdx.x;
    }
}

// link (mu, idx) of system k: from its own field (LI = 0), or a_k U0 + b_k U1
// of the shared endpoints (LI = 1: U0 alone where the endpoints agree; LI =
// 2: always both, no flag and no divergent branch)
template <class SL, int LI, class E>
__device__ __forceinline__ SU3<typename SL::R> hop_link(const HopArgs<E> &a, const typename SL::elem *U, int k, int mu,
                                                       long long idx) {
    if constexpr (LI == 2 && SL::VSH == 1) {
        SU3<float> u = load_link<SL>(a.li.U0, a.g.V, mu, idx);
        const SU3<float> u1 = load_link<SL>(a.li.U1, a.g.V, mu, idx);
        const float2 ab = __ldg(a.li.ab + k);
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                u.e[i][j].re = fmaf(ab.y, u1.e[i][j].re, ab.x * u.e[i][j].re);
                u.e[i][j].im = fmaf(ab.y, u1.e[i][j].im, ab.x * u.e[i][j].im);
            }
        return u;
    } else if constexpr (LI == 1 && SL::VSH == 1) {
        {
            SU3<float> u = load_link<SL>(a.li.U0, a.g.V, mu, idx);
            if (__ldg(a.li.flag + (long long)mu * a.g.V + idx)) {
                const SU3<float> u1 = load_link<SL>(a.li.U1, a.g.V, mu, idx);
                const float2 ab = __ldg(a.li.ab + k);
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int j = 0; j < 3; ++j) {
                        u.e[i][j].re = fmaf(ab.y, u1.e[i][j].re, ab.x * u.e[i][j].re);
                        u.e[i][j].im = fmaf(ab.y, u1.e[i][j].im, ab.x * u.e[i][j].im);
                    }
            }
            return u;
        }
    }
    return load_link<SL>(U, a.g.V, mu, idx);
}

template <int NT>
__device__ __forceinline__ double block_sum(double v, double *sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    __syncthreads();
    double t = 0;
    if (threadIdx.x == 0) {
        for (int i = 0; i < NT / 32; ++i) t += sh[i];
    }
    return t;  // valid in thread 0
}

// Directions [D0, D1) of the branch-free whole-lattice hop of one output
// site (d = 2 mu + (0 forward, 1 backward)), accumulated into acc.
template <int D0, int D1, class S, class SL, int LI, class E>
__device__ __forceinline__ void hop_dirs(const HopArgs<E> &a, const Geom &g, const BlockInfo &bi, int r, int p,
                                         const int y[4], int ll, long long s, int k, const E *in,
                                         const typename SL::elem *U, typename SL::R sg,
                                         Spinor<typename SL::R> &acc) {
    using R = typename SL::R;
    long long snb[8];
    int bsg[8];
#pragma unroll
    for (int d = D0; d < D1; ++d) neighbour(g, bi, r, p, y, ll, d >> 1, (d & 1) ? -1 : 1, HOP_ALL, snb[d], bsg[d]);
#pragma unroll
    for (int d = D0; d < D1; ++d) {
        const int mu = d >> 1;
        const bool fwd = (d & 1) == 0;
        Spinor<R> v = load_spinor_ro<S>(in, a.in.cs, snb[d] - a.in.off);
        const R tt = fwd ? -sg : sg;
        Half<R> h = project(mu, tt, v);
        if (mu == 0) {
            // antiperiodic time boundary: sign on the hop
            const R bsr = R(bsg[d]);
#pragma unroll
            for (int q = 0; q < 2; ++q)
#pragma unroll
                for (int c = 0; c < 3; ++c) h.c[q][c] = bsr * h.c[q][c];
        }
        SU3<R> u = hop_link<SL, LI>(a, U, k, mu, fwd ? s : snb[d]);
        reconstruct_add(mu, tt, fwd ? su3_mul(u, h) : su3_dag_mul(u, h), acc);
    }
}

// ALL = 1: specialised for HOP_ALL (every neighbour exists): the eight
// neighbour indices are computed first and the eight hops run as one
// branch-free sequence, so the compiler can issue later directions' loads
// before earlier directions' arithmetic (more loads in flight per thread).
// LI = 1: links from the shared endpoints (FP32 links only).
// SPLIT = 1 (whole lattice, FP32 arithmetic): two threads per output site in
// a CTA of NT = 256 (128 sites), the first half of the CTA summing the
// directions mu = 0, 1 and the second mu = 2, 3 (halves of whole warps, so
// no divergence); the second half's partial spinors join the first's
// through shared memory and the first half finishes the site -- half the
// per-thread state, twice the threads in flight.
template <class S, class SL, int NT, int MINB, int ALL, int LI = 0, int SPLIT = 0>
__global__ void __launch_bounds__(NT, MINB) hop_kernel(const HopArgs<typename S::elem> a) {
    using R = typename SL::R;
    using E = typename S::elem;
    using EL = typename SL::elem;
    static_assert(!SPLIT || (ALL && NT == 256 && sizeof(R) == 4), "split form: whole lattice, 256 threads, FP32");
    constexpr int SN = SPLIT ? NT / 2 : NT;  // output sites per CTA
    __shared__ double sh[NT / 32];
    int ks, bx;
    hop_cta(a.nsf, ks, bx);
    const int k = a.sys_map ? a.sys_map[ks] : ks;
    if (a.active && !a.active[k]) {
        if (a.partial && threadIdx.x == 0) a.partial[(long long)k * a.nct + bx] = 0.0;
        return;
    }
    const Geom &g = a.g;
    const long long per_p = (long long)a.n_ranks * g.Vbh;
    const long long total = (a.p < 0 ? 2 : 1) * per_p;
    const int half = SPLIT ? (int)(threadIdx.x >= SN) : 0;
    const long long t = (long long)bx * SN + (threadIdx.x - half * SN);
    double nrm = 0.0;
    double d_re = 0.0, d_im = 0.0, d_aa = 0.0;  // fused BiCGStab dot partials
    bool work = t < total;
    int p = 0, r = 0, j = 0;
    if (work) {
        // both parities: block-major order (block, parity, site) so that the
        // two endpoints of a block's links are processed close in time and
        // each link is fetched from HBM about once per launch
        if (a.p < 0) {
            r = a.rank_lo + (int)(t >> (g.vbh_sh + 1));
            p = (int)((t >> g.vbh_sh) & 1);
            j = (int)(t & (g.Vbh - 1));
            if (a.n_ranks == g.nblocks) {
                // whole lattice: walk the blocks in lexicographic order, so
                // that a block's neighbours (opposite colour) are processed
                // soon after it and face data is still in L2
                int B[4], rem = r;
                for (int m = 3; m >= 0; --m) {
                    B[m] = rem % g.nb[m];
                    rem /= g.nb[m];
                }
                r = rank_of_lex(g, r, B);
            }
        } else {
            p = a.p;
            r = a.rank_lo + (int)(t >> g.vbh_sh);
            j = (int)(t & (g.Vbh - 1));
            if (a.n_ranks == g.nblocks && g.coloured) {
                // whole lattice, one parity: walk the blocks in lexicographic
                // order (colours interleaved), so that the faces a block
                // reads from its neighbours were loaded by CTAs that ran
                // just before and are still in L2
                int B[4], rem = r;
                for (int m = 3; m >= 0; --m) {
                    B[m] = rem % g.nb[m];
                    rem /= g.nb[m];
                }
                r = rank_of_lex(g, r, B);
            }
        }
        work = !a.rank_active || a.rank_active[r];
    }
    if (a.prof_sites) {
        // output sites this warp computes (algorithmic-byte accounting)
        const unsigned cnt = __popc(__ballot_sync(0xffffffffu, work && !half));
        if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(a.prof_sites, (unsigned long long)cnt);
    }
    const long long s = (long long)p * g.Vh + (long long)r * g.Vbh + j;
    Spinor<R> acc;
    zero(acc);
    if (work) {
        int y[4];
        const int ll = local_lex(g, p, j, y);
        const BlockInfo &bi = a.binfo[r];
        const E *in = a.in.p + k * a.in.bs;
        const EL *U = (const EL *)a.U + k * a.U_bs;
        const R sg = a.dag ? R(-1) : R(1);
        if constexpr (SPLIT) {
            // warp-uniform halves: mu = 0, 1 in the first, mu = 2, 3 in the second
            if (half)
                hop_dirs<4, 8, S, SL, LI>(a, g, bi, r, p, y, ll, s, k, in, U, sg, acc);
            else
                hop_dirs<0, 4, S, SL, LI>(a, g, bi, r, p, y, ll, s, k, in, U, sg, acc);
        } else if constexpr (ALL) {
            hop_dirs<0, 8, S, SL, LI>(a, g, bi, r, p, y, ll, s, k, in, U, sg, acc);
        } else {
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) {
            long long sn;
            int bs;
            if (neighbour(g, bi, r, p, y, ll, mu, +1, a.mode, sn, bs)) {
                Spinor<R> v = load_spinor_ro<S>(in, a.in.cs, sn - a.in.off);
                const R tf = -sg;
                Half<R> h = project(mu, tf, v);
                if (bs < 0) {
#pragma unroll
                    for (int q = 0; q < 2; ++q)
#pragma unroll
                        for (int c = 0; c < 3; ++c) h.c[q][c] = R(-1) * h.c[q][c];
                }
                SU3<R> u = hop_link<SL, LI>(a, U, k, mu, s);
                reconstruct_add(mu, tf, su3_mul(u, h), acc);
            }
            if (neighbour(g, bi, r, p, y, ll, mu, -1, a.mode, sn, bs)) {
                Spinor<R> v = load_spinor_ro<S>(in, a.in.cs, sn - a.in.off);
                const R tb = sg;
                Half<R> h = project(mu, tb, v);
                if (bs < 0) {
#pragma unroll
                    for (int q = 0; q < 2; ++q)
#pragma unroll
                        for (int c = 0; c < 3; ++c) h.c[q][c] = R(-1) * h.c[q][c];
                }
                SU3<R> u = hop_link<SL, LI>(a, U, k, mu, sn);
                reconstruct_add(mu, tb, su3_dag_mul(u, h), acc);
            }
        }
        }
    }
    if constexpr (SPLIT) {
        // join the halves: the second half's partial spinor goes through
        // shared memory to the first, which finishes the site
        __shared__ float red[24][SN];
        if (half && work) {
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    red[2 * (3 * q + c)][threadIdx.x - SN] = acc.c[q][c].re;
                    red[2 * (3 * q + c) + 1][threadIdx.x - SN] = acc.c[q][c].im;
                }
        }
        __syncthreads();
        if (!half && work) {
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    acc.c[q][c].re += red[2 * (3 * q + c)][threadIdx.x];
                    acc.c[q][c].im += red[2 * (3 * q + c) + 1][threadIdx.x];
                }
        }
        work = work && !half;
    }
    if (work) {
        const R cb = (R)a.b;
        Spinor<R> o;
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int c = 0; c < 3; ++c) o.c[q][c] = cb * acc.c[q][c];
        if (a.y.p) {
            const R ca = (R)a.a;
            Spinor<R> v = load_spinor<S>(a.y.p + k * a.y.bs, a.y.cs, s - a.y.off);
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int c = 0; c < 3; ++c) o.c[q][c] = o.c[q][c] + ca * v.c[q][c];
        }
        if (a.y2.p) {
            const R ca = (R)a.a2;
            Spinor<R> v = load_spinor<S>(a.y2.p + k * a.y2.bs, a.y2.cs, s - a.y2.off);
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int c = 0; c < 3; ++c) o.c[q][c] = o.c[q][c] + ca * v.c[q][c];
        }
        store_spinor<S>(a.out.p + k * a.out.bs, a.out.cs, s - a.out.off, o);
        if (a.dot) {
            // the BiCGStab dot product of the output: the 12 components
            // summed in the inner precision (threads and CTAs in FP64)
            const Spinor<R> w = a.dot == 1 ? load_spinor<S>(a.dx.p + k * a.dx.bs, a.dx.cs, s - a.dx.off)
                                           : load_spinor<S>(a.y.p + k * a.y.bs, a.y.cs, s - a.y.off);
            R tre = 0, tim = 0, taa = 0;
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const cpx<R> x = a.dot == 1 ? w.c[q][c] : o.c[q][c];
                    const cpx<R> y = a.dot == 1 ? o.c[q][c] : w.c[q][c];
                    tre += x.re * y.re + x.im * y.im;
                    tim += x.re * y.im - x.im * y.re;
                    taa += x.re * x.re + x.im * x.im;
                }
            d_re = (double)tre;
            d_im = (double)tim;
            d_aa = (double)taa;
        }
        if (a.partial) {
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int c = 0; c < 3; ++c) nrm += (double)norm2(o.c[q][c]);
        }
    }
    if (a.partial) {
        double tot = block_sum<NT>(nrm, sh);
        if (threadIdx.x == 0) a.partial[(long long)k * a.nct + bx] = tot;
    }
    if (a.dot) {
        __shared__ double shd[3][NT / 32];
        bcg_partials_and_stage<NT>(a.dst, d_re, d_im, d_aa, a.dre, a.dim, a.daa, a.dcnt, a.dstage, a.dmaxit,
                                   a.dflags, shd, k, bx, a.nct);
    }
}

// Staged variant for whole-lattice launches on blocks of 2 x 128 sites (4^4):
// one CTA per (block, output parity, system).  The block's own input sites
// of the other parity (the neighbours of 3/4 of the hops) are copied into
// shared memory with asynchronous 16-byte copies (cp.async, past the
// registers and L1), then every direction reads its neighbour through one
// generic load sequence from shared memory (inside the block) or global
// memory (across a face), so the two cases do not split the warp.  Blocks
// are walked in lexicographic order (colours interleaved) as in the
// unstaged kernel.  Links are read from global memory as there.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// TMA = 1: the block's input rows (one contiguous 16-byte unit row of NT
// sites per spinor unit) are moved by the bulk-copy engine
// (cp.async.bulk, completion counted in bytes on an mbarrier) instead of
// per-thread 16-byte copies.  The wait is bounded; if it ran out, the
// neighbours are read from global memory instead (same values), after a
// second bounded wait for the copies in flight.
__device__ __forceinline__ bool bulk_wait(uint32_t bar, uint32_t parity) {
    for (int it = 0; it < (1 << 22); ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred q;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, q;\n\t}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

template <class S, class SL, int NT, int MINB, int TMA = 0>
__global__ void __launch_bounds__(NT, MINB) hop_staged_kernel(const HopArgs<typename S::elem> a) {
    using R = typename SL::R;
    using E = typename S::elem;
    using EL = typename SL::elem;
    constexpr int NU = 12 >> S::VSH;  // 16-byte units per site
    __shared__ int4 stage[NU * NT];
    __shared__ double sh[NT / 32];
    const Geom &g = a.g;
    const int k = a.sys_map ? a.sys_map[blockIdx.y] : (int)blockIdx.y;
    if (a.active && !a.active[k]) {
        if (a.partial && threadIdx.x == 0) a.partial[(long long)k * gridDim.x + blockIdx.x] = 0.0;
        return;
    }
    // CTA -> (block, parity): both parities in block-major order, or one
    int p, bl;
    if (a.p < 0) {
        bl = blockIdx.x >> 1;
        p = blockIdx.x & 1;
    } else {
        bl = blockIdx.x;
        p = a.p;
    }
    int B[4], rem = bl;
    for (int m = 3; m >= 0; --m) {
        B[m] = rem % g.nb[m];
        rem /= g.nb[m];
    }
    const int r = rank_of_lex(g, bl, B);
    if (a.rank_active && !a.rank_active[r]) {
        if (a.partial && threadIdx.x == 0) a.partial[(long long)k * gridDim.x + blockIdx.x] = 0.0;
        return;
    }
    if (a.prof_sites && threadIdx.x == 0) atomicAdd(a.prof_sites, (unsigned long long)NT);
    const E *in = a.in.p + k * a.in.bs;
    // stage the block's input sites of the other parity (unit u of site s at
    // 16-byte unit u * cs + s - off)
    bool staged_ok = true;
    {
        const long long s0 = (long long)(1 - p) * g.Vh + (long long)r * g.Vbh - a.in.off;
        const int4 *src = reinterpret_cast<const int4 *>(in);
        if constexpr (TMA) {
            __shared__ __align__(8) uint64_t bar;
            const uint32_t sbar = (uint32_t)__cvta_generic_to_shared(&bar);
            if (threadIdx.x == 0) {
                asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(sbar) : "memory");
                asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(sbar),
                             "r"((uint32_t)(NU * NT * 16))
                             : "memory");
#pragma unroll
                for (int u = 0; u < NU; ++u) {
                    const uint32_t dst = (uint32_t)__cvta_generic_to_shared(&stage[u * NT]);
                    asm volatile(
                        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                            dst),
                        "l"(src + u * a.in.cs + s0), "r"((uint32_t)(NT * 16)), "r"(sbar)
                        : "memory");
                }
            }
            staged_ok = bulk_wait(sbar, 0);
            if (!staged_ok) bulk_wait(sbar, 0);
            staged_ok = __syncthreads_and(staged_ok);
            if (threadIdx.x == 0) asm volatile("mbarrier.inval.shared::cta.b64 [%0];\n" ::"r"(sbar) : "memory");
        } else {
#pragma unroll
            for (int u = 0; u < NU; ++u)
                cp_async16(&stage[u * NT + threadIdx.x], src + u * a.in.cs + s0 + threadIdx.x);
            cp_async_wait_all();
            __syncthreads();
        }
    }
    const int j = threadIdx.x;
    int y[4];
    const int ll = local_lex(g, p, j, y);
    const BlockInfo &bi = a.binfo[r];
    const long long s = (long long)p * g.Vh + (long long)r * g.Vbh + j;
    const EL *U = (const EL *)a.U + k * a.U_bs;
    const R sg = a.dag ? R(-1) : R(1);
    const E *sm = reinterpret_cast<const E *>(stage);
    // lattice volumes stay below 2^31 sites: 32-bit indices keep the eight
    // neighbours in registers
    const int base_opp = (int)((long long)(1 - p) * g.Vh + (long long)r * g.Vbh);
    int snb[8], idx_[8];
    unsigned inside = 0, neg = 0;
#pragma unroll
    for (int d = 0; d < 8; ++d) {
        const int mu = d >> 1, sgn = (d & 1) ? -1 : 1;
        long long sn;
        int bs;
        neighbour(g, bi, r, p, y, ll, mu, sgn, HOP_ALL, sn, bs);
        snb[d] = (int)sn;
        if (bs < 0) neg |= 1u << d;
        const int yn = y[mu] + sgn;
        if (staged_ok && (unsigned)yn < (unsigned)g.l[mu]) {
            inside |= 1u << d;
            idx_[d] = snb[d] - base_opp;
        } else {
            idx_[d] = snb[d] - (int)a.in.off;
        }
    }
    Spinor<R> acc;
    zero(acc);
#pragma unroll
    for (int d = 0; d < 8; ++d) {
        const int mu = d >> 1;
        const bool fwd = (d & 1) == 0;
        const bool ins = (inside >> d) & 1;
        Spinor<R> v = load_spinor<S>(ins ? sm : in, ins ? (long long)NT : a.in.cs, idx_[d]);
        const R tt = fwd ? -sg : sg;
        Half<R> h = project(mu, tt, v);
        if (mu == 0 && ((neg >> d) & 1)) {
#pragma unroll
            for (int q = 0; q < 2; ++q)
#pragma unroll
                for (int c = 0; c < 3; ++c) h.c[q][c] = R(-1) * h.c[q][c];
        }
        SU3<R> u = load_link<SL>(U, g.V, mu, fwd ? s : (long long)snb[d]);
        reconstruct_add(mu, tt, fwd ? su3_mul(u, h) : su3_dag_mul(u, h), acc);
    }
    const R cb = (R)a.b;
    Spinor<R> o;
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int c = 0; c < 3; ++c) o.c[q][c] = cb * acc.c[q][c];
    if (a.y.p) {
        const R ca = (R)a.a;
        Spinor<R> v = load_spinor<S>(a.y.p + k * a.y.bs, a.y.cs, s - a.y.off);
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int c = 0; c < 3; ++c) o.c[q][c] = o.c[q][c] + ca * v.c[q][c];
    }
    if (a.y2.p) {
        const R ca = (R)a.a2;
        Spinor<R> v = load_spinor<S>(a.y2.p + k * a.y2.bs, a.y2.cs, s - a.y2.off);
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int c = 0; c < 3; ++c) o.c[q][c] = o.c[q][c] + ca * v.c[q][c];
    }
    store_spinor<S>(a.out.p + k * a.out.bs, a.out.cs, s - a.out.off, o);
    if (a.partial) {
        double nrm = 0.0;
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int c = 0; c < 3; ++c) nrm += (double)norm2(o.c[q][c]);
        double tot = block_sum<NT>(nrm, sh);
        if (threadIdx.x == 0) a.partial[(long long)k * gridDim.x + blockIdx.x] = tot;
    }
}

static constexpr int HOP_NT = 128;

int hop_ctas(psms_ctx *c, const HopCall &h) {
    const int nr = h.n_ranks < 0 ? c->g.nblocks : h.n_ranks;
    const long long total = (h.p < 0 ? 2LL : 1LL) * nr * c->g.Vbh;
    return (int)((total + HOP_NT - 1) / HOP_NT);
}

template <class S, class SL>
static int hop_launch_t(psms_ctx *c, const HopCall &h) {
    using E = typename S::elem;
    HopArgs<E> a;
    a.g = c->g;
    a.binfo = c->d_binfo;
    auto cv = [](const View<void> &v) {
        View<E> w;
        w.p = (E *)v.p;
        w.cs = v.cs;
        w.off = v.off;
        w.bs = v.bs;
        return w;
    };
    a.in = cv(h.in);
    a.out = cv(h.out);
    a.y = cv(h.y);
    a.y2 = cv(h.y2);
    a.a = h.a;
    a.a2 = h.a2;
    a.b = h.b;
    a.U = h.U;
    a.U_bs = h.U_bs;
    a.p = h.p;
    a.rank_lo = h.rank_lo;
    a.n_ranks = h.n_ranks < 0 ? c->g.nblocks : h.n_ranks;
    a.mode = h.mode;
    a.dag = h.dag;
    a.active = h.active;
    a.partial = h.partial;
    a.prof_sites = nullptr;
    a.sys_map = h.sys_map;
    a.rank_active = h.rank_active;
    const bool shared_links = h.li.U0 != nullptr;
    a.li = h.li;
    a.dot = h.dot.dot;
    a.dx = cv(h.dot.x);
    a.dst = h.dot.st;
    a.dre = h.dot.re;
    a.dim = h.dot.im;
    a.daa = h.dot.aa;
    a.dcnt = h.dot.cnt;
    a.dstage = h.dot.stage;
    a.dmaxit = h.dot.maxit;
    a.dflags = h.dot.flags;
    if (a.dot && (h.prec != P32 || h.p < 0 || !h.dot.st || !h.dot.cnt || (a.dot == 2 && !h.y.p) ||
                  (a.dot == 1 && !h.dot.x.p)))
        fail(PSMS_EINVAL, "hop_launch: a fused reduction needs FP32 storage, one parity and its vectors");
    if (shared_links) {
        if (h.prec == P64 || !h.li.U1 || !h.li.ab || !h.li.flag)
            fail(PSMS_EINVAL, "hop_launch: shared-endpoint links need FP32 storage, U1, ab and flags");
        a.U = h.li.U0;
        a.U_bs = 0;
    }
    const int nct = hop_ctas(c, h);
    const int nsys = h.sys_map ? h.n_map : h.n_sys;
    if (nct == 0 || nsys == 0) return 0;
    a.nct = nct;
    // shared-endpoint links: the systems of a launch run side by side (CTA
    // index = cta * nsys + system), so each endpoint link leaves HBM once
    a.nsf = shared_links ? nsys : 0;
    const dim3 grid = shared_links ? dim3((unsigned)((long long)nct * nsys), 1) : dim3(nct, nsys);
    double bytes = 0;
    int slot = -1;
    if (c->prof && h.mode == HOP_ALL && (c->prof_prec < 0 || c->prof_prec == h.prec)) {
        // algorithmic bytes per output site of an active system: in + out
        // (+ y, y2, + the fused reduction's vector) spinors and 4 links
        // (both parities) or 8 (one parity) of that system's field -- also
        // with shared-endpoint links, whose HBM traffic is lower (the
        // systems share the endpoint links through L2); the device counts
        // the output sites of the systems still active
        const double sp = 12.0 * sizeof(E), lk = 9.0 * sizeof(typename SL::elem);
        const double links = 4 * lk * (h.p < 0 ? 1 : 2);
        bytes = 2 * sp + (h.y.p ? sp : 0) + (h.y2.p ? sp : 0) + (a.dot == 1 ? sp : 0) + links;
        slot = prof_begin(c);
        a.prof_sites = prof_counter(c, slot);
    }
    // Register cap (minimum resident CTAs per SM) chosen by the autotuner:
    // on the first launch of each (precision, parity shape) every variant is
    // timed twice with CUDA events and the fastest is kept.  All variants do
    // identical arithmetic; a launch is idempotent (out is a function of in, y,
    // y2, U only), so the extra tuning launches leave the result unchanged.
    using KFn = void (*)(const HopArgs<E>);
    constexpr bool f32 = sizeof(typename SL::R) == 4;
    // FP32 links: register caps 2, 6, 7, 8 CTAs/SM; for the whole lattice
    // (HOP_ALL) the branch-free specialisation with caps 4, 5, 6, 7 besides
    const bool all = h.mode == HOP_ALL;
    // the staged kernel: whole lattice, 128 sites of each parity per block
    const bool staged = all && a.n_ranks == c->g.nblocks && h.rank_lo == 0 && c->g.Vbh == HOP_NT;
    const KFn *vars;
    const int *thr = nullptr;  // threads per CTA of each variant (null: all HOP_NT)
    int nvar;
    if constexpr (f32) {
        static const KFn v32[] = {hop_kernel<S, SL, HOP_NT, 2, 0>, hop_kernel<S, SL, HOP_NT, 6, 0>,
                                  hop_kernel<S, SL, HOP_NT, 7, 0>, hop_kernel<S, SL, HOP_NT, 8, 0>};
        static const KFn v32all[] = {hop_kernel<S, SL, HOP_NT, 2, 0>, hop_kernel<S, SL, HOP_NT, 6, 0>,
                                     hop_kernel<S, SL, HOP_NT, 7, 0>, hop_kernel<S, SL, HOP_NT, 8, 0>,
                                     hop_kernel<S, SL, HOP_NT, 4, 1>, hop_kernel<S, SL, HOP_NT, 5, 1>,
                                     hop_kernel<S, SL, HOP_NT, 6, 1>, hop_kernel<S, SL, HOP_NT, 7, 1>,
                                     hop_kernel<S, SL, 2 * HOP_NT, 3, 1, 0, 1>, hop_kernel<S, SL, 2 * HOP_NT, 4, 1, 0, 1>,
                                     hop_staged_kernel<S, SL, HOP_NT, 4>, hop_staged_kernel<S, SL, HOP_NT, 6>,
                                     hop_staged_kernel<S, SL, HOP_NT, 4, 1>, hop_staged_kernel<S, SL, HOP_NT, 6, 1>};
        static const int t32all[] = {HOP_NT, HOP_NT, HOP_NT, HOP_NT, HOP_NT, HOP_NT, HOP_NT,
                                     HOP_NT, 2 * HOP_NT, 2 * HOP_NT, HOP_NT, HOP_NT, HOP_NT, HOP_NT};
        // shared-endpoint links (whole lattice): register caps 2-8 CTAs/SM,
        // general and branch-free forms, flagged or unconditional U1 reads
        static const KFn v32li[] = {hop_kernel<S, SL, HOP_NT, 2, 0, 1>, hop_kernel<S, SL, HOP_NT, 4, 0, 1>,
                                    hop_kernel<S, SL, HOP_NT, 2, 1, 1>, hop_kernel<S, SL, HOP_NT, 3, 1, 1>,
                                    hop_kernel<S, SL, HOP_NT, 4, 1, 1>, hop_kernel<S, SL, HOP_NT, 5, 1, 1>,
                                    hop_kernel<S, SL, HOP_NT, 6, 0, 1>, hop_kernel<S, SL, HOP_NT, 8, 0, 1>,
                                    hop_kernel<S, SL, HOP_NT, 6, 1, 1>, hop_kernel<S, SL, HOP_NT, 4, 0, 2>,
                                    hop_kernel<S, SL, HOP_NT, 6, 0, 2>, hop_kernel<S, SL, HOP_NT, 4, 1, 2>,
                                    hop_kernel<S, SL, HOP_NT, 6, 1, 2>,
                                    hop_kernel<S, SL, 2 * HOP_NT, 2, 1, 1, 1>, hop_kernel<S, SL, 2 * HOP_NT, 3, 1, 1, 1>};
        static const int t32li[] = {HOP_NT, HOP_NT, HOP_NT, HOP_NT, HOP_NT, HOP_NT, HOP_NT, HOP_NT,
                                    HOP_NT, HOP_NT, HOP_NT, HOP_NT, HOP_NT, 2 * HOP_NT, 2 * HOP_NT};
        if (shared_links && !all) fail(PSMS_EINVAL, "hop_launch: shared-endpoint links on whole-lattice hops only");
        vars = shared_links ? v32li : (all ? v32all : v32);
        thr = shared_links ? t32li : (all ? t32all : nullptr);
        // two-threads-per-site forms: v32all entries 8, 9 and v32li 13, 14;
        // staged forms: v32all 10 to 13 (blocks of 2 x 128 sites only)
        nvar = shared_links ? 15 : (all ? (staged ? 14 : 10) : 4);
    } else {
        // FP64 (ALU bound): the general form, and for the whole lattice the
        // branch-free form, register caps 3 and 4 CTAs/SM
        static const KFn v64[] = {hop_kernel<S, SL, HOP_NT, 2, 0>};
        static const KFn v64all[] = {hop_kernel<S, SL, HOP_NT, 2, 0>, hop_kernel<S, SL, HOP_NT, 2, 1>,
                                     hop_kernel<S, SL, HOP_NT, 4, 0>, hop_kernel<S, SL, HOP_NT, 3, 1>};
        vars = all ? v64all : v64;
        nvar = all ? 4 : 1;
    }
    int &choice = c->hop_variant[h.prec][h.p < 0 ? 1 : 0][all ? 1 : 0][shared_links ? 1 : 0];
    // (launches with a fused reduction are not used for tuning: they advance
    // the solver's scalars)
    if (choice < 0 && c->autotune && nvar > 1 && slot < 0 && c->forced_hop_variant < 0 && !a.dot) {
        cudaEvent_t e0, e1;
        cuda_check(cudaEventCreate(&e0), "tune event");
        cuda_check(cudaEventCreate(&e1), "tune event");
        float best = 1e30f;
        for (int v = 0; v < nvar; ++v) {
            vars[v]<<<grid, thr ? thr[v] : HOP_NT, 0, c->stream>>>(a);
            cuda_check(cudaEventRecord(e0, c->stream), "tune record");
            vars[v]<<<grid, thr ? thr[v] : HOP_NT, 0, c->stream>>>(a);
            vars[v]<<<grid, thr ? thr[v] : HOP_NT, 0, c->stream>>>(a);
            cuda_check(cudaEventRecord(e1, c->stream), "tune record");
            cuda_check(cudaEventSynchronize(e1), "tune sync");
            launch_counter() += 3;
            float ms = 0;
            cuda_check(cudaEventElapsedTime(&ms, e0, e1), "tune elapsed");
            if (ms < best) {
                best = ms;
                choice = v;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        PSMS_LAUNCH_CHECK("hop_kernel (autotune)");
    }
    int v = (choice >= 0 && choice < nvar) ? choice : (f32 ? 1 : 0);
    if (c->forced_hop_variant >= 0) v = c->forced_hop_variant % nvar;
    // the staged kernels (v32all entries 10 to 13) carry no fused reduction
    if (a.dot && !shared_links && all && v >= 10) v = 6;
    vars[v]<<<grid, thr ? thr[v] : HOP_NT, 0, c->stream>>>(a);
    PSMS_LAUNCH_CHECK("hop_kernel");
    if (slot >= 0) prof_end(c, slot, bytes);
    return nct;
}

int hop_launch(psms_ctx *c, const HopCall &h) {
    switch (h.prec) {
        case P64: return hop_launch_t<Store<double>, Store<double>>(c, h);
        case P32: return hop_launch_t<Store<float>, Store<float>>(c, h);
        case PB16: return hop_launch_t<Store<__nv_bfloat16>, Store<float>>(c, h);
    }
    fail(PSMS_EINVAL, "hop_launch: bad precision");
}

// --- deterministic reductions ------------------------------------------------

template <int NT>
__global__ void __launch_bounds__(NT) reduce_partials_kernel(const double *partial, int n, double *out) {
    __shared__ double sh[NT / 32];
    const int k = blockIdx.x;
    double v = 0;
    for (int i = threadIdx.x; i < n; i += NT) v += partial[(long long)k * n + i];
    double t = block_sum<NT>(v, sh);
    if (threadIdx.x == 0) out[k] = t;
}

void reduce_partials(psms_ctx *c, const double *partial, int n, int n_sys, double *out) {
    reduce_partials_kernel<256><<<n_sys, 256, 0, c->stream>>>(partial, n, out);
    PSMS_LAUNCH_CHECK("reduce_partials");
}

template <class S, int NT>
__global__ void __launch_bounds__(NT) norm2_kernel(View<typename S::elem> v, long long s_lo, long long n,
                                                   double *partial) {
    __shared__ double sh[NT / 32];
    const int k = blockIdx.y;
    double acc = 0;
    for (long long i = (long long)blockIdx.x * NT + threadIdx.x; i < n; i += (long long)gridDim.x * NT) {
        const long long s = s_lo + i;
        for (int q = 0; q < 12; ++q) acc += (double)norm2(S::ld(v.p + k * v.bs, q, v.cs, s - v.off));
    }
    double t = block_sum<NT>(acc, sh);
    if (threadIdx.x == 0) partial[(long long)k * gridDim.x + blockIdx.x] = t;
}

void norm2_batch(psms_ctx *c, int prec, View<void> v, long long s_lo, long long n, int n_sys, double *out) {
    const int NT = 256;
    int nct = (int)std::min<long long>((n + NT - 1) / NT, 1024);
    if (nct < 1) nct = 1;
    double *partial = (double *)scratch(c, "norm2_partial", sizeof(double) * (size_t)nct * n_sys);
    dim3 grid(nct, n_sys);
    switch (prec) {
        case P64: {
            View<double2> w{(double2 *)v.p, v.cs, v.off, v.bs};
            norm2_kernel<Store<double>, NT><<<grid, NT, 0, c->stream>>>(w, s_lo, n, partial);
            break;
        }
        case P32: {
            View<float2> w{(float2 *)v.p, v.cs, v.off, v.bs};
            norm2_kernel<Store<float>, NT><<<grid, NT, 0, c->stream>>>(w, s_lo, n, partial);
            break;
        }
        default: {
            View<__nv_bfloat162> w{(__nv_bfloat162 *)v.p, v.cs, v.off, v.bs};
            norm2_kernel<Store<__nv_bfloat16>, NT><<<grid, NT, 0, c->stream>>>(w, s_lo, n, partial);
            break;
        }
    }
    PSMS_LAUNCH_CHECK("norm2_kernel");
    reduce_partials(c, partial, nct, n_sys, out);
}

}  // namespace psms
