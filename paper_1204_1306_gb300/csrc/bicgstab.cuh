// Shared state and scalar steps of the batched BiCGStab on Dhat (one system
// per interpolation step): the per-system scalars, the stage that turns a
// finished reduction into alpha, omega or (rho, beta, convergence), and the
// deterministic "last CTA finishes the reduction" pattern used by the BLAS
// kernels of the solver and by Wilson hops that fuse their dot products.
#pragma once

#include "common.cuh"

namespace psms {

struct BCS {
    double2 rho, alpha, omega, beta;
    double rr, target;
    int active, iters;
};

__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
    const double d = b.x * b.x + b.y * b.y;
    return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
__device__ __forceinline__ double2 cmul2(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// stage: 0 alpha = rho / <rh, v>; 1 omega = <t, s> / <t, t>;
//        2 rho_new = <rh, r>, rr = |r|^2, beta, convergence
__device__ __forceinline__ void bcg_stage(BCS *st, int k, double re, double im, double aa, int stage, int maxit, int *flags) {
    BCS s = st[k];
    const double2 d = make_double2(re, im);
    if (stage == 0) {
        if (!(re * re + im * im > 0.0)) {
            s.active = 0;  // breakdown: <rh, v> = 0
        } else {
            s.alpha = cdiv(s.rho, d);
        }
    } else if (stage == 1) {
        s.omega = aa > 0.0 ? make_double2(re / aa, im / aa) : make_double2(0.0, 0.0);
    } else {
        // the partials are sum conj(r) rh = conj(<rh, r>) and |r|^2 of the
        // new residual
        const double2 dr = make_double2(re, -im);
        s.iters += 1;
        s.rr = aa;
        const bool stalled = !(s.omega.x * s.omega.x + s.omega.y * s.omega.y > 0.0) ||
                             !(re * re + im * im > 0.0);
        if (!stalled) s.beta = cmul2(cdiv(dr, s.rho), cdiv(s.alpha, s.omega));
        s.rho = dr;
        if (aa <= s.target || s.iters >= maxit || stalled || !(aa == aa)) s.active = 0;
    }
    st[k] = s;
    flags[k] = s.active;
}

// Writes this CTA's partials of system k; the last CTA of the system to
// finish (a counter per system, no waiting) sums all partials in a fixed
// order and applies the scalar stage, so the result does not depend on
// which CTA finishes last.
template <int NT>
__device__ __forceinline__ void bcg_partials_and_stage(BCS *st, double re, double im, double aa, double *p_re,
                                                       double *p_im, double *p_aa, unsigned int *counters, int stage,
                                                       int maxit, int *flags, double (*sh)[NT / 32], int k,
                                                       int cta, int nct) {
    const long long slot = (long long)k * nct + cta;
    __shared__ int last;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        re += __shfl_xor_sync(0xffffffffu, re, o);
        im += __shfl_xor_sync(0xffffffffu, im, o);
        aa += __shfl_xor_sync(0xffffffffu, aa, o);
    }
    if ((threadIdx.x & 31) == 0) {
        sh[0][threadIdx.x >> 5] = re;
        sh[1][threadIdx.x >> 5] = im;
        sh[2][threadIdx.x >> 5] = aa;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t0 = 0, t1 = 0, t2 = 0;
        for (int w = 0; w < NT / 32; ++w) {
            t0 += sh[0][w];
            t1 += sh[1][w];
            t2 += sh[2][w];
        }
        p_re[slot] = t0;
        p_im[slot] = t1;
        p_aa[slot] = t2;
        __threadfence();
        last = atomicAdd(&counters[k], 1u) == (unsigned int)nct - 1u;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    // the other CTAs' partials, read past L1 (written by other SMs)
    const int m = nct;
    double v[3] = {0, 0, 0};
    for (int i = threadIdx.x; i < m; i += NT) {
        const long long q = (long long)k * m + i;
        v[0] += __ldcg(p_re + q);
        v[1] += __ldcg(p_im + q);
        v[2] += __ldcg(p_aa + q);
    }
    double tot[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double x = v[a];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        __syncthreads();
        if ((threadIdx.x & 31) == 0) sh[a][threadIdx.x >> 5] = x;
        __syncthreads();
        double t = 0;
        for (int w = 0; w < NT / 32; ++w) t += sh[a][w];
        tot[a] = t;
    }
    const double r0 = tot[0], r1 = tot[1], r2 = tot[2];
    if (threadIdx.x == 0) {
        counters[k] = 0;
        bcg_stage(st, k, r0, r1, r2, stage, maxit, flags);
    }
}

}  // namespace psms
