// BF16 GEMM on Blackwell's fifth-generation tensor cores (tcgen05, TMEM
// accumulators), used by the learned level's MLP (App. C's auxiliary action):
//
//   C[m][n] = alpha * sum_k A(m,k) B(n,k) + beta * C[m][n] + bias[n]
//             (then optional ReLU; FP32 and/or BF16 copies of C)
//
// A(m,k) = A[m*sAm + k*sAk] and B(n,k) = B[n*sBn + k*sBk], FP32 or BF16 in
// global memory with arbitrary strides (the MLP's forward and backward
// products read row-major and transposed operands alike).
//
// One CTA of 128 threads computes a 128 x TN tile (TN = 64 or 256):
//   * the tile's accumulator lives in TMEM (TN columns x 128 lanes, FP32),
//     allocated by warp 0 with tcgen05.alloc and freed before exit;
//   * K runs in chunks of 64 through two shared-memory stages: all threads
//     convert their share of the chunk to BF16 and store it in the
//     canonical no-swizzle K-major layout (8 x 16-byte core matrices:
//     element (r, k) at ((r/8)*8 + k/8)*128 + (r%8)*16 + (k%8)*2 bytes),
//     make it visible to the tensor core's async proxy, and one thread
//     issues four tcgen05.mma (M = 128, N = TN, K = 16 each) and commits
//     them to the stage's mbarrier; the next chunk is staged meanwhile in
//     the other buffer, which is reused only after its own commit arrived;
//   * epilogue: warp w reads TMEM lanes 32w..32w+31 (rows of the tile)
//     with tcgen05.ld, applies alpha, beta, bias and ReLU, and stores.
// Every mbarrier wait is bounded; a wait that runs out sets *err, waits
// (bounded again) for the MMAs in flight, frees the TMEM and returns.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

#include "tc_layout.hpp"

namespace psms {
namespace tc {

constexpr int NTHR = 128;

struct Args {
    int M, N, K;
    const void *A;
    long long sAm, sAk;
    int a_f32;
    const void *B;
    long long sBn, sBk;
    int b_f32;
    float *Cf;
    long long ldc;
    __nv_bfloat16 *Cb;
    long long ldcb;
    const float *bias;
    float alpha, beta;
    int relu;
    int *err;  // set to 1 when a bounded wait runs out
};

// dynamic shared memory of one CTA: two stages of A (128 x 64) and B (TN x 64)
// BF16 tiles, then two mbarriers and the TMEM address slot
template <int TN>
constexpr int smem_bytes() {
    return 2 * (TM + TN) * TK * 2 + 64;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, long long limit) {
    for (long long it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ float ld_elem(const void *p, long long i, int f32) {
    return f32 ? ((const float *)p)[i] : __bfloat162float(((const __nv_bfloat16 *)p)[i]);
}

// rows [r0, r0 + rows) x k-chunk [k0, k0 + TK) of X(r, k) = X[r*sr + k*sk]
// into the canonical layout at dst (zero outside [0, R) x [0, K))
template <int ROWS>
__device__ __forceinline__ void stage_tile(uint8_t *dst, const void *X, long long sr, long long sk, int f32, int r0,
                                           int R, int k0, int K) {
    const bool kfast = (sk == 1);
    for (int e = threadIdx.x; e < ROWS * TK; e += NTHR) {
        const int r = kfast ? e / TK : e % ROWS;
        const int k = kfast ? e % TK : e / ROWS;
        const int gr = r0 + r, gk = k0 + k;
        const float v = (gr < R && gk < K) ? ld_elem(X, (long long)gr * sr + (long long)gk * sk, f32) : 0.f;
        *(__nv_bfloat16 *)(dst + canon_off(r, k)) = __float2bfloat16(v);
    }
}

template <int TN>
__global__ void __launch_bounds__(NTHR) gemm_kernel(const Args a) {
    extern __shared__ __align__(1024) uint8_t tc_smem[];
    constexpr int A_BYTES = TM * TK * 2, B_BYTES = TN * TK * 2;
    uint8_t *sA[2] = {tc_smem, tc_smem + A_BYTES};
    uint8_t *sB[2] = {tc_smem + 2 * A_BYTES, tc_smem + 2 * A_BYTES + B_BYTES};
    uint64_t *bars = (uint64_t *)(tc_smem + 2 * (A_BYTES + B_BYTES));
    uint32_t *tslot = (uint32_t *)(bars + 2);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
    const uint32_t bar0 = smem_u32(&bars[0]), bar1 = smem_u32(&bars[1]);
    constexpr long long WAIT = 1ll << 24;  // try_wait polls (each suspends briefly): far above any chunk's MMA time

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tslot)),
                     "r"(TN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar0) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = *tslot;

    const int nc = (a.K + TK - 1) / TK;
    const uint32_t idesc = instr_desc<TN>();
    bool ok = true;
    for (int c = 0; c < nc; ++c) {
        const int s = c & 1;
        // the stage was last read by the MMAs of chunk c - 2: thread 0 waits
        // for their commit, the barrier hands the outcome to every thread
        int late = 0;
        if (c >= 2 && tid == 0) late = !mbar_wait(s ? bar1 : bar0, (uint32_t)(((c - 2) >> 1) & 1), WAIT);
        if (__syncthreads_or(late)) {
            ok = false;
            break;
        }
        stage_tile<TM>(sA[s], a.A, a.sAm, a.sAk, a.a_f32, m0, a.M, c * TK, a.K);
        stage_tile<TN>(sB[s], a.B, a.sBn, a.sBk, a.b_f32, n0, a.N, c * TK, a.K);
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            const uint32_t abase = smem_u32(sA[s]), bbase = smem_u32(sB[s]);
#pragma unroll
            for (int j = 0; j < TK / 16; ++j) {
                // K = 16 per MMA: two core matrices along K (256 bytes)
                const uint64_t ad = smem_desc(abase + j * 2 * LBO, LBO, SBO);
                const uint64_t bd = smem_desc(bbase + j * 2 * LBO, LBO, SBO);
                const uint32_t acc = (c > 0 || j > 0) ? 1u : 0u;
                asm volatile(
                    "{\n\t.reg .pred p;\n\t"
                    "setp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                             s ? bar1 : bar0)
                         : "memory");
        }
    }
    // the last commit covers every MMA issued before it; every thread polls
    // it, and the barrier makes the outcome uniform
    const uint32_t last_bar = ((nc - 1) & 1) ? bar1 : bar0, last_par = (uint32_t)(((nc - 1) >> 1) & 1);
    if (ok && nc > 0) ok = !__syncthreads_or(!mbar_wait(last_bar, last_par, WAIT));
    if (!ok) {
        // wait, bounded, for what was issued, then leave without the epilogue
        if (tid == 0 && a.err) atomicExch(a.err, 1);
        if (nc > 0) mbar_wait(last_bar, last_par, WAIT);
    } else {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        const int m = m0 + warp * 32 + lane;
        const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
        for (int col = 0; col < TN; col += 8) {
            uint32_t v[8];
            if (nc > 0) {
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                    : "r"(trow + (uint32_t)col));
                asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
            } else {
#pragma unroll
                for (int q = 0; q < 8; ++q) v[q] = 0u;
            }
            if (m >= a.M) continue;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int n = n0 + col + q;
                if (n >= a.N) continue;
                float x = a.alpha * __uint_as_float(v[q]);
                if (a.beta != 0.f && a.Cf) x += a.beta * a.Cf[(long long)m * a.ldc + n];
                if (a.bias) x += a.bias[n];
                if (a.relu) x = fmaxf(x, 0.f);
                if (a.Cf) a.Cf[(long long)m * a.ldc + n] = x;
                if (a.Cb) a.Cb[(long long)m * a.ldcb + n] = __float2bfloat16(x);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TN) : "memory");
    }
}

}  // namespace tc
}  // namespace psms
