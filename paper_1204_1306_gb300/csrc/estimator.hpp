// Estimator and filter-level interfaces.
#pragma once

#include "kernels.hpp"

namespace psms {

// number of interpolation steps batched per launch, from a per-system
// device-memory estimate (bytes per lattice site), a 64 GB budget and the
// context's cap (psms_max_chunk), balanced so that the chunks of N have
// equal sizes (the last one at most one smaller)
int chunk_size(psms_ctx *c, int N, double bytes_per_site);
// noise fields xi_i (i = 0..n-1) for `level`, FP64 full layout, optional P projection
void noise(psms_ctx *c, double2 *out, int n, uint64_t seed, uint64_t counter, int level, int proj, int i0);
// d_delta[b * N + i] (b = lexicographic block index); returns total inner iterations
long long block_level(psms_ctx *c, const double2 *U, const double2 *Up, int N, int mode, uint64_t seed,
                      uint64_t counter, double tol, int inner, double *d_delta, const int *d_block_mask = nullptr);
// d_delta[i]
long long global_level(psms_ctx *c, const double2 *U, const double2 *Up, int N, int mode, uint64_t seed,
                       uint64_t counter, double tol, int inner, double *d_delta);
// accept decisions: per block (or one decision on the sum), d_dsum[b] = Delta_b
// (+ d_dsum[nb] = total when not per block)
void decide(psms_ctx *c, const double *d_delta, int nb, int N, int per_block, uint64_t seed, uint64_t step, int level,
            double extra_sum, const double *d_extra_pb, double coef, double *d_dsum, int *d_acc,
            const int *d_mask = nullptr);
// h (float, per block) -> FP64 copy
void float_to_double(psms_ctx *c, const float *a, double *b, int n);

// FP32 copies of the two endpoint fields of Eq. (gfparam) (ends64: U then U',
// 36 V complex each, masked as the caller needs) and the per-link flags
// where they differ: the shared-endpoint links of whole-lattice FP32 solves
struct SharedEnds {
    float2 *u0 = nullptr, *u1 = nullptr;
    unsigned char *flag = nullptr;
};
SharedEnds shared_ends(psms_ctx *c, const double2 *ends64, const char *tag);
// the links of a chunk's n systems: system k uses field i0 + k + shift of
// Eq. (gfparam), a_k = (N - i)/N, b_k = i/N (independent mode: U for
// shift 0, U' for shift 1)
LinkInterp link_interp(psms_ctx *c, const SharedEnds &e, int N, int i0, int n, int shift, int mode,
                       const char *tag);

}  // namespace psms
