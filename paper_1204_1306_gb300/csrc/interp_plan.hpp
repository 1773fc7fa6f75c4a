// Host-side planning of the estimators' batched interpolation steps, pure
// arithmetic (no CUDA calls) so that host tests can check it against the
// oracle: the per-system coefficients of the shared-endpoint links and the
// balanced chunk sizes.
#pragma once

namespace psms {

// (a_k, b_k) of system k = 0..n-1 of a chunk starting at interpolation step
// i0: the links of field i = i0 + k + shift of Eq. (gfparam),
// U_i = ((N - i)/N) U + (i/N) U' (shift 0: the first operator of the pair,
// 1: the second); in the independent mode every system pairs U (shift 0)
// with U' (shift 1).  ab holds 2n floats.
inline void interp_coefs(int N, int i0, int n, int shift, bool independent, float *ab) {
    for (int k = 0; k < n; ++k) {
        if (independent) {
            ab[2 * k] = shift ? 0.f : 1.f;
            ab[2 * k + 1] = shift ? 1.f : 0.f;
        } else {
            const int i = i0 + k + shift;
            ab[2 * k] = (float)((double)(N - i) / N);
            ab[2 * k + 1] = (float)((double)i / N);
        }
    }
}

// systems per chunk when at most k fit: as many chunks as needed, of equal
// size (the last at most one smaller)
inline int balanced_chunk(int N, int k) {
    if (k < 1) k = 1;
    if (k > N) k = N;
    const int n_chunks = (N + k - 1) / k;
    return (N + n_chunks - 1) / n_chunks;
}

}  // namespace psms
