// Learned-level interfaces (domain features and the MLP surrogate).
#pragma once

#include "kernels.hpp"

namespace psms {

constexpr int N_FEAT = 32;
// features of every block of U into out[lex * stride + offset + 0..31]
void domain_features(psms_ctx *c, const double2 *U, float *out, int stride, int offset);
// rows [f(U_b), f(U'_b)] with the block distance d_b in slots 18 and 50
void pair_features(psms_ctx *c, const double2 *U, const double2 *Up, float *out);
// h[b] = ys (n(z_b) - n(swap z_b)) / 2 for rows z_b = feats[b * 64 ..]
void mlp_predict(psms_ctx *c, const float *feats, int B, float *h_out);
// throws PSMS_ETIMEOUT if a tensor-core GEMM's bounded wait ran out since the
// last check (synchronises the stream)
void mlp_check(psms_ctx *c);

}  // namespace psms
