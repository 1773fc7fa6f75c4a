// Exact determinants of the Dirichlet block operators (Sec. 3).
#pragma once

#include "kernels.hpp"

namespace psms {

// ln|det D_b(U)| for every block into d_out[n_blocks] (lexicographic block
// index): batched FP64 LU of the even-odd reduced block operators
void block_logdet(psms_ctx *c, const double2 *U, double *d_out);
// blocks factorised per batch (device-memory estimate, psms_max_chunk cap)
int block_logdet_batch(const psms_ctx *c);

}  // namespace psms
