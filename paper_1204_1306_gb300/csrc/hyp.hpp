// HYP-smeared links and the block HYP plaquette action (App. C, Sec. 5).
#pragma once

#include "kernels.hpp"

namespace psms {

// Fat links of one level of HYP smearing of U (internal layout [mu][e][s])
// into `out` (same layout); alpha = (a1, a2, a3).  Returns the device
// pointer it wrote (out, or a context scratch buffer when out is null).
double2 *hyp_smear(psms_ctx *c, const double2 *U, const double alpha[3], double2 *out);
// S_HYP,b per block (lexicographic block index) into d_out[n_blocks]:
// Eq. (Sw) on the fat links over the plaquettes with all four corners in b.
void hyp_block_action(psms_ctx *c, const double2 *U, const double alpha[3], double *d_out);

}  // namespace psms
