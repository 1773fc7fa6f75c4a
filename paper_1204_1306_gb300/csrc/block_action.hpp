// Per-block change of the plaquette action (App. C beta terms, block level).
#pragma once

#include "kernels.hpp"

namespace psms {

// dS_w,b (Eq. (Sw) without beta) of U -> Up for every block, lexicographic
// block index, into d_out[n_blocks]; plaquettes attributed to the block of
// their first changed link (block_action.cuh)
void block_action_change(psms_ctx *c, const double2 *U, const double2 *Up, double *d_out);
// d_out[b] = a x[b] + b y[b] + e z[b], null terms left out (in that order)
void block_lincomb(psms_ctx *c, double a, const double *x, double b, const double *y, double e, const double *z,
                   double *d_out);

}  // namespace psms
