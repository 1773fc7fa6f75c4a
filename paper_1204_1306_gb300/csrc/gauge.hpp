// Gauge-field kernel interfaces.
#pragma once

#include "kernels.hpp"

namespace psms {

void link_init(psms_ctx *c, double2 *U, double eps, uint64_t seed);
// returns the number of SU(2) draws that hit the attempt limit
int gauge_sweep(psms_ctx *c, double2 *U, int active_set, int n_iter, int n_or, double beta, uint64_t seed,
                uint64_t sweep0);
void plaquette_sum(psms_ctx *c, const double2 *U, double *d_out);
void translate(psms_ctx *c, const double2 *src, double2 *dst, const int sh[4]);
void interpolate(psms_ctx *c, const double2 *U, const double2 *Up, double2 *out64, float2 *out32, int N, int i0, int n);
void links_to_f32(psms_ctx *c, const double2 *a, float2 *b, long long n_el);
void merge_blocks(psms_ctx *c, const double2 *old, const double2 *prop, double2 *dst, const int *d_accept);
void gauge_canonical(psms_ctx *c, const double2 *canon, double2 *U, int to_internal);
void spinor_canonical(psms_ctx *c, const double2 *canon, void *nat, int prec, int to_native);

}  // namespace psms
