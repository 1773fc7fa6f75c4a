// Recursive domain decomposition (Eq. (ddrec)): outer blocks tiled by the
// context's blocks.
#pragma once

#include "kernels.hpp"

namespace psms {

bool has_outer(const psms_ctx *c);
// d_flag[b] (lexicographic block index) = 1 when a link starting in block b
// differs between U and Up, else 0
void block_changed(psms_ctx *c, const double2 *U, const double2 *Up, int *d_flag);
int n_outer(const psms_ctx *c);
// B = null or B[0] == 0 switches the outer level off
void set_outer(psms_ctx *c, const int *B);
// Stage 2: Delta contributions of the outer blocks' Schur complements,
// h_delta[b * N + i] (host, lexicographic outer block index b)
long long sub_level(psms_ctx *c, const double2 *U, const double2 *Up, int N, int mode, uint64_t seed,
                    uint64_t counter, double tol, int inner, double *h_delta);
// Global Schur complement of the outer decomposition, h_delta[i] (host)
long long outer_global_level(psms_ctx *c, const double2 *U, const double2 *Up, int N, int mode, uint64_t seed,
                             uint64_t counter, double tol, int inner, double *h_delta);

}  // namespace psms
