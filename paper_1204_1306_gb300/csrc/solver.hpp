// Requests for the block and whole-lattice solvers.
#pragma once

#include "kernels.hpp"

namespace psms {

// Solve D_b x = b for the blocks of rank [rank_lo, rank_lo + n_ranks) of
// n_sys systems (system k uses links U64 + k*U64_bs / U32 + k*U64_bs).
// Outputs per (system, block): iterations, relative true residual,
// |x_block|^2 (nullable) and status (0 ok, 1 not converged).
struct BlockSolveReq {
    int rank_lo = 0, n_ranks = 0, n_sys = 1;
    View<double2> b, x;
    const double2 *U64 = nullptr;
    const float2 *U32 = nullptr;
    long long U64_bs = 0;  // elements (complex) between the systems' link fields
    double tol = 1e-13;
    int maxit = 100000;
    int inner_prec = P64;
    const int *sys_active = nullptr;
    const int *block_active = nullptr;  // per lexicographic block (nullable)
    int *iters = nullptr;
    double *resid = nullptr;
    double *xnorm2 = nullptr;
    int *status = nullptr;
};
void block_solve(psms_ctx *c, const BlockSolveReq &q);

// Solve D x = b on the whole lattice for n_sys systems.
struct FullSolveReq {
    int n_sys = 1;
    View<double2> b, x;
    const double2 *U64 = nullptr;
    const float2 *U32 = nullptr;
    long long U64_bs = 0;
    double tol = 1e-13;
    int maxit = 100000;
    int inner_prec = P64;
    double *rel_out = nullptr;  // device, per system (nullable)
    // per rank (device, nullable): the operator is block-diagonal between the
    // flagged and unflagged ranks (links across are zero) and b vanishes on
    // the unflagged ones, so x vanishes there too and those sites are skipped
    const int *rank_active = nullptr;
    // optional: the FP32/BF16 inner iterations take system k's links as
    // a_k U0 + b_k U1 of two shared FP32 endpoint fields (U32 unused)
    LinkInterp li32;
};
void solve_full_batch(psms_ctx *c, const FullSolveReq &q, psms_solve_info *info);

}  // namespace psms
