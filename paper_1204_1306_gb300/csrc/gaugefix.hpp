// Relative gauge fixing of a pair of gauge fields (Sec. 4.2, App. B).
#pragma once

#include "kernels.hpp"

namespace psms {

struct GaugeFixParams {
    double alpha0 = 0.15, alpha_min = 0.10, dalpha = 0.01, theta_tol = 1e-3;
    int max_iter = 1000;
    int prec = P32;  // arithmetic of the iteration (P64 or P32)
};

// device results of the last gauge_fix_pair (context scratch, valid until
// the next call): transformations G1, G2 ([e][s], FP64, identity off the
// block interiors) and per-block (lexicographic order) steps, alpha, mean
// theta and canonical swap flag
struct GaugeFixInfo {
    double2 *G1 = nullptr, *G2 = nullptr;
    int *d_steps = nullptr;
    double *d_alpha = nullptr, *d_theta = nullptr;
    int *d_swap = nullptr;
};

// out0 = U^{g_1}, outN = U'^{g_2} (FP64, internal layout).  out0 may alias
// U and outN may alias Up; out0 must not alias Up nor outN alias U.
void gauge_fix_pair(psms_ctx *c, const double2 *U, const double2 *Up, double2 *out0, double2 *outN,
                    const GaugeFixParams &prm, GaugeFixInfo *info);
// canonical [lex][3][3] complex copy of an [e][s] transformation field
void gauge_fix_export(psms_ctx *c, const double2 *G, double2 *canon);

}  // namespace psms
