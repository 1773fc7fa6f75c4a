// Kernel launch interfaces shared between the translation units.
#pragma once

#include "ctx.hpp"

namespace psms {

// A batch of fields in the structure-of-arrays layout: system k, component c,
// internal site s live at p[k * bs + c * cs + (s - off)].  Full-lattice
// fields have cs = V, off = 0; single-parity fields cs = V/2, off = parity*V/2.
template <class E>
struct View {
    E *p = nullptr;
    long long cs = 0, off = 0, bs = 0;
};

enum Prec : int { P64 = PSMS_PREC_F64, P32 = PSMS_PREC_F32, PB16 = PSMS_PREC_BF16 };

// FP32 links of system k given as a_k U0 + b_k U1 of two endpoint fields
// (Eq. (gfparam): every interpolation step's links lie on the line between
// the endpoints), formed in the hop instead of read from a materialised
// field per system.  Links where U0 and U1 agree (flag 0: outside the
// updated blocks) are read from U0 alone.  A launch then walks its systems
// fastest, so all systems read each endpoint link from HBM about once and
// from L2 afterwards.
struct LinkInterp {
    const float2 *U0 = nullptr, *U1 = nullptr;  // canonical FP32 link layout
    const float2 *ab = nullptr;                 // device, per system: (a_k, b_k)
    const unsigned char *flag = nullptr;        // device, per link mu * V + s
};

struct BCS;
// A BiCGStab reduction fused into a single-parity hop (FP32 storage):
// dot = 1 sums conj(x) out (x = the vector `x`), dot = 2 sums conj(out) y and
// |out|^2; per-CTA partials go to re/im/aa (n_cta per system) and the last
// CTA of each system applies the scalar `stage` to st (counters cnt).
struct HopDot {
    int dot = 0;
    View<void> x;
    BCS *st = nullptr;
    double *re = nullptr, *im = nullptr, *aa = nullptr;
    unsigned int *cnt = nullptr;
    int stage = 0, maxit = 0;
    int *flags = nullptr;
};

// out = a*y + a2*y2 + b*H(in), H the hopping term of Eq. (Dw) (sum over the
// 8 neighbours of U (1 -/+ gamma) psi), restricted by `mode`, for output
// parity p (-1: both) on the blocks of rank [rank_lo, rank_lo + n_ranks).
// Batched over gridDim.y = n_sys systems with per-system strides.  Optional
// per-CTA partial sums of |out|^2 in partial[k * n_cta + cta].
struct HopCall {
    int prec = P64;  // storage of in/out/y/y2 (links: FP64 for P64, FP32 otherwise)
    View<void> in, out, y, y2;
    double a = 0, a2 = 0, b = 1;
    const void *U = nullptr;
    long long U_bs = 0;
    int p = -1, rank_lo = 0, n_ranks = -1, mode = HOP_ALL, dag = 0, n_sys = 1;
    const int *active = nullptr;
    double *partial = nullptr;
    // optional list of the systems to launch (device, n_map entries): the
    // launch covers only them (system k = sys_map[blockIdx.y])
    const int *sys_map = nullptr;
    int n_map = 0;
    // optional per-rank flags (device): output sites of ranks flagged 0 are
    // skipped (left unwritten)
    const int *rank_active = nullptr;
    // optional shared-endpoint FP32 links (replace U / U_bs; FP32 links only)
    LinkInterp li;
    // optional fused BiCGStab reduction of the output
    HopDot dot;
};
// returns the number of CTAs per system (for the partial sums)
int hop_launch(psms_ctx *c, const HopCall &h);
int hop_ctas(psms_ctx *c, const HopCall &h);

// deterministic reductions: sums partial[k * n + i] over i -> out[k]
void reduce_partials(psms_ctx *c, const double *partial, int n, int n_sys, double *out);
// sum_{c,s} |v|^2 per system over internal sites [s_lo, s_lo + n) (one parity
// range or a whole field), FP64 result out[k]
void norm2_batch(psms_ctx *c, int prec, View<void> v, long long s_lo, long long n, int n_sys, double *out);

}  // namespace psms
