// Per-block change of the plaquette action between a field and its proposal
// (the beta terms of App. C at the block level); arithmetic in
// block_action.cuh.  One CTA per block with a fixed-order reduction, so the
// sums are reproducible bit for bit.
#include "block_action.cuh"
#include "block_action.hpp"

namespace psms {
namespace {

struct PairLd {
    Geom g;
    const double2 *U0, *U1;

    __device__ hyp::M operator()(int f, int mu, const int x[4]) const {
        int y[4];
        for (int m = 0; m < 4; ++m) y[m] = act::wrap(x[m], g.L[m]);
        const long long s = site_index(g, y);
        const double2 *q = (f ? U1 : U0) + (long long)mu * 9 * g.V + s;
        hyp::M m;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                const double2 v = q[(long long)(3 * a + b) * g.V];
                m.e[a][b] = {v.x, v.y};
            }
        return m;
    }
};

constexpr int kNT = 128;

__global__ void __launch_bounds__(kNT) block_change_kernel(Geom g, const BlockInfo *binfo, const double2 *U0,
                                                           const double2 *U1, double *out) {
    __shared__ double sh[kNT / 32];
    const int r = blockIdx.x;
    act::Grid gr;
    for (int m = 0; m < 4; ++m) {
        gr.L[m] = g.L[m];
        gr.l[m] = g.l[m];
        gr.nb[m] = g.nb[m];
    }
    const PairLd ld{g, U0, U1};
    double acc = act::block_change_partial(ld, gr, binfo[r].B, binfo[r].lex, threadIdx.x, kNT);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < kNT / 32; ++w) tot += sh[w];
        out[binfo[r].lex] = tot;
    }
}

__global__ void lincomb_kernel(double a, const double *x, double b, const double *y, double e, const double *z,
                               double *out, int nb) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nb) return;
    double v = 0.0;
    if (x) v += a * x[k];
    if (y) v += b * y[k];
    if (z) v += e * z[k];
    out[k] = v;
}

}  // namespace

void block_action_change(psms_ctx *c, const double2 *U, const double2 *Up, double *d_out) {
    block_change_kernel<<<c->g.nblocks, kNT, 0, c->stream>>>(c->g, c->d_binfo, U, Up, d_out);
    PSMS_LAUNCH_CHECK("block_action_change");
}

void block_lincomb(psms_ctx *c, double a, const double *x, double b, const double *y, double e, const double *z,
                   double *d_out) {
    const int nb = c->g.nblocks;
    lincomb_kernel<<<(nb + 127) / 128, 128, 0, c->stream>>>(a, x, b, y, e, z, d_out, nb);
    PSMS_LAUNCH_CHECK("block_lincomb");
}

}  // namespace psms
