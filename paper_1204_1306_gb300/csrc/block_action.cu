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

__global__ void combine_kernel(const double *ds, double beta, const double *h, double *out, int nb) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nb) out[b] = beta * ds[b] - (h ? h[b] : 0.0);
}

}  // namespace

void block_action_change(psms_ctx *c, const double2 *U, const double2 *Up, double *d_out) {
    block_change_kernel<<<c->g.nblocks, kNT, 0, c->stream>>>(c->g, c->d_binfo, U, Up, d_out);
    PSMS_LAUNCH_CHECK("block_action_change");
}

void block_extra(psms_ctx *c, const double *d_ds, double beta, const double *d_h, double *d_out) {
    const int nb = c->g.nblocks;
    combine_kernel<<<(nb + 127) / 128, 128, 0, c->stream>>>(d_ds, beta, d_h, d_out, nb);
    PSMS_LAUNCH_CHECK("block_extra");
}

}  // namespace psms
