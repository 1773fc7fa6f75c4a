// Kernels of one level of HYP smearing and of the block HYP plaquette
// action (App. C, Sec. 5); the per-link arithmetic is in hyp.cuh.
//
// Each smearing level is one launch with a thread per (decorated field,
// site): 12 fields at levels 3 and 2 (direction mu times the one extra
// direction that labels the decoration), 4 at level 1.  The levels keep
// their fields in scratch in the links' layout [field][element][site]; a
// level reads the previous one at its own site and at the three neighbours
// of each staple.  FP64 throughout: the fat links feed an exact filter
// level whose Delta is compared across devices.
#include "hyp.cuh"
#include "hyp.hpp"

namespace psms {
namespace {

struct DevLd {
    Geom g;
    const double2 *U, *F3, *F2, *F1;

    __device__ hyp::M operator()(int lev, int mu, int k, const int x[4]) const {
        int y[4];
        for (int m = 0; m < 4; ++m) {
            y[m] = x[m];
            if (y[m] < 0) y[m] += g.L[m];
            if (y[m] >= g.L[m]) y[m] -= g.L[m];
        }
        const long long s = site_index(g, y);
        const double2 *base = U;
        int f = mu;
        if (lev == 3) {
            base = F3;
            f = hyp::key_of(mu, k);
        } else if (lev == 2) {
            base = F2;
            f = hyp::key_of(mu, k);
        } else if (lev == 1) {
            base = F1;
        }
        const double2 *q = base + (long long)f * 9 * g.V + s;
        hyp::M m;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                const double2 v = q[(long long)(3 * a + b) * g.V];
                m.e[a][b] = {v.x, v.y};
            }
        return m;
    }
};

__global__ void hyp_level_kernel(Geom g, const BlockInfo *binfo, int lev, int n_keys, const double2 *U,
                                 const double2 *F3, const double2 *F2, double2 *out, double a1, double a2,
                                 double a3) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)n_keys * g.V) return;
    const int key = (int)(t / g.V);
    const long long s = t - (long long)key * g.V;
    int p, r, j, y[4], x[4];
    decode(g, binfo, s, p, r, j, y, x);
    const int mu = lev == 1 ? key : key / 3;
    const int k = lev == 1 ? 0 : hyp::dir_of_key(key);
    const DevLd ld{g, U, F3, F2, nullptr};
    const hyp::M m = hyp::fat_link(ld, lev, mu, k, x, a1, a2, a3);
    double2 *q = out + (long long)key * 9 * g.V + s;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) q[(long long)(3 * a + b) * g.V] = make_double2(m.e[a][b].re, m.e[a][b].im);
}

constexpr int kActNT = 128;

// one CTA per block (rank); fixed-order reduction, so the sums are
// reproducible bit for bit
__global__ void __launch_bounds__(kActNT) hyp_block_action_kernel(Geom g, const BlockInfo *binfo,
                                                                  const double2 *F1, double *out) {
    __shared__ double sh[kActNT / 32];
    const int r = blockIdx.x;
    const DevLd ld{g, nullptr, nullptr, nullptr, F1};
    double acc = 0.0;
    for (int t = threadIdx.x; t < 2 * g.Vbh; t += kActNT) {
        const int p = t >= g.Vbh ? 1 : 0;
        const int j = t - p * g.Vbh;
        int y[4], x[4];
        local_lex(g, p, j, y);
        for (int m = 0; m < 4; ++m) x[m] = binfo[r].B[m] * g.l[m] + y[m];
        for (int mu = 0; mu < 4; ++mu)
            for (int nu = mu + 1; nu < 4; ++nu)
                if (y[mu] <= g.l[mu] - 2 && y[nu] <= g.l[nu] - 2) acc += hyp::plaquette_term(ld, 1, mu, nu, x);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < kActNT / 32; ++w) tot += sh[w];
        out[binfo[r].lex] = tot;
    }
}

}  // namespace

double2 *hyp_smear(psms_ctx *c, const double2 *U, const double alpha[3], double2 *out) {
    const long long V = c->g.V;
    double2 *F3 = (double2 *)scratch(c, "hyp_f3", sizeof(double2) * 12 * 9 * V);
    double2 *F2 = (double2 *)scratch(c, "hyp_f2", sizeof(double2) * 12 * 9 * V);
    double2 *F1 = out ? out : (double2 *)scratch(c, "hyp_f1", sizeof(double2) * 4 * 9 * V);
    const int NT = 128;
    const int levels[3] = {3, 2, 1};
    for (int lev : levels) {
        const int n_keys = lev == 1 ? 4 : 12;
        double2 *dst = lev == 3 ? F3 : (lev == 2 ? F2 : F1);
        const long long n = (long long)n_keys * V;
        hyp_level_kernel<<<(unsigned)((n + NT - 1) / NT), NT, 0, c->stream>>>(
            c->g, c->d_binfo, lev, n_keys, U, F3, F2, dst, alpha[0], alpha[1], alpha[2]);
        PSMS_LAUNCH_CHECK("hyp_level");
    }
    return F1;
}

void hyp_block_action(psms_ctx *c, const double2 *U, const double alpha[3], double *d_out) {
    const double2 *F1 = hyp_smear(c, U, alpha, nullptr);
    hyp_block_action_kernel<<<c->g.nblocks, kActNT, 0, c->stream>>>(c->g, c->d_binfo, F1, d_out);
    PSMS_LAUNCH_CHECK("hyp_block_action");
}

}  // namespace psms
