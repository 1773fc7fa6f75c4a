// Exact determinants of the Dirichlet block operators (Sec. 3: the paper
// computes small-block determinants exactly by LU; Tables 1 and 2 put
// coefficients on this exact action).
//
// For a block b, D_b = [[A, D_eo], [D_oe, A]] over its even and odd sites
// (A = 4 + m0, D_eo = -H_eo / 2 the hops of Eq. (Dw) that stay in the block),
// so det D_b = A^{n_e} det(A - D_oe D_eo / A): the even-odd reduced operator
// Dhat_b on the block's odd sites, an n x n complex matrix with
// n = 12 Vb / 2 (1536 for a 4^4 block).  For all blocks of a batch:
//   1. assemble Dhat_b column by column (a thread per column applies the two
//      hops to a unit vector and scatters the result; column-major storage);
//   2. LU with partial pivoting, right-looking in panels of width kNb (16):
//      lu_panel_kernel (one CTA per matrix) factors the panel, swaps rows
//      across the trailing columns and solves for the panel's block row of
//      U; lu_update_kernel subtracts L21 U12 from the trailing matrix in
//      64 x 64 tiles staged through shared memory (GB300's FP64 rate, not
//      memory, bounds it: 16 complex FMAs per element and panel);
//   3. ln|det D_b| = n_e ln A + sum_j ln|u_jj|, summed in a fixed order.
// FP64 throughout: the level built on it is exact, and its Delta is
// compared across devices.
#include <cmath>
#include <string>
#include <vector>

#include "blockdet.hpp"

namespace psms {
namespace {

constexpr int kNb = 16;       // panel width (two 16 x 64 complex tiles fit the static shared memory)
constexpr int kPanelNT = 512;
constexpr int kTile = 64;     // trailing-update tile (rows and columns)
constexpr int kUpdNT = 256;   // 16 x 16 threads, 4 x 4 outputs each
constexpr int kMaxBlockSites = 1024;  // n <= 6144: at most 0.6 GB and 6e11 flop per block

__device__ __forceinline__ cpx<double> ld(const double2 *p) {
    const double2 v = *p;
    return {v.x, v.y};
}
__device__ __forceinline__ void st(double2 *p, cpx<double> v) { *p = make_double2(v.re, v.im); }

// Column col of Dhat_b for rank r = rank_lo + blockIdx-derived matrix index.
// Row / column index of (odd site with half-block index j, component c):
// 12 j + c.
__global__ void assemble_kernel(Geom g, const BlockInfo *binfo, const double2 *U, int rank_lo, int n_mat, double A,
                                double2 *M) {
    const int n = 12 * g.Vbh;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)n_mat * n) return;
    const int m = (int)(t / n), col = (int)(t - (long long)m * n);
    const int r = rank_lo + m;
    const BlockInfo &bi = binfo[r];
    double2 *out = M + (long long)m * n * n + (long long)col * n;  // zeroed by the caller
    const int jy = col / 12, cy = col % 12;
    int y[4];
    const int lly = local_lex(g, 1, jy, y);
    const long long sy = (long long)g.Vh + (long long)r * g.Vbh + jy;
    Spinor<double> e;
    zero(e);
    e.c[cy / 3][cy % 3] = mk<double>(1.0, 0.0);
    const double f = -0.25 / A;  // -(1/A) (1/2)(1/2): Dhat = A - (H_oe/2)(H_eo/2)/A
    for (int mu = 0; mu < 4; ++mu)
        for (int sg = -1; sg <= 1; sg += 2) {
            // w = (H e)(z) at the even neighbour z = y + sg mu inside the block
            long long sz;
            int bsg;
            if (!neighbour(g, bi, r, 1, y, lly, mu, sg, HOP_INTRA, sz, bsg)) continue;
            Spinor<double> w;
            zero(w);
            if (sg > 0) {  // z - mu = y: backward term U(y,mu)^dag (1 + gamma_mu) e
                const Half<double> h = su3_dag_mul(load_link<Store<double>>(U, g.V, mu, sy), project(mu, 1.0, e));
                reconstruct_add(mu, 1.0, h, w);
            } else {       // z + mu = y: forward term U(z,mu) (1 - gamma_mu) e
                const Half<double> h = su3_mul(load_link<Store<double>>(U, g.V, mu, sz), project(mu, -1.0, e));
                reconstruct_add(mu, -1.0, h, w);
            }
            int z[4] = {y[0], y[1], y[2], y[3]};
            z[mu] += sg;
            const int llz = lly + sg * g.lstride[mu];
            for (int nu = 0; nu < 4; ++nu)
                for (int sh = -1; sh <= 1; sh += 2) {
                    long long sx;
                    int bsx;
                    if (!neighbour(g, bi, r, 0, z, llz, nu, sh, HOP_INTRA, sx, bsx)) continue;
                    Spinor<double> v;
                    zero(v);
                    if (sh > 0) {  // x - nu = z: U(z,nu)^dag (1 + gamma_nu) w
                        const Half<double> h =
                            su3_dag_mul(load_link<Store<double>>(U, g.V, nu, sz), project(nu, 1.0, w));
                        reconstruct_add(nu, 1.0, h, v);
                    } else {       // x + nu = z: U(x,nu) (1 - gamma_nu) w
                        const Half<double> h = su3_mul(load_link<Store<double>>(U, g.V, nu, sx), project(nu, -1.0, w));
                        reconstruct_add(nu, -1.0, h, v);
                    }
                    const int jx = (int)(sx - (long long)g.Vh - (long long)r * g.Vbh);
                    double2 *o = out + 12 * jx;
#pragma unroll
                    for (int q = 0; q < 12; ++q) {
                        const cpx<double> a = ld(o + q);
                        st(o + q, a + f * v.c[q / 3][q % 3]);
                    }
                }
        }
    double2 *d = out + col;
    const cpx<double> a = ld(d);
    st(d, a + mk<double>(A, 0.0));
}

// deterministic argmax of |a|^2 over a CTA: larger value wins, the lower
// row index on ties
__device__ __forceinline__ void argmax_pair(double &v, int &i, double v2, int i2) {
    if (v2 > v || (v2 == v && i2 < i)) {
        v = v2;
        i = i2;
    }
}

// Panel k (columns [k, k + w), w = min(kNb, n - k)) of matrix blockIdx.x:
// partial pivoting, row swaps over columns [k, n), multipliers, the rank-1
// updates inside the panel, then U12 = L11^-1 A12 for the trailing columns.
// logu[m * n + j] = ln|u_jj|.
__global__ void __launch_bounds__(kPanelNT) lu_panel_kernel(double2 *Mall, int n, int k, double *logu) {
    __shared__ double sv[kPanelNT / 32];
    __shared__ int si[kPanelNT / 32];
    __shared__ int piv_s;
    __shared__ double2 L11[kNb * kNb];
    const int m = blockIdx.x, tid = threadIdx.x;
    double2 *M = Mall + (long long)m * n * n;
    const int w = min(kNb, n - k);
    for (int jj = 0; jj < w; ++jj) {
        const int j = k + jj;
        double2 *cj = M + (long long)j * n;
        // pivot search in column j, rows [j, n)
        double bv = -1.0;
        int bi = n;
        for (int i = j + tid; i < n; i += kPanelNT) {
            const double2 a = cj[i];
            argmax_pair(bv, bi, a.x * a.x + a.y * a.y, i);
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double v2 = __shfl_xor_sync(0xffffffffu, bv, o);
            const int i2 = __shfl_xor_sync(0xffffffffu, bi, o);
            argmax_pair(bv, bi, v2, i2);
        }
        if ((tid & 31) == 0) {
            sv[tid >> 5] = bv;
            si[tid >> 5] = bi;
        }
        __syncthreads();
        if (tid == 0) {
            double v = sv[0];
            int i = si[0];
            for (int q = 1; q < kPanelNT / 32; ++q) argmax_pair(v, i, sv[q], si[q]);
            piv_s = i;
        }
        __syncthreads();
        const int p = piv_s;
        // swap rows j and p over columns [k, n)
        if (p != j && p < n)
            for (int c = k + tid; c < n; c += kPanelNT) {
                double2 *cc = M + (long long)c * n;
                const double2 t = cc[j];
                cc[j] = cc[p];
                cc[p] = t;
            }
        __syncthreads();
        const double2 pv = cj[j];
        const double pn = pv.x * pv.x + pv.y * pv.y;
        if (tid == 0) logu[(long long)m * n + j] = 0.5 * log(pn);
        // multipliers l_ij = a_ij / u_jj (a singular pivot gives non-finite values the host detects)
        const cpx<double> inv = {pv.x / pn, -pv.y / pn};
        for (int i = j + 1 + tid; i < n; i += kPanelNT) st(cj + i, cmul(ld(cj + i), inv));
        __syncthreads();
        // rank-1 update of the panel columns to the right of j
        const int rows = n - j - 1, cols = w - jj - 1;
        for (long long q = tid; q < (long long)rows * cols; q += kPanelNT) {
            const int i = j + 1 + (int)(q % rows);
            const int c = j + 1 + (int)(q / rows);
            double2 *cc = M + (long long)c * n;
            const cpx<double> u = ld(cc + j);
            st(cc + i, ld(cc + i) - cmul(ld(cj + i), u));
        }
        __syncthreads();
    }
    // U12 = L11^-1 A12: forward substitution with the unit lower L11 for
    // every trailing column (a thread per column)
    for (int q = tid; q < w * w; q += kPanelNT) {
        const int rr = q % w, cc = q / w;
        L11[rr * kNb + cc] = M[(long long)(k + cc) * n + k + rr];
    }
    __syncthreads();
    for (int c = k + w + tid; c < n; c += kPanelNT) {
        double2 *col = M + (long long)c * n + k;
        cpx<double> x[kNb];
        for (int rr = 0; rr < w; ++rr) x[rr] = ld(col + rr);
        for (int rr = 1; rr < w; ++rr) {
            cpx<double> s = x[rr];
            for (int q = 0; q < rr; ++q) {
                const double2 l = L11[rr * kNb + q];
                s = s - cmul(mk<double>(l.x, l.y), x[q]);
            }
            x[rr] = s;
        }
        for (int rr = 1; rr < w; ++rr) st(col + rr, x[rr]);
    }
}

// A22 -= L21 U12 on the trailing matrix [k + w, n) x [k + w, n):
// tile (blockIdx.x: rows, blockIdx.y: columns) of matrix blockIdx.z
__global__ void __launch_bounds__(kUpdNT) lu_update_kernel(double2 *Mall, int n, int k, int w) {
    __shared__ double2 Ls[kNb][kTile];  // Ls[q][i]: L21 rows of the tile
    __shared__ double2 Us[kNb][kTile];  // Us[q][c]: U12 columns of the tile
    const int m = blockIdx.z;
    double2 *M = Mall + (long long)m * n * n;
    const int t0 = k + w;
    const int i0 = t0 + blockIdx.x * kTile, c0 = t0 + blockIdx.y * kTile;
    const int tid = threadIdx.x;
    for (int q = tid; q < w * kTile; q += kUpdNT) {
        const int qq = q / kTile, ii = q % kTile;
        const int i = i0 + ii;
        Ls[qq][ii] = i < n ? M[(long long)(k + qq) * n + i] : make_double2(0.0, 0.0);
        const int c = c0 + ii;
        Us[qq][ii] = c < n ? M[(long long)c * n + k + qq] : make_double2(0.0, 0.0);
    }
    __syncthreads();
    const int tr = tid % 16, tc = tid / 16;  // rows tr + 16 a, columns tc + 16 b
    cpx<double> acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = mk<double>(0.0, 0.0);
    for (int q = 0; q < w; ++q) {
        cpx<double> l[4], u[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const double2 v = Ls[q][tr + 16 * a];
            l[a] = {v.x, v.y};
            const double2 z = Us[q][tc + 16 * a];
            u[a] = {z.x, z.y};
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] = cfma(l[a], u[b], acc[a][b]);
    }
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        const int c = c0 + tc + 16 * b;
        if (c >= n) continue;
        double2 *col = M + (long long)c * n;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const int i = i0 + tr + 16 * a;
            if (i < n) st(col + i, ld(col + i) - acc[a][b]);
        }
    }
}

// out[lex(rank_lo + m)] = n_e ln A + sum_j logu[m * n + j] (fixed order)
__global__ void logdet_sum_kernel(const BlockInfo *binfo, const double *logu, int n, int n_mat, int rank_lo,
                                  double base, double *out) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n_mat) return;
    double s = base;
    for (int j = 0; j < n; ++j) s += logu[(long long)m * n + j];
    out[binfo[rank_lo + m].lex] = s;
}

}  // namespace

int block_logdet_batch(const psms_ctx *c) {
    const long long n = 12LL * c->g.Vbh;
    const double per = 16.0 * (double)n * (double)n;
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    const double budget = std::min(8e9, 0.25 * (double)tot);
    int k = (int)(budget / per);
    if (c->max_chunk > 0) k = std::min(k, c->max_chunk);
    return std::max(1, std::min(k, c->g.nblocks));
}

void block_logdet(psms_ctx *c, const double2 *U, double *d_out) {
    const Geom &g = c->g;
    if (2 * g.Vbh > kMaxBlockSites)
        fail(PSMS_EINVAL, "exact block determinants are for blocks of at most " + std::to_string(kMaxBlockSites) +
                              " sites (Sec. 3: small blocks)");
    const int n = 12 * g.Vbh;
    const int batch = block_logdet_batch(c);
    double2 *M = (double2 *)scratch(c, "bd_mat", sizeof(double2) * (size_t)n * n * batch);
    double *logu = (double *)scratch(c, "bd_logu", sizeof(double) * (size_t)n * batch);
    const double base = 12.0 * g.Vbh * std::log(c->A);
    for (int r0 = 0; r0 < g.nblocks; r0 += batch) {
        const int nm = std::min(batch, g.nblocks - r0);
        const long long nt = (long long)nm * n;
        cuda_check(cudaMemsetAsync(M, 0, sizeof(double2) * (size_t)n * n * nm, c->stream), "blockdet memset");
        assemble_kernel<<<(unsigned)((nt + 127) / 128), 128, 0, c->stream>>>(g, c->d_binfo, U, r0, nm, c->A, M);
        PSMS_LAUNCH_CHECK("blockdet assemble");
        for (int k = 0; k < n; k += kNb) {
            const int w = std::min(kNb, n - k);
            lu_panel_kernel<<<nm, kPanelNT, 0, c->stream>>>(M, n, k, logu);
            PSMS_LAUNCH_CHECK("blockdet panel");
            const int rest = n - k - w;
            if (rest > 0) {
                const unsigned tiles = (unsigned)((rest + kTile - 1) / kTile);
                lu_update_kernel<<<dim3(tiles, tiles, nm), kUpdNT, 0, c->stream>>>(M, n, k, w);
                PSMS_LAUNCH_CHECK("blockdet update");
            }
        }
        logdet_sum_kernel<<<(nm + 127) / 128, 128, 0, c->stream>>>(c->d_binfo, logu, n, nm, r0, base, d_out);
        PSMS_LAUNCH_CHECK("blockdet sum");
    }
}

}  // namespace psms
