// Learned delayed-acceptance level: domain features (plaquettes and clover
// field strength per block) and a 64 -> 256 -> 256 -> 1 MLP with BF16
// tensor-core GEMMs and FP32 accumulation, trained on the GPU (forward,
// backward, AdamW).  The surrogate h = (n(f, f') - n(f', f))/2 is
// antisymmetric, so inserting it as a level with min{1, exp(-h)} and
// subtracting it at the next level keeps the chain exact (App. C: an
// auxiliary action whose coefficients sum to zero over the later levels).
#include <algorithm>
#include <cmath>
#include <numeric>
#include <random>
#include <vector>

#include "mlp.hpp"
#include "tc_gemm.cuh"

namespace psms {

// ---------------------------------------------------------------------------
// domain features, 32 per block (see oracle documentation of the same names)
// ---------------------------------------------------------------------------
using C = cpx<double>;
struct M3f {
    C e[3][3];
};

__device__ __forceinline__ C fcm(C a, C b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }

__device__ __forceinline__ M3f fmul(const M3f &a, const M3f &b) {
    M3f r;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            C z = fcm(a.e[i][0], b.e[0][j]);
            C z1 = fcm(a.e[i][1], b.e[1][j]);
            C z2 = fcm(a.e[i][2], b.e[2][j]);
            r.e[i][j] = {z.re + z1.re + z2.re, z.im + z1.im + z2.im};
        }
    return r;
}

__device__ __forceinline__ M3f fdag(const M3f &a) {
    M3f r;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) r.e[i][j] = {a.e[j][i].re, -a.e[j][i].im};
    return r;
}

__device__ __forceinline__ M3f fld(const double2 *U, const Geom &g, int mu, const int x[4], int d0, int m0, int d1,
                                   int m1) {
    int y[4] = {x[0], x[1], x[2], x[3]};
    y[m0] += d0;
    y[m1] += d1;
    for (int m = 0; m < 4; ++m) {
        if (y[m] < 0) y[m] += g.L[m];
        if (y[m] >= g.L[m]) y[m] -= g.L[m];
    }
    const long long s = site_index(g, y);
    M3f r;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double2 v = U[((long long)mu * 9 + 3 * a + b) * g.V + s];
            r.e[a][b] = {v.x, v.y};
        }
    return r;
}

template <int NT>
__device__ __forceinline__ double cta_sum_f(double v, double *sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0;
        for (int i = 0; i < NT / 32; ++i) t += sh[i];
        sh[NT / 32] = t;
    }
    __syncthreads();
    return sh[NT / 32];
}

template <int NT>
__global__ void __launch_bounds__(NT) features_kernel(Geom g, const BlockInfo *binfo, const double2 *U, float *out,
                                                      int stride, int offset) {
    __shared__ double sh[NT / 32 + 1];
    const int r = blockIdx.x;
    const BlockInfo &bi = binfo[r];
    const int Vb = 2 * g.Vbh;
    const int planes[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
    float *o = out + (long long)bi.lex * stride + offset;
    for (int k = 0; k < 6; ++k) {
        const int mu = planes[k][0], nu = planes[k][1];
        double s1 = 0, cnt = 0, s3 = 0, c3 = 0;
        // pass 1: plaquette mean and clover Tr F^2
        for (int ll = threadIdx.x; ll < Vb; ll += NT) {
            int y[4], rem = ll;
            for (int m = 3; m >= 0; --m) {
                y[m] = rem % g.l[m];
                rem /= g.l[m];
            }
            int x[4];
            for (int m = 0; m < 4; ++m) x[m] = bi.B[m] * g.l[m] + y[m];
            if (y[mu] < g.l[mu] - 1 && y[nu] < g.l[nu] - 1) {
                M3f P = fmul(fmul(fmul(fld(U, g, mu, x, 0, 0, 0, 0), fld(U, g, nu, x, 1, mu, 0, nu)),
                                  fdag(fld(U, g, mu, x, 1, nu, 0, mu))),
                             fdag(fld(U, g, nu, x, 0, 0, 0, 0)));
                s1 += (P.e[0][0].re + P.e[1][1].re + P.e[2][2].re) / 3.0;
                cnt += 1;
            }
            if (y[mu] >= 1 && y[mu] <= g.l[mu] - 2 && y[nu] >= 1 && y[nu] <= g.l[nu] - 2) {
                M3f Um = fld(U, g, mu, x, 0, 0, 0, 0), Un = fld(U, g, nu, x, 0, 0, 0, 0);
                M3f L1 = fmul(fmul(fmul(Um, fld(U, g, nu, x, 1, mu, 0, nu)), fdag(fld(U, g, mu, x, 1, nu, 0, mu))),
                              fdag(Un));
                M3f Umm = fld(U, g, mu, x, -1, mu, 0, nu);
                M3f L2 = fmul(fmul(fmul(Un, fdag(fld(U, g, mu, x, -1, mu, 1, nu))), fdag(fld(U, g, nu, x, -1, mu, 0, nu))),
                              Umm);
                M3f Unn = fld(U, g, nu, x, -1, nu, 0, mu);
                M3f L3 = fmul(fmul(fmul(fdag(Umm), fdag(fld(U, g, nu, x, -1, mu, -1, nu))), fld(U, g, mu, x, -1, mu, -1, nu)),
                              Unn);
                M3f L4 = fmul(fmul(fmul(fdag(Unn), fld(U, g, mu, x, -1, nu, 0, mu)), fld(U, g, nu, x, 1, mu, -1, nu)),
                              fdag(Um));
                M3f F;
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) {
                        C q = {L1.e[a][b].re + L2.e[a][b].re + L3.e[a][b].re + L4.e[a][b].re,
                               L1.e[a][b].im + L2.e[a][b].im + L3.e[a][b].im + L4.e[a][b].im};
                        C qt = {L1.e[b][a].re + L2.e[b][a].re + L3.e[b][a].re + L4.e[b][a].re,
                                -(L1.e[b][a].im + L2.e[b][a].im + L3.e[b][a].im + L4.e[b][a].im)};
                        // (Q - Q^dag) / (8 i)
                        C d = {q.re - qt.re, q.im - qt.im};
                        F.e[a][b] = {d.im / 8.0, -d.re / 8.0};
                    }
                C tr = {(F.e[0][0].re + F.e[1][1].re + F.e[2][2].re) / 3.0,
                        (F.e[0][0].im + F.e[1][1].im + F.e[2][2].im) / 3.0};
                for (int a = 0; a < 3; ++a) F.e[a][a] = {F.e[a][a].re - tr.re, F.e[a][a].im - tr.im};
                double t2 = 0;
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) {
                        C z = fcm(F.e[a][b], F.e[b][a]);
                        t2 += z.re;
                    }
                s3 += t2;
                c3 += 1;
            }
        }
        s1 = cta_sum_f<NT>(s1, sh);
        cnt = cta_sum_f<NT>(cnt, sh);
        s3 = cta_sum_f<NT>(s3, sh);
        c3 = cta_sum_f<NT>(c3, sh);
        const double mean = s1 / fmax(cnt, 1.0);
        // pass 2: variance
        double s2 = 0;
        for (int ll = threadIdx.x; ll < Vb; ll += NT) {
            int y[4], rem = ll;
            for (int m = 3; m >= 0; --m) {
                y[m] = rem % g.l[m];
                rem /= g.l[m];
            }
            if (!(y[mu] < g.l[mu] - 1 && y[nu] < g.l[nu] - 1)) continue;
            int x[4];
            for (int m = 0; m < 4; ++m) x[m] = bi.B[m] * g.l[m] + y[m];
            M3f P = fmul(fmul(fmul(fld(U, g, mu, x, 0, 0, 0, 0), fld(U, g, nu, x, 1, mu, 0, nu)),
                              fdag(fld(U, g, mu, x, 1, nu, 0, mu))),
                         fdag(fld(U, g, nu, x, 0, 0, 0, 0)));
            const double v = (P.e[0][0].re + P.e[1][1].re + P.e[2][2].re) / 3.0 - mean;
            s2 += v * v;
        }
        s2 = cta_sum_f<NT>(s2, sh);
        if (threadIdx.x == 0) {
            o[k] = (float)mean;
            o[6 + k] = (float)(s2 / fmax(cnt, 1.0));
            o[12 + k] = (float)(s3 / fmax(c3, 1.0));
        }
    }
    for (int k = 18 + threadIdx.x; k < 32; k += NT) o[k] = 0.0f;
}

void domain_features(psms_ctx *c, const double2 *U, float *out, int stride, int offset) {
    features_kernel<128><<<c->g.nblocks, 128, 0, c->stream>>>(c->g, c->d_binfo, U, out, stride, offset);
    PSMS_LAUNCH_CHECK("features_kernel");
}

// distance of two gauge fields on a block (the scalar product of Sec. 4.2,
// Eq. (sprodgf), restricted to the links starting in the block):
// d_b = sum_{x in b, mu} ReTr(1 - U(x,mu)^dagger U'(x,mu)) / (12 * 4 * Vb),
// written to slots 18 and 18 + 32 of the pair's row (same value in both
// halves, so the surrogate stays antisymmetric)
template <int NT>
__global__ void __launch_bounds__(NT) distance_kernel(Geom g, const BlockInfo *binfo, const double2 *U,
                                                      const double2 *Up, float *out) {
    __shared__ double sh[NT / 32 + 1];
    const int r = blockIdx.x;
    double acc = 0;
    for (int p = 0; p < 2; ++p)
        for (int j = threadIdx.x; j < g.Vbh; j += NT) {
            const long long s = (long long)p * g.Vh + (long long)r * g.Vbh + j;
            for (int mu = 0; mu < 4; ++mu) {
                double tr = 0;
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) {
                        const long long i = ((long long)mu * 9 + 3 * a + b) * g.V + s;
                        const double2 u = U[i], v = Up[i];
                        tr += u.x * v.x + u.y * v.y;  // Re(conj(U_ab) U'_ab)
                    }
                acc += 3.0 - tr;
            }
        }
    acc = cta_sum_f<NT>(acc, sh);
    if (threadIdx.x == 0) {
        const float d = (float)(acc / (12.0 * 4.0 * 2.0 * g.Vbh));
        const long long row = (long long)binfo[r].lex * 2 * N_FEAT;
        out[row + 18] = d;
        out[row + N_FEAT + 18] = d;
    }
}

void pair_features(psms_ctx *c, const double2 *U, const double2 *Up, float *out) {
    domain_features(c, U, out, 2 * N_FEAT, 0);
    domain_features(c, Up, out, 2 * N_FEAT, N_FEAT);
    distance_kernel<128><<<c->g.nblocks, 128, 0, c->stream>>>(c->g, c->d_binfo, U, Up, out);
    PSMS_LAUNCH_CHECK("distance_kernel");
}

// ---------------------------------------------------------------------------
// BF16 tensor-core GEMM: C[m][n] = alpha * sum_k A(m,k) B(n,k) + beta*C + bias[n]
// (optional ReLU and BF16 copy), FP32 accumulation in TMEM (tc_gemm.cuh).
// A(m,k) = A[m*sAm + k*sAk] (FP32 or BF16), B(n,k) likewise.
// ---------------------------------------------------------------------------
struct GemmArgs {
    int M, N, K;
    const void *A;
    long long sAm, sAk;
    int a_f32;
    const void *B;
    long long sBn, sBk;
    int b_f32;
    float *Cf;
    long long ldc;
    __nv_bfloat16 *Cb;
    long long ldcb;
    const float *bias;
    float alpha, beta;
    int relu;
};

template <int TN>
static void gemm_tn(psms_ctx *c, const tc::Args &t) {
    constexpr int smem = tc::smem_bytes<TN>();
    cuda_check(cudaFuncSetAttribute(tc::gemm_kernel<TN>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem),
               "tc gemm smem");
    dim3 grid((t.N + TN - 1) / TN, (t.M + tc::TM - 1) / tc::TM);
    tc::gemm_kernel<TN><<<grid, tc::NTHR, smem, c->stream>>>(t);
    PSMS_LAUNCH_CHECK("tc::gemm_kernel");
}

static void gemm(psms_ctx *c, const GemmArgs &a, int *err) {
    if (a.M < 1 || a.N < 1) return;
    const tc::Args t{a.M, a.N, a.K, a.A, a.sAm, a.sAk, a.a_f32, a.B, a.sBn, a.sBk, a.b_f32, a.Cf, a.ldc,
                     a.Cb, a.ldcb, a.bias, a.alpha, a.beta, a.relu, err};
    // N = 64 (the input layer's weight gradient) takes the narrow tile
    if (a.N <= 64)
        gemm_tn<64>(c, t);
    else
        gemm_tn<256>(c, t);
}

// ---------------------------------------------------------------------------
// MLP parameters (FP32 master) and kernels
// ---------------------------------------------------------------------------
// parameter block offsets (floats)
constexpr int NI = 64, NH = 256;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + NH * NI, OFF_W2 = OFF_B1 + NH, OFF_B2 = OFF_W2 + NH * NH,
              OFF_W3 = OFF_B2 + NH, OFF_B3 = OFF_W3 + NH, N_TRAIN = OFF_B3 + 1;
constexpr int OFF_MU = N_TRAIN, OFF_SIG = OFF_MU + NI, OFF_YS = OFF_SIG + NI, N_PARAM = OFF_YS + 1;

struct Mlp {
    float *p = nullptr;         // N_PARAM floats (trainable first, then normalisation)
    float *m = nullptr, *v = nullptr;  // Adam moments (N_TRAIN)
    float *g = nullptr;         // gradient (N_TRAIN)
    __nv_bfloat16 *w1b = nullptr, *w2b = nullptr;
    int *err = nullptr;  // set by a tensor-core GEMM whose bounded wait ran out
    long long step = 0;
};

static Mlp &mlp_of(psms_ctx *c) {
    if (!c->mlp) {
        Mlp *m = new Mlp();
        cuda_check(cudaMalloc(&m->p, sizeof(float) * N_PARAM), "mlp alloc");
        cuda_check(cudaMalloc(&m->m, sizeof(float) * N_TRAIN), "mlp alloc");
        cuda_check(cudaMalloc(&m->v, sizeof(float) * N_TRAIN), "mlp alloc");
        cuda_check(cudaMalloc(&m->g, sizeof(float) * N_TRAIN), "mlp alloc");
        cuda_check(cudaMalloc(&m->w1b, sizeof(__nv_bfloat16) * NH * NI), "mlp alloc");
        cuda_check(cudaMalloc(&m->w2b, sizeof(__nv_bfloat16) * NH * NH), "mlp alloc");
        cuda_check(cudaMalloc(&m->err, sizeof(int)), "mlp alloc");
        cuda_check(cudaMemset(m->err, 0, sizeof(int)), "mlp alloc");
        c->mlp = m;
        c->mlp_free = [](void *q) {
            Mlp *mm = (Mlp *)q;
            cudaFree(mm->p);
            cudaFree(mm->m);
            cudaFree(mm->v);
            cudaFree(mm->g);
            cudaFree(mm->w1b);
            cudaFree(mm->w2b);
            cudaFree(mm->err);
            delete mm;
        };
    }
    return *(Mlp *)c->mlp;
}

__global__ void mlp_init_kernel(float *p, uint64_t seed) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N_PARAM) return;
    float v = 0.f;
    auto normal = [&](int i) {
        uni4 u = uniforms(seed, 6, (uint64_t)i, 0, 0, 0);
        return (float)(sqrt(-2.0 * log(u.u[0])) * cos(2.0 * M_PI * u.u[1]));
    };
    if (t < OFF_B1) v = normal(t) * sqrtf(2.f / NI);
    else if (t >= OFF_W2 && t < OFF_B2) v = normal(t) * sqrtf(2.f / NH);
    else if (t >= OFF_W3 && t < OFF_B3) v = normal(t) * sqrtf(1.f / NH);
    else if (t >= OFF_SIG && t < OFF_YS) v = 1.f;
    else if (t == OFF_YS) v = 1.f;
    p[t] = v;
}

__global__ void to_bf16_kernel(const float *a, __nv_bfloat16 *b, int n) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) b[t] = __float2bfloat16(a[t]);
}

static void refresh_bf16(psms_ctx *c, Mlp &m) {
    to_bf16_kernel<<<(NH * NI + 255) / 256, 256, 0, c->stream>>>(m.p + OFF_W1, m.w1b, NH * NI);
    PSMS_LAUNCH_CHECK("to_bf16");
    to_bf16_kernel<<<(NH * NH + 255) / 256, 256, 0, c->stream>>>(m.p + OFF_W2, m.w2b, NH * NH);
    PSMS_LAUNCH_CHECK("to_bf16");
}

// X[r] = (z - mu)/sigma for rows r < B (z = feats[idx[r]]) and the swapped
// pair for rows B + r
__global__ void prep_kernel(const float *feats, const int *idx, int B, const float *p, float *X) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 2 * B * NI) return;
    const int row = t / NI, col = t % NI;
    const int b = row < B ? row : row - B;
    const int src = idx ? idx[b] : b;
    int cs = col;
    if (row >= B) cs = col < NI / 2 ? col + NI / 2 : col - NI / 2;
    const float z = feats[(long long)src * NI + cs];
    X[t] = (z - p[OFF_MU + col]) / p[OFF_SIG + col];
}

// n[r] = h2[r] . w3 + b3
__global__ void out_kernel(const float *H2, const float *p, int R, float *n) {
    const int r = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= R) return;
    float s = 0.f;
    for (int j = lane; j < NH; j += 32) s += H2[(long long)r * NH + j] * p[OFF_W3 + j];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) n[r] = s + p[OFF_B3];
}

// h = ys (n_a - n_b)/2 ; r = h - y ; dn_a = ys r / B (scaled so that the loss
// is the MSE of h), dn_b = -dn_a ; per-row squared residual
__global__ void loss_kernel(const float *n, const double *labels, const int *idx, int B, const float *p, float *dn,
                            float *res2, float *h_out) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const float ys = p[OFF_YS];
    const float h = ys * 0.5f * (n[b] - n[B + b]);
    if (h_out) h_out[b] = h;
    if (!labels) return;
    const float y = (float)labels[idx ? idx[b] : b];
    const float r = h - y;
    res2[b] = r * r;
    const float d = ys * r / (float)B;
    dn[b] = d;
    dn[B + b] = -d;
}

// D2[r][j] = dn[r] * w3[j] * (H2[r][j] > 0)
__global__ void d2_kernel(const float *dn, const float *H2, const float *p, int R, float *D2) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)R * NH) return;
    const int r = (int)(t / NH), j = (int)(t % NH);
    D2[t] = H2[t] > 0.f ? dn[r] * p[OFF_W3 + j] : 0.f;
}

__global__ void mask_kernel(float *D, const float *H, long long n) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n && !(H[t] > 0.f)) D[t] = 0.f;
}

// g[off + j] = sum_r A[r][j] * (w ? w[r] : 1)   (column sums, deterministic)
__global__ void colsum_kernel(const float *A, const float *w, int R, int ncol, float *g) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= ncol) return;
    double s = 0;
    for (int r = 0; r < R; ++r) s += (double)A[(long long)r * ncol + j] * (w ? (double)w[r] : 1.0);
    g[j] = (float)s;
}

__global__ void sum_kernel(const float *a, int n, float *out) {
    if (blockIdx.x || threadIdx.x) return;
    double s = 0;
    for (int i = 0; i < n; ++i) s += a[i];
    *out = (float)s;
}

__global__ void adamw_kernel(float *p, const float *g, float *m, float *v, int n, float lr, float b1, float b2,
                             float eps, float wd, float c1, float c2) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const float gr = g[t];
    const float mm = b1 * m[t] + (1.f - b1) * gr;
    const float vv = b2 * v[t] + (1.f - b2) * gr * gr;
    m[t] = mm;
    v[t] = vv;
    const bool decay = (t < OFF_B1) || (t >= OFF_W2 && t < OFF_B2) || (t >= OFF_W3 && t < OFF_B3);
    float w = p[t];
    if (decay) w -= lr * wd * w;
    w -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
    p[t] = w;
}

struct Work {
    float *X, *H1, *H2, *n, *dn, *res2, *D2, *D1;
    __nv_bfloat16 *Xb, *H1b;
    int *idx;
};

static Work work(psms_ctx *c, int B) {
    const int R = 2 * B;
    Work w;
    w.X = (float *)scratch(c, "mlp_X", sizeof(float) * R * NI);
    w.H1 = (float *)scratch(c, "mlp_H1", sizeof(float) * R * NH);
    w.H2 = (float *)scratch(c, "mlp_H2", sizeof(float) * R * NH);
    w.n = (float *)scratch(c, "mlp_n", sizeof(float) * R);
    w.dn = (float *)scratch(c, "mlp_dn", sizeof(float) * R);
    w.res2 = (float *)scratch(c, "mlp_res2", sizeof(float) * B);
    w.D2 = (float *)scratch(c, "mlp_D2", sizeof(float) * R * NH);
    w.D1 = (float *)scratch(c, "mlp_D1", sizeof(float) * R * NH);
    w.Xb = (__nv_bfloat16 *)scratch(c, "mlp_Xb", sizeof(__nv_bfloat16) * R * NI);
    w.H1b = (__nv_bfloat16 *)scratch(c, "mlp_H1b", sizeof(__nv_bfloat16) * R * NH);
    w.idx = (int *)scratch(c, "mlp_idx", sizeof(int) * B);
    return w;
}

// forward of rows [z; swap(z)]: H1, H2 (FP32, ReLU'd), n
static void forward(psms_ctx *c, Mlp &m, const Work &w, const float *feats, const int *idx, int B) {
    const int R = 2 * B;
    prep_kernel<<<(R * NI + 255) / 256, 256, 0, c->stream>>>(feats, idx, B, m.p, w.X);
    PSMS_LAUNCH_CHECK("prep_kernel");
    to_bf16_kernel<<<(R * NI + 255) / 256, 256, 0, c->stream>>>(w.X, w.Xb, R * NI);
    PSMS_LAUNCH_CHECK("to_bf16");
    GemmArgs g1{R, NH, NI, w.Xb, NI, 1, 0, m.w1b, NI, 1, 0, w.H1, NH, w.H1b, NH, m.p + OFF_B1, 1.f, 0.f, 1};
    gemm(c, g1, m.err);
    GemmArgs g2{R, NH, NH, w.H1b, NH, 1, 0, m.w2b, NH, 1, 0, w.H2, NH, nullptr, 0, m.p + OFF_B2, 1.f, 0.f, 1};
    gemm(c, g2, m.err);
    out_kernel<<<(R + 3) / 4, 128, 0, c->stream>>>(w.H2, m.p, R, w.n);
    PSMS_LAUNCH_CHECK("out_kernel");
}

// gradient of the MSE of h over the B rows into m.g; returns nothing (loss
// partials in w.res2)
static void backward(psms_ctx *c, Mlp &m, const Work &w, int B) {
    const int R = 2 * B;
    float *g = m.g;
    // output layer
    colsum_kernel<<<(NH + 127) / 128, 128, 0, c->stream>>>(w.H2, w.dn, R, NH, g + OFF_W3);
    PSMS_LAUNCH_CHECK("colsum");
    sum_kernel<<<1, 1, 0, c->stream>>>(w.dn, R, g + OFF_B3);
    PSMS_LAUNCH_CHECK("sum");
    d2_kernel<<<(unsigned)(((long long)R * NH + 255) / 256), 256, 0, c->stream>>>(w.dn, w.H2, m.p, R, w.D2);
    PSMS_LAUNCH_CHECK("d2");
    // dW2[j][i] = sum_r D2[r][j] H1[r][i]
    GemmArgs gw2{NH, NH, R, w.D2, 1, NH, 1, w.H1b, 1, NH, 0, g + OFF_W2, NH, nullptr, 0, nullptr, 1.f, 0.f, 0};
    gemm(c, gw2, m.err);
    colsum_kernel<<<(NH + 127) / 128, 128, 0, c->stream>>>(w.D2, nullptr, R, NH, g + OFF_B2);
    PSMS_LAUNCH_CHECK("colsum");
    // D1 = (D2 W2) * (H1 > 0)
    GemmArgs gd1{R, NH, NH, w.D2, NH, 1, 1, m.w2b, 1, NH, 0, w.D1, NH, nullptr, 0, nullptr, 1.f, 0.f, 0};
    gemm(c, gd1, m.err);
    mask_kernel<<<(unsigned)(((long long)R * NH + 255) / 256), 256, 0, c->stream>>>(w.D1, w.H1, (long long)R * NH);
    PSMS_LAUNCH_CHECK("mask");
    // dW1[i][c] = sum_r D1[r][i] X[r][c]
    GemmArgs gw1{NH, NI, R, w.D1, 1, NH, 1, w.X, 1, NI, 1, g + OFF_W1, NI, nullptr, 0, nullptr, 1.f, 0.f, 0};
    gemm(c, gw1, m.err);
    colsum_kernel<<<(NH + 127) / 128, 128, 0, c->stream>>>(w.D1, nullptr, R, NH, g + OFF_B1);
    PSMS_LAUNCH_CHECK("colsum");
}

// a tensor-core GEMM whose bounded wait ran out leaves the flag set: report
// it once (PSMS_ETIMEOUT) and clear it
void mlp_check(psms_ctx *c) {
    if (!c->mlp) return;
    Mlp &m = *(Mlp *)c->mlp;
    int h = 0;
    cuda_check(cudaMemcpyAsync(&h, m.err, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "mlp status");
    cuda_check(cudaStreamSynchronize(c->stream), "mlp status");
    if (h) {
        cuda_check(cudaMemsetAsync(m.err, 0, sizeof(int), c->stream), "mlp status");
        fail(PSMS_ETIMEOUT, "tensor-core GEMM of the MLP: a bounded mbarrier wait ran out");
    }
}

void mlp_predict(psms_ctx *c, const float *feats, int B, float *h_out) {
    Mlp &m = mlp_of(c);
    Work w = work(c, B);
    forward(c, m, w, feats, nullptr, B);
    loss_kernel<<<(B + 127) / 128, 128, 0, c->stream>>>(w.n, nullptr, nullptr, B, m.p, nullptr, nullptr, h_out);
    PSMS_LAUNCH_CHECK("loss_kernel");
}

}  // namespace psms

using namespace psms;

#define MLP_TRY(ctx)                \
    if (!(ctx)) return PSMS_EINVAL; \
    try {
#define MLP_CATCH(ctx)       \
    }                        \
    catch (const Error &e) { \
        (ctx)->err = e.msg;  \
        return e.st;         \
    }                        \
    return PSMS_OK;

extern "C" {

psms_status psms_domain_features(psms_ctx *ctx, int field, float *out_dev) {
    MLP_TRY(ctx)
    check_field(ctx, field);
    if (!out_dev) fail(PSMS_EINVAL, "null output");
    domain_features(ctx, ctx->U64[field], out_dev, N_FEAT, 0);
    MLP_CATCH(ctx)
}

psms_status psms_domain_features_pair(psms_ctx *ctx, int field_old, int field_new, float *out_dev) {
    MLP_TRY(ctx)
    check_field(ctx, field_old);
    check_field(ctx, field_new);
    if (!out_dev) fail(PSMS_EINVAL, "null output");
    pair_features(ctx, ctx->U64[field_old], ctx->U64[field_new], out_dev);
    MLP_CATCH(ctx)
}

psms_status psms_mlp_init(psms_ctx *ctx, uint64_t seed) {
    MLP_TRY(ctx)
    Mlp &m = mlp_of(ctx);
    mlp_init_kernel<<<(N_PARAM + 255) / 256, 256, 0, ctx->stream>>>(m.p, seed);
    PSMS_LAUNCH_CHECK("mlp_init");
    cuda_check(cudaMemsetAsync(m.m, 0, sizeof(float) * N_TRAIN, ctx->stream), "mlp");
    cuda_check(cudaMemsetAsync(m.v, 0, sizeof(float) * N_TRAIN, ctx->stream), "mlp");
    m.step = 0;
    refresh_bf16(ctx, m);
    MLP_CATCH(ctx)
}

size_t psms_mlp_param_count(void) { return N_PARAM; }

psms_status psms_mlp_params(psms_ctx *ctx, float *host, int set) {
    MLP_TRY(ctx)
    if (!host) fail(PSMS_EINVAL, "null buffer");
    Mlp &m = mlp_of(ctx);
    if (set) {
        cuda_check(cudaMemcpyAsync(m.p, host, sizeof(float) * N_PARAM, cudaMemcpyHostToDevice, ctx->stream), "set");
        refresh_bf16(ctx, m);
    } else {
        cuda_check(cudaMemcpyAsync(host, m.p, sizeof(float) * N_PARAM, cudaMemcpyDeviceToHost, ctx->stream), "get");
    }
    cuda_check(cudaStreamSynchronize(ctx->stream), "mlp params");
    MLP_CATCH(ctx)
}

psms_status psms_mlp_predict(psms_ctx *ctx, const float *feats_dev, int n, float *h_dev) {
    MLP_TRY(ctx)
    if (!feats_dev || !h_dev || n < 1) fail(PSMS_EINVAL, "bad arguments");
    mlp_predict(ctx, feats_dev, n, h_dev);
    mlp_check(ctx);
    MLP_CATCH(ctx)
}

psms_status psms_mlp_grad(psms_ctx *ctx, const float *feats_dev, const double *labels_dev, int n, float *grad_host,
                          double *loss) {
    MLP_TRY(ctx)
    if (!feats_dev || !labels_dev || n < 1) fail(PSMS_EINVAL, "bad arguments");
    Mlp &m = mlp_of(ctx);
    Work w = work(ctx, n);
    forward(ctx, m, w, feats_dev, nullptr, n);
    loss_kernel<<<(n + 127) / 128, 128, 0, ctx->stream>>>(w.n, labels_dev, nullptr, n, m.p, w.dn, w.res2, nullptr);
    PSMS_LAUNCH_CHECK("loss_kernel");
    backward(ctx, m, w, n);
    float *d_l = (float *)scratch(ctx, "mlp_loss", sizeof(float));
    sum_kernel<<<1, 1, 0, ctx->stream>>>(w.res2, n, d_l);
    PSMS_LAUNCH_CHECK("sum");
    float hl = 0;
    cuda_check(cudaMemcpyAsync(&hl, d_l, sizeof(float), cudaMemcpyDeviceToHost, ctx->stream), "loss");
    if (grad_host)
        cuda_check(cudaMemcpyAsync(grad_host, m.g, sizeof(float) * N_TRAIN, cudaMemcpyDeviceToHost, ctx->stream), "g");
    cuda_check(cudaStreamSynchronize(ctx->stream), "grad");
    mlp_check(ctx);
    if (loss) *loss = hl / n;
    MLP_CATCH(ctx)
}

psms_status psms_mlp_train(psms_ctx *ctx, const float *feats_dev, const double *labels_dev, int n,
                           const psms_train_params *tp, double *loss_per_epoch) {
    MLP_TRY(ctx)
    if (!feats_dev || !labels_dev || n < 1 || !tp) fail(PSMS_EINVAL, "bad arguments");
    if (tp->batch < 1 || tp->epochs < 1) fail(PSMS_EINVAL, "batch, epochs >= 1");
    Mlp &m = mlp_of(ctx);
    if (tp->normalise) {
        // feature mean / scale and label scale from the training set (host, FP64)
        std::vector<float> hf((size_t)n * N_FEAT * 2);
        std::vector<double> hy(n);
        cuda_check(cudaMemcpyAsync(hf.data(), feats_dev, sizeof(float) * hf.size(), cudaMemcpyDeviceToHost, ctx->stream),
                   "norm");
        cuda_check(cudaMemcpyAsync(hy.data(), labels_dev, sizeof(double) * n, cudaMemcpyDeviceToHost, ctx->stream),
                   "norm");
        cuda_check(cudaStreamSynchronize(ctx->stream), "norm");
        std::vector<float> hp(N_PARAM);
        cuda_check(cudaMemcpy(hp.data(), m.p, sizeof(float) * N_PARAM, cudaMemcpyDeviceToHost), "norm");
        for (int col = 0; col < NI; ++col) {
            // both halves of z share the statistics of the 32 features
            const int f = col % N_FEAT;
            double s = 0, s2 = 0;
            for (int i = 0; i < n; ++i)
                for (int half = 0; half < 2; ++half) {
                    const double v = hf[(size_t)i * NI + half * N_FEAT + f];
                    s += v;
                    s2 += v * v;
                }
            const double mean = s / (2.0 * n), var = std::max(0.0, s2 / (2.0 * n) - mean * mean);
            hp[OFF_MU + col] = (float)mean;
            hp[OFF_SIG + col] = var > 1e-20 ? (float)std::sqrt(var) : 1.f;
        }
        // output scale: the spread of the labels about their mean (an
        // antisymmetric h cannot represent the mean, so scaling by the RMS
        // would inflate h when the labels sit far from zero); the RMS if
        // the labels do not vary
        double sm = 0, ss = 0;
        for (int i = 0; i < n; ++i) sm += hy[i];
        const double mean = sm / n;
        for (int i = 0; i < n; ++i) ss += (hy[i] - mean) * (hy[i] - mean);
        double scale = std::sqrt(ss / n);
        if (!(scale > 1e-12)) {
            ss = 0;
            for (int i = 0; i < n; ++i) ss += hy[i] * hy[i];
            scale = std::sqrt(ss / n);
        }
        hp[OFF_YS] = scale > 0 ? (float)scale : 1.f;
        cuda_check(cudaMemcpy(m.p, hp.data(), sizeof(float) * N_PARAM, cudaMemcpyHostToDevice), "norm");
    }
    const int B = std::min(tp->batch, n);
    Work w = work(ctx, B);
    std::mt19937_64 rng(tp->seed);
    std::vector<int> perm(n);
    std::iota(perm.begin(), perm.end(), 0);
    int *d_perm = (int *)scratch(ctx, "mlp_perm", sizeof(int) * n);
    float *d_l = (float *)scratch(ctx, "mlp_loss", sizeof(float));
    const float b1 = (float)tp->beta1, b2 = (float)tp->beta2;
    for (int ep = 0; ep < tp->epochs; ++ep) {
        std::shuffle(perm.begin(), perm.end(), rng);
        cuda_check(cudaMemcpyAsync(d_perm, perm.data(), sizeof(int) * n, cudaMemcpyHostToDevice, ctx->stream), "perm");
        double eloss = 0;
        int nb = 0;
        for (int s0 = 0; s0 + B <= n; s0 += B, ++nb) {
            forward(ctx, m, w, feats_dev, d_perm + s0, B);
            loss_kernel<<<(B + 127) / 128, 128, 0, ctx->stream>>>(w.n, labels_dev, d_perm + s0, B, m.p, w.dn, w.res2,
                                                                  nullptr);
            PSMS_LAUNCH_CHECK("loss_kernel");
            backward(ctx, m, w, B);
            m.step += 1;
            const float c1 = 1.f - std::pow(b1, (float)m.step), c2 = 1.f - std::pow(b2, (float)m.step);
            adamw_kernel<<<(N_TRAIN + 255) / 256, 256, 0, ctx->stream>>>(m.p, m.g, m.m, m.v, N_TRAIN, (float)tp->lr, b1,
                                                                         b2, (float)tp->eps, (float)tp->weight_decay,
                                                                         c1, c2);
            PSMS_LAUNCH_CHECK("adamw");
            refresh_bf16(ctx, m);
            sum_kernel<<<1, 1, 0, ctx->stream>>>(w.res2, B, d_l);
            PSMS_LAUNCH_CHECK("sum");
            float hl = 0;
            cuda_check(cudaMemcpyAsync(&hl, d_l, sizeof(float), cudaMemcpyDeviceToHost, ctx->stream), "loss");
            cuda_check(cudaStreamSynchronize(ctx->stream), "loss");
            eloss += hl / B;
        }
        if (loss_per_epoch) loss_per_epoch[ep] = nb ? eloss / nb : 0.0;
        mlp_check(ctx);
    }
    MLP_CATCH(ctx)
}

}  // extern "C"
