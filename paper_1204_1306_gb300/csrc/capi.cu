// C ABI of the library (declared in include/psms.h): context management and
// the entry points.  Every entry point catches internal errors and returns a
// psms_status; the message is kept in the context.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#if __has_include(<nvtx3/nvToolsExt.h>)
#include <nvtx3/nvToolsExt.h>
#define PSMS_HAVE_NVTX 1
#endif
#include "estimator.hpp"
#include "gauge.hpp"
#include "gaugefix.hpp"
#include "hyp.hpp"
#include "block_action.hpp"
#include "blockdet.hpp"
#include "outer.hpp"
#include "mlp.hpp"
#include "solver.hpp"

namespace psms {

long long &launch_counter() {
    static long long n = 0;
    return n;
}

void *scratch(psms_ctx *c, const std::string &name, size_t bytes) {
    if (bytes == 0) bytes = 16;
    DevBuf &b = c->scratch[name];
    if (b.bytes < bytes) {
        if (b.p) {
            cuda_check(cudaStreamSynchronize(c->stream), "scratch sync");
            cuda_check(cudaFree(b.p), "scratch free");
            b.p = nullptr;
            b.bytes = 0;
        }
        cuda_check(cudaMalloc(&b.p, bytes), ("scratch alloc " + name).c_str());
        b.bytes = bytes;
    }
    return b.p;
}

void check_field(psms_ctx *c, int f) {
    if (f < 0 || f >= c->n_fields) fail(PSMS_EINVAL, "gauge field index out of range");
}

float2 *links32(psms_ctx *c, int f) {
    check_field(c, f);
    if (!c->U32[f]) cuda_check(cudaMalloc(&c->U32[f], sizeof(float2) * 36 * c->g.V), "alloc FP32 links");
    if (!c->u32_ok[f]) {
        links_to_f32(c, c->U64[f], c->U32[f], 36 * c->g.V);
        c->u32_ok[f] = 1;
    }
    return c->U32[f];
}

int prof_begin(psms_ctx *c) {
    const int slot = (int)c->prof_pending.size();
    while ((int)c->ev_pool.size() < 2 * (slot + 1)) {
        cudaEvent_t e;
        cuda_check(cudaEventCreate(&e), "event create");
        c->ev_pool.push_back(e);
    }
    cuda_check(cudaEventRecord(c->ev_pool[2 * slot], c->stream), "event record");
    c->prof_pending.push_back({slot, 0.0});
    return slot;
}

void prof_end(psms_ctx *c, int slot, double bytes) {
    cuda_check(cudaEventRecord(c->ev_pool[2 * slot + 1], c->stream), "event record");
    c->prof_pending[slot].second = bytes;
}

unsigned long long *prof_counter(psms_ctx *c, int slot) {
    if (slot >= c->prof_cap) {
        // grow the per-launch site counters (profiling mode only)
        std::vector<unsigned long long> keep(c->prof_cap);
        if (c->prof_cap) {
            cuda_check(cudaStreamSynchronize(c->stream), "prof sync");
            cuda_check(cudaMemcpy(keep.data(), c->d_prof_sites, sizeof(unsigned long long) * c->prof_cap,
                                  cudaMemcpyDeviceToHost),
                       "prof copy");
            cudaFree(c->d_prof_sites);
        }
        int cap = std::max(4096, 2 * c->prof_cap);
        cuda_check(cudaMalloc(&c->d_prof_sites, sizeof(unsigned long long) * cap), "prof alloc");
        cuda_check(cudaMemset(c->d_prof_sites, 0, sizeof(unsigned long long) * cap), "prof memset");
        if (c->prof_cap)
            cuda_check(cudaMemcpy(c->d_prof_sites, keep.data(), sizeof(unsigned long long) * c->prof_cap,
                                  cudaMemcpyHostToDevice),
                       "prof copy");
        c->prof_cap = cap;
    }
    return c->d_prof_sites + slot;
}

int prof_block_begin(psms_ctx *c) {
    const int slot = (int)c->prof_b_pending.size();
    while ((int)c->ev_pool_b.size() < 2 * (slot + 1)) {
        cudaEvent_t e;
        cuda_check(cudaEventCreate(&e), "event create");
        c->ev_pool_b.push_back(e);
    }
    cuda_check(cudaEventRecord(c->ev_pool_b[2 * slot], c->stream), "event record");
    c->prof_b_pending.push_back({slot, 0.0});
    return slot;
}

void prof_block_end(psms_ctx *c, int slot) {
    cuda_check(cudaEventRecord(c->ev_pool_b[2 * slot + 1], c->stream), "event record");
    c->last_block_slot = slot;
}

// algorithmic bytes of one block-CG iteration per half-block site: 4 half
// hops (in, out, 8 links per output site, y on the second hop of each pair)
// and 12 half-vector passes = 4416 B in FP32, twice that in FP64
void prof_block_bytes(psms_ctx *c, long long block_iters, int inner_prec) {
    if (!c->prof || c->last_block_slot < 0) return;
    const double per = (inner_prec == P64 ? 8832.0 : 4416.0) * c->g.Vbh;
    c->prof_b_pending[c->last_block_slot].second += per * (double)block_iters;
    c->last_block_slot = -1;
}

static void prof_collect(psms_ctx *c) {
    if (c->prof_pending.empty()) return;
    cuda_check(cudaStreamSynchronize(c->stream), "prof sync");
    const int n = (int)c->prof_pending.size();
    std::vector<unsigned long long> sites(n);
    cuda_check(cudaMemcpy(sites.data(), c->d_prof_sites, sizeof(unsigned long long) * n, cudaMemcpyDeviceToHost),
               "prof sites");
    for (int i = 0; i < n; ++i) {
        const auto &pp = c->prof_pending[i];
        float ms = 0;
        cuda_check(cudaEventElapsedTime(&ms, c->ev_pool[2 * pp.first], c->ev_pool[2 * pp.first + 1]), "elapsed");
        c->prof_ms += ms;
        c->prof_bytes += pp.second * (double)sites[i];
        c->prof_launches += 1;
    }
    cuda_check(cudaMemset(c->d_prof_sites, 0, sizeof(unsigned long long) * c->prof_cap), "prof reset");
    c->prof_pending.clear();
}

static void prof_collect_block(psms_ctx *c) {
    if (c->prof_b_pending.empty()) return;
    cuda_check(cudaStreamSynchronize(c->stream), "prof sync");
    for (auto &pp : c->prof_b_pending) {
        float ms = 0;
        cuda_check(cudaEventElapsedTime(&ms, c->ev_pool_b[2 * pp.first], c->ev_pool_b[2 * pp.first + 1]), "elapsed");
        c->prof_b_ms += ms;
        c->prof_b_bytes += pp.second;
        c->prof_b_launches += 1;
        if (c->prof_b_list.size() < 4096) c->prof_b_list.push_back({ms, pp.second});
    }
    c->prof_b_pending.clear();
    c->last_block_slot = -1;
}

__global__ void unit_links_kernel(double2 *U, long long V) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 36 * V) return;
    const int e = (int)((t / V) % 9);
    U[t] = make_double2((e == 0 || e == 4 || e == 8) ? 1.0 : 0.0, 0.0);
}

static bool pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }
static int ilog2(int v) {
    int r = 0;
    while ((1 << r) < v) ++r;
    return r;
}

static void build_geometry(psms_ctx *c, const psms_lattice_desc *d) {
    Geom &g = c->g;
    long long V = 1, Vb = 1;
    for (int m = 0; m < 4; ++m) {
        const int L = d->dims[m], l = d->block[m];
        if (L <= 0 || l < 2 || !pow2(l) || L % l) fail(PSMS_EINVAL, "block extents must be powers of two >= 2 dividing L");
        g.L[m] = L;
        g.l[m] = l;
        g.lsh[m] = ilog2(l);
        g.nb[m] = L / l;
        V *= L;
        Vb *= l;
    }
    if (V / 2 > (1LL << 30)) fail(PSMS_EINVAL, "lattice too large");
    g.V = V;
    g.Vh = (int)(V / 2);
    g.Vbh = (int)(Vb / 2);
    g.vbh_sh = ilog2(g.Vbh);
    g.lstride[3] = 1;
    g.lstride[2] = g.l[3];
    g.lstride[1] = g.l[3] * g.l[2];
    g.lstride[0] = g.l[3] * g.l[2] * g.l[1];
    g.bstride[3] = 1;
    g.bstride[2] = g.nb[3];
    g.bstride[1] = g.nb[3] * g.nb[2];
    g.bstride[0] = g.nb[3] * g.nb[2] * g.nb[1];
    g.nblocks = g.nb[0] * g.nb[1] * g.nb[2] * g.nb[3];
    g.coloured = (g.nb[0] % 2 == 0 && g.nb[1] % 2 == 0 && g.nb[2] % 2 == 0 && g.nb[3] % 2 == 0) ? 1 : 0;
    g.nbh = g.coloured ? g.nblocks / 2 : 0;
    c->h_binfo.assign(g.nblocks, BlockInfo{});
    for (int b = 0; b < g.nblocks; ++b) {
        int B[4];
        int rem = b;
        for (int m = 3; m >= 0; --m) {
            B[m] = rem % g.nb[m];
            rem /= g.nb[m];
        }
        const int r = rank_of_lex(g, b, B);
        BlockInfo bi;
        for (int m = 0; m < 4; ++m) bi.B[m] = B[m];
        bi.lex = b;
        for (int mu = 0; mu < 4; ++mu)
            for (int sg = 0; sg < 2; ++sg) {
                int Bn[4] = {B[0], B[1], B[2], B[3]};
                Bn[mu] = (Bn[mu] + (sg == 0 ? 1 : -1) + g.nb[mu]) % g.nb[mu];
                const int bn = ((Bn[0] * g.nb[1] + Bn[1]) * g.nb[2] + Bn[2]) * g.nb[3] + Bn[3];
                bi.nbr[2 * mu + sg] = rank_of_lex(g, bn, Bn);
            }
        c->h_binfo[r] = bi;
    }
    cuda_check(cudaMalloc(&c->d_binfo, sizeof(BlockInfo) * g.nblocks), "binfo alloc");
    cuda_check(cudaMemcpy(c->d_binfo, c->h_binfo.data(), sizeof(BlockInfo) * g.nblocks, cudaMemcpyHostToDevice),
               "binfo copy");
}

static void free_ctx(psms_ctx *c) {
    for (auto p : c->U64)
        if (p) cudaFree(p);
    for (auto p : c->U32)
        if (p) cudaFree(p);
    for (auto &kv : c->scratch)
        if (kv.second.p) cudaFree(kv.second.p);
    for (auto e : c->ev_pool) cudaEventDestroy(e);
    for (auto e : c->ev_pool_b) cudaEventDestroy(e);
    if (c->d_prof_sites) cudaFree(c->d_prof_sites);
    if (c->d_binfo) cudaFree(c->d_binfo);
    if (c->mlp && c->mlp_free) c->mlp_free(c->mlp);
    delete c;
}

static const void *links_for(psms_ctx *c, int f, int prec) {
    check_field(c, f);
    return prec == P64 ? (const void *)c->U64[f] : (const void *)links32(c, f);
}

static size_t elem_size(int prec) {
    switch (prec) {
        case P64: return sizeof(double2);
        case P32: return sizeof(float2);
        case PB16: return sizeof(__nv_bfloat162);
    }
    fail(PSMS_EINVAL, "unknown precision");
}

static int rank_of_block(psms_ctx *c, int b) {
    if (b < 0 || b >= c->g.nblocks) fail(PSMS_EINVAL, "block index out of range");
    int B[4], rem = b;
    for (int m = 3; m >= 0; --m) {
        B[m] = rem % c->g.nb[m];
        rem /= c->g.nb[m];
    }
    return rank_of_lex(c->g, b, B);
}

}  // namespace psms

using namespace psms;

#define PSMS_TRY(ctx)                         \
    if (!(ctx)) return PSMS_EINVAL;           \
    try {
#define PSMS_CATCH(ctx)                       \
    }                                         \
    catch (const Error &e) {                  \
        (ctx)->err = e.msg;                   \
        return e.st;                          \
    }                                         \
    catch (const std::exception &e) {         \
        (ctx)->err = e.what();                \
        return PSMS_EINVAL;                   \
    }                                         \
    return PSMS_OK;

extern "C" {

psms_status psms_create(const psms_lattice_desc *desc, psms_ctx **out) {
    if (!desc || !out) return PSMS_EINVAL;
    *out = nullptr;
    psms_ctx *c = new psms_ctx();
    try {
        if (!(desc->kappa > 0)) fail(PSMS_EINVAL, "kappa must be positive");
        if (desc->n_fields < 1 || desc->n_fields > 64) fail(PSMS_EINVAL, "n_fields must be in 1..64");
        build_geometry(c, desc);
        c->kappa = desc->kappa;
        c->A = 1.0 / (2.0 * desc->kappa);
        c->n_fields = desc->n_fields;
        c->U64.assign(c->n_fields, nullptr);
        c->U32.assign(c->n_fields, nullptr);
        c->u32_ok.assign(c->n_fields, 0);
        const long long n = 36 * c->g.V;
        for (int f = 0; f < c->n_fields; ++f) {
            cuda_check(cudaMalloc(&c->U64[f], sizeof(double2) * n), "gauge alloc");
            unit_links_kernel<<<(unsigned)((n + 255) / 256), 256>>>(c->U64[f], c->g.V);
            PSMS_LAUNCH_CHECK("unit links");
        }
        cuda_check(cudaDeviceSynchronize(), "create sync");
    } catch (const Error &e) {
        psms_status st = e.st;
        free_ctx(c);
        return st;
    }
    *out = c;
    return PSMS_OK;
}

psms_status psms_destroy(psms_ctx *ctx) {
    if (!ctx) return PSMS_EINVAL;
    cudaStreamSynchronize(ctx->stream);
    free_ctx(ctx);
    return PSMS_OK;
}

const char *psms_last_error(const psms_ctx *ctx) {
    if (!ctx) return "null context";
    return ctx->err.c_str();
}

psms_status psms_set_stream(psms_ctx *ctx, void *stream) {
    PSMS_TRY(ctx)
    ctx->stream = (cudaStream_t)stream;
    PSMS_CATCH(ctx)
}

psms_status psms_geometry_info(const psms_ctx *cctx, long long *n_blocks, long long *dim_P, long long *n_active) {
    psms_ctx *ctx = const_cast<psms_ctx *>(cctx);
    PSMS_TRY(ctx)
    const Geom &g = ctx->g;
    long long dimP = 0, act = 0;
    const int lv = g.l[0] * g.l[1] * g.l[2] * g.l[3];
    for (int ll = 0; ll < lv; ++ll) {
        int y[4], rem = ll;
        for (int m = 3; m >= 0; --m) {
            y[m] = rem % g.l[m];
            rem /= g.l[m];
        }
        int nf = 0;
        for (int m = 0; m < 4; ++m) nf += (y[m] == 0 || y[m] == g.l[m] - 1) ? 1 : 0;
        dimP += nf == 0 ? 0 : (nf == 1 ? 6 : 12);
        for (int mu = 0; mu < 4; ++mu) act += link_active(g, y, mu, 0) ? 1 : 0;
    }
    if (n_blocks) *n_blocks = g.nblocks;
    if (dim_P) *dim_P = g.coloured ? dimP * g.nbh : 0;
    if (n_active) *n_active = act * g.nblocks;
    PSMS_CATCH(ctx)
}

psms_status psms_gauge_init(psms_ctx *ctx, int field, double eps, uint64_t seed) {
    PSMS_TRY(ctx)
    check_field(ctx, field);
    link_init(ctx, ctx->U64[field], eps, seed);
    touch_field(ctx, field);
    PSMS_CATCH(ctx)
}

__global__ void nonfinite_kernel(const double *p, long long n, unsigned int *count) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        if (!isfinite(p[i])) {
            atomicAdd(count, 1u);
            return;
        }
}

// PSMS_EINVAL when any of the n doubles at p (device) is NaN or infinite
static void require_finite(psms_ctx *c, const double *p, long long n, const char *what) {
    unsigned int *d = (unsigned int *)scratch(c, "nonfinite", sizeof(unsigned int));
    cuda_check(cudaMemsetAsync(d, 0, sizeof(unsigned int), c->stream), "nonfinite");
    const long long blocks = std::min<long long>((n + 255) / 256, 152 * 16);
    nonfinite_kernel<<<(unsigned)std::max<long long>(blocks, 1), 256, 0, c->stream>>>(p, n, d);
    PSMS_LAUNCH_CHECK("nonfinite");
    unsigned int h = 0;
    cuda_check(cudaMemcpyAsync(&h, d, sizeof(h), cudaMemcpyDeviceToHost, c->stream), "nonfinite");
    cuda_check(cudaStreamSynchronize(c->stream), "nonfinite");
    if (h) fail(PSMS_EINVAL, std::string(what) + " holds NaN or infinite values");
}

psms_status psms_gauge_set(psms_ctx *ctx, int field, const double *links) {
    PSMS_TRY(ctx)
    check_field(ctx, field);
    if (!links) fail(PSMS_EINVAL, "null links");
    require_finite(ctx, links, 72 * ctx->g.V, "the gauge field");
    gauge_canonical(ctx, (const double2 *)links, ctx->U64[field], 1);
    touch_field(ctx, field);
    PSMS_CATCH(ctx)
}

psms_status psms_gauge_get(psms_ctx *ctx, int field, double *links) {
    PSMS_TRY(ctx)
    check_field(ctx, field);
    if (!links) fail(PSMS_EINVAL, "null links");
    gauge_canonical(ctx, (const double2 *)links, ctx->U64[field], 0);
    PSMS_CATCH(ctx)
}

// HYP smearing parameters: the caller's (each in [0, 1]) or those of the
// HYP construction, (0.75, 0.6, 0.3)
static void hyp_alpha(const double *alpha, double a[3]) {
    const double def[3] = {0.75, 0.6, 0.3};
    for (int i = 0; i < 3; ++i) {
        a[i] = alpha ? alpha[i] : def[i];
        if (!(a[i] >= 0.0 && a[i] <= 1.0)) fail(PSMS_EINVAL, "HYP parameters must lie in [0, 1]");
    }
}

psms_status psms_hyp_smear(psms_ctx *ctx, int field, const double *alpha, double *links_dev) {
    PSMS_TRY(ctx)
    check_field(ctx, field);
    if (!links_dev) fail(PSMS_EINVAL, "null links");
    double a[3];
    hyp_alpha(alpha, a);
    const double2 *F1 = hyp_smear(ctx, ctx->U64[field], a, nullptr);
    gauge_canonical(ctx, (const double2 *)links_dev, const_cast<double2 *>(F1), 0);
    PSMS_CATCH(ctx)
}

psms_status psms_hyp_block_action(psms_ctx *ctx, int field, const double *alpha, double *s_host) {
    PSMS_TRY(ctx)
    check_field(ctx, field);
    if (!s_host) fail(PSMS_EINVAL, "null output");
    double a[3];
    hyp_alpha(alpha, a);
    const int nb = ctx->g.nblocks;
    double *d = (double *)scratch(ctx, "hyp_action", sizeof(double) * nb);
    hyp_block_action(ctx, ctx->U64[field], a, d);
    cuda_check(cudaMemcpyAsync(s_host, d, sizeof(double) * nb, cudaMemcpyDeviceToHost, ctx->stream), "hyp action");
    cuda_check(cudaStreamSynchronize(ctx->stream), "hyp action");
    for (int b = 0; b < nb; ++b)
        if (!std::isfinite(s_host[b])) fail(PSMS_ESPECTRUM, "non-finite HYP action (singular smearing sum)");
    PSMS_CATCH(ctx)
}

psms_status psms_block_logdet(psms_ctx *ctx, int field, double *out_host) {
    PSMS_TRY(ctx)
    check_field(ctx, field);
    if (!out_host) fail(PSMS_EINVAL, "null output");
    const int nb = ctx->g.nblocks;
    double *d = (double *)scratch(ctx, "bd_out", sizeof(double) * nb);
    block_logdet(ctx, ctx->U64[field], d);
    cuda_check(cudaMemcpyAsync(out_host, d, sizeof(double) * nb, cudaMemcpyDeviceToHost, ctx->stream), "logdet");
    cuda_check(cudaStreamSynchronize(ctx->stream), "logdet");
    for (int b = 0; b < nb; ++b)
        if (!std::isfinite(out_host[b])) fail(PSMS_ESPECTRUM, "singular block operator (non-finite ln|det|)");
    PSMS_CATCH(ctx)
}

psms_status psms_set_outer_blocks(psms_ctx *ctx, const int *outer) {
    PSMS_TRY(ctx)
    set_outer(ctx, outer);
    PSMS_CATCH(ctx)
}

psms_status psms_block_action_change(psms_ctx *ctx, int field_old, int field_new, double *ds_host) {
    PSMS_TRY(ctx)
    check_field(ctx, field_old);
    check_field(ctx, field_new);
    if (!ds_host) fail(PSMS_EINVAL, "null output");
    const int nb = ctx->g.nblocks;
    double *d = (double *)scratch(ctx, "bac_out", sizeof(double) * nb);
    block_action_change(ctx, ctx->U64[field_old], ctx->U64[field_new], d);
    cuda_check(cudaMemcpyAsync(ds_host, d, sizeof(double) * nb, cudaMemcpyDeviceToHost, ctx->stream), "dS_w");
    cuda_check(cudaStreamSynchronize(ctx->stream), "dS_w");
    PSMS_CATCH(ctx)
}

psms_status psms_gauge_copy(psms_ctx *ctx, int dst, int src) {
    PSMS_TRY(ctx)
    check_field(ctx, dst);
    check_field(ctx, src);
    if (dst != src) {
        cuda_check(cudaMemcpyAsync(ctx->U64[dst], ctx->U64[src], sizeof(double2) * 36 * ctx->g.V,
                                   cudaMemcpyDeviceToDevice, ctx->stream),
                   "gauge copy");
        touch_field(ctx, dst);
    }
    PSMS_CATCH(ctx)
}

psms_status psms_plaquette(psms_ctx *ctx, int field, double *mean_plaq, double *s_w) {
    PSMS_TRY(ctx)
    check_field(ctx, field);
    double *d = (double *)scratch(ctx, "plaq_out", sizeof(double));
    plaquette_sum(ctx, ctx->U64[field], d);
    double h = 0;
    cuda_check(cudaMemcpyAsync(&h, d, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream), "plaq");
    cuda_check(cudaStreamSynchronize(ctx->stream), "plaq");
    const double V = (double)ctx->g.V;
    if (mean_plaq) *mean_plaq = h / (18.0 * V);
    if (s_w) *s_w = (18.0 * V - h) / 3.0;
    PSMS_CATCH(ctx)
}

psms_status psms_gauge_sweep(psms_ctx *ctx, int field, int active_set, int n_iter, int n_or, double beta,
                             uint64_t seed, uint64_t sweep0, int *failed_out) {
    PSMS_TRY(ctx)
    check_field(ctx, field);
    if (n_iter < 0 || n_or < 0) fail(PSMS_EINVAL, "negative sweep count");
    if (active_set != PSMS_ACTIVE_BLOCKS && active_set != PSMS_ACTIVE_ALL) fail(PSMS_EINVAL, "bad active set");
    int f = gauge_sweep(ctx, ctx->U64[field], active_set, n_iter, n_or, beta, seed, sweep0);
    touch_field(ctx, field);
    if (failed_out) *failed_out = f;
    if (f) fail(PSMS_EHEATBATH, "an SU(2) heatbath draw hit its attempt limit");
    PSMS_CATCH(ctx)
}

psms_status psms_gauge_translate(psms_ctx *ctx, int field, const int shift[4]) {
    PSMS_TRY(ctx)
    check_field(ctx, field);
    double2 *tmp = (double2 *)scratch(ctx, "translate_tmp", sizeof(double2) * 36 * ctx->g.V);
    translate(ctx, ctx->U64[field], tmp, shift);
    cuda_check(cudaMemcpyAsync(ctx->U64[field], tmp, sizeof(double2) * 36 * ctx->g.V, cudaMemcpyDeviceToDevice,
                               ctx->stream),
               "translate copy");
    touch_field(ctx, field);
    PSMS_CATCH(ctx)
}

size_t psms_spinor_bytes(const psms_ctx *ctx, int prec) {
    if (!ctx) return 0;
    size_t e = prec == P64 ? sizeof(double2) : (prec == P32 ? sizeof(float2) : sizeof(__nv_bfloat162));
    return e * 12 * (size_t)ctx->g.V;
}

psms_status psms_spinor_import(psms_ctx *ctx, const double *canon, void *nat, int prec) {
    PSMS_TRY(ctx)
    if (!canon || !nat) fail(PSMS_EINVAL, "null pointer");
    elem_size(prec);
    require_finite(ctx, canon, 24 * ctx->g.V, "the spinor field");
    spinor_canonical(ctx, (const double2 *)canon, nat, prec, 1);
    PSMS_CATCH(ctx)
}

psms_status psms_spinor_export(psms_ctx *ctx, const void *nat, double *canon, int prec) {
    PSMS_TRY(ctx)
    if (!canon || !nat) fail(PSMS_EINVAL, "null pointer");
    elem_size(prec);
    spinor_canonical(ctx, (const double2 *)canon, (void *)nat, prec, 0);
    PSMS_CATCH(ctx)
}

psms_status psms_dw_apply(psms_ctx *ctx, int field, int op, const void *in, void *out, int prec) {
    PSMS_TRY(ctx)
    if (!in || !out || in == out) fail(PSMS_EINVAL, "in / out must be distinct non-null buffers");
    const size_t es = elem_size(prec);
    const long long V = ctx->g.V;
    HopCall h;
    h.prec = prec;
    h.U = links_for(ctx, field, prec);
    h.in = View<void>{(void *)in, V, 0, 12 * V};
    h.out = View<void>{out, V, 0, 12 * V};
    h.y = h.in;
    h.a = ctx->A;
    h.b = -0.5;
    h.p = -1;
    if (op == PSMS_OP_FULL) {
        h.mode = HOP_ALL;
    } else if (op == PSMS_OP_BLOCKS) {
        h.mode = HOP_INTRA;
    } else {
        const int r = rank_of_block(ctx, op);
        cuda_check(cudaMemsetAsync(out, 0, es * 12 * V, ctx->stream), "dw memset");
        h.mode = HOP_INTRA;
        h.rank_lo = r;
        h.n_ranks = 1;
    }
    hop_launch(ctx, h);
    PSMS_CATCH(ctx)
}

psms_status psms_solve(psms_ctx *ctx, int field, int op, const void *b, void *x, double tol, int maxit,
                       int inner_prec, psms_solve_info *info) {
    PSMS_TRY(ctx)
    check_field(ctx, field);
    if (!b || !x || b == x) fail(PSMS_EINVAL, "b / x must be distinct non-null buffers");
    if (!(tol > 0) || maxit < 1) fail(PSMS_EINVAL, "tol must be > 0 and maxit >= 1");
    elem_size(inner_prec);
    const long long V = ctx->g.V;
    require_finite(ctx, (const double *)b, 24 * V, "the right-hand side");
    const float2 *U32 = inner_prec == P64 ? nullptr : links32(ctx, field);
    if (op == PSMS_OP_FULL) {
        FullSolveReq q;
        q.b = View<double2>{(double2 *)b, V, 0, 12 * V};
        q.x = View<double2>{(double2 *)x, V, 0, 12 * V};
        q.U64 = ctx->U64[field];
        q.U32 = U32;
        q.tol = tol;
        q.maxit = maxit;
        q.inner_prec = inner_prec;
        solve_full_batch(ctx, q, info);
    } else {
        if (inner_prec == PB16) fail(PSMS_EINVAL, "block solves support FP64 and FP32 inner iterations");
        int lo = 0, nr = ctx->g.nblocks;
        if (op != PSMS_OP_BLOCKS) {
            lo = rank_of_block(ctx, op);
            nr = 1;
        }
        cuda_check(cudaMemsetAsync(x, 0, sizeof(double2) * 12 * V, ctx->stream), "solve memset");
        int *iters = (int *)scratch(ctx, "api_iters", sizeof(int) * nr);
        double *resid = (double *)scratch(ctx, "api_resid", sizeof(double) * nr);
        int *status = (int *)scratch(ctx, "api_status", sizeof(int) * nr);
        BlockSolveReq q;
        q.rank_lo = lo;
        q.n_ranks = nr;
        q.n_sys = 1;
        q.b = View<double2>{(double2 *)b, V, 0, 12 * V};
        q.x = View<double2>{(double2 *)x, V, 0, 12 * V};
        q.U64 = ctx->U64[field];
        q.U32 = U32;
        q.tol = tol;
        q.maxit = maxit;
        q.inner_prec = inner_prec;
        q.iters = iters;
        q.resid = resid;
        q.status = status;
        block_solve(ctx, q);
        std::vector<int> hi(nr), hs(nr);
        std::vector<double> hr(nr);
        cuda_check(cudaMemcpyAsync(hi.data(), iters, sizeof(int) * nr, cudaMemcpyDeviceToHost, ctx->stream), "it");
        cuda_check(cudaMemcpyAsync(hr.data(), resid, sizeof(double) * nr, cudaMemcpyDeviceToHost, ctx->stream), "res");
        cuda_check(cudaMemcpyAsync(hs.data(), status, sizeof(int) * nr, cudaMemcpyDeviceToHost, ctx->stream), "st");
        cuda_check(cudaStreamSynchronize(ctx->stream), "solve sync");
        long long tot = 0;
        double worst = 0;
        int bad = 0;
        for (int i = 0; i < nr; ++i) {
            tot += hi[i];
            worst = std::max(worst, hr[i]);
            bad |= hs[i];
        }
        prof_block_bytes(ctx, tot, inner_prec);
        if (info) {
            info->outer_iters = 0;
            info->inner_iters = tot;
            info->true_residual = worst;
            info->n_systems = nr;
        }
        if (bad) fail(PSMS_ENOCONV, "a block solve missed its tolerance");
    }
    PSMS_CATCH(ctx)
}

psms_status psms_logdet_ratio(psms_ctx *ctx, int level, int field_old, int field_new, int n, int mode,
                              uint64_t seed, uint64_t counter, double tol, int inner_prec, double *delta_out) {
    PSMS_TRY(ctx)
    check_field(ctx, field_old);
    check_field(ctx, field_new);
    if (n < 1 || !delta_out) fail(PSMS_EINVAL, "n >= 1 and delta_out required");
    if (mode != PSMS_EST_INTERP && mode != PSMS_EST_INDEPENDENT) fail(PSMS_EINVAL, "bad estimator mode");
    if (inner_prec != P64 && inner_prec != P32) fail(PSMS_EINVAL, "estimators use FP64 or FP32 inner iterations");
    const int nb = ctx->g.nblocks;
    if (level == PSMS_LEVEL_BLOCK) {
        double *d = (double *)scratch(ctx, "ld_delta", sizeof(double) * nb * n);
        block_level(ctx, ctx->U64[field_old], ctx->U64[field_new], n, mode, seed, counter, tol, inner_prec, d);
        cuda_check(cudaMemcpyAsync(delta_out, d, sizeof(double) * nb * n, cudaMemcpyDeviceToHost, ctx->stream), "out");
    } else if (level == PSMS_LEVEL_OUTER_GLOBAL) {
        outer_global_level(ctx, ctx->U64[field_old], ctx->U64[field_new], n, mode, seed, counter, tol, inner_prec,
                           delta_out);
    } else if (level == PSMS_LEVEL_GLOBAL) {
        double *d = (double *)scratch(ctx, "ld_delta", sizeof(double) * n);
        global_level(ctx, ctx->U64[field_old], ctx->U64[field_new], n, mode, seed, counter, tol, inner_prec, d);
        cuda_check(cudaMemcpyAsync(delta_out, d, sizeof(double) * n, cudaMemcpyDeviceToHost, ctx->stream), "out");
    } else if (level == PSMS_LEVEL_SUB) {
        sub_level(ctx, ctx->U64[field_old], ctx->U64[field_new], n, mode, seed, counter, tol, inner_prec, delta_out);
    } else {
        fail(PSMS_EINVAL, "level must be PSMS_LEVEL_BLOCK, PSMS_LEVEL_GLOBAL, PSMS_LEVEL_SUB or "
                          "PSMS_LEVEL_OUTER_GLOBAL");
    }
    cuda_check(cudaStreamSynchronize(ctx->stream), "logdet sync");
    PSMS_CATCH(ctx)
}

static GaugeFixParams gf_params(const psms_relgf_params &p) {
    if (!(p.alpha0 > 0) || !(p.alpha_min > 0) || p.alpha_min > p.alpha0 || !(p.dalpha > 0) || !(p.theta_tol >= 0) ||
        p.max_iter < 0 || p.max_iter > 1000000 || (p.prec != P64 && p.prec != P32))
        fail(PSMS_EINVAL, "gauge fixing: need alpha0 >= alpha_min > 0, dalpha > 0, theta_tol >= 0, "
                          "0 <= max_iter <= 1e6, prec FP64 or FP32");
    GaugeFixParams q;
    q.alpha0 = p.alpha0;
    q.alpha_min = p.alpha_min;
    q.dalpha = p.dalpha;
    q.theta_tol = p.theta_tol;
    q.max_iter = p.max_iter;
    q.prec = p.prec;
    return q;
}

// NVTX range for one level of the filter step (visible to Nsight tools, a
// no-op otherwise)
struct Range {
    explicit Range(const char *name) {
#ifdef PSMS_HAVE_NVTX
        nvtxRangePushA(name);
#else
        (void)name;
#endif
    }
    ~Range() {
#ifdef PSMS_HAVE_NVTX
        nvtxRangePop();
#endif
    }
};

psms_status psms_relative_gauge_fix(psms_ctx *ctx, int field_old, int field_new, int out_old, int out_new,
                                    const psms_relgf_params *prm, int *steps, double *alpha, double *theta,
                                    int *swapped, void *g_dev) {
    PSMS_TRY(ctx)
    check_field(ctx, field_old);
    check_field(ctx, field_new);
    check_field(ctx, out_old);
    check_field(ctx, out_new);
    if (!prm) fail(PSMS_EINVAL, "null parameters");
    if (out_old == field_new || out_new == field_old || out_old == out_new)
        fail(PSMS_EINVAL, "output slots overlap the other input");
    const GaugeFixParams q = gf_params(*prm);
    GaugeFixInfo gi;
    gauge_fix_pair(ctx, ctx->U64[field_old], ctx->U64[field_new], ctx->U64[out_old], ctx->U64[out_new], q, &gi);
    touch_field(ctx, out_old);
    touch_field(ctx, out_new);
    if (g_dev) {
        gauge_fix_export(ctx, gi.G1, (double2 *)g_dev);
        gauge_fix_export(ctx, gi.G2, (double2 *)g_dev + 9 * ctx->g.V);
    }
    const int nb = ctx->g.nblocks;
    if (steps) cuda_check(cudaMemcpyAsync(steps, gi.d_steps, sizeof(int) * nb, cudaMemcpyDeviceToHost, ctx->stream), "gf");
    if (alpha)
        cuda_check(cudaMemcpyAsync(alpha, gi.d_alpha, sizeof(double) * nb, cudaMemcpyDeviceToHost, ctx->stream), "gf");
    if (theta)
        cuda_check(cudaMemcpyAsync(theta, gi.d_theta, sizeof(double) * nb, cudaMemcpyDeviceToHost, ctx->stream), "gf");
    if (swapped)
        cuda_check(cudaMemcpyAsync(swapped, gi.d_swap, sizeof(int) * nb, cudaMemcpyDeviceToHost, ctx->stream), "gf");
    cuda_check(cudaStreamSynchronize(ctx->stream), "gf");
    PSMS_CATCH(ctx)
}

psms_status psms_filter_step(psms_ctx *ctx, int field, const psms_filter_params *prm, psms_filter_result *res,
                             double *delta_block_out, int *accept_block_out) {
    PSMS_TRY(ctx)
    check_field(ctx, field);
    if (!prm) fail(PSMS_EINVAL, "null parameters");
    if (prm->n_block < 1 || prm->n_global < 1) fail(PSMS_EINVAL, "n_block, n_global >= 1");
    if (prm->inner_prec != P64 && prm->inner_prec != P32) fail(PSMS_EINVAL, "inner precision FP64 or FP32");
    const Geom &g = ctx->g;
    const long long nel = 36 * g.V;
    const size_t fb = sizeof(double2) * nel;
    double2 *cur = ctx->U64[field];
    for (auto *v : {&ctx->rec_h, &ctx->rec_dhyp, &ctx->rec_acc1, &ctx->rec_dsub, &ctx->rec_acc_sub}) v->clear();
    double2 *old = (double2 *)scratch(ctx, "fs_old", fb);
    double2 *prop = (double2 *)scratch(ctx, "fs_prop", fb);
    double2 *mid = (double2 *)scratch(ctx, "fs_mid", fb);
    cuda_check(cudaMemcpyAsync(old, cur, fb, cudaMemcpyDeviceToDevice, ctx->stream), "copy");
    // level 0: proposal (domain sweep, or an external proposal slot)
    Range r_step("psms_filter_step");
    int failed = 0;
    std::unique_ptr<Range> r_lvl(new Range("level 0: proposal"));
    if (prm->proposal_field >= 0) {
        check_field(ctx, prm->proposal_field);
        if (prm->proposal_field == field) fail(PSMS_EINVAL, "the proposal slot must differ from the field");
        cuda_check(cudaMemcpyAsync(prop, ctx->U64[prm->proposal_field], fb, cudaMemcpyDeviceToDevice, ctx->stream),
                   "copy");
    } else {
        cuda_check(cudaMemcpyAsync(prop, cur, fb, cudaMemcpyDeviceToDevice, ctx->stream), "copy");
        failed = gauge_sweep(ctx, prop, PSMS_ACTIVE_BLOCKS, prm->n_iter, prm->n_or, prm->beta0, prm->seed,
                             prm->step << 20);
        if (failed) fail(PSMS_EHEATBATH, "an SU(2) heatbath draw hit its attempt limit");
    }
    const int nb = g.nblocks, N1 = prm->n_block;
    bool per_block = true;
    for (int m = 0; m < 4; ++m) per_block &= g.l[m] >= 3;
    if (!std::isfinite(prm->beta_block) || !std::isfinite(prm->beta_block_hyp) ||
        !std::isfinite(prm->beta_global_hyp) || !std::isfinite(prm->hyp_beta[0]) || !std::isfinite(prm->hyp_beta[1]))
        fail(PSMS_EINVAL, "filter coefficients must be finite");
    r_lvl.reset();  // pop before the next push (NVTX ranges nest as a stack)
    r_lvl.reset(new Range("HYP level"));
    // per-block action changes of the proposal: dS_w,b (beta_block and the
    // HYP level) and dS_HYP,b (the HYP terms, App. C)
    const bool recursive = prm->n_sub > 0;
    if (recursive) {
        if (!has_outer(ctx)) fail(PSMS_EINVAL, "n_sub >= 1 needs outer blocks (psms_set_outer_blocks)");
        if (prm->hyp_level || prm->beta_block_hyp != 0.0 || prm->beta_global_hyp != 0.0)
            fail(PSMS_EINVAL, "the recursive filter does not combine with the HYP options");
        if (!std::isfinite(prm->beta_sub)) fail(PSMS_EINVAL, "beta_sub must be finite");
        if (prm->exact_block || prm->beta_global_blockdet != 0.0)
            fail(PSMS_EINVAL, "the recursive filter does not combine with the exact block level");
    }
    if (!std::isfinite(prm->beta_block_det) || !std::isfinite(prm->beta_global_blockdet))
        fail(PSMS_EINVAL, "filter coefficients must be finite");
    // exact change of the block-determinant action S_b = -2 ln|det D_b|
    double *d_dsb = nullptr;
    if (prm->exact_block || prm->beta_global_blockdet != 0.0) {
        double *d_l0 = (double *)scratch(ctx, "fs_ld0", sizeof(double) * nb);
        double *d_l1 = (double *)scratch(ctx, "fs_ld1", sizeof(double) * nb);
        d_dsb = (double *)scratch(ctx, "fs_dsb", sizeof(double) * nb);
        block_logdet(ctx, old, d_l0);
        block_logdet(ctx, prop, d_l1);
        block_lincomb(ctx, 2.0, d_l0, -2.0, d_l1, 0.0, nullptr, d_dsb);
        std::vector<double> chk(nb);
        cuda_check(cudaMemcpyAsync(chk.data(), d_dsb, sizeof(double) * nb, cudaMemcpyDeviceToHost, ctx->stream), "dsb");
        cuda_check(cudaStreamSynchronize(ctx->stream), "dsb");
        for (double v : chk)
            if (!std::isfinite(v)) fail(PSMS_ESPECTRUM, "singular block operator (non-finite ln|det|)");
    }
    const bool need_dsw = prm->beta_block != 0.0 || prm->hyp_level || (recursive && prm->beta_sub != 0.0);
    const bool need_hyp = prm->hyp_level || prm->beta_block_hyp != 0.0 || prm->beta_global_hyp != 0.0;
    double *d_dsw = nullptr, *d_dhyp = nullptr;
    if (need_dsw) {
        d_dsw = (double *)scratch(ctx, "fs_dsw", sizeof(double) * nb);
        block_action_change(ctx, old, prop, d_dsw);
    }
    if (need_hyp) {
        const double alpha[3] = {0.75, 0.6, 0.3};
        double *d_s0 = (double *)scratch(ctx, "fs_hyp0", sizeof(double) * nb);
        double *d_s1 = (double *)scratch(ctx, "fs_hyp1", sizeof(double) * nb);
        d_dhyp = (double *)scratch(ctx, "fs_dhyp", sizeof(double) * nb);
        hyp_block_action(ctx, old, alpha, d_s0);
        hyp_block_action(ctx, prop, alpha, d_s1);
        block_lincomb(ctx, 1.0, d_s1, -1.0, d_s0, 0.0, nullptr, d_dhyp);
    }
    // HYP level: Delta_b = b0 dS_w,b + b1 dS_HYP,b, decision counter (step, 5, b)
    const int *d_mask = nullptr;
    int n_hyp = -1;
    if (prm->hyp_level) {
        double *d_dl = (double *)scratch(ctx, "fs_dhl", sizeof(double) * nb);
        block_lincomb(ctx, prm->hyp_beta[0], d_dsw, prm->hyp_beta[1], d_dhyp, 0.0, nullptr, d_dl);
        double *d_hs5 = (double *)scratch(ctx, "fs_hs5", sizeof(double) * (nb + 1));
        int *d_acc5 = (int *)scratch(ctx, "fs_acc5", sizeof(int) * nb);
        decide(ctx, d_dl, nb, 1, per_block ? 1 : 0, prm->seed, prm->step, 5, 0.0, nullptr, 0.0, d_hs5, d_acc5);
        std::vector<int> h5(nb);
        ctx->rec_dhyp.assign(nb, 0.0);
        cuda_check(cudaMemcpyAsync(h5.data(), d_acc5, sizeof(int) * nb, cudaMemcpyDeviceToHost, ctx->stream), "l5");
        cuda_check(cudaMemcpyAsync(ctx->rec_dhyp.data(), d_dl, sizeof(double) * nb, cudaMemcpyDeviceToHost,
                                   ctx->stream),
                   "l5");
        cuda_check(cudaStreamSynchronize(ctx->stream), "l5");
        n_hyp = 0;
        for (int v : h5) n_hyp += v;
        d_mask = d_acc5;
    }
    r_lvl.reset();  // pop before the next push (NVTX ranges nest as a stack)
    r_lvl.reset(new Range("learned level"));
    // learned level (before level 1): h_b, accept with min{1, exp(-h_b)}
    double *d_h = nullptr;
    int n_learned = -1;
    if (prm->learned) {
        if (!per_block) fail(PSMS_EINVAL, "the learned level needs per-block decisions (block extents >= 3)");
        if (!ctx->mlp) fail(PSMS_EINVAL, "the learned level needs a trained MLP (psms_mlp_init / psms_mlp_train)");
        float *z = (float *)scratch(ctx, "fs_feat", sizeof(float) * nb * 2 * N_FEAT);
        pair_features(ctx, old, prop, z);
        float *hf = (float *)scratch(ctx, "fs_hf", sizeof(float) * nb);
        mlp_predict(ctx, z, nb, hf);
        d_h = (double *)scratch(ctx, "fs_h", sizeof(double) * nb);
        float_to_double(ctx, hf, d_h, nb);
        int *d_acc3 = (int *)scratch(ctx, "fs_acc3", sizeof(int) * nb);
        double *d_hs = (double *)scratch(ctx, "fs_hsum", sizeof(double) * (nb + 1));
        decide(ctx, d_h, nb, 1, 1, prm->seed, prm->step, 3, 0.0, nullptr, 0.0, d_hs, d_acc3, d_mask);
        std::vector<int> h3(nb);
        ctx->rec_h.assign(nb, 0.0);
        cuda_check(cudaMemcpyAsync(h3.data(), d_acc3, sizeof(int) * nb, cudaMemcpyDeviceToHost, ctx->stream), "l3");
        cuda_check(cudaMemcpyAsync(ctx->rec_h.data(), d_h, sizeof(double) * nb, cudaMemcpyDeviceToHost, ctx->stream),
                   "l3");
        cuda_check(cudaStreamSynchronize(ctx->stream), "l3");
        mlp_check(ctx);
        n_learned = 0;
        for (int v : h3) n_learned += v;
        d_mask = d_acc3;
    }
    r_lvl.reset();  // pop before the next push (NVTX ranges nest as a stack)
    r_lvl.reset(new Range("relative gauge fixing"));
    // relative gauge fixing: the estimators interpolate between U^{g_1} and
    // U'^{g_2} (Sec. 4.2); blocks decouple, so the level-2 endpoints are the
    // level-1 ones on accepted blocks and U elsewhere
    double2 *e0 = old, *eN = prop;
    long long gf_steps = 0;
    if (prm->gauge_fix) {
        const GaugeFixParams q = gf_params(prm->relgf);
        e0 = (double2 *)scratch(ctx, "fs_e0", fb);
        eN = (double2 *)scratch(ctx, "fs_en", fb);
        GaugeFixInfo gi;
        gauge_fix_pair(ctx, old, prop, e0, eN, q, &gi);
        std::vector<int> hs(nb);
        cuda_check(cudaMemcpyAsync(hs.data(), gi.d_steps, sizeof(int) * nb, cudaMemcpyDeviceToHost, ctx->stream), "gf");
        cuda_check(cudaStreamSynchronize(ctx->stream), "gf");
        for (int v : hs) gf_steps += v;
    }
    r_lvl.reset();  // pop before the next push (NVTX ranges nest as a stack)
    r_lvl.reset(new Range("level 1: block det ratios"));
    // level 1: block det ratios (blocks that passed the learned level)
    double *d_db = (double *)scratch(ctx, "fs_dblk", sizeof(double) * nb * N1);
    long long iters = 0;
    const int n_pass = n_learned >= 0 ? n_learned : n_hyp;  // -1: every block
    int N1d = N1;  // Delta terms per block in d_db
    if (prm->exact_block) {
        N1d = 1;
        block_lincomb(ctx, prm->beta_block_det, d_dsb, 0.0, nullptr, 0.0, nullptr, d_db);
    } else if (n_pass != 0) {
        iters = block_level(ctx, e0, eN, N1, PSMS_EST_INTERP, prm->seed, prm->step, prm->tol, prm->inner_prec,
                            d_db, d_mask);
    } else {
        cuda_check(cudaMemsetAsync(d_db, 0, sizeof(double) * nb * N1, ctx->stream), "dblk");
    }
    double *d_dsum = (double *)scratch(ctx, "fs_dsum", sizeof(double) * (nb + 1));
    int *d_acc = (int *)scratch(ctx, "fs_acc", sizeof(int) * nb);
    // per-block extra term: beta_block dS_w,b + beta_block_hyp dS_HYP,b
    // (App. C) minus the learned h_b
    const double *d_extra = d_h;
    double coef = -1.0;
    if (prm->beta_block != 0.0 || prm->beta_block_hyp != 0.0) {
        double *d_ex = (double *)scratch(ctx, "fs_extra", sizeof(double) * nb);
        block_lincomb(ctx, prm->beta_block, prm->beta_block != 0.0 ? d_dsw : nullptr, prm->beta_block_hyp,
                      prm->beta_block_hyp != 0.0 ? d_dhyp : nullptr, -1.0, d_h, d_ex);
        d_extra = d_ex;
        coef = 1.0;
    }
    decide(ctx, d_db, nb, N1d, per_block ? 1 : 0, prm->seed, prm->step, PSMS_LEVEL_BLOCK, 0.0, d_extra, coef, d_dsum,
           d_acc, d_mask);
    if (!per_block && n_hyp == 0)  // one decision on the sum: a rejected HYP level rejects the step
        cuda_check(cudaMemsetAsync(d_acc, 0, sizeof(int) * nb, ctx->stream), "reject");
    merge_blocks(ctx, old, prop, mid, d_acc);
    std::vector<double> hd(nb + 1);
    std::vector<int> ha(nb);
    cuda_check(cudaMemcpyAsync(hd.data(), d_dsum, sizeof(double) * (nb + 1), cudaMemcpyDeviceToHost, ctx->stream), "d");
    cuda_check(cudaMemcpyAsync(ha.data(), d_acc, sizeof(int) * nb, cudaMemcpyDeviceToHost, ctx->stream), "a");
    cuda_check(cudaStreamSynchronize(ctx->stream), "filter sync");
    int nacc = 0;
    double dsum = 0;
    for (int b = 0; b < nb; ++b) {
        nacc += ha[b];
        dsum += hd[b];
    }
    if (ctx->rec_h.empty()) ctx->rec_h.assign(nb, 0.0);
    if (ctx->rec_dhyp.empty()) ctx->rec_dhyp.assign(nb, 0.0);
    ctx->rec_acc1.assign(ha.begin(), ha.end());
    // stage 2 of the recursive decomposition (Eq. (4step)): the Schur
    // complements of the outer blocks that changed, between U and the field
    // after the block level
    int n_sub_acc = -1;
    if (recursive) {
        r_lvl.reset();
        r_lvl.reset(new Range("stage 2: outer-block Schur ratios"));
        const int no = n_outer(ctx);
        std::vector<int> oo(nb);  // outer block of every block (lexicographic indices)
        for (int b = 0; b < nb; ++b) {
            int B[4], q = b;
            for (int m = 3; m >= 0; --m) {
                B[m] = q % g.nb[m];
                q /= g.nb[m];
            }
            int o = 0;
            for (int m = 0; m < 4; ++m) o = o * (g.L[m] / ctx->outer[m]) + B[m] * g.l[m] / ctx->outer[m];
            oo[b] = o;
        }
        // an outer block changes when one of its accepted blocks changed a
        // link; the others keep det D-hat_b (Eq. (ddrec)) and Delta_b = 0
        int *d_chg = (int *)scratch(ctx, "fs_chg", sizeof(int) * nb);
        block_changed(ctx, old, prop, d_chg);
        std::vector<int> chg(nb);
        cuda_check(cudaMemcpyAsync(chg.data(), d_chg, sizeof(int) * nb, cudaMemcpyDeviceToHost, ctx->stream), "chg");
        cuda_check(cudaStreamSynchronize(ctx->stream), "chg");
        std::vector<char> changed(no, 0);
        bool any = false;
        for (int b = 0; b < nb; ++b)
            if (ha[b] && chg[b]) changed[oo[b]] = 1, any = true;
        std::vector<double> dsub(no, 0.0);
        if (any) {
            // between U and the field after stage 1, or their relatively
            // gauge-fixed pair: the stage-1 endpoints merged on the accepted
            // inner blocks (the inner blocks decouple)
            const double2 *s0 = old, *s1 = mid;
            if (prm->gauge_fix) {
                merge_blocks(ctx, old, e0, e0, d_acc);
                merge_blocks(ctx, old, eN, eN, d_acc);
                s0 = e0;
                s1 = eN;
            }
            std::vector<double> hs((long long)no * prm->n_sub);
            iters += sub_level(ctx, s0, s1, prm->n_sub, PSMS_EST_INTERP, prm->seed, prm->step, prm->tol,
                               prm->inner_prec, hs.data());
            for (int o = 0; o < no; ++o)
                if (changed[o])
                    for (int i = 0; i < prm->n_sub; ++i) dsub[o] += hs[(long long)o * prm->n_sub + i];
        }
        if (prm->beta_sub != 0.0) {
            std::vector<double> dw(nb);
            cuda_check(cudaMemcpyAsync(dw.data(), d_dsw, sizeof(double) * nb, cudaMemcpyDeviceToHost, ctx->stream),
                       "dS_w");
            cuda_check(cudaStreamSynchronize(ctx->stream), "dS_w");
            std::vector<double> acc_ds(no, 0.0);
            for (int b = 0; b < nb; ++b)
                if (ha[b]) acc_ds[oo[b]] += dw[b];
            for (int o = 0; o < no; ++o) dsub[o] += prm->beta_sub * acc_ds[o];
        }
        for (int o = 0; o < no; ++o)
            if (!std::isfinite(dsub[o])) fail(PSMS_ESPECTRUM, "non-finite outer-block estimate");
        std::vector<char> acc_o(no, 1);
        if (per_block) {
            for (int o = 0; o < no; ++o)
                if (changed[o]) {
                    const double u = uniforms(prm->seed, TAG_ACCEPT, prm->step, PSMS_LEVEL_SUB, (uint64_t)o, 0).u[0];
                    acc_o[o] = (dsub[o] <= 0.0 || u < std::exp(-dsub[o])) ? 1 : 0;
                }
        } else if (any) {
            double tot = 0.0;
            for (int o = 0; o < no; ++o) tot += dsub[o];
            const double u = uniforms(prm->seed, TAG_ACCEPT, prm->step, PSMS_LEVEL_SUB, 0, 0).u[0];
            const char a = (tot <= 0.0 || u < std::exp(-tot)) ? 1 : 0;
            for (int o = 0; o < no; ++o) acc_o[o] = a;
        }
        n_sub_acc = 0;
        for (int o = 0; o < no; ++o) n_sub_acc += changed[o] && acc_o[o];
        ctx->rec_dsub.assign(dsub.begin(), dsub.end());
        ctx->rec_acc_sub.assign(acc_o.begin(), acc_o.end());
        nacc = 0;
        for (int b = 0; b < nb; ++b) {
            ha[b] = ha[b] && acc_o[oo[b]];
            nacc += ha[b];
        }
        cuda_check(cudaMemcpyAsync(d_acc, ha.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, ctx->stream), "acc2");
        merge_blocks(ctx, old, prop, mid, d_acc);
    }
    r_lvl.reset();  // pop before the next push (NVTX ranges nest as a stack)
    r_lvl.reset(new Range("level 2: global det ratio"));
    // level 2: global Schur det ratio (a field equal to the old one has
    // Delta = 0 exactly: every M_i is the identity)
    double dglob = 0;
    int accg = 1;
    double2 *fin = mid;
    if (prm->global_level && nacc > 0) {
        const int N2 = prm->n_global;
        double *d_dg = (double *)scratch(ctx, "fs_dg", sizeof(double) * N2);
        if (prm->gauge_fix) {
            merge_blocks(ctx, old, e0, e0, d_acc);
            merge_blocks(ctx, old, eN, eN, d_acc);
        }
        std::vector<double> hg(N2);
        if (recursive) {
            iters += outer_global_level(ctx, e0, prm->gauge_fix ? eN : mid, N2, PSMS_EST_INTERP, prm->seed,
                                        prm->step, prm->tol, prm->inner_prec, hg.data());
        } else {
            iters += global_level(ctx, e0, prm->gauge_fix ? eN : mid, N2, PSMS_EST_INTERP, prm->seed, prm->step,
                                  prm->tol, prm->inner_prec, d_dg);
            cuda_check(cudaMemcpyAsync(hg.data(), d_dg, sizeof(double) * N2, cudaMemcpyDeviceToHost, ctx->stream),
                       "dg");
            cuda_check(cudaStreamSynchronize(ctx->stream), "dg");
        }
        for (int i = 0; i < N2; ++i) dglob += hg[i];
        if (prm->beta_global != 0.0) {
            double *pd = (double *)scratch(ctx, "fs_plaq", sizeof(double) * 2);
            plaquette_sum(ctx, mid, pd);
            plaquette_sum(ctx, old, pd + 1);
            double hp[2];
            cuda_check(cudaMemcpyAsync(hp, pd, sizeof(hp), cudaMemcpyDeviceToHost, ctx->stream), "plaq");
            cuda_check(cudaStreamSynchronize(ctx->stream), "plaq");
            dglob += prm->beta_global * (-(hp[0] - hp[1]) / 3.0);
        }
        if (prm->beta_global_hyp != 0.0) {
            // S_HYP changes on the accepted blocks only (it factorises over blocks)
            std::vector<double> hh(nb);
            cuda_check(cudaMemcpyAsync(hh.data(), d_dhyp, sizeof(double) * nb, cudaMemcpyDeviceToHost, ctx->stream),
                       "dS_HYP");
            cuda_check(cudaStreamSynchronize(ctx->stream), "dS_HYP");
            double sh = 0.0;
            for (int b = 0; b < nb; ++b)
                if (ha[b]) sh += hh[b];
            dglob += prm->beta_global_hyp * sh;
        }
        if (prm->beta_global_blockdet != 0.0) {
            // S_b changes on the accepted blocks only (the blocks decouple)
            std::vector<double> hb(nb);
            cuda_check(cudaMemcpyAsync(hb.data(), d_dsb, sizeof(double) * nb, cudaMemcpyDeviceToHost, ctx->stream),
                       "dS_b");
            cuda_check(cudaStreamSynchronize(ctx->stream), "dS_b");
            double sb = 0.0;
            for (int b = 0; b < nb; ++b)
                if (ha[b]) sb += hb[b];
            dglob += prm->beta_global_blockdet * sb;
        }
        if (!std::isfinite(dglob)) fail(PSMS_ESPECTRUM, "non-finite global estimate");
        const double u = uniforms(prm->seed, TAG_ACCEPT, prm->step, PSMS_LEVEL_GLOBAL, 0, 0).u[0];
        accg = (dglob <= 0.0 || u < std::exp(-dglob)) ? 1 : 0;
        if (!accg) fin = old;
    }
    r_lvl.reset();
    // random translation
    int sh[4] = {0, 0, 0, 0};
    if (prm->translate) {
        uni4 u = uniforms(prm->seed, TAG_SHIFT, prm->step, 0, 0, 0);
        for (int m = 0; m < 4; ++m) {
            int v = (int)std::floor(u.u[m] * g.L[m]);
            sh[m] = v > g.L[m] - 1 ? g.L[m] - 1 : v;
        }
    }
    translate(ctx, fin, cur, sh);
    touch_field(ctx, field);
    cuda_check(cudaStreamSynchronize(ctx->stream), "filter end");
    if (res) {
        res->n_blocks = nb;
        res->n_accept_blocks = nacc;
        res->accept_global = accg;
        for (int m = 0; m < 4; ++m) res->shift[m] = sh[m];
        res->delta_global = dglob;
        res->delta_block_sum = per_block ? dsum : hd[nb];
        res->solver_iters = iters;
        res->hb_failed = failed;
        res->n_accept_learned = n_learned;
        res->gf_steps = gf_steps;
        res->n_accept_hyp = n_hyp;
        res->n_accept_sub = n_sub_acc;
    }
    if (delta_block_out)
        for (int b = 0; b < nb; ++b) delta_block_out[b] = hd[b];
    if (accept_block_out)
        for (int b = 0; b < nb; ++b) accept_block_out[b] = ha[b];
    PSMS_CATCH(ctx)
}

psms_status psms_filter_record(psms_ctx *ctx, int what, double *out, int n, int *n_out) {
    PSMS_TRY(ctx)
    const std::vector<double> *v = nullptr;
    switch (what) {
        case PSMS_REC_H: v = &ctx->rec_h; break;
        case PSMS_REC_DELTA_HYP: v = &ctx->rec_dhyp; break;
        case PSMS_REC_ACCEPT_BLOCK: v = &ctx->rec_acc1; break;
        case PSMS_REC_DELTA_SUB: v = &ctx->rec_dsub; break;
        case PSMS_REC_ACCEPT_SUB: v = &ctx->rec_acc_sub; break;
        default: fail(PSMS_EINVAL, "unknown filter record");
    }
    if (v->empty()) fail(PSMS_EINVAL, "no filter step has produced this record");
    if (n_out) *n_out = (int)v->size();
    if (!out || n < (int)v->size()) fail(PSMS_EINVAL, "record output too small");
    for (size_t i = 0; i < v->size(); ++i) out[i] = (*v)[i];
    PSMS_CATCH(ctx)
}

psms_status psms_scratch_bytes(const psms_ctx *cctx, size_t *bytes) {
    if (!cctx || !bytes) return PSMS_EINVAL;
    size_t t = 0;
    for (const auto &kv : cctx->scratch) t += kv.second.bytes;
    *bytes = t;
    return PSMS_OK;
}

psms_status psms_max_chunk(psms_ctx *ctx, int n) {
    PSMS_TRY(ctx)
    if (n < 0) fail(PSMS_EINVAL, "the chunk cap must be >= 0");
    ctx->max_chunk = n;
    PSMS_CATCH(ctx)
}

psms_status psms_profile_enable(psms_ctx *ctx, int enable) {
    PSMS_TRY(ctx)
    prof_collect(ctx);
    prof_collect_block(ctx);
    ctx->prof = enable != 0;
    ctx->prof_prec = enable >= 10 ? enable - 10 : -1;
    ctx->prof_launches = 0;
    ctx->prof_ms = 0;
    ctx->prof_bytes = 0;
    ctx->prof_b_launches = 0;
    ctx->prof_b_ms = 0;
    ctx->prof_b_bytes = 0;
    ctx->prof_b_list.clear();
    PSMS_CATCH(ctx)
}

long long psms_kernel_launches(void) { return launch_counter(); }

// checkpoint file: magic, version, dims[4], block[4], kappa, step, seed,
// has_mlp, then the FP64 links in the canonical layout, then (if has_mlp)
// the MLP parameter block as float32
static const char PSMS_MAGIC[8] = {'P', 'S', 'M', 'S', 'C', 'K', 'P', '1'};

psms_status psms_full_solver(psms_ctx *ctx, int kind) {
    PSMS_TRY(ctx)
    if (kind != PSMS_SOLVER_CGNR && kind != PSMS_SOLVER_BICGSTAB) fail(PSMS_EINVAL, "unknown solver");
    ctx->full_solver = kind;
    PSMS_CATCH(ctx)
}

psms_status psms_inner_reduction(psms_ctx *ctx, double delta) {
    PSMS_TRY(ctx)
    if (!(delta == 0.0 || (delta >= 1e-8 && delta <= 0.5))) fail(PSMS_EINVAL, "delta must be 0 or in [1e-8, 0.5]");
    ctx->inner_delta = delta;
    PSMS_CATCH(ctx)
}

psms_status psms_shared_links(psms_ctx *ctx, int on) {
    PSMS_TRY(ctx)
    if (on != 0 && on != 1) fail(PSMS_EINVAL, "on must be 0 or 1");
    ctx->shared_links = on;
    PSMS_CATCH(ctx)
}

psms_status psms_block_krylov(psms_ctx *ctx, int kind) {
    PSMS_TRY(ctx)
    if (kind != PSMS_SOLVER_CGNR && kind != PSMS_SOLVER_BICGSTAB) fail(PSMS_EINVAL, "unknown solver");
    ctx->block_krylov = kind;
    PSMS_CATCH(ctx)
}

psms_status psms_hop_variant(psms_ctx *ctx, int variant, int *n_variants) {
    PSMS_TRY(ctx)
    if (variant < -1 || variant > 14) fail(PSMS_EINVAL, "hop variant must be -1 or 0..14");
    ctx->forced_hop_variant = variant;
    if (n_variants) *n_variants = 15;
    PSMS_CATCH(ctx)
}

psms_status psms_checkpoint_save(psms_ctx *ctx, int field, const char *path, uint64_t step, uint64_t seed) {
    PSMS_TRY(ctx)
    check_field(ctx, field);
    if (!path) fail(PSMS_EINVAL, "null path");
    const long long n = 36 * ctx->g.V;
    std::vector<double2> host(n);
    double2 *canon = (double2 *)scratch(ctx, "ckpt", sizeof(double2) * n);
    gauge_canonical(ctx, canon, ctx->U64[field], 0);
    cuda_check(cudaMemcpyAsync(host.data(), canon, sizeof(double2) * n, cudaMemcpyDeviceToHost, ctx->stream), "ckpt");
    std::vector<float> mlp;
    if (ctx->mlp) {
        mlp.resize(psms_mlp_param_count());
        psms_status st = psms_mlp_params(ctx, mlp.data(), 0);
        if (st) return st;
    }
    cuda_check(cudaStreamSynchronize(ctx->stream), "ckpt");
    FILE *f = std::fopen(path, "wb");
    if (!f) fail(PSMS_EINVAL, std::string("cannot open ") + path);
    int hdr[10] = {1, ctx->g.L[0], ctx->g.L[1], ctx->g.L[2], ctx->g.L[3], ctx->g.l[0], ctx->g.l[1], ctx->g.l[2],
                   ctx->g.l[3], mlp.empty() ? 0 : 1};
    bool ok = std::fwrite(PSMS_MAGIC, 1, 8, f) == 8 && std::fwrite(hdr, sizeof(int), 10, f) == 10 &&
              std::fwrite(&ctx->kappa, sizeof(double), 1, f) == 1 && std::fwrite(&step, sizeof(step), 1, f) == 1 &&
              std::fwrite(&seed, sizeof(seed), 1, f) == 1 &&
              std::fwrite(host.data(), sizeof(double2), n, f) == (size_t)n &&
              (mlp.empty() || std::fwrite(mlp.data(), sizeof(float), mlp.size(), f) == mlp.size());
    ok = (std::fclose(f) == 0) && ok;
    if (!ok) fail(PSMS_EINVAL, std::string("write failed: ") + path);
    PSMS_CATCH(ctx)
}

psms_status psms_checkpoint_load(psms_ctx *ctx, int field, const char *path, uint64_t *step, uint64_t *seed) {
    PSMS_TRY(ctx)
    check_field(ctx, field);
    if (!path) fail(PSMS_EINVAL, "null path");
    FILE *f = std::fopen(path, "rb");
    if (!f) fail(PSMS_EINVAL, std::string("cannot open ") + path);
    char magic[8];
    int hdr[10];
    double kappa = 0;
    uint64_t st_step = 0, st_seed = 0;
    bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, PSMS_MAGIC, 8) == 0 &&
              std::fread(hdr, sizeof(int), 10, f) == 10 && std::fread(&kappa, sizeof(double), 1, f) == 1 &&
              std::fread(&st_step, sizeof(st_step), 1, f) == 1 && std::fread(&st_seed, sizeof(st_seed), 1, f) == 1;
    for (int m = 0; ok && m < 4; ++m) ok = hdr[1 + m] == ctx->g.L[m] && hdr[5 + m] == ctx->g.l[m];
    ok = ok && hdr[0] == 1 && kappa == ctx->kappa;
    if (!ok) {
        std::fclose(f);
        fail(PSMS_EINVAL, "checkpoint does not match this context (format, lattice, blocks or kappa)");
    }
    const long long n = 36 * ctx->g.V;
    std::vector<double2> host(n);
    ok = std::fread(host.data(), sizeof(double2), n, f) == (size_t)n;
    std::vector<float> mlp;
    if (ok && hdr[9]) {
        mlp.resize(psms_mlp_param_count());
        ok = std::fread(mlp.data(), sizeof(float), mlp.size(), f) == mlp.size();
    }
    std::fclose(f);
    if (!ok) fail(PSMS_EINVAL, "truncated checkpoint");
    double2 *canon = (double2 *)scratch(ctx, "ckpt", sizeof(double2) * n);
    cuda_check(cudaMemcpyAsync(canon, host.data(), sizeof(double2) * n, cudaMemcpyHostToDevice, ctx->stream), "ckpt");
    gauge_canonical(ctx, canon, ctx->U64[field], 1);
    touch_field(ctx, field);
    cuda_check(cudaStreamSynchronize(ctx->stream), "ckpt");
    if (!mlp.empty()) {
        psms_status st = psms_mlp_params(ctx, mlp.data(), 1);
        if (st) return st;
    }
    if (step) *step = st_step;
    if (seed) *seed = st_seed;
    PSMS_CATCH(ctx)
}

psms_status psms_profile_block_launches(psms_ctx *ctx, int n_max, int *n_out, double *ms, double *bytes) {
    PSMS_TRY(ctx)
    if (n_max < 0 || !n_out) fail(PSMS_EINVAL, "n_max >= 0 and n_out required");
    prof_collect_block(ctx);
    const int n = std::min(n_max, (int)ctx->prof_b_list.size());
    for (int i = 0; i < n; ++i) {
        if (ms) ms[i] = ctx->prof_b_list[i].first;
        if (bytes) bytes[i] = ctx->prof_b_list[i].second;
    }
    *n_out = n;
    PSMS_CATCH(ctx)
}

psms_status psms_profile_read_block(psms_ctx *ctx, long long *launches, double *total_ms, double *bytes) {
    PSMS_TRY(ctx)
    prof_collect_block(ctx);
    if (launches) *launches = ctx->prof_b_launches;
    if (total_ms) *total_ms = ctx->prof_b_ms;
    if (bytes) *bytes = ctx->prof_b_bytes;
    PSMS_CATCH(ctx)
}

psms_status psms_autotune(psms_ctx *ctx, int enable, int block_variant) {
    PSMS_TRY(ctx)
    if (block_variant < -1 || block_variant > 20) fail(PSMS_EINVAL, "block_variant must be -1 or 0..20");
    ctx->autotune = enable != 0;
    ctx->forced_block_variant = block_variant;
    ctx->block_variant.clear();
    for (auto &plane : ctx->hop_variant)
        for (auto &row : plane)
            for (auto &cell : row) cell[0] = cell[1] = -1;
    PSMS_CATCH(ctx)
}

psms_status psms_profile_read(psms_ctx *ctx, long long *launches, double *total_ms, double *bytes) {
    PSMS_TRY(ctx)
    prof_collect(ctx);
    if (launches) *launches = ctx->prof_launches;
    if (total_ms) *total_ms = ctx->prof_ms;
    if (bytes) *bytes = ctx->prof_bytes;
    PSMS_CATCH(ctx)
}

}  // extern "C"
