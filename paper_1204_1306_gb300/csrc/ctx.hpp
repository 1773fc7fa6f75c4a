// Host-side context of the library: geometry, gauge-field slots, scratch
// buffers, stream and error state.  Shared by the translation units.
#pragma once

#include <cuda_runtime.h>

#include <map>
#include <string>
#include <vector>

#include "../../include/psms.h"
#include "common.cuh"

namespace psms {

struct Error {
    psms_status st;
    std::string msg;
};

[[noreturn]] inline void fail(psms_status st, const std::string &m) { throw Error{st, m}; }

inline void cuda_check(cudaError_t e, const char *what) {
    if (e != cudaSuccess) {
        cudaGetLastError();  // clear a non-sticky error so later launch checks do not report it
        psms_status st = (e == cudaErrorMemoryAllocation) ? PSMS_ENOMEM : PSMS_ECUDA;
        fail(st, std::string(what) + ": " + cudaGetErrorString(e));
    }
}

// process-wide count of kernel launches issued by the library
long long &launch_counter();
#define PSMS_LAUNCH_CHECK(what) (++::psms::launch_counter(), ::psms::cuda_check(cudaGetLastError(), what))

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

}  // namespace psms

struct psms_ctx {
    psms::Geom g;
    double kappa = 0;
    double A = 0;  // 4 + m0 = 1 / (2 kappa)
    int n_fields = 0;
    std::vector<double2 *> U64;   // FP64 links per slot, [mu][e][s]
    std::vector<float2 *> U32;    // FP32 copies, valid when u32_ok
    std::vector<int> u32_ok;
    std::vector<psms::BlockInfo> h_binfo;
    psms::BlockInfo *d_binfo = nullptr;
    cudaStream_t stream = nullptr;
    std::string err;
    std::map<std::string, psms::DevBuf> scratch;
    // profiling of Wilson-operator launches
    bool prof = false;
    int prof_prec = -1;  // profile hop launches of this storage precision only (-1: all)
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<int, double>> prof_pending;  // (event pair index, bytes per output site)
    unsigned long long *d_prof_sites = nullptr;         // per pending launch: active output sites
    int prof_cap = 0;
    long long prof_launches = 0;
    // autotuned hop-kernel variant per (storage precision, both parities,
    // whole lattice or not, shared-endpoint links or not); -1 untuned
    int hop_variant[3][2][2][2] = {{{{-1, -1}, {-1, -1}}, {{-1, -1}, {-1, -1}}},
                                   {{{-1, -1}, {-1, -1}}, {{-1, -1}, {-1, -1}}},
                                   {{{-1, -1}, {-1, -1}}, {{-1, -1}, {-1, -1}}}};
    bool autotune = true;
    int forced_hop_variant = -1;  // -1: autotuned; else the variant index (mod the variant count)
    double inner_delta = 0;       // inner relative reduction of whole-lattice solves (0: defaults)
    int shared_links = 1;         // estimators' whole-lattice FP32 solves: shared-endpoint links
    int full_solver = 1;          // inner Krylov method of whole-lattice solves: 0 CGNR, 1 BiCGStab
    int block_krylov = 0;         // inner Krylov method of block solves: 0 CGNR, 1 BiCGStab
    int outer[4] = {0, 0, 0, 0};  // outer blocks of the recursive decomposition (0: none)
    int max_chunk = 0;            // cap on systems per estimator launch (0: from the memory estimate)
    // per-block records of the last filter step (psms_filter_record); empty
    // until a step has produced them
    std::vector<double> rec_h, rec_dhyp, rec_acc1, rec_dsub, rec_acc_sub;
    // autotuned block-solver variant per (precision, block size, batched)
    std::map<long long, int> block_variant;
    int forced_block_variant = -1;
    // learned level: MLP state (owned, freed with mlp_free)
    void *mlp = nullptr;
    void (*mlp_free)(void *) = nullptr;
    double prof_ms = 0, prof_bytes = 0;
    // profiling of block-solver launches: (event pair, algorithmic bytes)
    std::vector<cudaEvent_t> ev_pool_b;
    std::vector<std::pair<int, double>> prof_b_pending;
    int last_block_slot = -1;
    long long prof_b_launches = 0;
    double prof_b_ms = 0, prof_b_bytes = 0;
    std::vector<std::pair<float, double>> prof_b_list;  // per launch: (ms, algorithmic bytes), first 4096
};

namespace psms {

// grow-only named scratch buffer
void *scratch(psms_ctx *c, const std::string &name, size_t bytes);
// FP32 copy of a gauge slot (converted on first use after a change)
float2 *links32(psms_ctx *c, int field);
inline void touch_field(psms_ctx *c, int f) { c->u32_ok[f] = 0; }
void check_field(psms_ctx *c, int f);

// profiling hooks around Wilson-operator launches
int prof_begin(psms_ctx *c);
void prof_end(psms_ctx *c, int slot, double bytes_per_site);
unsigned long long *prof_counter(psms_ctx *c, int slot);
// block-solver launches: events around the launch; bytes set afterwards from
// the iterations the solve reports
int prof_block_begin(psms_ctx *c);
void prof_block_end(psms_ctx *c, int slot);
void prof_block_bytes(psms_ctx *c, long long block_iters, int inner_prec);

}  // namespace psms
