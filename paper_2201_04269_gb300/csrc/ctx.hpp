// ctx.hpp - the library context shared by the ABI files (internal).
#pragma once
#include <map>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "mbc.h"
#include "device.cuh"

namespace mbc {

// A growable device buffer of the context's pool.
struct Buf {
    void* p = nullptr;
    size_t n = 0;
};

}  // namespace mbc

struct mbc_ctx {
    int device = 0;
    std::string err;
    int64_t launches = 0;
    int sms = 0;
    mbc::Buf partials, site_tmp, scratch, exps, counter, hU, hD, hC;
    // mbc_correlator_host: a copy stream and one event per slice chunk (created on first use)
    static constexpr int kHostChunks = 8;
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t h2d_start = nullptr, h2d_done[kHostChunks] = {};
    std::vector<mbc_plan*> plans;
    std::vector<mbc_block_plan*> block_plans;
    std::map<std::string, mbc_schedule> tune_cache;
    // batched launches: item tables per precision (device) and the reserved item list
    mbc::Buf batch_items, batch_parts, batch_k;
    std::vector<mbc_work> batch_reserved;
    std::vector<mbc::BatchItem> batch_host[2];
    size_t batch_smem[2] = {0, 0};
    int64_t batch_units[2] = {0, 0}, batch_kslot = 0;
    int batch_grid = 0, batch_threads = 384;
    // hadron blocks: per-tile partial blocks, projected blocks, tree partials
    mbc::Buf blk_part, blk_F, blk_tree;
    // FP32 e-graph: one B table per cluster, the list of sites to recompute, the sites'
    // error scales
    mbc::Buf bslot, flags, gscale;
    // batched FP32 items: their FP32 and double-float item tables (device) and launch shape
    mbc::Buf batch32_items, batch32_scale;
    std::vector<mbc::BatchItem32> batch32_host;
    std::vector<int> batch32_src;              // the mbc_work index of each FP32 table entry
    std::vector<mbc::BatchItem> batch32_df_host;
    int64_t batch32_units = 0, batch32_slices = 0, batch32_bvals = 0;
    int batch32_cs = 1, batch32_walkers = 1, batch32_smem = 0, batch32_nj = 1, batch32_df_threads = 384;
    bool batch32_real = true;
    size_t batch32_df_smem = 0;
};

namespace mbc {

mbc_status fail(mbc_ctx* c, mbc_status s, const std::string& m);
mbc_status cuda_fail(mbc_ctx* c, cudaError_t e, const char* what);
bool capturing(cudaStream_t s);
// Grow a pool buffer to at least `bytes` (never during a stream capture).
mbc_status ensure(mbc_ctx* c, Buf& b, size_t bytes, cudaStream_t s);
// Free every block plan of the context (blocks_api.cu).
void destroy_block_plans(mbc_ctx* c);

// NVTX range around an ABI call (a no-op unless a profiler is attached): the planner and
// every evaluation show up by name on a profiler's timeline, and `ncu --clock-control
// none --nvtx --nvtx-include "mbc_correlator/"` captures only the kernels of that call
// (always with --clock-control none on a shared GPU: ncu otherwise locks the clocks).
struct Range {
    explicit Range(const char* name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range&) = delete;
    Range& operator=(const Range&) = delete;
};

}  // namespace mbc
