// noalloc.cu - correlator evaluation that allocates no device memory.
//
// Some callers cannot call cudaMalloc at the moment they need a correlator: services
// whose device memory is carved out once at start up and must not grow afterwards (an
// allocation could fail, or take memory another tenant of the GPU was promised),
// plug-ins running inside a host application that owns every device allocation, and
// real-time loops where an allocation's latency and implicit synchronisation are not
// acceptable.  mbc_correlator normally takes its temporaries (the per-block K slots of
// the e-graph kernel, the per-site partial sums and the work counter) from the
// context's pool, growing it with cudaMalloc when a call needs more.  This file offers
// the same e-graph kernel with every temporary taken from one fixed array compiled into
// the library instead.
//
// The array is a file-scope __device__ variable of MBC_NOALLOC_SCRATCH_BYTES bytes:
// every GPU that loads this part of the library holds it until the process exits.
// Its host-side name is not a device address, so the device address is looked up with
// cudaGetSymbolAddress once per device, on the first call made on that device, and
// kept for the life of the process (a device reset invalidates it: after
// cudaDeviceReset the entry point is not usable again in that process).
#include <algorithm>
#include <cstdio>
#include <mutex>
#include <string>

#include "device.cuh"
#include "mbc.h"

#include "noalloc.hpp"
#include "ctx.hpp"

using namespace mbc;

namespace {

static __device__ __align__(256) unsigned char g_scratch[MBC_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
void* g_scratch_ptr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mutex;

// Device address of g_scratch on the current device (looked up once per device).
cudaError_t scratch_address(int device, void** out) {
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_ptr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[device] = p;
    }
    *out = g_scratch_ptr[device];
    return cudaSuccess;
}

size_t align256(size_t n) { return (n + 255) / 256 * 256; }

}  // namespace

extern "C" mbc_status mbc_correlator_noalloc(mbc_plan* plan, const void* U, const void* D, int n_sets, int T,
                                             int64_t V3, void* C, mbc_stream stream) {
    Range range_("mbc_correlator_noalloc");
    if (!plan) return MBC_INVALID_ARG;
    NoallocView v;
    if (!noalloc_view(plan, &v)) return MBC_INVALID_ARG;
    auto fail = [&](mbc_status s, const std::string& m) { *v.err = m; return s; };
    if (v.device < 0) return fail(MBC_UNSUPPORTED, "host-only context (device -1) cannot evaluate");
    if (v.device >= kMaxDevices) return fail(MBC_UNSUPPORTED, "device index beyond the no-allocation table");
    if (v.algo != MBC_ALGO_EGRAPH) return fail(MBC_UNSUPPORTED, "mbc_correlator_noalloc needs an MBC_ALGO_EGRAPH plan");
    if (n_sets < 0 || T < 0 || V3 < 0) return fail(MBC_INVALID_ARG, "negative size");
    const int64_t n_sites = (int64_t)n_sets * T * V3;
    if ((int64_t)n_sets * T > 0 && !C) return fail(MBC_INVALID_ARG, "null output");
    if (n_sites > 0 && (!U || !D)) return fail(MBC_INVALID_ARG, "null propagator field");
    cudaError_t e = cudaSetDevice(v.device);
    if (e != cudaSuccess) return fail(MBC_CUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
    cudaStream_t s = (cudaStream_t)stream;
    // plans whose canonical term set is empty give C = 0 without a kernel (as
    // mbc_correlator does), whatever the size
    if (v.empty || n_sites == 0) {
        if ((int64_t)n_sets * T > 0) {
            e = cudaMemsetAsync(C, 0, sizeof(double2) * (size_t)n_sets * T, s);
            if (e != cudaSuccess) return fail(MBC_CUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
        }
        v.err->clear();
        return MBC_OK;
    }
    // scratch layout: [work counter | per-site partials | K slots]
    const size_t counter_bytes = 256;
    const size_t part_bytes = align256(sizeof(d4) * (size_t)n_sites);
    const size_t kslot = egraph_kslot_bytes(v.ed);
    const size_t need_min = counter_bytes + part_bytes + kslot;
    if (need_min > (size_t)MBC_NOALLOC_SCRATCH_BYTES) {
        char buf[256];
        snprintf(buf, sizeof buf,
                 "mbc_correlator_noalloc: %lld sites need %zu bytes of scratch (one K slot %zu, partials %zu); "
                 "the fixed array holds %zu bytes",
                 (long long)n_sites, need_min, kslot, part_bytes, (size_t)MBC_NOALLOC_SCRATCH_BYTES);
        return fail(MBC_UNSUPPORTED, buf);
    }
    void* base = nullptr;
    e = scratch_address(v.device, &base);
    if (e != cudaSuccess) return fail(MBC_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    unsigned char* p = static_cast<unsigned char*>(base);
    unsigned int* counter = reinterpret_cast<unsigned int*>(p);
    d4* parts = reinterpret_cast<d4*>(p + counter_bytes);
    void* kscratch = p + counter_bytes + part_bytes;
    // as many blocks as K slots fit (each block owns one slot)
    const int64_t slots = (int64_t)(((size_t)MBC_NOALLOC_SCRATCH_BYTES - counter_bytes - part_bytes) / kslot);
    const int64_t max_blocks = std::min<int64_t>(n_sites, (int64_t)v.sms * v.blocks_per_sm);
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(max_blocks, slots));
    Geometry g{n_sets, T, V3};
    Partials pt{parts, 1};
    // the work counter is the only scratch that must start at zero (launch_egraph clears
    // it on the stream); K slots are written before they are read, partials fully written.
    // MBC_PREC_FP32 plans are evaluated here with the double-float kernel.
    e = launch_egraph(v.ed, v.prec == MBC_PREC_FP64 ? 0 : 1, (const double*)U, (const double*)D, g, pt, v.threads, grid, counter, kscratch, s,
                      v.launches);
    if (e != cudaSuccess) return fail(MBC_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
    e = launch_reduce(pt, g, v.scale, (double2*)C, nullptr, nullptr, s, v.launches);
    if (e != cudaSuccess) return fail(MBC_CUDA, std::string("reduction launch: ") + cudaGetErrorString(e));
    v.err->clear();
    return MBC_OK;
}
