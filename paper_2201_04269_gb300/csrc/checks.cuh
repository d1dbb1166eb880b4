// checks.cuh - device bounds checks of the bounds-checking build (internal).
//
// Built with -DMBC_DEVICE_CHECKS, MBC_BAD(cond, code, value, bound) is true when an index
// is out of range: the first failure (check code, offending value, the bound it broke)
// is recorded in the translation unit's g_check and the caller skips the access instead
// of faulting; the unit's read_checks() copies the record to the host and clears it.  In
// the normal build MBC_BAD is constant false and compiles away.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace mbc {
struct CheckRecord {
    int code;
    int count;
    long long value;
    long long bound;
};
}  // namespace mbc

#ifdef MBC_DEVICE_CHECKS
static __device__ mbc::CheckRecord g_check;
static inline cudaError_t read_checks(mbc::CheckRecord* out) {
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpyFromSymbol(out, g_check, sizeof(mbc::CheckRecord));
    mbc::CheckRecord zero = {0, 0, 0, 0};
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_check, &zero, sizeof zero);
    return e;
}
__device__ __forceinline__ bool mbc_check_fail(int code, long long value, long long bound) {
    if (atomicAdd(&g_check.count, 1) == 0) {
        g_check.code = code;
        g_check.value = value;
        g_check.bound = bound;
    }
    return true;
}
#define MBC_BAD(cond, code, value, bound) (!(cond) && mbc_check_fail((code), (long long)(value), (long long)(bound)))
#else
#define MBC_BAD(cond, code, value, bound) false
static inline cudaError_t read_checks(mbc::CheckRecord* out) {
    *out = mbc::CheckRecord{0, 0, 0, 0};
    return cudaSuccess;
}
#endif
