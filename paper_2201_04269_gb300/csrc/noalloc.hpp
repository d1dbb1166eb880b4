// noalloc.hpp - the plan fields that the allocation-free entry point (noalloc.cu) reads
// (internal; filled by api.cu, which owns the plan structure).
#pragma once
#include <string>

#include "device.cuh"
#include "mbc.h"

namespace mbc {
struct NoallocView {
    int device, algo, prec, threads, blocks_per_sm, sms;
    cd scale;
    EgraphDev ed;
    bool empty;
    std::string* err;
    int64_t* launches;
};
bool noalloc_view(mbc_plan* plan, NoallocView* v);
}  // namespace mbc
