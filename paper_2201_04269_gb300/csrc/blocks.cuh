// blocks.cuh - device views and launchers of the hadron-block kernels (internal).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "numeric.cuh"

namespace mbc {

// One block type on the device: flavour of q1 (0 = u, 1 = d) and the nonzeros of G.
struct BlockTypeDev {
    int q1;
    int n;
    int be[4], ga[4];
    double g_re[4], g_im[4];
};

// The block entries one launch computes.  entry[f] packs (slot << 16) | (s1 << 12) |
// (s2 << 8) | (s3 << 4) | alpha, where slot indexes t[]; entry == nullptr means all
// 6912 entries of slot 0 in eta order.
struct BlockDev {
    int n_f;
    const uint32_t* entry;
    int n_types;
    BlockTypeDev t[6];
};

// Factor tree of a block plan on the device (see BlockHostPlan).
struct BlockTreeDev {
    int A;
    int n_f;
    int64_t n_units;
    const uint16_t* unit_pre;      // [n_units][A - 1]
    const int32_t* unit_leaf;      // [n_units + 1]
    const uint16_t* leaf_f;        // [leaves]
    const float2* leaf_w;          // [leaves] integer-valued weights (exact in float): double-float tree
    const double2* leaf_wd;        // [leaves] the same in double: FP64 tree
    int n_chunks;
    const int64_t* chunk_unit;     // [n_chunks + 1]
};

// Largest entry count one block of the projected kernel holds in shared memory.
int block_entries_per_cta(int n_types);
size_t block_kernel_smem(int n_f, int n_types, bool projected);

// Per-site blocks: out [n_sites][b.n_f] complex double.
cudaError_t launch_blocks_site(const BlockDev& b, const double* U, const double* D, int64_t n_sites, cd* out,
                               int sms, cudaStream_t s, int64_t* launches);
// Projected blocks: F [n_slices][b.n_f] = sum over the V3 sites of each slice of
// e^{-i 2 pi p.x / L} f(x), in complex double (prec 0) or double-float (prec 1, block
// types with G entries in {0, +1, -1}); part: scratch of block_project_scratch(...)
// complex doubles.
int64_t block_project_scratch(int n_f, int n_types, int64_t n_slices, int64_t V3, int sms);
cudaError_t launch_blocks_projected(const BlockDev& b, int prec, const double* U, const double* D, int64_t n_slices,
                                    int64_t V3, int L, const int* p, cd* part, cd* F, int sms, cudaStream_t s,
                                    int64_t* launches);
// Local-sink block form: part [n_sites] = per-site compensated sums of the block factor
// tree over the site's own blocks (complex double); cudaErrorInvalidValue when the
// plan's block entries do not fit shared memory.
cudaError_t launch_block_local(const BlockDev& b, const BlockTreeDev& t, const double* U, const double* D,
                               int64_t n_sites, d4* part, int sms, cudaStream_t s, int64_t* launches);
// Factor tree over projected blocks: part [n_slices][t.n_chunks] compensated partial sums;
// prec 0 in complex double, 1 in double-float (the slice's blocks scaled by a power of two).
cudaError_t launch_block_tree(const BlockTreeDev& t, int prec, const cd* F, int64_t n_slices, d4* part,
                              cudaStream_t s, int64_t* launches);

}  // namespace mbc
