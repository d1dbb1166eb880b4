// device.cuh - device-side views of a plan and the launch interfaces between the
// C ABI (api.cu) and the kernel files (internal).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "numeric.cuh"
#include "walk.hpp"

namespace mbc {

// Shared-memory leading dimension of a staged 12x12 block: 13 values per row so that
// 16-byte reads of one column by 8 consecutive rows hit 8 different bank groups.
static constexpr int kLd = 13;
static constexpr int kBlk = 12 * kLd;

// Work geometry shared by every algorithm: n_sets x T x V3 sites, fields laid out
// [set][t][site][12][12] complex double; a "site" below is the flat index
// (set * T + t) * V3 + x.
struct Geometry {
    int n_sets, T;
    int64_t V3;
    __host__ __device__ int64_t n_sites() const { return (int64_t)n_sets * T * V3; }
};

// Partial sums: one per (site, chunk); each holds a compensated complex double
// (re.hi, re.lo, im.hi, im.lo).
struct Partials {
    d4* part;          // [n_sites * n_chunks]
    int n_chunks;
};

// ---------------------------------------------------------------- direct sweep
struct DirectDev {
    int n_u, n_d;
    int explicit_terms;
    // factored: blocks of sink range x source range with coefficient P
    int n_blocks;
    const int64_t* blk_start;      // [n_blocks + 1] prefix sums of pairs
    const int64_t* blk_s0; const int64_t* blk_r0; const int64_t* blk_nr; const int64_t* blk_ns;
    // weights below are 16-byte values of the plan's precision (cd or cdf)
    const void* blk_p;
    const int8_t* snk_idx; const void* snk_w;
    const int8_t* src_idx; const void* src_w;
    // explicit: term t = (ex_snk[t], ex_src[t], ex_w[t])
    const int8_t* ex_snk; const int8_t* ex_src; const void* ex_w;
    int64_t index_size;
};

// ---------------------------------------------------------------- factor tree
struct TreeDev {
    int n_u, n_d;
    int64_t n_minors[2];
    const int8_t* minor_rows[2];   // [m][n_f]
    const int8_t* minor_cols[2];
    int64_t n_nodes;
    const int32_t* factors;
    const int32_t* children;
    const void* coefficients;      // precision-P values
    int n_chunks;
    const int64_t* chunk_node;
    const int64_t* chunk_leaf;
    const int32_t* chunk_count;
};

// ---------------------------------------------------------------- e-graph plan
struct MinorDev {
    int n;
    int size[7];                   // |F_k|, k = 0..6 (size[0] = 1)
    int off[7];                    // offset of level k in a stacked table
    const uint16_t* child[7];      // [e * k + i]
    const uint8_t* row[7];
    const uint32_t* pack[7];       // [i * size[k] + e] = child | row << 16 (one entry's words strided,
                                   // so the threads of a warp read consecutive words)
    int n_nodes;
    const uint8_t* node_level;
    const uint8_t* node_col;
    const int8_t* node_sign;
    const int32_t* node_leaf;
};

struct EgraphDev {
    int flav_a, n_j;
    int real_w;                      // every G weight and pair coefficient is real
    int compact;                     // ... and exact in float: g_ws / pair_cs hold them as
    const void* g_ws;                // scalars of the precision (double or float): [entry]
    const void* pair_cs;             // [pair * n_j + j]
    MinorDev A, B;
    int n_rows_b, n_cols_b;          // K is n_cols_b x n_rows_b per block slot
    const int32_t* g_off; const int32_t* g_a; const void* g_w;           // g_w, pair_coef:
    const int32_t* pair_off; const int32_t* pair_b; const uint8_t* pair_first;
    const void* pair_coef;                                               // precision-P values
    int stack_a;                     // values in the A stack (levels 0..n_A)
    int stack_b;                     // values in the B stack (levels 0..n_B)
    int smem_values;                 // total complex values in dynamic shared memory
    int stage_pk;                    // copy the leaf-level packed tables to shared memory
    // G entries of the fused leaf path in sliced-ELL form: for the 32 B row sets of slice
    // s and free index j, entry k of lane l at sell[sell_off[s * n_j + j] + k * 32 + l]
    // (k < sell_w[s * n_j + j]; padding entries have weight 0), so the loads of a warp are
    // consecutive 8-byte records
    const int2* sell;                // (T index, float weight bits)
    const int32_t* sell_off;
    const int32_t* sell_w;
    // pairs of the fused leaf path (n_j <= 2, weights exact in float): (B column |
    // first update << 31, float bits of coef_0, of coef_1, 0)
    const int4* pair_rec;
    // per A leaf: bit j set when some pair of the leaf has coef_j != 0 (fused leaf path)
    const uint8_t* leaf_jmask;
};

// ---------------------------------------------------------------- FP32 e-graph plan
// Walker programs of one flavour (walk.hpp) with the level tables they use.
struct WalkDev {
    int n;                           // minor size
    int size[7];                     // entries of the level-k table (size[0] = 1)
    int off[7];                      // offset of level k (0..n-1) in a walker's table stack
    int pk_off[7];                   // offset of level k's packed words in the staged word array
    const WalkStep* steps;
    const int32_t* step_off;         // [walkers + 1]
    const WalkLeaf* leaves;
    int n_steps, n_leaves;           // array sizes (bounds-checking build)
};

// The e-graph plan of the FP32 kernel: the same column trees, G entries and pairs as
// EgraphDev, arranged for walkers of 128 threads and FP32 values.
struct Eg32Dev {
    int flav_a, n_j, real_w;
    int walkers, lb;                 // walkers per block, leaf batch size of the A flavour
    int cs;                          // blocks per site (a thread-block cluster when > 1)
    int n_rows_b, n_cols_b;          // the B table of a site is n_cols_b x n_rows_b
    int stack_vals;                  // float2 values of a walker's table stack
    int leafbuf_vals;                // lb x size_A[n_A]
    int pk_words;                    // packed Laplace words staged in shared memory (A, then B)
    const uint32_t* pk;              // their global copy
    WalkDev A, B;
    // G entries in sliced-ELL form (slices of 32 B row sets; entry k of lane l of slice s
    // and free index j at [sell_off[s * n_j + j] + 32 k + l], k < sell_w[s * n_j + j])
    const int32_t* sell_off;
    const int32_t* sell_w;
    const int2* sell;                // real weights: (A row-set index, float weight bits)
    const int4* sellc;               // complex weights: (A row-set index, re bits, im bits, 0)
    int g_small;                     // every G weight a real number with at most 8 significant
                                     // bits (a bfloat16) and every A row-set index < 65536:
    const uint32_t* sell1;           // ... then the entries are (index | bf16 weight << 16)
    // pair terms, one per pair (C_a, C_b) and free index j with coef_j != 0, coef_j =
    // sum_j' P_jj' conj(r_j'(C_a, C_b)); the terms of A leaf C_a are [term_off[C_a],
    // term_off[C_a + 1]); x = 4 (C_b n_rows_b) + j
    const int32_t* term_off;         // [|cols_A| + 1]
    const int2* term2;               // real coefficients: (x, float bits of coef_j)
    const int4* term4;               // complex coefficients: (x, re bits, im bits, 0)
    const uint8_t* leaf_jmask;       // per A leaf: bit j set when a pair of the leaf has coef_j != 0
    // B row sets in the order of the leaf stage (and of the site's B table): sorted by their
    // G entry count, so that the 32 row sets of a sliced-ELL slice have similar widths;
    // b_pos[e] = position of the B leaf level's row set e
    const int32_t* b_pos;
    float guard;                     // a site whose error estimate exceeds this is recomputed
    int smem_bytes;                  // dynamic shared memory of the kernel
    int n_cols_a;                    // A leaves (column sets)
    int64_t n_terms, n_sell;         // array sizes (bounds-checking build)
};

// One item of a batched FP32 launch: the plan's FP32 view, its fields and geometry, where
// its per-site partials and error scales go, its first work unit and first time slice
// (numbered item by item), and its guards.
struct BatchItem32 {
    Eg32Dev d;
    const double* U;
    const double* D;
    d4* part;
    double* scale;
    Geometry g;
    int64_t unit_begin;
    int64_t slice_begin;
    float site_guard;
    double slice_tol;
};

// One item of a batched launch: a plan's device view, its fields, where its per-site
// partials go, and the number of the item's first work unit (site).
struct BatchItem {
    EgraphDev d;
    const double* U;
    const double* D;
    d4* part;
    int64_t unit_begin;
    int64_t n_sites;
};

// ---------------------------------------------------------------- launchers
cudaError_t launch_direct(const DirectDev& d, int prec, const double* U, const double* D, Geometry g,
                          int64_t chunk, Partials out, int threads, cudaStream_t s, int64_t* launches);
cudaError_t launch_tree(const TreeDev& d, int prec, const double* U, const double* D, Geometry g,
                        void* scratch, int64_t scratch_sites, int* exps, Partials out, int threads,
                        cudaStream_t s, int64_t* launches);
size_t tree_value_bytes(int prec);
cudaError_t launch_egraph(const EgraphDev& d, int prec, const double* U, const double* D, Geometry g,
                          Partials out, int threads, int grid, unsigned int* counter, void* kscratch,
                          cudaStream_t s, int64_t* launches);
size_t egraph_smem_bytes(const EgraphDev& d, int prec);
cudaError_t launch_egraph_batch(const BatchItem* items, int n_items, int64_t n_units, int prec, int threads, int grid,
                                size_t smem, unsigned int* counter, void* kscratch, int64_t kslot_values, cudaStream_t s,
                                int64_t* launches);
size_t egraph_kslot_bytes(const EgraphDev& d);
// Batched FP32 launch over items (device table) sharing one cluster size, walker count
// and shared-memory layout size (smem bytes): the FP32 kernel over every (item, site)
// unit, then the slice guard of every item's time slices (n_slices in all).  Units to
// recompute go to flag_list.  bslots: one bslot_values float2 table per cluster.
cudaError_t launch_egraph32_batch(const BatchItem32* items, int n_items, int64_t n_units, int64_t n_slices, bool real,
                                  int nj, int cs, int walkers, int smem, int max_grid, void* bslots,
                                  int64_t bslot_values, unsigned int* flag_count, unsigned int* flag_list,
                                  cudaStream_t s, int64_t* launches);
// The double-float batched kernel over a device list of units (list_n: device count).
cudaError_t launch_egraph_batch_list(const BatchItem* items, int n_items, int64_t n_units, int threads, int grid,
                                     size_t smem, unsigned int* counter, void* kscratch, int64_t kslot_values,
                                     const unsigned int* list, const unsigned int* list_n, cudaStream_t s,
                                     int64_t* launches);
// The double-float e-graph kernel over a device list of sites (list_n: device count).
cudaError_t launch_egraph_list(const EgraphDev& d, const double* U, const double* D, Partials out, int threads,
                               int grid, unsigned int* counter, void* kscratch, const unsigned int* list,
                               const unsigned int* list_n, int64_t n_sites, cudaStream_t s, int64_t* launches);
// Bounds-checking build (-DMBC_DEVICE_CHECKS): the first failed device check of the
// FP32 kernels (egraph32.cu) and of the double-float e-graph kernels (egraph.cu); both
// synchronise the device and clear the record.  Normal build: always empty.
struct CheckRecord;
cudaError_t egraph32_checks(CheckRecord* out);
cudaError_t egraph_checks(CheckRecord* out);

// Sink momentum of the site sum: p in units of 2 pi / L, site x of a slice at
// (x mod L, (x / L) mod L, x / L^2); p = 0 is the plain sum.
struct Momentum {
    int L = 1, px = 0, py = 0, pz = 0;
    __host__ __device__ bool nonzero() const { return (px | py | pz) != 0; }
};
// FP32 e-graph kernel (egraph32.cu): one block per SM, one site per cluster of d.cs
// blocks at a time, at most max_grid blocks; then the slice guard (unless slice_tol is
// +inf).  Writes every site's partial and its error scale (scale, [n_sites] double, 0
// for a site already listed); sites whose error estimate exceeds site_guard, and the
// remaining sites of every time slice whose C(t) error estimate exceeds slice_tol |C(t)|,
// are appended to flag_list (flag_count counts them) for the double-float kernel to
// recompute.  bslots: one n_cols_b x n_rows_b float2 table per cluster (max_grid / d.cs).
cudaError_t launch_egraph32(const Eg32Dev& d, const double* U, const double* D, Geometry g, d4* part, int max_grid,
                            void* bslots, unsigned int* flag_count, unsigned int* flag_list, float site_guard,
                            double slice_tol, double* scale, Momentum mom, cudaStream_t s, int64_t* launches);
// C[set][t] = scale * sum_x e^{-i 2 pi p.x / L} (sum over chunks of the site's partials);
// site_out (optional) receives scale * the site values without the phase.
cudaError_t launch_reduce(Partials in, Geometry g, cd scale, double2* C, double2* site_out, d4* site_tmp,
                          cudaStream_t s, int64_t* launches, Momentum mom = Momentum());

}  // namespace mbc
