// egraph.cu - evaluation of the plan extracted from the tensor e-graph
// (arXiv 2201.04269 Sec. 5) for the canonical correlator (Sec. 3).
//
// Per site the correlator is
//   C_x = sum_{(j, j')} P_jj' sum_{(R_a, R_b)} s_j sum_{(C_a, C_b)} conj(r_j') A[R_a, C_a] B[R_b, C_b]
// with A, B the minors of the two flavours.  The extracted plan stages it as
//   K(C_b, R_b) = sum_{C_a} sum_j coef_j(C_a, C_b) G_j(C_a, R_b),
//   G_j(C_a, R_b) = sum_{R_a} s_j(R_a, R_b) A[R_a, C_a],   coef_j = sum_j' P_jj' conj(r_j'),
//   C_x = sum_{C_b} sum_{R_b} K(C_b, R_b) B[R_b, C_b],
// so every minor of either flavour is formed once per site.  Minors come from the
// extracted column trees: a node's table det M[R, C] (every needed row set R of the
// level) follows from its parent's table by one Laplace step along the added column c,
//   det M[R, C] = sum_i (-1)^{i+q} M[r_i, c] det M[R \ r_i, C \ c],
// and a depth-first walk keeps one table per level in shared memory.
//
// Phase 1 walks the A tree; at each leaf (a needed A column set) it forms G_j in
// shared memory and adds coef_j-weighted G_j into the K columns of the paired B column
// sets.  K lives in a per-block slot of global scratch memory (|cols_B| x |rows_B|
// values, written first by the plan-known first update of each column, so it needs no
// clearing).  Phase 2 walks the B tree and, at each leaf, takes the dot product of the
// B column with the matching K column.  One block owns one site at a time and takes
// sites from an atomic work counter (persistent grid, no inter-block waiting).
// Mixed precision: the site's 12x12 blocks are scaled by exact powers of two and every
// product and sum is a double-float operation; the scale is restored in double.
#include "common.cuh"
#include "checks.cuh"

namespace mbc {

// One Laplace step for every row set of level K: dest[e] = sum_i (-1)^(i+q) M[r_i, col] parent[c_i].
template <class P, int K>
__device__ __forceinline__ void laplace_k(const MinorDev& m, const uint32_t* pk, int col, int sign,
                                          const typename P::V* mat, const typename P::V* parent, typename P::V* dest) {
    const int n = m.size[K];
    const typename P::V* mc = mat + col;
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
        uint32_t w[K];
#pragma unroll
        for (int i = 0; i < K; ++i) {
            w[i] = pk[i * n + e];
            if (MBC_BAD((w[i] >> 16) < 12u && (w[i] & 0xFFFFu) < (uint32_t)m.size[K - 1], 53, w[i], m.size[K - 1]))
                w[i] = 0;
        }
        typename P::A acc;
        P::acc_zero(acc);
#pragma unroll
        for (int i = 0; i < K; ++i) {
            // the term's sign (-1)^(i+q) goes into the parent value's sign bits, so every
            // term is one multiply-add
            const typename P::V a = mc[(w[i] >> 16) * kLd];
            const typename P::V p = P::flip(parent[w[i] & 0xFFFFu], (i & 1) ? -sign : sign);
            P::fma(acc, a, p);
        }
        dest[e] = P::get(acc);
    }
}

// The leaf level's packed table is read from leaf_pk (a shared-memory copy when the plan stages it); the other
// levels from global memory.
template <class P>
__device__ __forceinline__ void laplace_level(const MinorDev& m, int k, int col, int sign, const typename P::V* mat,
                                              const typename P::V* parent, typename P::V* dest,
                                              const uint32_t* leaf_pk) {
    const uint32_t* pk = k == m.n ? leaf_pk : m.pack[k];
    switch (k) {
        case 1: laplace_k<P, 1>(m, pk, col, sign, mat, parent, dest); break;
        case 2: laplace_k<P, 2>(m, pk, col, sign, mat, parent, dest); break;
        case 3: laplace_k<P, 3>(m, pk, col, sign, mat, parent, dest); break;
        case 4: laplace_k<P, 4>(m, pk, col, sign, mat, parent, dest); break;
        case 5: laplace_k<P, 5>(m, pk, col, sign, mat, parent, dest); break;
        default: laplace_k<P, 6>(m, pk, col, sign, mat, parent, dest); break;
    }
}

// Leaf work with G kept in registers (NJ free indices, real float weights): each thread
// owns row sets R_b of the B flavour, forms G_j(R_b) and applies it to every pair.
template <class P, int NJ>
__device__ __forceinline__ void leaf_fused(const EgraphDev& d, int leaf, const typename P::V* T,
                                           typename P::V* __restrict__ K) {
    typedef typename P::V V;
    typedef typename P::S S;
    const int n_rb = d.n_rows_b;
    const int p0 = __ldg(d.pair_off + leaf), p1 = __ldg(d.pair_off + leaf + 1);
    const int lane = threadIdx.x & 31;
    // free indices whose G the leaf's pairs use (the others are skipped)
    const int jmask = __ldg(d.leaf_jmask + leaf);
    for (int b = threadIdx.x; b < n_rb; b += blockDim.x) {
        V g[NJ];
        const int sl = b >> 5;      // slice of 32 row sets (blockDim is a multiple of 32)
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
            typename P::A acc;
            P::acc_zero(acc);
            if (!((jmask >> j) & 1)) {
                g[j] = P::zero();
                continue;
            }
            if (P::kind == 1) {
                // double-float: issue-bound, coalesced sliced-ELL records (padding is cheap)
                const int2* ent = d.sell + __ldg(d.sell_off + sl * NJ + j) + lane;
                const int width = __ldg(d.sell_w + sl * NJ + j);
                for (int k = 0; k < width; ++k) {
                    const int2 r = __ldg(ent + k * 32);
                    P::fma_s(acc, (S)__int_as_float(r.y), T[r.x]);
                }
            } else {
                // FP64: bound by the FP64 pipe, so no padded entries (row-wise lists)
                const S* gws = reinterpret_cast<const S*>(d.g_ws);
                const int e1 = __ldg(d.g_off + b * NJ + j + 1);
                for (int e = __ldg(d.g_off + b * NJ + j); e < e1; ++e) P::fma_s(acc, __ldg(gws + e), T[__ldg(d.g_a + e)]);
            }
            g[j] = P::get_s(acc);
        }
        // K(C_b, R_b) (+)= sum_j coef_j G_j, accumulated onto the stored value
        if (P::kind == 1) {
            // double-float: one 16-byte record per pair (B column | first update << 31,
            // coef_0, coef_1 as float bits); two pairs at a time (the pairs of one leaf go
            // to distinct K columns, so both loads may precede both stores)
            int pr = p0;
            for (; pr + 1 < p1; pr += 2) {
                const int4 r0 = __ldg(d.pair_rec + pr), r1 = __ldg(d.pair_rec + pr + 1);
                V* k0 = K + (size_t)(r0.x & 0x7fffffff) * n_rb + b;
                V* k1 = K + (size_t)(r1.x & 0x7fffffff) * n_rb + b;
                const V v0 = r0.x < 0 ? P::zero() : *k0;
                const V v1 = r1.x < 0 ? P::zero() : *k1;
                typename P::A h0, h1;
                P::acc_set(h0, v0);
                P::acc_set(h1, v1);
                // zero coefficients are skipped: the branches are uniform (every thread of
                // the block handles the same pair)
                if (r0.y) P::fma_s(h0, (S)__int_as_float(r0.y), g[0]);
                if (r1.y) P::fma_s(h1, (S)__int_as_float(r1.y), g[0]);
                if (NJ > 1) {
                    if (r0.z) P::fma_s(h0, (S)__int_as_float(r0.z), g[NJ - 1]);
                    if (r1.z) P::fma_s(h1, (S)__int_as_float(r1.z), g[NJ - 1]);
                }
                *k0 = P::get_s(h0);
                *k1 = P::get_s(h1);
            }
            if (pr < p1) {
                const int4 rec = __ldg(d.pair_rec + pr);
                V* kp = K + (size_t)(rec.x & 0x7fffffff) * n_rb + b;
                typename P::A h;
                if (rec.x < 0) P::acc_zero(h);
                else P::acc_set(h, *kp);
                if (rec.y) P::fma_s(h, (S)__int_as_float(rec.y), g[0]);
                if (NJ > 1 && rec.z) P::fma_s(h, (S)__int_as_float(rec.z), g[NJ - 1]);
                *kp = P::get_s(h);
            }
        } else {
            // FP64: coefficients stored as doubles (a float-to-double conversion would take
            // a slot of the FP64 pipe that bounds this kernel)
            const S* pcs = reinterpret_cast<const S*>(d.pair_cs);
            for (int pr = p0; pr < p1; ++pr) {
                V* kp = K + (size_t)__ldg(d.pair_b + pr) * n_rb + b;
                typename P::A h;
                if (__ldg(d.pair_first + pr)) P::acc_zero(h);
                else P::acc_set(h, *kp);
#pragma unroll
                for (int j = 0; j < NJ; ++j) P::fma_s(h, __ldg(pcs + pr * NJ + j), g[j]);
                *kp = P::get_s(h);
            }
        }
    }
}

// One sink site: stage, phase 1 (A tree, K updates), phase 2 (B tree, dots), site sum.
template <class P>
__device__ __forceinline__ void egraph_site(const EgraphDev& d, const double* __restrict__ U,
                                            const double* __restrict__ D, int64_t site, d4* part,
                                            typename P::V* __restrict__ kslot, unsigned char* smem_raw, double* red,
                                            const uint32_t*& pk_owner) {
    typedef typename P::V V;
    V* sA = reinterpret_cast<V*>(smem_raw);
    V* sB = sA + kBlk;
    V* stA = sB + kBlk;
    V* stB = stA + d.stack_a;
    V* G = stB + d.stack_b;
    const int nA = d.A.n, nB = d.B.n;
    const int n_rb = d.n_rows_b, nj = d.n_j;
    const bool fused = d.compact && nj <= 2;
    V* K = kslot;
    // packed tables of the two leaf levels: copied to shared memory when the plan asks for
    // it (when that costs no resident block), else read through L1.  Where they sit depends
    // on the plan's stack and G sizes, so a site of another plan (batched items) overwrites
    // them: pk_owner (the same in every thread) names the plan whose copy is intact, and is
    // cleared by a site of a plan that does not stage
    const uint32_t* pkA = d.A.pack[nA];
    const uint32_t* pkB = d.B.pack[nB];
    if (d.stage_pk) {
        uint32_t* sa = reinterpret_cast<uint32_t*>(G + (fused ? 0 : nj * n_rb));
        uint32_t* sb = sa + d.A.size[nA] * nA;
        if (pk_owner != d.A.pack[nA]) {
            __syncthreads();
            for (int i = threadIdx.x; i < d.A.size[nA] * nA; i += blockDim.x) sa[i] = __ldg(d.A.pack[nA] + i);
            for (int i = threadIdx.x; i < d.B.size[nB] * nB; i += blockDim.x) sb[i] = __ldg(d.B.pack[nB] + i);
            __syncthreads();
            pk_owner = d.A.pack[nA];
        }
        pkA = sa;
        pkB = sb;
    } else {
        pk_owner = nullptr;
    }
    // ---- stage the site's blocks (A flavour first)
    const double* ma = (d.flav_a == 0 ? U : D) + site * 288;
    const double* mb = (d.flav_a == 0 ? D : U) + site * 288;
    int ea, eb;
    load_pair<P>(ma, mb, sA, sB, red, ea, eb);
    if (threadIdx.x == 0) {
        stA[0] = P::one();
        stB[0] = P::one();
    }
    __syncthreads();
    // ---- phase 1: A column tree, G_j per leaf, K updates per pair
    int parity = 0;
    for (int nd = 0; nd < d.A.n_nodes; ++nd) {
        const int k = __ldg(d.A.node_level + nd);
        // leaf-level tables alternate between two buffers, so the next leaf's Laplace
        // step may start while slower threads still read this leaf's table
        V* dest = stA + d.A.off[k] + (k == nA ? parity * d.A.size[nA] : 0);
        laplace_level<P>(d.A, k, __ldg(d.A.node_col + nd), __ldg(d.A.node_sign + nd), sA, stA + d.A.off[k - 1],
                         dest, pkA);
        __syncthreads();
        const int leaf = __ldg(d.A.node_leaf + nd);
        if (leaf < 0) continue;
        const V* T = dest;
        parity ^= 1;
        if (fused) {
            if (nj == 1) leaf_fused<P, 1>(d, leaf, T, K);
            else leaf_fused<P, 2>(d, leaf, T, K);
            // no barrier: the next leaf writes the other buffer, and the barrier after
            // the next Laplace step orders these K writes before later K updates
            continue;
        }
        {   // G_j(R_b) = sum_{R_a} s_j(R_a, R_b) T(R_a); flat index it = b * nj + j
            const int total = n_rb * nj, stride = blockDim.x;
            int b = threadIdx.x / nj, j = threadIdx.x - (threadIdx.x / nj) * nj;
            const int db = stride / nj, dj = stride - db * nj;
            for (int it = threadIdx.x; it < total; it += stride) {
                typename P::A gj;
                P::acc_zero(gj);
                const int e1 = __ldg(d.g_off + it + 1);
                if (d.real_w) {
                    for (int e = __ldg(d.g_off + it); e < e1; ++e) P::fma_real(gj, ldv<V>(d.g_w, e), T[__ldg(d.g_a + e)]);
                } else {
                    for (int e = __ldg(d.g_off + it); e < e1; ++e) P::fma(gj, ldv<V>(d.g_w, e), T[__ldg(d.g_a + e)]);
                }
                G[j * n_rb + b] = P::get(gj);
                b += db;
                j += dj;
                if (j >= nj) { j -= nj; ++b; }
            }
        }
        __syncthreads();
        {   // K(C_b, :) += sum_j coef_j G_j for each pair of this leaf; flat index bi * n_rb + b
            const int p0 = __ldg(d.pair_off + leaf), np = __ldg(d.pair_off + leaf + 1) - p0;
            int bi = threadIdx.x / n_rb, b = threadIdx.x - (threadIdx.x / n_rb) * n_rb;
            const int dbi = blockDim.x / n_rb, db = blockDim.x - dbi * n_rb;
            for (int it = threadIdx.x; it < np * n_rb; it += blockDim.x) {
                const int pr = p0 + bi;
                typename P::A h;
                P::acc_zero(h);
                if (d.real_w) {
                    for (int j = 0; j < nj; ++j) P::fma_real(h, ldv<V>(d.pair_coef, (int64_t)pr * nj + j), G[j * n_rb + b]);
                } else {
                    for (int j = 0; j < nj; ++j) P::fma(h, ldv<V>(d.pair_coef, (int64_t)pr * nj + j), G[j * n_rb + b]);
                }
                V* kp = K + (size_t)__ldg(d.pair_b + pr) * n_rb + b;
                const V hv = P::get(h);
                *kp = __ldg(d.pair_first + pr) ? hv : P::vadd(*kp, hv);
                bi += dbi;
                b += db;
                if (b >= n_rb) { b -= n_rb; ++bi; }
            }
        }
        // G is rewritten by the next leaf only after the barrier that follows the next
        // Laplace step, which also orders these K writes before later K updates
    }
    __syncthreads();
    // ---- phase 2: B column tree, <K(C_b, :), det B[:, C_b]> per leaf
    typename P::A acc;
    P::acc_zero(acc);
    if (nB == 0) {
        if (threadIdx.x == 0) P::add(acc, K[0]);
    } else {
        int pb = 0;
        for (int nd = 0; nd < d.B.n_nodes; ++nd) {
            const int k = __ldg(d.B.node_level + nd);
            V* dest = stB + d.B.off[k] + (k == nB ? pb * d.B.size[nB] : 0);
            laplace_level<P>(d.B, k, __ldg(d.B.node_col + nd), __ldg(d.B.node_sign + nd), sB, stB + d.B.off[k - 1],
                             dest, pkB);
            __syncthreads();
            const int leaf = __ldg(d.B.node_leaf + nd);
            if (leaf < 0) continue;
            pb ^= 1;
            const V* kc = K + (size_t)leaf * n_rb;
            for (int b = threadIdx.x; b < n_rb; b += blockDim.x) P::fma(acc, kc[b], dest[b]);
        }
    }
    // ---- site value
    const cd v = P::to_cd(P::get(acc));
    kacc re, im;
    block_sum(v, re, im, red);
    if (threadIdx.x == 0) store_partial(part, re, im, ea * nA + eb * nB);
    __syncthreads();
}

template <class P>
__global__ void __launch_bounds__(384) egraph_kernel(EgraphDev d, const double* __restrict__ U,
                                                     const double* __restrict__ D, Geometry g, Partials out,
                                                     unsigned int* __restrict__ counter,
                                                     typename P::V* __restrict__ kscratch,
                                                     const unsigned int* __restrict__ list,
                                                     const unsigned int* __restrict__ list_n, int64_t n_sites_list) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[4 * 32];
    __shared__ unsigned int s_unit;
    const uint32_t* pk_owner = nullptr;
    typename P::V* K = kscratch + (size_t)blockIdx.x * d.n_cols_b * d.n_rows_b;      // this block's K slot
    // every site of the geometry, or (list mode) the sites of a device list
    const int64_t n_units = list ? (int64_t)*list_n : g.n_sites();
    for (;;) {
        if (threadIdx.x == 0) s_unit = atomicAdd(counter, 1u);
        __syncthreads();
        const int64_t unit = s_unit;
        if (unit >= n_units) break;
        const int64_t site = list ? (int64_t)list[unit] : unit;
        if (list && MBC_BAD(site >= 0 && site < n_sites_list, 50, site, n_sites_list)) continue;
        egraph_site<P>(d, U, D, site, out.part + site, K, smem_raw, red, pk_owner);
    }
}

// Several (plan, fields) items in one persistent launch: work units are (item, site),
// numbered item by item; a block takes units from the counter, finds the item by a
// search over the unit offsets and evaluates the site with that item's plan.  Three
// resident blocks of up to 384 threads per SM: the register cap this implies (56) costs a
// few spills of the per-item plan view, which the occupancy more than repays.
template <class P>
__global__ void __launch_bounds__(384, 3) egraph_batch_kernel(const BatchItem* __restrict__ items, int n_items,
                                                           int64_t n_units, unsigned int* __restrict__ counter,
                                                           typename P::V* __restrict__ kscratch, int64_t kslot_values,
                                                           const unsigned int* __restrict__ list,
                                                           const unsigned int* __restrict__ list_n,
                                                           int64_t n_units_list) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[4 * 32];
    __shared__ unsigned int s_unit;
    const uint32_t* pk_owner = nullptr;
    typename P::V* K = kscratch + (size_t)blockIdx.x * kslot_values;
    // every unit, or (list mode) the units of a device list
    const int64_t n_work = list ? (int64_t)*list_n : n_units;
    for (;;) {
        if (threadIdx.x == 0) s_unit = atomicAdd(counter, 1u);
        __syncthreads();
        const int64_t work = s_unit;
        if (work >= n_work) break;
        const int64_t unit = list ? (int64_t)list[work] : work;
        if (list && MBC_BAD(unit >= 0 && unit < n_units_list, 51, unit, n_units_list)) continue;
        int lo = 0, hi = n_items - 1;
        while (lo < hi) {                  // last item whose first unit is <= unit
            const int mid = (lo + hi + 1) >> 1;
            if (items[mid].unit_begin <= unit) lo = mid; else hi = mid - 1;
        }
        const BatchItem& it = items[lo];
        const int64_t site = unit - it.unit_begin;
        if (MBC_BAD(site >= 0 && site < it.n_sites, 52, site, it.n_sites)) continue;
        egraph_site<P>(it.d, it.U, it.D, site, it.part + site, K, smem_raw, red, pk_owner);
    }
}

size_t egraph_smem_bytes(const EgraphDev& d, int) { return (size_t)d.smem_values * 16; }
size_t egraph_kslot_bytes(const EgraphDev& d) { return (size_t)d.n_cols_b * d.n_rows_b * 16; }

cudaError_t launch_egraph_batch(const BatchItem* items, int n_items, int64_t n_units, int prec, int threads, int grid,
                                size_t smem, unsigned int* counter, void* kscratch, int64_t kslot_values, cudaStream_t s,
                                int64_t* launches) {
    if (n_units == 0) return cudaSuccess;
    cudaError_t e;
    if (prec == 0) e = cudaFuncSetAttribute(egraph_batch_kernel<FP64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    else e = cudaFuncSetAttribute(egraph_batch_kernel<MIXED>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    grid = (int)std::min<int64_t>(n_units, grid);
    e = cudaMemsetAsync(counter, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
    if (prec == 0)
        egraph_batch_kernel<FP64><<<grid, threads, smem, s>>>(items, n_items, n_units, counter, (cd*)kscratch, kslot_values,
                                                              nullptr, nullptr, 0);
    else
        egraph_batch_kernel<MIXED><<<grid, threads, smem, s>>>(items, n_items, n_units, counter, (cdf*)kscratch,
                                                               kslot_values, nullptr, nullptr, 0);
    ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_egraph_batch_list(const BatchItem* items, int n_items, int64_t n_units, int threads, int grid,
                                     size_t smem, unsigned int* counter, void* kscratch, int64_t kslot_values,
                                     const unsigned int* list, const unsigned int* list_n, cudaStream_t s,
                                     int64_t* launches) {
    if (n_items == 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(egraph_batch_kernel<MIXED>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(counter, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
    egraph_batch_kernel<MIXED><<<grid, threads, smem, s>>>(items, n_items, 0, counter, (cdf*)kscratch, kslot_values,
                                                           list, list_n, n_units);
    ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_egraph(const EgraphDev& d, int prec, const double* U, const double* D, Geometry g, Partials out,
                          int threads, int grid, unsigned int* counter, void* kscratch, cudaStream_t s,
                          int64_t* launches) {
    const int64_t units = g.n_sites();
    if (units == 0) return cudaSuccess;
    const size_t smem = egraph_smem_bytes(d, prec);
    cudaError_t e;
    if (prec == 0) e = cudaFuncSetAttribute(egraph_kernel<FP64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    else e = cudaFuncSetAttribute(egraph_kernel<MIXED>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    grid = (int)std::min<int64_t>(units, grid);
    e = cudaMemsetAsync(counter, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
    if (prec == 0)
        egraph_kernel<FP64><<<grid, threads, smem, s>>>(d, U, D, g, out, counter, (cd*)kscratch, nullptr, nullptr, 0);
    else
        egraph_kernel<MIXED><<<grid, threads, smem, s>>>(d, U, D, g, out, counter, (cdf*)kscratch, nullptr, nullptr, 0);
    ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_egraph_list(const EgraphDev& d, const double* U, const double* D, Partials out, int threads,
                               int grid, unsigned int* counter, void* kscratch, const unsigned int* list,
                               const unsigned int* list_n, int64_t n_sites, cudaStream_t s, int64_t* launches) {
    const size_t smem = egraph_smem_bytes(d, 1);
    cudaError_t e = cudaFuncSetAttribute(egraph_kernel<MIXED>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(counter, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
    // the list's length is known on the device only: the full persistent grid is
    // launched and blocks without work exit at once
    egraph_kernel<MIXED><<<grid, threads, smem, s>>>(d, U, D, Geometry{0, 0, 0}, out, counter, (cdf*)kscratch, list,
                                                     list_n, n_sites);
    ++*launches;
    return cudaGetLastError();
}

cudaError_t egraph_checks(CheckRecord* out) { return read_checks(out); }

}  // namespace mbc
