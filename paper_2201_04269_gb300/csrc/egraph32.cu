// egraph32.cu - the e-graph plan (arXiv 2201.04269 Sec. 5) evaluated in FP32 with a
// per-site error guard.
//
// Same staged contraction as egraph.cu, per sink site
//   C_x = sum_{C_a} sum_{C_b paired} sum_{R_b} (sum_j coef_j(C_a, C_b) G_j(C_a, R_b)) B[R_b, C_b],
//   G_j(C_a, R_b) = sum_{R_a} s_j(R_a, R_b) A[R_a, C_a],
// with A, B the minors of the two flavours, but arranged for FP32 arithmetic and with no
// K scratch in global memory:
//  1. the site's 12x12 blocks are scaled by exact powers of two (largest |re|, |im| in
//     [0.5, 1)) and rounded to FP32 in shared memory;
//  2. the block's walkers (groups of 128 threads, named barriers) walk their parts of
//     the B column tree and write every B leaf table det B[:, C_b] to the block's B
//     table (n_cols_b x n_rows_b FP32 values in global memory, L2 resident);
//  3. the walkers walk their parts of the A column tree; the children of a level-(n-1)
//     node are formed in batches that share the parent's values in registers; for each
//     leaf C_a and B row set R_b a thread forms G_j(C_a, R_b) and the leaf's part
//        sum_{pairs (C_a, C_b)} (sum_j coef_j G_j) B[R_b, C_b]
//     in FP32, and adds it to its running sum with TwoSum (Knuth) compensation;
//  4. the block sum is taken in compensated double; the scale is restored in double.
// Minors, G and pair products carry FP32 rounding (relative 2^-24 per operation), which
// the site sum can amplify where it cancels (the floating-point cancellation the paper
// cites in Sec. 1).  Each thread therefore also sums |part|^2 over its (leaf, R_b)
// parts, and the site's estimate
//        est = sqrt(sum |part|^2) / |C_x|
// measures how much the site sum cancels relative to its parts.  A site whose estimate
// exceeds the plan's guard (or is not finite) is appended to a list, and the
// double-float kernel (egraph.cu) recomputes exactly those sites afterwards.
#include "common.cuh"

namespace mbc {
namespace {

constexpr int kWalker = 128;         // threads per walker

__device__ __forceinline__ void walker_sync(int w) {
    asm volatile("bar.sync %0, %1;" ::"r"(w + 1), "r"(kWalker) : "memory");
}

__device__ __forceinline__ float2 cfma(float2 acc, float2 a, float2 b) {
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(-a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y);
    acc.y = fmaf(a.y, b.x, acc.y);
    return acc;
}

// x with both parts negated when the bit is set (sign bits, integer operations only)
__device__ __forceinline__ float2 flip_bits(float2 x, unsigned m) {
    return make_float2(__uint_as_float(__float_as_uint(x.x) ^ m), __uint_as_float(__float_as_uint(x.y) ^ m));
}

// compensated FP32 sum of complex values: s + c, TwoSum of every addend (Knuth)
struct CAcc {
    float sr, cr, si, ci;
};
__device__ __forceinline__ void two_sum_add(float& s, float& c, float x) {
    const float t = __fadd_rn(s, x);
    const float bp = __fsub_rn(t, s);
    c = __fadd_rn(c, __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(x, bp)));
    s = t;
}
__device__ __forceinline__ void cacc_add(CAcc& a, float2 x) {
    two_sum_add(a.sr, a.cr, x.x);
    two_sum_add(a.si, a.ci, x.y);
}

// Stage the site's two 12x12 blocks as FP32 values scaled by exact powers of two (the
// largest |re|, |im| of each block in [0.5, 1)); entry (r, c) at [r * kLd + c].
__device__ __forceinline__ void stage_f32(const double* __restrict__ a, const double* __restrict__ b, float2* sa,
                                          float2* sb, double* red, int& ea, int& eb) {
    double ma = 0.0, mb = 0.0;
    for (int i = threadIdx.x; i < 288; i += blockDim.x) {
        const int e = i < 144 ? i : i - 144;
        const double2 v = __ldg(reinterpret_cast<const double2*>(i < 144 ? a : b) + e);
        const double m = fmax(fabs(v.x), fabs(v.y));
        if (i < 144) ma = fmax(ma, m);
        else mb = fmax(mb, m);
    }
    ma = block_max(ma, red);
    mb = block_max(mb, red);
    ea = block_exponent(ma);
    eb = block_exponent(mb);
    for (int i = threadIdx.x; i < 288; i += blockDim.x) {
        const int e = i < 144 ? i : i - 144;
        const double2 v = __ldg(reinterpret_cast<const double2*>(i < 144 ? a : b) + e);
        const int sc = i < 144 ? -ea : -eb;
        const float2 f = make_float2((float)ldexp(v.x, sc), (float)ldexp(v.y, sc));
        (i < 144 ? sa : sb)[(e / 12) * kLd + e % 12] = f;
    }
}

// One Laplace step of a walker: dest[e] = sum_i (-1)^(i+q) M[r_i, col] parent[c_i] for
// every row set e of level K (packed words transposed: word i of entry e at [i n + e]).
template <int K>
__device__ __forceinline__ void lap_node(const float2* M, const uint32_t* pk, int n, int col, int sign,
                                         const float2* parent, float2* dest, int wt) {
    const float2* mc = M + col;
    const unsigned qm = sign < 0 ? 0x80000000u : 0u;
    for (int e = wt; e < n; e += kWalker) {
        uint32_t w[K];
#pragma unroll
        for (int i = 0; i < K; ++i) w[i] = pk[i * n + e];
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int i = 0; i < K; ++i) {
            const float2 p = flip_bits(parent[w[i] & 0xFFFFu], qm ^ ((i & 1) ? 0x80000000u : 0u));
            acc = cfma(acc, mc[(w[i] >> 16) * kLd], p);
        }
        dest[e] = acc;
    }
}

// A batch of leaves sharing one parent table: for every row set e the K parent values
// (with the row-position signs) are loaded once and reused for each leaf of the batch.
// Leaf l's table goes to out + l * n (A: shared memory) or, when to_cols, to
// out + leaf * n (B: the block's B table, column-major by B column set).
template <int K>
__device__ __forceinline__ void lap_leaves(const float2* M, const uint32_t* pk, int n, const WalkLeaf* lv,
                                           int nleaf, const float2* parent, float2* out, bool to_cols, int wt) {
    for (int e = wt; e < n; e += kWalker) {
        float2 p[K];
        int r[K];
#pragma unroll
        for (int i = 0; i < K; ++i) {
            const uint32_t w = pk[i * n + e];
            r[i] = (int)(w >> 16) * kLd;
            p[i] = flip_bits(parent[w & 0xFFFFu], (i & 1) ? 0x80000000u : 0u);
        }
        for (int l = 0; l < nleaf; ++l) {
            const WalkLeaf L = lv[l];
            float2 acc = make_float2(0.f, 0.f);
#pragma unroll
            for (int i = 0; i < K; ++i) acc = cfma(acc, M[r[i] + L.col], p[i]);
            acc = flip_bits(acc, L.sign < 0 ? 0x80000000u : 0u);
            out[(size_t)(to_cols ? L.leaf : l) * n + e] = acc;
        }
    }
}

__device__ __forceinline__ void lap_node_k(int k, const float2* M, const uint32_t* pk, int n, int col, int sign,
                                           const float2* parent, float2* dest, int wt) {
    switch (k) {
        case 1: lap_node<1>(M, pk, n, col, sign, parent, dest, wt); break;
        case 2: lap_node<2>(M, pk, n, col, sign, parent, dest, wt); break;
        case 3: lap_node<3>(M, pk, n, col, sign, parent, dest, wt); break;
        case 4: lap_node<4>(M, pk, n, col, sign, parent, dest, wt); break;
        case 5: lap_node<5>(M, pk, n, col, sign, parent, dest, wt); break;
        default: lap_node<6>(M, pk, n, col, sign, parent, dest, wt); break;
    }
}

__device__ __forceinline__ void lap_leaves_k(int k, const float2* M, const uint32_t* pk, int n, const WalkLeaf* lv,
                                             int nleaf, const float2* parent, float2* out, bool to_cols, int wt) {
    switch (k) {
        case 1: lap_leaves<1>(M, pk, n, lv, nleaf, parent, out, to_cols, wt); break;
        case 2: lap_leaves<2>(M, pk, n, lv, nleaf, parent, out, to_cols, wt); break;
        case 3: lap_leaves<3>(M, pk, n, lv, nleaf, parent, out, to_cols, wt); break;
        case 4: lap_leaves<4>(M, pk, n, lv, nleaf, parent, out, to_cols, wt); break;
        case 5: lap_leaves<5>(M, pk, n, lv, nleaf, parent, out, to_cols, wt); break;
        default: lap_leaves<6>(M, pk, n, lv, nleaf, parent, out, to_cols, wt); break;
    }
}

// The leaf stage of a batch of A leaves: items (leaf l, B row set b).  Per item: G_j(b)
// for the free indices the leaf's pairs use, then the leaf's part
//   sum_pairs (sum_j coef_j G_j(b)) B[b, C_b],
// added to the thread's compensated sum; |part|^2 goes to the guard sum.
template <bool REAL, int NJ>
__device__ __forceinline__ void leaf_stage(const Eg32Dev& d, const WalkLeaf* lv, int nleaf, const float2* leafbuf,
                                           int n_e, const float2* __restrict__ bt, CAcc& acc, float& guard, int wt) {
    const int n_rb = d.n_rows_b;
    const int total = nleaf * n_rb;
    int l = wt / n_rb, b = wt - (wt / n_rb) * n_rb;
    for (int it = wt; it < total; it += kWalker) {
        const int leaf = lv[l].leaf;
        const float2* T = leafbuf + l * n_e;
        const int jm = __ldg(d.leaf_jmask + leaf);
        const int sl = b >> 5, lane = b & 31;
        float2 g[NJ];
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
            g[j] = make_float2(0.f, 0.f);
            if (!((jm >> j) & 1)) continue;
            const int o = __ldg(d.sell_off + sl * NJ + j) + lane;
            const int wd = __ldg(d.sell_w + sl * NJ + j);
            if (REAL) {
                for (int k = 0; k < wd; ++k) {
                    const int2 rec = __ldg(d.sell + o + k * 32);
                    const float w = __int_as_float(rec.y);
                    const float2 t = T[rec.x];
                    g[j].x = fmaf(w, t.x, g[j].x);
                    g[j].y = fmaf(w, t.y, g[j].y);
                }
            } else {
                for (int k = 0; k < wd; ++k) {
                    const int4 rec = __ldg(d.sellc + o + k * 32);
                    g[j] = cfma(g[j], make_float2(__int_as_float(rec.y), __int_as_float(rec.z)), T[rec.x]);
                }
            }
        }
        const int p0 = __ldg(d.pair_off + leaf), p1 = __ldg(d.pair_off + leaf + 1);
        float2 part = make_float2(0.f, 0.f);
        for (int pr = p0; pr < p1; ++pr) {
            const int cb = __ldg(d.pair_cb + pr);
            float2 h = make_float2(0.f, 0.f);
#pragma unroll
            for (int j = 0; j < NJ; ++j) {
                const float2 c = __ldg(d.pair_cf + pr * NJ + j);
                if (REAL) {
                    if (c.x != 0.f) {
                        h.x = fmaf(c.x, g[j].x, h.x);
                        h.y = fmaf(c.x, g[j].y, h.y);
                    }
                } else {
                    h = cfma(h, c, g[j]);
                }
            }
            part = cfma(part, h, bt[(size_t)cb * n_rb + b]);
        }
        cacc_add(acc, part);
        guard = fmaf(part.x, part.x, fmaf(part.y, part.y, guard));
        b += kWalker;
        while (b >= n_rb) {
            b -= n_rb;
            ++l;
        }
    }
}

// Run one flavour's walker program: B (to_cols: leaf tables to the block's B table) or
// A (leaf tables to the walker's batch buffer, then the leaf stage).
template <bool REAL, int NJ>
__device__ __forceinline__ void walk(const Eg32Dev& d, const WalkDev& f, bool is_a, const float2* M,
                                     const uint32_t* spk, float2* stack, float2* leafbuf, float2* bt, CAcc& acc,
                                     float& guard, int w, int wt) {
    const int n = f.n;
    const int s0 = __ldg(f.step_off + w), s1 = __ldg(f.step_off + w + 1);
    for (int s = s0; s < s1; ++s) {
        const WalkStep st = f.steps[s];
        if (st.level > 0) {
            const int k = st.level;
            lap_node_k(k, M, spk + f.pk_off[k], f.size[k], st.col, st.sign, stack + f.off[k - 1], stack + f.off[k], wt);
            walker_sync(w);
        }
        if (st.nleaf > 0) {
            if (st.level == 0) walker_sync(w);     // the previous batch may still be read
            const WalkLeaf* lv = f.leaves + st.leaf0;
            lap_leaves_k(n, M, spk + f.pk_off[n], f.size[n], lv, st.nleaf, stack + f.off[n - 1],
                         is_a ? leafbuf : bt, !is_a, wt);
            walker_sync(w);
            if (is_a) leaf_stage<REAL, NJ>(d, lv, st.nleaf, leafbuf, f.size[n], bt, acc, guard, wt);
        }
    }
}

template <bool REAL, int NJ>
__global__ void __launch_bounds__(1024, 1) egraph32_kernel(Eg32Dev d, const double* __restrict__ U,
                                                           const double* __restrict__ D, Geometry g,
                                                           d4* __restrict__ part, float2* __restrict__ bslots,
                                                           unsigned int* __restrict__ counter,
                                                           unsigned int* __restrict__ flag_count,
                                                           unsigned int* __restrict__ flag_list) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[4 * 32];
    __shared__ unsigned int s_unit;
    float2* sA = reinterpret_cast<float2*>(smem_raw);
    float2* sB = sA + kBlk;
    uint32_t* spk = reinterpret_cast<uint32_t*>(sB + kBlk);
    const int w = threadIdx.x / kWalker, wt = threadIdx.x % kWalker;
    float2* stack = reinterpret_cast<float2*>(spk + d.pk_words) + (size_t)w * (d.stack_vals + d.leafbuf_vals);
    float2* leafbuf = stack + d.stack_vals;
    float2* bt = bslots + (size_t)blockIdx.x * d.n_cols_b * d.n_rows_b;
    for (int i = threadIdx.x; i < d.pk_words; i += blockDim.x) spk[i] = __ldg(d.pk + i);
    if (wt == 0) stack[0] = make_float2(1.f, 0.f);          // level 0: the empty minor
    const int64_t n_units = g.n_sites();
    const int nA = d.A.n, nB = d.B.n;
    for (;;) {
        if (threadIdx.x == 0) s_unit = atomicAdd(counter, 1u);
        __syncthreads();
        const int64_t site = s_unit;
        if (site >= n_units) break;
        const double* ma = (d.flav_a == 0 ? U : D) + site * 288;
        const double* mb = (d.flav_a == 0 ? D : U) + site * 288;
        int ea, eb;
        stage_f32(ma, mb, sA, sB, red, ea, eb);
        __syncthreads();
        CAcc acc = {0.f, 0.f, 0.f, 0.f};
        float guard = 0.f;
        if (nB == 0) {
            if (threadIdx.x == 0) bt[0] = make_float2(1.f, 0.f);
        } else {
            walk<REAL, NJ>(d, d.B, false, sB, spk, stack, leafbuf, bt, acc, guard, w, wt);
        }
        __syncthreads();                                   // the B table is complete
        walk<REAL, NJ>(d, d.A, true, sA, spk, stack, leafbuf, bt, acc, guard, w, wt);
        // site value: compensated double block sums of the parts and of |part|^2
        kacc re, im, gs, gz;
        block_sum(cd_make((double)acc.sr + (double)acc.cr, (double)acc.si + (double)acc.ci), re, im, red);
        block_sum(cd_make((double)guard, 0.0), gs, gz, red);
        if (threadIdx.x == 0) {
            store_partial(part + site, re, im, ea * nA + eb * nB);
            const double cr = re.hi + re.lo, ci = im.hi + im.lo;
            const double est = sqrt(gs.hi + gs.lo) / sqrt(cr * cr + ci * ci);
            if (!(est <= (double)d.guard)) flag_list[atomicAdd(flag_count, 1u)] = (unsigned int)site;
        }
    }
}

template <bool REAL, int NJ>
cudaError_t launch_t(const Eg32Dev& d, const double* U, const double* D, Geometry g, d4* part, int grid, void* bslots,
                     unsigned int* counter, unsigned int* flag_count, unsigned int* flag_list, cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(egraph32_kernel<REAL, NJ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         d.smem_bytes);
    if (e != cudaSuccess) return e;
    egraph32_kernel<REAL, NJ><<<grid, d.walkers * kWalker, d.smem_bytes, s>>>(d, U, D, g, part, (float2*)bslots,
                                                                             counter, flag_count, flag_list);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_egraph32(const Eg32Dev& d, const double* U, const double* D, Geometry g, d4* part, int grid,
                            void* bslots, unsigned int* counter, unsigned int* flag_count, unsigned int* flag_list,
                            cudaStream_t s, int64_t* launches) {
    const int64_t units = g.n_sites();
    if (units == 0) return cudaSuccess;
    grid = (int)std::min<int64_t>(units, grid);
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
    switch (d.n_j * 2 + (d.real_w ? 1 : 0)) {
        case 3: e = launch_t<true, 1>(d, U, D, g, part, grid, bslots, counter, flag_count, flag_list, s); break;
        case 5: e = launch_t<true, 2>(d, U, D, g, part, grid, bslots, counter, flag_count, flag_list, s); break;
        case 7: e = launch_t<true, 3>(d, U, D, g, part, grid, bslots, counter, flag_count, flag_list, s); break;
        case 9: e = launch_t<true, 4>(d, U, D, g, part, grid, bslots, counter, flag_count, flag_list, s); break;
        case 2: e = launch_t<false, 1>(d, U, D, g, part, grid, bslots, counter, flag_count, flag_list, s); break;
        case 4: e = launch_t<false, 2>(d, U, D, g, part, grid, bslots, counter, flag_count, flag_list, s); break;
        case 6: e = launch_t<false, 3>(d, U, D, g, part, grid, bslots, counter, flag_count, flag_list, s); break;
        case 8: e = launch_t<false, 4>(d, U, D, g, part, grid, bslots, counter, flag_count, flag_list, s); break;
        default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    ++*launches;
    return cudaSuccess;
}

}  // namespace mbc
