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
//  2. the walkers (groups of 128 threads, named barriers) of the site's block, or of
//     the d.cs blocks of its thread-block cluster, walk their parts of the B column tree
//     and write every B leaf table det B[:, C_b] to the site's B table (n_cols_b x
//     n_rows_b FP32 values in global memory: a cluster shares one, so that the tables
//     of every site in flight stay in L2);
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
#include "checks.cuh"

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

// Block sum of every thread's compensated complex sum and guard sum: TwoSum merges across
// each warp in FP32, the warp results in compensated double by thread 0 (fixed order).
// Results valid in thread 0; red holds 5 doubles per warp.
__device__ __forceinline__ void block_sum_site(const CAcc& a, float guard, kacc& re, kacc& im, double& gsum,
                                               double* red) {
    float sr = a.sr, cr = a.cr, si = a.si, ci = a.ci, g = guard;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const float osr = __shfl_down_sync(0xffffffffu, sr, off), ocr = __shfl_down_sync(0xffffffffu, cr, off);
        const float osi = __shfl_down_sync(0xffffffffu, si, off), oci = __shfl_down_sync(0xffffffffu, ci, off);
        g = __fadd_rn(g, __shfl_down_sync(0xffffffffu, g, off));
        cr = __fadd_rn(cr, ocr);
        two_sum_add(sr, cr, osr);
        ci = __fadd_rn(ci, oci);
        two_sum_add(si, ci, osi);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) {
        red[5 * warp + 0] = sr;
        red[5 * warp + 1] = cr;
        red[5 * warp + 2] = si;
        red[5 * warp + 3] = ci;
        red[5 * warp + 4] = g;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        kacc r = {0.0, 0.0}, i = {0.0, 0.0};
        double gg = 0.0;
        for (int w = 0; w < nw; ++w) {
            kacc_add(r, red[5 * w + 0]);
            kacc_add(r, red[5 * w + 1]);
            kacc_add(i, red[5 * w + 2]);
            kacc_add(i, red[5 * w + 3]);
            gg += red[5 * w + 4];
        }
        re = r;
        im = i;
        gsum = gg;
    }
    __syncthreads();
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
                                         const float2* parent, float2* dest, int wt, int n_parent) {
    const float2* mc = M + col;
    const unsigned qm = sign < 0 ? 0x80000000u : 0u;
    for (int e = wt; e < n; e += kWalker) {
        uint32_t w[K];
#pragma unroll
        for (int i = 0; i < K; ++i) w[i] = pk[i * n + e];
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int i = 0; i < K; ++i) {
            if (MBC_BAD((int)(w[i] >> 16) < 12 && (int)(w[i] & 0xFFFFu) < n_parent, 1, w[i], n_parent)) continue;
            const float2 p = flip_bits(parent[w[i] & 0xFFFFu], qm ^ ((i & 1) ? 0x80000000u : 0u));
            acc = cfma(acc, mc[(w[i] >> 16) * kLd], p);
        }
        dest[e] = acc;
    }
}

// A batch of leaves sharing one parent table: for every row set e the K parent values
// (with the row-position signs) are loaded once and reused for each leaf of the batch.
// Leaf l's table goes to out + l * n (A: shared memory) or, when to_cols, to
// out + leaf * n (B: the site's B table, column-major by B column set, row set e at
// position opos[e]).  A batch holds
// at most kMaxLeafBatch leaves; their columns, signs and output offsets stay in registers.
constexpr int kMaxBatch = kMaxLeafBatch;
template <int K>
__device__ __forceinline__ void lap_leaves(const float2* M, const uint32_t* pk, int n, const WalkLeaf* lv,
                                           int nleaf, const float2* parent, float2* out, bool to_cols, int wt,
                                           int n_parent, int64_t out_bound, const int32_t* __restrict__ opos) {
    int col[kMaxBatch], obase[kMaxBatch];
    unsigned sm[kMaxBatch];
#pragma unroll
    for (int l = 0; l < kMaxBatch; ++l) {
        col[l] = 0;
        obase[l] = 0;
        sm[l] = 0u;
        if (l < nleaf) {
            const WalkLeaf L = lv[l];
            col[l] = L.col;
            sm[l] = L.sign < 0 ? 0x80000000u : 0u;
            obase[l] = (to_cols ? L.leaf : l) * n;
            if (MBC_BAD(L.col < 12 && (int64_t)obase[l] + n <= out_bound, 2, obase[l] + n, out_bound)) nleaf = l;
        }
    }
    for (int e = wt; e < n; e += kWalker) {
        int eo = to_cols ? __ldg(opos + e) : e;
        if (MBC_BAD(eo >= 0 && eo < n, 4, eo, n)) eo = e;
        float2 p[K];
        const float2* mr[K];
#pragma unroll
        for (int i = 0; i < K; ++i) {
            uint32_t w = pk[i * n + e];
            if (MBC_BAD((int)(w >> 16) < 12 && (int)(w & 0xFFFFu) < n_parent, 3, w, n_parent)) w = 0;
            mr[i] = M + (int)(w >> 16) * kLd;
            p[i] = flip_bits(parent[w & 0xFFFFu], (i & 1) ? 0x80000000u : 0u);
        }
#pragma unroll
        for (int l = 0; l < kMaxBatch; ++l) {
            if (l < nleaf) {
                float2 acc = make_float2(0.f, 0.f);
#pragma unroll
                for (int i = 0; i < K; ++i) acc = cfma(acc, mr[i][col[l]], p[i]);
                out[obase[l] + eo] = flip_bits(acc, sm[l]);
            }
        }
    }
}

__device__ __forceinline__ void lap_node_k(int k, const float2* M, const uint32_t* pk, int n, int col, int sign,
                                           const float2* parent, float2* dest, int wt, int n_parent) {
    switch (k) {
        case 1: lap_node<1>(M, pk, n, col, sign, parent, dest, wt, n_parent); break;
        case 2: lap_node<2>(M, pk, n, col, sign, parent, dest, wt, n_parent); break;
        case 3: lap_node<3>(M, pk, n, col, sign, parent, dest, wt, n_parent); break;
        case 4: lap_node<4>(M, pk, n, col, sign, parent, dest, wt, n_parent); break;
        case 5: lap_node<5>(M, pk, n, col, sign, parent, dest, wt, n_parent); break;
        default: lap_node<6>(M, pk, n, col, sign, parent, dest, wt, n_parent); break;
    }
}

__device__ __forceinline__ void lap_leaves_k(int k, const float2* M, const uint32_t* pk, int n, const WalkLeaf* lv,
                                             int nleaf, const float2* parent, float2* out, bool to_cols, int wt,
                                             int n_parent, int64_t out_bound, const int32_t* opos) {
    switch (k) {
        case 1: lap_leaves<1>(M, pk, n, lv, nleaf, parent, out, to_cols, wt, n_parent, out_bound, opos); break;
        case 2: lap_leaves<2>(M, pk, n, lv, nleaf, parent, out, to_cols, wt, n_parent, out_bound, opos); break;
        case 3: lap_leaves<3>(M, pk, n, lv, nleaf, parent, out, to_cols, wt, n_parent, out_bound, opos); break;
        case 4: lap_leaves<4>(M, pk, n, lv, nleaf, parent, out, to_cols, wt, n_parent, out_bound, opos); break;
        case 5: lap_leaves<5>(M, pk, n, lv, nleaf, parent, out, to_cols, wt, n_parent, out_bound, opos); break;
        default: lap_leaves<6>(M, pk, n, lv, nleaf, parent, out, to_cols, wt, n_parent, out_bound, opos); break;
    }
}

template <int NJ>
__device__ __forceinline__ float2 pick(const float2* g, int j) {
    float2 v = g[0];
#pragma unroll
    for (int q = 1; q < NJ; ++q)
        if (j == q) v = g[q];
    return v;
}

__device__ __forceinline__ void add_part(CAcc& acc, float& guard, float2 part) {
    cacc_add(acc, part);
    guard = fmaf(part.x, part.x, fmaf(part.y, part.y, guard));
}

// The leaf stage of a batch of NL A leaves, row-major: each thread owns B row sets b (b =
// wt, wt + 128, ...; the 32 rows of a warp form one sliced-ELL slice).  For each of its
// rows it loads the G entries s_j(a, b) once and applies them to every leaf of the batch,
//   G_j(C_a, b) = sum_a s_j(a, b) T_{C_a}[a],
// then for each leaf takes the part
//   sum over the leaf's pair terms (C_b, j, coef_j) of coef_j G_j(C_a, b) B[b, C_b]
// (the term loop is the same for the whole walker: uniform loads, no divergence), adds
// it to its compensated sum and |part|^2 to the guard sum.  A term is (x, coef) with
// x = 4 (C_b n_rows_b) + j: the offset of column C_b in the B table and the free index.
// The B table is read through L2 only (another block of the cluster may have written it).
template <bool REAL, int NJ, int NL>
__device__ __forceinline__ void leaf_stage_n(const Eg32Dev& d, const WalkLeaf* lv, const float2* leafbuf, int n_e,
                                             const float2* __restrict__ bt, CAcc& acc, float& guard, int wt) {
    const int n_rb = d.n_rows_b;
    int lq0[NL], lnt[NL];
    int jm = 0;
#pragma unroll
    for (int l = 0; l < NL; ++l) {
        int id = lv[l].leaf;
        if (MBC_BAD(id >= 0 && id < d.n_cols_a, 20, id, d.n_cols_a)) id = 0;
        jm |= __ldg(d.leaf_jmask + id);
        lq0[l] = __ldg(d.term_off + id);
        lnt[l] = __ldg(d.term_off + id + 1) - lq0[l];
        if (MBC_BAD(lq0[l] >= 0 && lq0[l] + lnt[l] <= d.n_terms, 21, lq0[l] + lnt[l], d.n_terms)) lnt[l] = 0;
    }
    for (int b = wt; b < n_rb; b += kWalker) {
        const int sl = b >> 5, lane = b & 31;
        float2 g[NL][NJ];
#pragma unroll
        for (int l = 0; l < NL; ++l)
#pragma unroll
            for (int j = 0; j < NJ; ++j) g[l][j] = make_float2(0.f, 0.f);
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
            if (!((jm >> j) & 1)) continue;
            const int o = __ldg(d.sell_off + sl * d.n_j + j) + lane;
            int wd = __ldg(d.sell_w + sl * d.n_j + j);
            if (MBC_BAD(o >= 0 && o + (int64_t)(wd > 0 ? wd - 1 : 0) * 32 < d.n_sell, 22, o + (int64_t)wd * 32, d.n_sell))
                wd = 0;
            for (int k = 0; k < wd; ++k) {
                int a;
                float2 w;
                if (REAL && d.g_small) {
                    const uint32_t rec = __ldg(d.sell1 + o + k * 32);
                    a = (int)(rec & 0xFFFFu);
                    w = make_float2(__uint_as_float(rec & 0xFFFF0000u), 0.f);
                } else if (REAL) {
                    const int2 rec = __ldg(d.sell + o + k * 32);
                    a = rec.x;
                    w = make_float2(__int_as_float(rec.y), 0.f);
                } else {
                    const int4 rec = __ldg(d.sellc + o + k * 32);
                    a = rec.x;
                    w = make_float2(__int_as_float(rec.y), __int_as_float(rec.z));
                }
                if (MBC_BAD(a >= 0 && a < n_e, 23, a, n_e)) a = 0;
                const float2* ta = leafbuf + a;
#pragma unroll
                for (int l = 0; l < NL; ++l) {
                    const float2 t = ta[l * n_e];
                    if (REAL) {
                        g[l][j].x = fmaf(w.x, t.x, g[l][j].x);
                        g[l][j].y = fmaf(w.x, t.y, g[l][j].y);
                    } else {
                        g[l][j] = cfma(g[l][j], w, t);
                    }
                }
            }
        }
        const float2* btb = bt + b;
#pragma unroll
        for (int l = 0; l < NL; ++l) {
            float2 part = make_float2(0.f, 0.f);
            const int nt = lnt[l];
            if (REAL) {
                // four terms at a time: their records, then their B values, are independent loads
                const int2* tp = d.term2 + lq0[l];
#pragma unroll 1
                for (int q = 0; q < nt; q += 4) {
                    int2 r[4];
                    float2 bv[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        r[u] = q + u < nt ? __ldg(tp + q + u) : make_int2(0, 0);
                        if (MBC_BAD(r[u].x >= 0 && (int64_t)(r[u].x >> 2) + b < (int64_t)d.n_cols_b * n_rb, 24,
                                    (r[u].x >> 2) + b, (int64_t)d.n_cols_b * n_rb))
                            r[u] = make_int2(0, 0);
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) bv[u] = __ldcg(btb + (r[u].x >> 2));
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const float2 gj = pick<NJ>(g[l], r[u].x & 3);
                        const float c = __int_as_float(r[u].y);
                        part = cfma(part, make_float2(c * gj.x, c * gj.y), bv[u]);
                    }
                }
            } else {
                const int4* tp = d.term4 + lq0[l];
#pragma unroll 1
                for (int q = 0; q < nt; ++q) {
                    const int4 r = __ldg(tp + q);
                    const float2 bv = __ldcg(btb + (r.x >> 2));
                    const float2 gj = pick<NJ>(g[l], r.x & 3);
                    part = cfma(part, cfma(make_float2(0.f, 0.f), make_float2(__int_as_float(r.y), __int_as_float(r.z)), gj),
                                bv);
                }
            }
            add_part(acc, guard, part);
        }
    }
}

template <bool REAL, int NJ>
__device__ __forceinline__ void leaf_stage(const Eg32Dev& d, const WalkLeaf* lv, int nleaf, const float2* leafbuf,
                                           int n_e, const float2* __restrict__ bt, CAcc& acc, float& guard, int wt) {
    if (NJ > 2 || nleaf == 1) {         // one leaf at a time (G of more free indices per leaf)
        for (int l = 0; l < nleaf; ++l) leaf_stage_n<REAL, NJ, 1>(d, lv + l, leafbuf + l * n_e, n_e, bt, acc, guard, wt);
        return;
    }
    if (nleaf == 2) leaf_stage_n<REAL, NJ, NJ <= 2 ? 2 : 1>(d, lv, leafbuf, n_e, bt, acc, guard, wt);
    else if (nleaf == 3) leaf_stage_n<REAL, NJ, NJ <= 2 ? 3 : 1>(d, lv, leafbuf, n_e, bt, acc, guard, wt);
    else leaf_stage_n<REAL, NJ, NJ <= 2 ? 4 : 1>(d, lv, leafbuf, n_e, bt, acc, guard, wt);
}

// Run one flavour's walker program: B (to_cols: leaf tables to the block's B table) or
// A (leaf tables to the walker's batch buffer, then the leaf stage).
template <bool REAL, int NJ>
__device__ __forceinline__ void walk(const Eg32Dev& d, const WalkDev& f, bool is_a, const float2* M,
                                     const uint32_t* spk, float2* stack, float2* leafbuf, float2* bt, CAcc& acc,
                                     float& guard, int gw, int w, int wt) {
    const int n = f.n;
    const int s0 = __ldg(f.step_off + gw);
    int s1 = __ldg(f.step_off + gw + 1);
    if (MBC_BAD(s0 >= 0 && s1 <= f.n_steps, 10, s1, f.n_steps)) s1 = s0;
    for (int s = s0; s < s1; ++s) {
        WalkStep st = f.steps[s];
        if (MBC_BAD(st.level < n && st.leaf0 >= 0 && st.leaf0 + st.nleaf <= f.n_leaves && st.nleaf <= kMaxBatch, 11,
                    st.leaf0 + st.nleaf, f.n_leaves)) {
            st.level = 0;
            st.nleaf = 0;
        }
        if (st.level > 0) {
            const int k = st.level;
            lap_node_k(k, M, spk + f.pk_off[k], f.size[k], st.col, st.sign, stack + f.off[k - 1], stack + f.off[k], wt,
                       f.size[k - 1]);
            walker_sync(w);
        }
        if (st.nleaf > 0) {
            if (st.level == 0) walker_sync(w);     // the previous batch may still be read
            const WalkLeaf* lv = f.leaves + st.leaf0;
            lap_leaves_k(n, M, spk + f.pk_off[n], f.size[n], lv, st.nleaf, stack + f.off[n - 1],
                         is_a ? leafbuf : bt, !is_a, wt, f.size[n - 1],
                         is_a ? (int64_t)d.leafbuf_vals : (int64_t)d.n_cols_b * d.n_rows_b, d.b_pos);
            walker_sync(w);
            if (is_a) leaf_stage<REAL, NJ>(d, lv, st.nleaf, leafbuf, f.size[n], bt, acc, guard, wt);
        }
    }
}

// Cluster helpers (sm_90+): rank of this block in its cluster, a cluster-wide barrier
// with release/acquire ordering, and a store to another block's shared memory.
__device__ __forceinline__ int cluster_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return (int)r;
}
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ void st_cluster(double* local, int rank, double v) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(local);
    unsigned ra;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(rank));
    asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(ra), "d"(v) : "memory");
}

// Shared memory of the FP32 kernels and the per-block state of a walker.
struct Site32Smem {
    float2* sA;
    float2* sB;
    uint32_t* spk;
    float2* stack;
    float2* leafbuf;
    double* red;
    double* xpart;
};

__device__ __forceinline__ Site32Smem site32_smem(const Eg32Dev& d, unsigned char* raw, double* red, double* xpart) {
    Site32Smem m;
    m.sA = reinterpret_cast<float2*>(raw);
    m.sB = m.sA + kBlk;
    m.spk = reinterpret_cast<uint32_t*>(m.sB + kBlk);
    m.stack = reinterpret_cast<float2*>(m.spk + d.pk_words) + (size_t)(threadIdx.x / kWalker) *
                                                                  (d.stack_vals + d.leafbuf_vals);
    m.leafbuf = m.stack + d.stack_vals;
    m.red = red;
    m.xpart = xpart;
    return m;
}

// Copy the plan's packed Laplace words to shared memory and set level 0 of the walker
// stacks (the empty minor); block-wide barrier before and after.
__device__ __forceinline__ void site32_stage_plan(const Eg32Dev& d, const Site32Smem& m) {
    __syncthreads();
    for (int i = threadIdx.x; i < d.pk_words; i += blockDim.x) m.spk[i] = __ldg(d.pk + i);
    if (threadIdx.x % kWalker == 0 && threadIdx.x / kWalker < d.walkers) m.stack[0] = make_float2(1.f, 0.f);
    __syncthreads();
}

// One sink site on one block of its cluster (rank), d.cs blocks per site.  The cluster's
// blocks share the site's B table bt (global memory); their d.walkers walkers each are
// walkers rank * d.walkers + w of the plan's programs.  With d.cs > 1 every block sends
// its partial sums to block 0 of the cluster, which combines them in rank order
// (deterministic).  Block 0 writes the site's partial and error scale and, when the
// per-site estimate exceeds site_guard, appends `unit` to the recompute list.
template <bool REAL, int NJ>
__device__ __forceinline__ void site32(const Eg32Dev& d, const double* __restrict__ U, const double* __restrict__ D,
                                       int64_t site, int64_t unit, d4* __restrict__ part, double* __restrict__ scale_out,
                                       float2* __restrict__ bt, const Site32Smem& m, int rank, int cs,
                                       float site_guard, unsigned int* __restrict__ flag_count,
                                       unsigned int* __restrict__ flag_list, unsigned int flag_cap) {
    // cs: the launch's cluster size; blocks of rank >= d.cs (a batched item planned for
    // smaller clusters) and walkers w >= d.walkers (an item planned for fewer walkers than
    // the launch's blocks have) take part in the barriers and the exchange only
    const int w = threadIdx.x / kWalker, wt = threadIdx.x % kWalker;
    const bool active = rank < d.cs && w < d.walkers;
    const int gw = rank * d.walkers + w;
    const int nA = d.A.n, nB = d.B.n;
    const double* ma = (d.flav_a == 0 ? U : D) + site * 288;
    const double* mb = (d.flav_a == 0 ? D : U) + site * 288;
    int ea, eb;
    stage_f32(ma, mb, m.sA, m.sB, m.red, ea, eb);
    __syncthreads();
    CAcc acc = {0.f, 0.f, 0.f, 0.f};
    float guard = 0.f;
    if (nB == 0) {
        if (threadIdx.x == 0 && rank == 0) bt[0] = make_float2(1.f, 0.f);
    } else if (active) {
        walk<REAL, NJ>(d, d.B, false, m.sB, m.spk, m.stack, m.leafbuf, bt, acc, guard, gw, w, wt);
    }
    __syncthreads();                                   // the B table is complete
    if (cs > 1) cluster_sync_all();
    if (active) walk<REAL, NJ>(d, d.A, true, m.sA, m.spk, m.stack, m.leafbuf, bt, acc, guard, gw, w, wt);
    // site value: compensated block sums of the parts and of |part|^2
    kacc re = {0.0, 0.0}, im = {0.0, 0.0}, gs = {0.0, 0.0};
    block_sum_site(acc, guard, re, im, gs.hi, m.red);
    if (cs > 1) {
        if (threadIdx.x == 0) {
            st_cluster(m.xpart + 5 * rank + 0, 0, re.hi);
            st_cluster(m.xpart + 5 * rank + 1, 0, re.lo);
            st_cluster(m.xpart + 5 * rank + 2, 0, im.hi);
            st_cluster(m.xpart + 5 * rank + 3, 0, im.lo);
            st_cluster(m.xpart + 5 * rank + 4, 0, gs.hi + gs.lo);
        }
        cluster_sync_all();
        if (rank == 0 && threadIdx.x == 0) {
            kacc r2 = {0.0, 0.0}, i2 = {0.0, 0.0};
            double gsum = 0.0;
            for (int q = 0; q < cs; ++q) {
                kacc_merge(r2, kacc{m.xpart[5 * q + 0], m.xpart[5 * q + 1]});
                kacc_merge(i2, kacc{m.xpart[5 * q + 2], m.xpart[5 * q + 3]});
                gsum += m.xpart[5 * q + 4];
            }
            re = r2;
            im = i2;
            gs = kacc{gsum, 0.0};
        }
    }
    if (rank == 0 && threadIdx.x == 0) {
        const int sc = ea * nA + eb * nB;
        store_partial(part + site, re, im, sc);
        const double cr = re.hi + re.lo, ci = im.hi + im.lo;
        const double gsum = sqrt(gs.hi + gs.lo);
        const double est = gsum / sqrt(cr * cr + ci * ci);
        // per-site guard (when per-site values are returned); a site it sends to the
        // double-float kernel has no FP32 error left for the slice guard
        const bool flag = !(est <= (double)site_guard) || !isfinite(gsum);
        if (flag) {
            const unsigned k = atomicAdd(flag_count, 1u);
            if (!MBC_BAD(k < flag_cap, 30, k, flag_cap)) flag_list[k] = (unsigned int)unit;
        }
        scale_out[site] = flag ? 0.0 : ldexp(gsum, sc);
    }
}

// One plan: sites assigned round robin to the grid's clusters.
template <bool REAL, int NJ>
__global__ void __launch_bounds__(768, 1) egraph32_kernel(Eg32Dev d, const double* __restrict__ U,
                                                          const double* __restrict__ D, Geometry g,
                                                          d4* __restrict__ part, float2* __restrict__ bslots,
                                                          unsigned int* __restrict__ flag_count,
                                                          unsigned int* __restrict__ flag_list,
                                                          float site_guard, double* __restrict__ scale_out,
                                                          unsigned int flag_cap) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[5 * 32];
    __shared__ double xpart[5 * 16];      // block 0 of a cluster: the blocks' (re, im, guard) sums
    const Site32Smem m = site32_smem(d, smem_raw, red, xpart);
    const int rank = d.cs > 1 ? cluster_rank() : 0;
    const int64_t cid = blockIdx.x / d.cs, ncl = gridDim.x / d.cs;
    float2* bt = bslots + (size_t)cid * d.n_cols_b * d.n_rows_b;
    site32_stage_plan(d, m);
    const int64_t n_units = g.n_sites();
    for (int64_t site = cid; site < n_units; site += ncl)
        site32<REAL, NJ>(d, U, D, site, site, part, scale_out, bt, m, rank, d.cs, site_guard, flag_count, flag_list,
                         flag_cap);
}

// Several (plan, fields) items in one launch: units (item, site) numbered item by item,
// assigned round robin to the grid's clusters.  The launch takes the largest cluster size
// and walker count among the items (an item planned for fewer leaves the extra blocks or
// warps idle), their largest free-index count NJ, and complex weights if any item has
// them.  A block copies the item's plan view to shared memory and stages its packed words
// when the item changes.
template <bool REAL, int NJ>
__global__ void __launch_bounds__(768, 1) egraph32_batch_kernel(const BatchItem32* __restrict__ items, int n_items,
                                                                int64_t n_units, int cs, float2* __restrict__ bslots,
                                                                int64_t bslot_values,
                                                                unsigned int* __restrict__ flag_count,
                                                                unsigned int* __restrict__ flag_list) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[5 * 32];
    __shared__ double xpart[5 * 16];
    __shared__ Eg32Dev sd;
    const unsigned int flag_cap = (unsigned int)n_units;
    __shared__ int s_item;
    const int rank = cs > 1 ? cluster_rank() : 0;
    const int64_t cid = blockIdx.x / cs, ncl = gridDim.x / cs;
    float2* bt = bslots + (size_t)cid * bslot_values;
    int cur = -1;
    for (int64_t unit = cid; unit < n_units; unit += ncl) {
        if (threadIdx.x == 0) {
            int lo = 0, hi = n_items - 1;
            while (lo < hi) {                  // last item whose first unit is <= unit
                const int mid = (lo + hi + 1) >> 1;
                if (items[mid].unit_begin <= unit) lo = mid; else hi = mid - 1;
            }
            s_item = lo;
        }
        __syncthreads();
        int it = s_item;
        if (MBC_BAD(it >= 0 && it < n_items && unit - items[it].unit_begin < items[it].g.n_sites(), 40, unit, n_items))
            it = 0;
        if (it != cur) {
            if (threadIdx.x == 0) sd = items[it].d;
            __syncthreads();
            site32_stage_plan(sd, site32_smem(sd, smem_raw, red, xpart));
            cur = it;
        }
        const BatchItem32& item = items[it];
        const Site32Smem m = site32_smem(sd, smem_raw, red, xpart);
        site32<REAL, NJ>(sd, item.U, item.D, unit - item.unit_begin, unit, item.part, item.scale, bt, m, rank, cs,
                         item.site_guard, flag_count, flag_list, flag_cap);
    }
}

// The slice guard: one block per (set, t).  The FP32 error of C(t) is estimated as
//   err(t) = kSliceErr * sqrt(sum_x s_x^2),   s_x = sqrt(sum |part|^2) of site x,
// (the sites' rounding errors add like independent random numbers, so the slice's error
// is close to a complex Gaussian of rms r sqrt(sum_x s_x^2), r the rms ratio of a site's
// FP32 error to s_x, measured 1.5e-7 on the He-3 workloads; kSliceErr = 1.67 r.  It is an
// estimate, not a bound: 4e-7 (2.67 r) recomputed three times as many slices of the He-3
// workload at 24^3 x 48 without changing its largest C(t) error, 8.2e-7).  When
// err(t) > tol |C(t)|, the sites of the slice with the largest s_x are appended to the
// recompute list -- those with s_x above the largest threshold tau for which the sites at
// or below tau leave an estimate of at most tol |C(t)| / 2 (a recomputed site carries no
// FP32 error; tau by bisection) -- skipping sites the site guard listed already (s_x = 0).
// C(t) here is the FP32 estimate with the momentum phase of the site sum.
constexpr double kSliceErr = 2.5e-7;
constexpr int kTauSteps = 40;
__device__ __forceinline__ void slice_guard_body(const d4* __restrict__ part, const double* __restrict__ scale,
                                                 int64_t st, int64_t V3, Momentum mom, double tol, int64_t unit0,
                                                 unsigned int* __restrict__ flag_count,
                                                 unsigned int* __restrict__ flag_list, unsigned int flag_cap, double* red,
                                                 int* s_flag, double* s_tau) {
    double re = 0.0, im = 0.0, m = 0.0;
    for (int64_t x = threadIdx.x; x < V3; x += blockDim.x) {
        const d4 v = part[st * V3 + x];
        double vr = v.x + v.y, vi = v.z + v.w;
        if (mom.nonzero()) {
            const int64_t L = mom.L;
            int64_t k = ((int64_t)mom.px * (x % L) + (int64_t)mom.py * ((x / L) % L) + (int64_t)mom.pz * (x / (L * L))) % L;
            if (k < 0) k += L;
            double sn, cs;
            sincospi(-2.0 * (double)k / (double)L, &sn, &cs);
            const double tr = vr * cs - vi * sn;
            vi = vr * sn + vi * cs;
            vr = tr;
        }
        re += vr;
        im += vi;
        m = fmax(m, scale[st * V3 + x]);
    }
    kacc kr, ki;
    block_sum(cd_make(re, im), kr, ki, red);          // valid in thread 0
    m = block_max(m, red);
    double q = 0.0;
    if (m > 0.0)
        for (int64_t x = threadIdx.x; x < V3; x += blockDim.x) {
            const double r = scale[st * V3 + x] / m;
            q += r * r;
        }
    kacc kq, kz;
    block_sum(cd_make(q, 0.0), kq, kz, red);
    // the remaining sum of (s_x / m)^2 allowed after the recompute: (tol |C| / (2 kSliceErr m))^2
    __shared__ double s_allow;
    if (threadIdx.x == 0) {
        const double cr = kr.hi + kr.lo, ci = ki.hi + ki.lo;
        const double cabs = sqrt(cr * cr + ci * ci);
        const double err = kSliceErr * m * sqrt(kq.hi + kq.lo);
        *s_flag = m > 0.0 && !(err <= tol * cabs);
        const double a = m > 0.0 ? tol * cabs / (2.0 * kSliceErr * m) : 0.0;
        s_allow = isfinite(a) ? a * a : 0.0;
        s_tau[0] = 0.0;                              // sum over s_x <= tau within the allowance
        s_tau[1] = 1.0;                              // (every site: above it)
    }
    __syncthreads();
    if (!*s_flag) return;
    for (int it = 0; it < kTauSteps; ++it) {
        const double mid = 0.5 * (s_tau[0] + s_tau[1]);
        double qb = 0.0;
        for (int64_t x = threadIdx.x; x < V3; x += blockDim.x) {
            const double r = scale[st * V3 + x] / m;
            if (r <= mid) qb += r * r;
        }
        kacc kb, kbz;
        block_sum(cd_make(qb, 0.0), kb, kbz, red);
        if (threadIdx.x == 0) {
            if (kb.hi + kb.lo <= s_allow) s_tau[0] = mid;
            else s_tau[1] = mid;
        }
        __syncthreads();
    }
    const double tau = s_tau[0];
    for (int64_t x = threadIdx.x; x < V3; x += blockDim.x) {
        const double sx = scale[st * V3 + x];
        if (sx > 0.0 && sx / m > tau) {
            const unsigned k = atomicAdd(flag_count, 1u);
            if (!MBC_BAD(k < flag_cap, 31, k, flag_cap)) flag_list[k] = (unsigned int)(unit0 + st * V3 + x);
        }
    }
}

__global__ void slice_guard_kernel(const d4* __restrict__ part, const double* __restrict__ scale, int64_t V3,
                                   Momentum mom, double tol, unsigned int* __restrict__ flag_count,
                                   unsigned int* __restrict__ flag_list, unsigned int flag_cap) {
    __shared__ double red[4 * 32];
    __shared__ int s_flag;
    __shared__ double s_tau[2];
    slice_guard_body(part, scale, blockIdx.x, V3, mom, tol, 0, flag_count, flag_list, flag_cap, red, &s_flag, s_tau);
}

// Batched slice guard: block b is slice b - slice_begin of the item whose slices contain it.
__global__ void slice_guard_batch_kernel(const BatchItem32* __restrict__ items, int n_items,
                                         unsigned int* __restrict__ flag_count, unsigned int* __restrict__ flag_list,
                                         unsigned int flag_cap) {
    __shared__ double red[4 * 32];
    __shared__ int s_flag;
    __shared__ double s_tau[2];
    int lo = 0, hi = n_items - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (items[mid].slice_begin <= (int64_t)blockIdx.x) lo = mid; else hi = mid - 1;
    }
    const BatchItem32& it = items[lo];
    if (std::isinf(it.slice_tol) && it.slice_tol > 0) return;
    slice_guard_body(it.part, it.scale, (int64_t)blockIdx.x - it.slice_begin, it.g.V3, Momentum(), it.slice_tol,
                     it.unit_begin, flag_count, flag_list, flag_cap, red, &s_flag, s_tau);
}

// Cluster launch of kern with as many clusters as can be resident at once (at most
// `want` clusters).
template <class K, class... Args>
cudaError_t launch_clusters(K kern, int cs, int walkers, int smem, int64_t want, int max_grid, cudaStream_t s,
                            Args... args) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(walkers * kWalker);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cs;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int clusters = max_grid / cs;
    if (cs > 1) {
        cfg.gridDim = dim3(cs * clusters);
        int active = 0;
        e = cudaOccupancyMaxActiveClusters(&active, kern, &cfg);
        if (e != cudaSuccess) return e;
        if (active < 1) return cudaErrorInvalidConfiguration;
        clusters = std::min(clusters, active);
    }
    clusters = (int)std::max<int64_t>(1, std::min<int64_t>(clusters, want));
    cfg.gridDim = dim3(cs * clusters);
    e = cudaLaunchKernelEx(&cfg, kern, args...);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

template <bool REAL, int NJ>
cudaError_t launch_t(const Eg32Dev& d, const double* U, const double* D, Geometry g, d4* part, int max_grid,
                     void* bslots, unsigned int* flag_count, unsigned int* flag_list, float site_guard,
                     double* scale_out, cudaStream_t s) {
    return launch_clusters(egraph32_kernel<REAL, NJ>, d.cs, d.walkers, d.smem_bytes, g.n_sites(), max_grid, s, d, U,
                           D, g, part, (float2*)bslots, flag_count, flag_list, site_guard, scale_out,
                           (unsigned int)g.n_sites());
}

template <bool REAL, int NJ>
cudaError_t launch_batch_t(const BatchItem32* items, int n_items, int64_t n_units, int cs, int walkers, int smem,
                           int max_grid, void* bslots, int64_t bslot_values, unsigned int* flag_count,
                           unsigned int* flag_list, cudaStream_t s) {
    return launch_clusters(egraph32_batch_kernel<REAL, NJ>, cs, walkers, smem, n_units, max_grid, s, items, n_items,
                           n_units, cs, (float2*)bslots, bslot_values, flag_count, flag_list);
}

}  // namespace

cudaError_t launch_egraph32(const Eg32Dev& d, const double* U, const double* D, Geometry g, d4* part, int max_grid,
                            void* bslots, unsigned int* flag_count, unsigned int* flag_list, float site_guard,
                            double slice_tol, double* scale, Momentum mom, cudaStream_t s, int64_t* launches) {
    if (g.n_sites() == 0) return cudaSuccess;
    cudaError_t e;
#define MBC_E32_ARGS d, U, D, g, part, max_grid, bslots, flag_count, flag_list, site_guard, scale, s
    switch (d.n_j * 2 + (d.real_w ? 1 : 0)) {
        case 3: e = launch_t<true, 1>(MBC_E32_ARGS); break;
        case 5: e = launch_t<true, 2>(MBC_E32_ARGS); break;
        case 7: e = launch_t<true, 3>(MBC_E32_ARGS); break;
        case 9: e = launch_t<true, 4>(MBC_E32_ARGS); break;
        case 2: e = launch_t<false, 1>(MBC_E32_ARGS); break;
        case 4: e = launch_t<false, 2>(MBC_E32_ARGS); break;
        case 6: e = launch_t<false, 3>(MBC_E32_ARGS); break;
        case 8: e = launch_t<false, 4>(MBC_E32_ARGS); break;
        default: return cudaErrorInvalidValue;
    }
#undef MBC_E32_ARGS
    if (e != cudaSuccess) return e;
    ++*launches;
    if (std::isinf(slice_tol) && slice_tol > 0) return cudaSuccess;      // slice guard off
    slice_guard_kernel<<<(unsigned)((int64_t)g.n_sets * g.T), 256, 0, s>>>(part, scale, g.V3, mom, slice_tol,
                                                                          flag_count, flag_list,
                                                                          (unsigned int)g.n_sites());
    ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_egraph32_batch(const BatchItem32* items, int n_items, int64_t n_units, int64_t n_slices, bool real,
                                  int nj, int cs, int walkers, int smem, int max_grid, void* bslots,
                                  int64_t bslot_values, unsigned int* flag_count, unsigned int* flag_list,
                                  cudaStream_t s, int64_t* launches) {
    if (n_units == 0) return cudaSuccess;
    cudaError_t e;
#define MBC_E32B_ARGS items, n_items, n_units, cs, walkers, smem, max_grid, bslots, bslot_values, flag_count, flag_list, s
    if (real) e = nj <= 2 ? launch_batch_t<true, 2>(MBC_E32B_ARGS) : launch_batch_t<true, 4>(MBC_E32B_ARGS);
    else e = nj <= 2 ? launch_batch_t<false, 2>(MBC_E32B_ARGS) : launch_batch_t<false, 4>(MBC_E32B_ARGS);
#undef MBC_E32B_ARGS
    if (e != cudaSuccess) return e;
    ++*launches;
    if (n_slices > 0) {
        slice_guard_batch_kernel<<<(unsigned)n_slices, 256, 0, s>>>(items, n_items, flag_count, flag_list,
                                                                     (unsigned int)n_units);
        ++*launches;
    }
    return cudaGetLastError();
}

cudaError_t egraph32_checks(CheckRecord* out) { return read_checks(out); }

}  // namespace mbc
