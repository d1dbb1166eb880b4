// tree.cu - factor-tree evaluation (arXiv 2201.04269 Sec. 4).
//
// The planner's linearised factor tree (factors in depth-first order, children counts,
// leaf coefficients; Fig. 5) has the up minors det U[R_u, C_u] at level 1 and the down
// minors det D[R_d, C_d] at the leaves.  Evaluation has two kernels per wave of sites:
//
//  1. minor_table_kernel: every factor (distinct minor) once per site, by pivoted LU,
//     into a scratch table laid out [minor][site] so that the tree walk's gathers for
//     32 consecutive sites are one contiguous 512-byte access.  A block stages the 12x12
//     blocks of its 32 sites in shared memory (row stride padded by 16 bytes, so that a
//     warp reading the same entry of 32 sites touches every bank once per phase).
//  2. tree_walk_kernel: one warp per (32 sites, chunk of level-1 subtrees); lane = site.
//     The tree arrays are read warp-uniformly (broadcast), the factor values gathered
//     from the table; a level-1 vertex multiplies the sum of its leaves
//     (coefficient x leaf factor) -- the sum over root-to-leaf paths of Sec. 4.
#include "common.cuh"

namespace mbc {

static constexpr int kTreeSites = 32;              // sites per block / warp
static constexpr int kPad = 145;                   // padded 12x12 block stride (values)

template <class P>
__global__ void __launch_bounds__(256) minor_table_kernel(TreeDev d, int flavour, const double* __restrict__ M,
                                                          int64_t site0, int64_t n_sites, int64_t wave,
                                                          typename P::V* __restrict__ table, int64_t table_off,
                                                          int* __restrict__ exps) {
    typedef typename P::V V;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V* sm = reinterpret_cast<V*>(smem_raw);        // [32][kPad]
    __shared__ int s_exp[kTreeSites];
    const int n = flavour == 0 ? d.n_u : d.n_d;
    const int64_t n_minors = d.n_minors[flavour];
    const int64_t g0 = (int64_t)blockIdx.y * kTreeSites;   // first site of this block within the wave
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    // stage 32 sites (one warp per site at a time), with the per-site exponent
    for (int s = warp; s < kTreeSites; s += nw) {
        const int64_t site = site0 + g0 + s;
        double m = 0.0;
        cd raw[5];
        for (int i = 0; i < 5; ++i) {
            const int e = lane + 32 * i;
            raw[i] = cd_make(0.0, 0.0);
            if (e < 144 && g0 + s < n_sites) {
                const double2 v = __ldg(reinterpret_cast<const double2*>(M + site * 288) + e);
                raw[i] = cd_make(v.x, v.y);
                m = fmax(m, fmax(fabs(v.x), fabs(v.y)));
            }
        }
        for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, off));
        const int e = P::scaled() ? block_exponent(m) : 0;
        for (int i = 0; i < 5; ++i) {
            const int k = lane + 32 * i;
            if (k < 144) sm[s * kPad + k] = P::from_cd(raw[i], -e);
        }
        if (lane == 0) s_exp[s] = e;
    }
    __syncthreads();
    if (blockIdx.x == 0 && threadIdx.x < kTreeSites && g0 + threadIdx.x < n_sites)
        exps[(g0 + threadIdx.x) * 2 + flavour] = s_exp[threadIdx.x];
    // minors: warp w takes minors blockIdx.x * nw + w, + gridDim.x * nw, ...
    const bool live = g0 + lane < n_sites;
    for (int64_t mi = (int64_t)blockIdx.x * nw + warp; mi < n_minors; mi += (int64_t)gridDim.x * nw) {
        int8_t rows[6], cols[6];
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            if (i < n) { rows[i] = d.minor_rows[flavour][mi * n + i]; cols[i] = d.minor_cols[flavour][mi * n + i]; }
        }
        const V v = det_n<P, 12>(n, sm + lane * kPad, rows, cols);
        if (live) table[(table_off + mi) * wave + g0 + lane] = v;
    }
}

template <class P>
__global__ void __launch_bounds__(256) tree_walk_kernel(TreeDev d, const typename P::V* __restrict__ table,
                                                        int64_t site0, int64_t n_sites, int64_t wave,
                                                        const int* __restrict__ exps, Partials out) {
    typedef typename P::V V;
    const int lane = threadIdx.x & 31;
    const int64_t warp_global = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t groups = (n_sites + 31) / 32;
    const int64_t n_items = groups * d.n_chunks;
    if (warp_global >= n_items) return;
    const int64_t grp = warp_global % groups;     // neighbouring warps share a chunk: tree reads hit L1
    const int c = (int)(warp_global / groups);
    const int64_t s = grp * 32 + lane;
    const bool live = s < n_sites;
    const int64_t col = live ? s : 0;
    int64_t k = d.chunk_node[c];
    int64_t leaf = d.chunk_leaf[c];
    const int count = d.chunk_count[c];
    typename P::A acc;
    P::acc_zero(acc);
    for (int v1 = 0; v1 < count; ++v1) {
        const int32_t f1 = __ldg(d.factors + k);
        const int32_t nch = __ldg(d.children + k);
        ++k;
        const V u = table[(int64_t)f1 * wave + col];
        typename P::A inner;
        P::acc_zero(inner);
        for (int i = 0; i < nch; ++i) {
            const int32_t f2 = __ldg(d.factors + k + i);
            P::fma(inner, ldv<V>(d.coefficients, leaf + i), table[(int64_t)f2 * wave + col]);
        }
        k += nch;
        leaf += nch;
        P::fma(acc, u, P::get(inner));
    }
    if (live) {
        const cd v = P::to_cd(P::get(acc));
        const int e = exps[s * 2 + 0] * d.n_u + exps[s * 2 + 1] * d.n_d;
        d4 r;
        r.x = ldexp(v.re, e); r.y = 0.0; r.z = ldexp(v.im, e); r.w = 0.0;
        out.part[(site0 + s) * out.n_chunks + c] = r;
    }
}

size_t tree_value_bytes(int) { return 16; }

cudaError_t launch_tree(const TreeDev& d, int prec, const double* U, const double* D, Geometry g, void* scratch,
                        int64_t scratch_sites, int* exps, Partials out, int threads, cudaStream_t s,
                        int64_t* launches) {
    const int64_t total = g.n_sites();
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t smem = (size_t)kTreeSites * kPad * 16;
    static bool attr_set[2] = {false, false};
    if (!attr_set[prec]) {
        if (prec == 0) cudaFuncSetAttribute(minor_table_kernel<FP64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        else cudaFuncSetAttribute(minor_table_kernel<MIXED>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr_set[prec] = true;
    }
    cudaMemsetAsync(exps, 0, sizeof(int) * 2 * (size_t)std::min(total, scratch_sites), s);
    for (int64_t site0 = 0; site0 < total; site0 += scratch_sites) {
        const int64_t n = std::min(scratch_sites, total - site0);
        const int64_t wave = (n + 31) / 32 * 32;
        const int64_t gy = wave / 32;
        for (int f = 0; f < 2; ++f) {
            if (d.n_minors[f] == 0) continue;
            const int64_t per_block = (int64_t)(threads / 32) * 16;            // minors per block (16 rounds)
            int64_t gx = (d.n_minors[f] + per_block - 1) / per_block;
            gx = std::max<int64_t>(1, std::min<int64_t>(gx, std::max<int64_t>(1, (int64_t)sms * 16 / gy)));
            dim3 grid((unsigned)gx, (unsigned)gy);
            const double* M = (f == 0 ? U : D) + site0 * 288;
            const int64_t off = f == 0 ? 0 : d.n_minors[0];
            if (prec == 0)
                minor_table_kernel<FP64><<<grid, threads, smem, s>>>(d, f, M, 0, n, wave, (cd*)scratch, off, exps);
            else
                minor_table_kernel<MIXED><<<grid, threads, smem, s>>>(d, f, M, 0, n, wave, (cdf*)scratch, off, exps);
            ++*launches;
        }
        const int64_t items = (n + 31) / 32 * d.n_chunks;
        const int64_t blocks = (items * 32 + threads - 1) / threads;
        if (prec == 0)
            tree_walk_kernel<FP64><<<(unsigned)blocks, threads, 0, s>>>(d, (const cd*)scratch, site0, n, wave, exps, out);
        else
            tree_walk_kernel<MIXED><<<(unsigned)blocks, threads, 0, s>>>(d, (const cdf*)scratch, site0, n, wave, exps, out);
        ++*launches;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

}  // namespace mbc
