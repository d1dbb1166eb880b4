// egraph.cu - evaluation of the plan extracted from the tensor e-graph
// (arXiv 2201.04269 Sec. 5) for the canonical correlator (Sec. 3).
//
// Per site the correlator is
//   C_x = sum_{(j, j')} P_jj' sum_{(R_a, R_b)} s_j sum_{(C_a, C_b)} conj(r_j') A[R_a, C_a] B[R_b, C_b]
// with A, B the minors of the two flavours (A = the flavour whose column tree is
// streamed).  The extracted plan evaluates it as
//   for every needed A column set C_a (a leaf of the A column tree, depth first):
//     A-column   T(R_a) = det A[R_a, C_a] for every needed row set R_a, from the parent
//                column subset's table by one Laplace step along the added column:
//                det M[R, C] = sum_i (-1)^{i+q} M[r_i, c] det M[R \ r_i, C \ c];
//     G_j(R_b)   = sum_{R_a} s_j(R_a, R_b) T(R_a)                   (shared by all pairs)
//     for every B column set C_b paired with C_a by the source:
//       B-column det B[R_b, C_b] from a cached level-L table of its column prefix and
//                the remaining Laplace steps;
//       acc     += sum_{R_b} (sum_j coef_j(C_a, C_b) G_j(R_b)) det B[R_b, C_b]
// with coef_j = sum_j' P_jj' conj(r_j'(C_a, C_b)).  Everything lives in shared memory:
// the A tables along the current tree path (one per level), the B prefix cache, the
// on-demand B columns of a batch of pairs and G.  One block owns one site at a time and
// takes sites from an atomic work counter (persistent grid, no inter-block waiting).
// Mixed precision: the site's 12x12 blocks are scaled by exact powers of two and every
// product and sum is a double-float operation; the scale is restored in double.
#include "common.cuh"

namespace mbc {

template <class P>
__device__ __forceinline__ void laplace_level(const MinorDev& m, int k, int col, int sign, const typename P::V* mat,
                                              const typename P::V* parent, typename P::V* dest) {
    const int n = m.size[k];
    const uint16_t* child = m.child[k];
    const uint8_t* row = m.row[k];
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
        typename P::A acc;
        P::acc_zero(acc);
        for (int i = 0; i < k; ++i) {
            const int r = __ldg(row + e * k + i);
            const int c = __ldg(child + e * k + i);
            const typename P::V a = mat[r * kLd + col];
            if (((i & 1) ? -sign : sign) > 0) P::fma(acc, a, parent[c]);
            else P::fms(acc, a, parent[c]);
        }
        dest[e] = P::get(acc);
    }
}

template <class P>
__global__ void __launch_bounds__(256) egraph_kernel(EgraphDev d, const double* __restrict__ U,
                                                     const double* __restrict__ D, Geometry g, Partials out,
                                                     unsigned int* __restrict__ counter) {
    typedef typename P::V V;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V* sA = reinterpret_cast<V*>(smem_raw);
    V* sB = sA + kBlk;
    V* stA = sB + kBlk;
    V* stB = stA + d.stack_a;
    const int L = d.cache_level;
    const int nA = d.A.n, nB = d.B.n;
    const int fL = nB ? d.B.size[L] : 1;
    V* cache = stB + d.stack_b;
    V* path = cache + (size_t)d.n_cache_slots * fL;
    V* G = path + (size_t)d.n_batch * d.path_b;
    __shared__ double red[4 * 32];
    __shared__ unsigned int s_unit;
    const int64_t n_units = g.n_sites();
    const int n_rb = d.n_rows_b;
    const V one = P::one();
    for (;;) {
        if (threadIdx.x == 0) s_unit = atomicAdd(counter, 1u);
        __syncthreads();
        const int64_t site = s_unit;
        if (site >= n_units) break;
        // ---- stage the site's blocks (A flavour first)
        const double* ma = (d.flav_a == 0 ? U : D) + site * 288;
        const double* mb = (d.flav_a == 0 ? D : U) + site * 288;
        int ea, eb;
        load_pair<P>(ma, mb, sA, sB, red, ea, eb);
        if (threadIdx.x == 0) {
            stA[d.A.off[0]] = one;
            if (nB) stB[d.B.off[0]] = one;
        }
        __syncthreads();
        // ---- B prefix cache: column-tree nodes of depth <= L
        for (int ci = 0; ci < d.n_cache_nodes; ++ci) {
            const int node = __ldg(d.cache_nodes + ci);
            const int k = d.B.node_level[node];
            const int slot = __ldg(d.cache_slot + ci);
            V* dest = slot >= 0 ? cache + (size_t)slot * fL : stB + d.B.off[k];
            laplace_level<P>(d.B, k, d.B.node_col[node], d.B.node_sign[node], sB, stB + d.B.off[k - 1], dest);
            __syncthreads();
        }
        typename P::A acc;
        P::acc_zero(acc);
        // ---- A column tree, depth first
        for (int nd = 0; nd < d.A.n_nodes; ++nd) {
            const int k = __ldg(d.A.node_level + nd);
            laplace_level<P>(d.A, k, __ldg(d.A.node_col + nd), __ldg(d.A.node_sign + nd), sA, stA + d.A.off[k - 1],
                             stA + d.A.off[k]);
            __syncthreads();
            const int leaf = __ldg(d.A.node_leaf + nd);
            if (leaf < 0) continue;
            const V* T = stA + d.A.off[nA];
            // G_j(R_b) = sum_{R_a} s_j(R_a, R_b) T(R_a)
            {
                // flat index it = b * n_j + j, stepped without division
                const int nj = d.n_j, total = n_rb * nj, stride = blockDim.x;
                int b = threadIdx.x / nj, j = threadIdx.x - (threadIdx.x / nj) * nj;
                const int db = stride / nj, dj = stride - db * nj;
                for (int it = threadIdx.x; it < total; it += stride) {
                    typename P::A gj;
                    P::acc_zero(gj);
                    const int e1 = __ldg(d.g_off + it + 1);
                    for (int e = __ldg(d.g_off + it); e < e1; ++e) P::fma(gj, ldv<V>(d.g_w, e), T[__ldg(d.g_a + e)]);
                    G[j * n_rb + b] = P::get(gj);
                    b += db;
                    j += dj;
                    if (j >= nj) { j -= nj; ++b; }
                }
            }
            __syncthreads();
            // paired B columns, in batches
            const int p0 = __ldg(d.pair_off + leaf), p1 = __ldg(d.pair_off + leaf + 1);
            for (int ps = p0; ps < p1; ps += d.n_batch) {
                const int nbt = min(d.n_batch, p1 - ps);
                if (nB > L) {
                    for (int k = L + 1; k <= nB; ++k) {
                        const int fk = d.B.size[k];
                        const int poff = d.B.off[k] - d.B.off[L + 1];       // offset of level k in a path
                        const int ppar = k - 1 == L ? -1 : d.B.off[k - 1] - d.B.off[L + 1];
                        const uint16_t* child = d.B.child[k];
                        const uint8_t* row = d.B.row[k];
                        // flat index it = bi * fk + e, stepped without division
                        int bi = threadIdx.x / fk, e = threadIdx.x - (threadIdx.x / fk) * fk;
                        const int dbi = blockDim.x / fk, de = blockDim.x - dbi * fk;
                        for (int it = threadIdx.x; it < nbt * fk; it += blockDim.x) {
                            const int cb = __ldg(d.pair_b + ps + bi);
                            const int step = (int)((int64_t)cb * (nB - L) + (k - L - 1));
                            const V* parent = ppar < 0 ? cache + (size_t)__ldg(d.bcol_slot + cb) * fL
                                                       : path + (size_t)bi * d.path_b + ppar;
                            const int col = __ldg(d.bcol_path_col + step);
                            const int sign = __ldg(d.bcol_path_sign + step);
                            typename P::A a;
                            P::acc_zero(a);
                            for (int i = 0; i < k; ++i) {
                                const int r = __ldg(row + e * k + i);
                                const int c = __ldg(child + e * k + i);
                                const V m = sB[r * kLd + col];
                                if (((i & 1) ? -sign : sign) > 0) P::fma(a, m, parent[c]);
                                else P::fms(a, m, parent[c]);
                            }
                            path[(size_t)bi * d.path_b + poff + e] = P::get(a);
                            bi += dbi;
                            e += de;
                            if (e >= fk) { e -= fk; ++bi; }
                        }
                        __syncthreads();
                    }
                }
                // accumulate: threads over (pair, R_b)
                const int last = nB > L ? d.B.off[nB] - d.B.off[L + 1] : 0;
                int bi = threadIdx.x / n_rb, b = threadIdx.x - (threadIdx.x / n_rb) * n_rb;
                const int dbi = blockDim.x / n_rb, db = blockDim.x - dbi * n_rb;
                for (int it = threadIdx.x; it < nbt * n_rb; it += blockDim.x) {
                    const int pr = ps + bi;
                    const int cb = __ldg(d.pair_b + pr);
                    V bv;
                    if (nB == 0) bv = one;
                    else if (nB == L) bv = cache[(size_t)__ldg(d.bcol_slot + cb) * fL + b];
                    else bv = path[(size_t)bi * d.path_b + last + b];
                    typename P::A h;
                    P::acc_zero(h);
                    for (int j = 0; j < d.n_j; ++j) P::fma(h, ldv<V>(d.pair_coef, (int64_t)pr * d.n_j + j), G[j * n_rb + b]);
                    P::fma(acc, P::get(h), bv);
                    bi += dbi;
                    b += db;
                    if (b >= n_rb) { b -= n_rb; ++bi; }
                }
                if (ps + d.n_batch < p1) __syncthreads();
            }
            __syncthreads();
        }
        // ---- site value
        const cd v = P::to_cd(P::get(acc));
        kacc re, im;
        block_sum(v, re, im, red);
        if (threadIdx.x == 0) store_partial(out.part + site, re, im, ea * nA + eb * nB);
        __syncthreads();
    }
}

size_t egraph_smem_bytes(const EgraphDev& d, int) { return (size_t)d.smem_values * 16; }

cudaError_t launch_egraph(const EgraphDev& d, int prec, const double* U, const double* D, Geometry g, Partials out,
                          int threads, int blocks_per_sm, unsigned int* counter, cudaStream_t s, int64_t* launches) {
    const int64_t units = g.n_sites();
    if (units == 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t smem = egraph_smem_bytes(d, prec);
    cudaError_t e;
    if (prec == 0) e = cudaFuncSetAttribute(egraph_kernel<FP64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    else e = cudaFuncSetAttribute(egraph_kernel<MIXED>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t grid = std::min<int64_t>(units, (int64_t)sms * blocks_per_sm);
    e = cudaMemsetAsync(counter, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
    if (prec == 0) egraph_kernel<FP64><<<(unsigned)grid, threads, smem, s>>>(d, U, D, g, out, counter);
    else egraph_kernel<MIXED><<<(unsigned)grid, threads, smem, s>>>(d, U, D, g, out, counter);
    ++*launches;
    return cudaGetLastError();
}

}  // namespace mbc
