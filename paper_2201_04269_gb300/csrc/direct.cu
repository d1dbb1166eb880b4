// direct.cu - the direct index-set sweep (arXiv 2201.04269 Eq. 1, Sec. 1).
//
// For every sink site x and every (a, a') in the index set I the kernel forms
// W(a, a') det U_x[a_u, a'_u] det D_x[a_d, a'_d] with one pivoted LU per determinant
// (the determinant formulation of the Wick contraction) and sums.  No symmetry is
// used: this is the unoptimised correlator the paper's algorithms are measured against.
//
// Work unit = (site, chunk of the flattened index set).  A block stages the site's
// two 12x12 blocks in shared memory (coalesced 16-byte loads), every thread takes pairs
// q = begin + tid, begin + tid + blockDim, ..., gathers its n_u x n_u and n_d x n_d
// submatrices from shared memory into registers and factorises them there.  Per-thread
// sums are combined by a deterministic compensated block reduction into one partial
// per unit.
#include "common.cuh"

namespace mbc {

template <class P>
__global__ void __launch_bounds__(256) direct_kernel(DirectDev d, const double* __restrict__ U,
                                                     const double* __restrict__ D, Geometry g, int64_t chunk,
                                                     Partials out) {
    typedef typename P::V V;
    __shared__ __align__(16) V su[kBlk];
    __shared__ __align__(16) V sd[kBlk];
    __shared__ double red[4 * 32];
    const int nq = d.n_u + d.n_d;
    const int64_t n_chunks = out.n_chunks;
    const int64_t n_units = g.n_sites() * n_chunks;
    for (int64_t unit = blockIdx.x; unit < n_units; unit += gridDim.x) {
        const int64_t site = unit / n_chunks, ch = unit % n_chunks;
        int eu, ed;
        load_pair<P>(U + site * 288, D + site * 288, su, sd, red, eu, ed);
        const int64_t begin = ch * chunk;
        const int64_t end = min(begin + chunk, d.index_size);
        typename P::A acc;
        P::acc_zero(acc);
        // pair q = blk_start[blk] + (a - s0) * nr + (r - r0): the thread steps (blk, a, r)
        // by blockDim without dividing
        int blk = 0;
        int64_t a = 0, r = 0, nr = 1;
        const int64_t q0 = begin + threadIdx.x;
        if (!d.explicit_terms && q0 < end) {
            while (q0 >= d.blk_start[blk + 1]) ++blk;
            const int64_t loc = q0 - d.blk_start[blk];
            nr = d.blk_nr[blk];
            a = d.blk_s0[blk] + loc / nr;
            r = d.blk_r0[blk] + loc % nr;
        }
        for (int64_t q = q0; q < end; q += blockDim.x) {
            const int8_t* ia;
            const int8_t* ib;
            V w;
            if (d.explicit_terms) {
                ia = d.ex_snk + q * nq;
                ib = d.ex_src + q * nq;
                w = ldv<V>(d.ex_w, q);
            } else {
                ia = d.snk_idx + a * nq;
                ib = d.src_idx + r * nq;
                // W = P_jj' s_j(a) conj(r_j'(a'))
                w = P::mul(P::mul(ldv<V>(d.blk_p, blk), ldv<V>(d.snk_w, a)), conj(ldv<V>(d.src_w, r)));
                // advance by blockDim pairs
                int64_t step = blockDim.x;
                while (step > 0) {
                    const int64_t room = (d.blk_r0[blk] + nr) - r;     // pairs left in this row of the block
                    if (step < room) { r += step; step = 0; break; }
                    step -= room;
                    ++a;
                    r = d.blk_r0[blk];
                    if (a - d.blk_s0[blk] >= d.blk_ns[blk]) {   // next block
                        ++blk;
                        if (blk >= d.n_blocks) break;
                        nr = d.blk_nr[blk];
                        a = d.blk_s0[blk];
                        r = d.blk_r0[blk];
                    }
                }
            }
            int8_t ra[12], rb[12];
#pragma unroll
            for (int i = 0; i < 12; ++i) {
                if (i < nq) { ra[i] = ia[i]; rb[i] = ib[i]; }
            }
            const V du = det_n<P, kLd>(d.n_u, su, ra, rb);
            const V dd = det_n<P, kLd>(d.n_d, sd, ra + d.n_u, rb + d.n_u);
            const V wd = P::mul(w, du);
            P::fma(acc, wd, dd);
        }
        const cd v = P::to_cd(P::get(acc));
        kacc re, im;
        block_sum(v, re, im, red);
        if (threadIdx.x == 0) store_partial(out.part + unit, re, im, eu * d.n_u + ed * d.n_d);
        __syncthreads();
    }
}

cudaError_t launch_direct(const DirectDev& d, int prec, const double* U, const double* D, Geometry g,
                          int64_t chunk, Partials out, int threads, cudaStream_t s, int64_t* launches) {
    const int64_t units = g.n_sites() * out.n_chunks;
    if (units == 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t grid = std::min<int64_t>(units, (int64_t)sms * 8);
    if (prec == 0) direct_kernel<FP64><<<(unsigned)grid, threads, 0, s>>>(d, U, D, g, chunk, out);
    else direct_kernel<MIXED><<<(unsigned)grid, threads, 0, s>>>(d, U, D, g, chunk, out);
    ++*launches;
    return cudaGetLastError();
}

}  // namespace mbc
