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
    __shared__ __align__(16) V su[144];
    __shared__ __align__(16) V sd[144];
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
        int blk = 0;
        for (int64_t q = begin + threadIdx.x; q < end; q += blockDim.x) {
            const int8_t* ia;
            const int8_t* ib;
            cd w;
            if (d.explicit_terms) {
                ia = d.ex_snk + q * nq;
                ib = d.ex_src + q * nq;
                w = d.ex_w[q];
            } else {
                while (q >= d.blk_start[blk + 1]) ++blk;      // q only grows within a thread
                const int64_t loc = q - d.blk_start[blk];
                const int64_t a = d.blk_s0[blk] + loc / d.blk_nr[blk];
                const int64_t r = d.blk_r0[blk] + loc % d.blk_nr[blk];
                ia = d.snk_idx + a * nq;
                ib = d.src_idx + r * nq;
                const cd p = d.blk_p[blk], s = d.snk_w[a], t = d.src_w[r];
                const cd ps = cd_make(p.re * s.re - p.im * s.im, p.re * s.im + p.im * s.re);
                w = cd_make(ps.re * t.re + ps.im * t.im, ps.im * t.re - ps.re * t.im);   // p s conj(t)
            }
            int8_t ra[12], rb[12];
#pragma unroll
            for (int i = 0; i < 12; ++i) {
                if (i < nq) { ra[i] = ia[i]; rb[i] = ib[i]; }
            }
            const V du = det_n<P>(d.n_u, su, ra, rb);
            const V dd = det_n<P>(d.n_d, sd, ra + d.n_u, rb + d.n_u);
            const V wd = P::mul(P::from_cd(w, 0), du);
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
