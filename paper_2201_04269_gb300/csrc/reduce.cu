// reduce.cu - site sum of the correlator (arXiv 2201.04269 Eq. 1 summed over the sink
// sites of a time slice), with the sink momentum phase e^{-i p.x} of the projection in
// Sec. 2 (zero momentum: the plain sum).
//
// Partials (one per (site, chunk), each a compensated complex double) are combined in a
// fixed order with TwoSum accumulation: first over the chunks of a site (one thread per
// site), then over the sites of each (set, t) (one block per (set, t), a fixed
// thread-to-site assignment and a fixed reduction tree), so the result does not depend
// on which block computed which unit.
#include "common.cuh"

namespace mbc {

__device__ __forceinline__ cd cmul(cd a, cd b) { return cd_make(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re); }

__global__ void site_reduce_kernel(Partials in, int64_t n_sites, int64_t V3, Momentum mom, cd scale, d4* site_tmp,
                                   double2* site_out) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_sites) return;
    kacc re = {0.0, 0.0}, im = {0.0, 0.0};
    for (int c = 0; c < in.n_chunks; ++c) {
        const d4 v = in.part[s * in.n_chunks + c];
        kacc_merge(re, kacc{v.x, v.y});
        kacc_merge(im, kacc{v.z, v.w});
    }
    if (site_out) {
        const cd v = cmul(scale, cd_make(re.hi + re.lo, im.hi + im.lo));
        site_out[s] = make_double2(v.re, v.im);
    }
    if (mom.nonzero()) {
        // e^{-i 2 pi p.x / L} with p.x reduced modulo L first (exact argument)
        const int64_t x = s % V3, L = mom.L;
        int64_t k = ((int64_t)mom.px * (x % L) + (int64_t)mom.py * ((x / L) % L) + (int64_t)mom.pz * (x / (L * L))) % L;
        if (k < 0) k += L;
        double sn, cs;
        sincospi(-2.0 * (double)k / (double)L, &sn, &cs);
        const cd v = cmul(cd_make(re.hi + re.lo, im.hi + im.lo), cd_make(cs, sn));
        site_tmp[s] = make_d4(v.re, 0.0, v.im, 0.0);
    } else {
        site_tmp[s] = make_d4(re.hi, re.lo, im.hi, im.lo);
    }
}

__global__ void slice_reduce_kernel(const d4* __restrict__ sites, int64_t V3, cd scale, double2* C) {
    __shared__ double red[4 * 32];
    const int64_t st = blockIdx.x;
    kacc re = {0.0, 0.0}, im = {0.0, 0.0};
    for (int64_t x = threadIdx.x; x < V3; x += blockDim.x) {
        const d4 v = sites[st * V3 + x];
        kacc_merge(re, kacc{v.x, v.y});
        kacc_merge(im, kacc{v.z, v.w});
    }
    for (int off = 16; off > 0; off >>= 1) {
        kacc_merge(re, kacc_shfl_down(re, off));
        kacc_merge(im, kacc_shfl_down(im, off));
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        red[4 * warp + 0] = re.hi; red[4 * warp + 1] = re.lo;
        red[4 * warp + 2] = im.hi; red[4 * warp + 3] = im.lo;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        kacc r = {0.0, 0.0}, i = {0.0, 0.0};
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            kacc_merge(r, kacc{red[4 * w + 0], red[4 * w + 1]});
            kacc_merge(i, kacc{red[4 * w + 2], red[4 * w + 3]});
        }
        const cd v = cmul(scale, cd_make(r.hi + r.lo, i.hi + i.lo));
        C[st] = make_double2(v.re, v.im);
    }
}

cudaError_t launch_reduce(Partials in, Geometry g, cd scale, double2* C, double2* site_out, d4* site_tmp,
                          cudaStream_t s, int64_t* launches, Momentum mom) {
    const int64_t n_sites = g.n_sites();
    const d4* sites = in.part;
    if (in.n_chunks > 1 || site_out || mom.nonzero()) {
        const int64_t blocks = (n_sites + 255) / 256;
        if (blocks > 0) {
            site_reduce_kernel<<<(unsigned)blocks, 256, 0, s>>>(in, n_sites, g.V3, mom, scale, site_tmp, site_out);
            ++*launches;
        }
        sites = site_tmp;
    }
    const int64_t slices = (int64_t)g.n_sets * g.T;
    if (slices > 0) {
        slice_reduce_kernel<<<(unsigned)slices, 256, 0, s>>>(sites, g.V3, scale, C);
        ++*launches;
    }
    return cudaGetLastError();
}

}  // namespace mbc
