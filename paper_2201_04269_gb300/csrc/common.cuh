// common.cuh - block reductions, site loading and small pivoted LU determinants shared by
// the kernels of libmbc (internal).
#pragma once
#include "device.cuh"
#include "numeric.cuh"

namespace mbc {

// --------------------------------------------------------------------- reductions
__device__ __forceinline__ kacc kacc_shfl_down(kacc v, int off) {
    kacc o;
    o.hi = __shfl_down_sync(0xffffffffu, v.hi, off);
    o.lo = __shfl_down_sync(0xffffffffu, v.lo, off);
    return o;
}

// Deterministic compensated block sum of one complex double per thread; the result is
// valid in thread 0.  red: shared scratch of 2 * 2 * (blockDim / 32) doubles x 2.
__device__ __forceinline__ void block_sum(cd v, kacc& out_re, kacc& out_im, double* red) {
    kacc re = {v.re, 0.0}, im = {v.im, 0.0};
    for (int off = 16; off > 0; off >>= 1) {
        kacc_merge(re, kacc_shfl_down(re, off));
        kacc_merge(im, kacc_shfl_down(im, off));
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) {
        red[4 * warp + 0] = re.hi; red[4 * warp + 1] = re.lo;
        red[4 * warp + 2] = im.hi; red[4 * warp + 3] = im.lo;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        kacc r = {0.0, 0.0}, i = {0.0, 0.0};
        for (int w = 0; w < nw; ++w) {
            kacc_merge(r, kacc{red[4 * w + 0], red[4 * w + 1]});
            kacc_merge(i, kacc{red[4 * w + 2], red[4 * w + 3]});
        }
        out_re = r;
        out_im = i;
    }
    __syncthreads();
}

__device__ __forceinline__ double block_max(double v, double* red) {
    for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, off));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double m = 0.0;
    for (int w = 0; w < nw; ++w) m = fmax(m, red[w]);
    __syncthreads();
    return m;
}

// Load two 12x12 complex double blocks (flavour matrices of one site) into shared memory
// as precision-P values; for the mixed precision each block is first scaled by an exact
// power of two so that its largest |re|, |im| lies in [0.5, 1); the exponents are
// returned (0, 0 for FP64).
template <class P>
__device__ __forceinline__ void load_pair(const double* __restrict__ a, const double* __restrict__ b,
                                          typename P::V* sa, typename P::V* sb, double* red, int& ea, int& eb) {
    // entry (r, c) goes to [r * kLd + c]
    cd* ra = reinterpret_cast<cd*>(sa);
    cd* rb = reinterpret_cast<cd*>(sb);
    double ma = 0.0, mb = 0.0;
    for (int i = threadIdx.x; i < 288; i += blockDim.x) {
        const int e = i < 144 ? i : i - 144;
        const int o = (e / 12) * kLd + e % 12;
        const double2 v = __ldg(reinterpret_cast<const double2*>(i < 144 ? a : b) + e);
        if (i < 144) { ra[o] = cd_make(v.x, v.y); ma = fmax(ma, fmax(fabs(v.x), fabs(v.y))); }
        else { rb[o] = cd_make(v.x, v.y); mb = fmax(mb, fmax(fabs(v.x), fabs(v.y))); }
    }
    if (!P::scaled()) { ea = eb = 0; __syncthreads(); return; }
    ma = block_max(ma, red);
    mb = block_max(mb, red);
    ea = block_exponent(ma);
    eb = block_exponent(mb);
    for (int i = threadIdx.x; i < 288; i += blockDim.x) {
        const int e = i < 144 ? i : i - 144;
        const int o = (e / 12) * kLd + e % 12;
        if (i < 144) sa[o] = P::from_cd(ra[o], -ea);
        else sb[o] = P::from_cd(rb[o], -eb);
    }
    __syncthreads();
}

// --------------------------------------------------------------------- LU determinants
// det of the N x N matrix m[rows[i]][cols[k]] gathered from a 12x12 block, by Gaussian
// elimination with partial pivoting (pivot = largest |re| + |im|, first on ties; a row
// swap flips the sign; an exactly zero pivot gives 0, and so does, in the mixed
// arithmetic, a pivot below P::tiny()).
template <class P, int N, int LD>
__device__ __forceinline__ typename P::V det_gather(const typename P::V* m, const int8_t* rows, const int8_t* cols) {
    typedef typename P::V V;
    V a[N][N];
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
        for (int k = 0; k < N; ++k) a[i][k] = m[rows[i] * LD + cols[k]];
    V det = P::zero();
    bool first = true;
    int sign = 1;
#pragma unroll
    for (int k = 0; k < N; ++k) {
        int p = k;
        auto best = P::mag(a[k][k]);
#pragma unroll
        for (int i = k + 1; i < N; ++i) {
            auto mg = P::mag(a[i][k]);
            if (mg > best) { best = mg; p = i; }
        }
        if (best <= P::tiny()) return P::zero();
#pragma unroll
        for (int i = k + 1; i < N; ++i) {
            if (i == p) {
#pragma unroll
                for (int c = k; c < N; ++c) { V t = a[k][c]; a[k][c] = a[i][c]; a[i][c] = t; }
                sign = -sign;
            }
        }
        det = first ? a[k][k] : P::mul(det, a[k][k]);
        first = false;
        if (k + 1 < N) {
            V inv = P::div(P::one(), a[k][k]);
#pragma unroll
            for (int i = k + 1; i < N; ++i) {
                V f = P::mul(a[i][k], inv);
#pragma unroll
                for (int c = k + 1; c < N; ++c) {
                    typename P::A acc;
                    P::acc_zero(acc);
                    P::add(acc, a[i][c]);
                    P::fms(acc, f, a[k][c]);
                    a[i][c] = P::get(acc);
                }
            }
        }
    }
    return sign < 0 ? P::neg(det) : det;
}

template <class P, int LD>
__device__ __forceinline__ typename P::V det_n(int n, const typename P::V* m, const int8_t* rows, const int8_t* cols) {
    switch (n) {
        case 1: return m[rows[0] * LD + cols[0]];
        case 2: return det_gather<P, 2, LD>(m, rows, cols);
        case 3: return det_gather<P, 3, LD>(m, rows, cols);
        case 4: return det_gather<P, 4, LD>(m, rows, cols);
        case 5: return det_gather<P, 5, LD>(m, rows, cols);
        case 6: return det_gather<P, 6, LD>(m, rows, cols);
        default: return P::one();   // n = 0: empty product
    }
}

__device__ __forceinline__ void store_partial(d4* dst, const kacc& re, const kacc& im, int scale_exp) {
    d4 v;
    v.x = ldexp(re.hi, scale_exp); v.y = ldexp(re.lo, scale_exp);
    v.z = ldexp(im.hi, scale_exp); v.w = ldexp(im.lo, scale_exp);
    *dst = v;
}

}  // namespace mbc
