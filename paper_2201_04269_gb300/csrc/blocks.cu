// blocks.cu - hadron blocks (arXiv 2201.04269 Sec. 2), their momentum projection, and
// the factor tree over projected blocks (Secs. 3-4).
//
// Block of a baryon eps_abc (q1_a^T G q2_b) q3_c^alpha (q3 = q1) at one sink site:
//     f(s1, s2, s3)_alpha = eps_abc G_{beta gamma} [ Q1[(a beta), s3] Q1[(c alpha), s1]
//                                      - Q1[(a beta), s1] Q1[(c alpha), s3] ] Q2[(b gamma), s2]
// Evaluated in two steps per site: the diquark table
//     Dq[c][s][s2] = sum_{a,b} eps_abc sum_{beta,gamma} G_{beta gamma} Q1[(a beta), s] Q2[(b gamma), s2]
// (432 entries per block type, two eps terms x nnz(G) products each), then every entry
//     f(s1, s2, s3)_alpha = sum_c Dq[c][s3][s2] Q1[(c alpha), s1] - Dq[c][s1][s2] Q1[(c alpha), s3]
// (6 complex multiply-adds).  The site's two propagators and the diquark tables live in
// shared memory; for the projection each thread owns a fixed set of entries and keeps
// their running sums over the block's sites in shared memory, so the kernel reads 4.6 KB
// per site and writes one partial block per tile of sites.  Arithmetic: complex double;
// the kernel is bound by the FP64 pipe.
#include "blocks.cuh"
#include "common.cuh"

namespace mbc {

namespace {

constexpr int kQ = 144;           // one 12 x 12 propagator
constexpr int kDq = 432;          // one diquark table [c][s][s2]
constexpr int kThreads = 512;
constexpr int kTreeThreads = 512;
constexpr size_t kSmemBudget = 200 * 1024;

__device__ __forceinline__ cd cmul(cd a, cd b) { return cd_make(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re); }
__device__ __forceinline__ void cfma(cd& acc, cd a, cd b) {
    acc.re = fma(a.re, b.re, acc.re);
    acc.re = fma(-a.im, b.im, acc.re);
    acc.im = fma(a.re, b.im, acc.im);
    acc.im = fma(a.im, b.re, acc.im);
}
__device__ __forceinline__ void cfms(cd& acc, cd a, cd b) {
    acc.re = fma(-a.re, b.re, acc.re);
    acc.re = fma(a.im, b.im, acc.re);
    acc.im = fma(-a.re, b.im, acc.im);
    acc.im = fma(-a.im, b.re, acc.im);
}

// U_x then D_x (complex double, 144 each) into shared memory
__device__ __forceinline__ void stage_site(const double* __restrict__ U, const double* __restrict__ D, int64_t site,
                                           cd* q) {
    const double2* u = reinterpret_cast<const double2*>(U + site * 288);
    const double2* d = reinterpret_cast<const double2*>(D + site * 288);
    for (int i = threadIdx.x; i < 2 * kQ; i += blockDim.x) {
        const double2 v = i < kQ ? __ldg(u + i) : __ldg(d + i - kQ);
        q[i] = cd_make(v.x, v.y);
    }
}

// the block types' tables, copied from the launch parameters to shared memory
__device__ __forceinline__ void load_types(const BlockDev& b, BlockTypeDev* ty) {
    if (threadIdx.x < b.n_types) ty[threadIdx.x] = b.t[threadIdx.x];
}

__device__ __forceinline__ void diquarks(int n_types, const BlockTypeDev* types, const cd* q, cd* dq) {
    for (int e = threadIdx.x; e < n_types * kDq; e += blockDim.x) {
        const int t = e / kDq, r = e - t * kDq;
        const int c = r / 144, s = (r / 12) % 12, s2 = r % 12;
        const BlockTypeDev& ty = types[t];
        const cd* q1 = q + ty.q1 * kQ;
        const cd* q2 = q + (1 - ty.q1) * kQ;
        const int a0 = (c + 1) % 3, b0 = (c + 2) % 3;   // eps_{a0 b0 c} = +1, eps_{b0 a0 c} = -1
        cd acc = cd_make(0.0, 0.0);
        for (int k = 0; k < ty.n; ++k) {
            const int rb = 3 * ty.be[k], rg = 3 * ty.ga[k];
            cd x = cmul(q1[(rb + a0) * 12 + s], q2[(rg + b0) * 12 + s2]);
            const cd y = cmul(q1[(rb + b0) * 12 + s], q2[(rg + a0) * 12 + s2]);
            x.re -= y.re;
            x.im -= y.im;
            cfma(acc, cd_make(ty.g_re[k], ty.g_im[k]), x);
        }
        dq[e] = acc;
    }
}

__device__ __forceinline__ uint32_t entry_code(const BlockDev& b, int f) {
    if (b.entry) return __ldg(b.entry + f);
    const int s1 = f / 576, s2 = (f / 48) % 12, s3 = (f / 4) % 12, al = f % 4;
    return (uint32_t)((s1 << 12) | (s2 << 8) | (s3 << 4) | al);
}

// v + f(entry): the entry's block value added to v (v = 0 for the value itself)
__device__ __forceinline__ cd block_entry(const BlockTypeDev* types, uint32_t code, const cd* q, const cd* dq,
                                          cd v = cd_make(0.0, 0.0)) {
    const int slot = code >> 16, s1 = (code >> 12) & 15, s2 = (code >> 8) & 15, s3 = (code >> 4) & 15, al = code & 15;
    const cd* q1 = q + types[slot].q1 * kQ + 3 * al * 12;
    const cd* d = dq + slot * kDq;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        cfma(v, d[c * 144 + s3 * 12 + s2], q1[c * 12 + s1]);
        cfms(v, d[c * 144 + s1 * 12 + s2], q1[c * 12 + s3]);
    }
    return v;
}

__global__ void __launch_bounds__(kThreads) block_site_kernel(BlockDev b, const double* __restrict__ U,
                                                               const double* __restrict__ D, int64_t n_sites,
                                                               cd* __restrict__ out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ BlockTypeDev ty[6];
    cd* q = reinterpret_cast<cd*>(smem_raw);
    cd* dq = q + 2 * kQ;
    load_types(b, ty);
    for (int64_t site = blockIdx.x; site < n_sites; site += gridDim.x) {
        __syncthreads();
        stage_site(U, D, site, q);
        __syncthreads();
        diquarks(b.n_types, ty, q, dq);
        __syncthreads();
        cd* o = out + site * b.n_f;
        for (int f = threadIdx.x; f < b.n_f; f += blockDim.x) o[f] = block_entry(ty, entry_code(b, f), q, dq);
    }
}

// unit = (slice, tile, entry chunk); part [slice][tile][n_f]
__global__ void __launch_bounds__(kThreads) block_project_kernel(BlockDev b, const double* __restrict__ U,
                                                                  const double* __restrict__ D, int64_t V3, int L,
                                                                  int px, int py, int pz, int tiles, int f_chunk,
                                                                  int n_fc, cd* __restrict__ part) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ BlockTypeDev ty[6];
    cd* q = reinterpret_cast<cd*>(smem_raw);
    cd* dq = q + 2 * kQ;
    cd* acc = dq + b.n_types * kDq;
    load_types(b, ty);
    const int64_t unit = blockIdx.x;
    const int fc = (int)(unit % n_fc);
    const int tile = (int)((unit / n_fc) % tiles);
    const int64_t slice = unit / ((int64_t)n_fc * tiles);
    const int f0 = fc * f_chunk;
    const int nf = min(f_chunk, b.n_f - f0);
    for (int f = threadIdx.x; f < nf; f += blockDim.x) acc[f] = cd_make(0.0, 0.0);
    const int64_t x0 = V3 * tile / tiles, x1 = V3 * (tile + 1) / tiles;
    const bool mom = (px | py | pz) != 0;
    for (int64_t x = x0; x < x1; ++x) {
        __syncthreads();
        stage_site(U, D, slice * V3 + x, q);
        __syncthreads();
        diquarks(b.n_types, ty, q, dq);
        __syncthreads();
        cd ph = cd_make(1.0, 0.0);
        if (mom) {
            const int64_t cx = x % L, cy = (x / L) % L, cz = x / ((int64_t)L * L);
            int64_t k = ((int64_t)px * cx + (int64_t)py * cy + (int64_t)pz * cz) % L;
            if (k < 0) k += L;
            double sn, cs;
            sincospi(-2.0 * (double)k / (double)L, &sn, &cs);
            ph = cd_make(cs, sn);
        }
        if (mom) {
            for (int f = threadIdx.x; f < nf; f += blockDim.x) {
                const cd v = cmul(block_entry(ty, entry_code(b, f0 + f), q, dq), ph);
                acc[f].re += v.re;
                acc[f].im += v.im;
            }
        } else {
            // the running sum is the first addend of the entry's multiply-add chain
            for (int f = threadIdx.x; f < nf; f += blockDim.x) acc[f] = block_entry(ty, entry_code(b, f0 + f), q, dq, acc[f]);
        }
    }
    cd* o = part + (slice * tiles + tile) * (int64_t)b.n_f + f0;
    for (int f = threadIdx.x; f < nf; f += blockDim.x) o[f] = acc[f];
}

// ---------------------------------------------------------------- double-float blocks
// The same projection in double-float arithmetic (complex FP32 pairs, error-free
// products and sums).  Each site's propagators are scaled by exact powers of two 2^-e
// (e from the exponent bits of the block's largest |re|, |im|) before the split into
// (hi, lo) floats, so the block values are of order one; a block entry then carries the
// factor 2^(2 e_q1 + e_q2).  Every tile first finds the largest such exponent over its
// sites, per q1 flavour, and adds each site's values times 2^(exponent - largest) (an
// exact power of two <= 1), so nothing overflows; the tile's sums are converted to
// double and rescaled once.  The G matrices of the library's block types have entries
// in {0, +1, -1} (Dirac basis), which the diquark step uses as signs.
__device__ __forceinline__ unsigned abs_hiword(double x) { return (unsigned)__double2hiint(x) & 0x7fffffffu; }
// frexp exponent of a double whose |x| has high word m (0 for x = 0)
__device__ __forceinline__ int exponent_of(unsigned m) { return m ? (int)(m >> 20) - 1022 : 0; }
// exact 2^k in double for |k| <= 1022
__device__ __forceinline__ double pow2d(int k) { return __hiloint2double((1023 + k) << 20, 0); }
// exact 2^k in float for -126 <= k <= 0, 0 below
__device__ __forceinline__ float pow2f_le0(int k) { return k < -126 ? 0.f : __int_as_float((127 + k) << 23); }

// max over the block of two unsigned values; red: 64 unsigned of shared scratch
__device__ __forceinline__ void block_max_u2(unsigned& a, unsigned& b, unsigned* red) {
    a = __reduce_max_sync(0xffffffffu, a);
    b = __reduce_max_sync(0xffffffffu, b);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) { red[warp] = a; red[32 + warp] = b; }
    __syncthreads();
    a = 0u;
    b = 0u;
    for (int w = 0; w < nw; ++w) { a = max(a, red[w]); b = max(b, red[32 + w]); }
    __syncthreads();
}

// U_x, D_x scaled and split (one value per thread: needs blockDim >= 288); returns their
// exponents
__device__ __forceinline__ void stage_site_df(const double* __restrict__ U, const double* __restrict__ D,
                                              int64_t site, cdf* q, unsigned* red, int& eU, int& eD) {
    const int i = threadIdx.x;
    double2 v = make_double2(0.0, 0.0);
    if (i < 144) v = __ldg(reinterpret_cast<const double2*>(U + site * 288) + i);
    else if (i < 288) v = __ldg(reinterpret_cast<const double2*>(D + site * 288) + (i - 144));
    const unsigned m = max(abs_hiword(v.x), abs_hiword(v.y));
    unsigned mu = i < 144 ? m : 0u, md = (i >= 144 && i < 288) ? m : 0u;
    block_max_u2(mu, md, red);
    eU = exponent_of(mu);
    eD = exponent_of(md);
    if (i < 288) {
        const double sc = pow2d(-(i < 144 ? eU : eD));
        cdf z;
        z.re = df_from_double(v.x * sc);
        z.im = df_from_double(v.y * sc);
        q[i] = z;
    }
}

__device__ __forceinline__ void diquarks_df(int n_types, const BlockTypeDev* types, const cdf* q, cdf* dq) {
    for (int e = threadIdx.x; e < n_types * kDq; e += blockDim.x) {
        const int t = e / kDq, r = e - t * kDq;
        const int c = r / 144, s = (r / 12) % 12, s2 = r % 12;
        const BlockTypeDev& ty = types[t];
        const cdf* q1 = q + ty.q1 * kQ;
        const cdf* q2 = q + (1 - ty.q1) * kQ;
        const int a0 = (c + 1) % 3, b0 = (c + 2) % 3;
        MIXED::A acc;
        MIXED::acc_zero(acc);
        for (int k = 0; k < ty.n; ++k) {
            const int rb = 3 * ty.be[k], rg = 3 * ty.ga[k];
            // + g Q1[(rb + a0), s] Q2[(rg + b0), s2] - g Q1[(rb + b0), s] Q2[(rg + a0), s2], g = +-1
            if (ty.g_re[k] > 0.0) {
                MIXED::fma(acc, q1[(rb + a0) * 12 + s], q2[(rg + b0) * 12 + s2]);
                MIXED::fms(acc, q1[(rb + b0) * 12 + s], q2[(rg + a0) * 12 + s2]);
            } else {
                MIXED::fms(acc, q1[(rb + a0) * 12 + s], q2[(rg + b0) * 12 + s2]);
                MIXED::fma(acc, q1[(rb + b0) * 12 + s], q2[(rg + a0) * 12 + s2]);
            }
        }
        dq[e] = MIXED::get(acc);
    }
}

__device__ __forceinline__ cdf block_entry_df(const BlockTypeDev* types, uint32_t code, const cdf* q, const cdf* dq) {
    const int slot = code >> 16, s1 = (code >> 12) & 15, s2 = (code >> 8) & 15, s3 = (code >> 4) & 15, al = code & 15;
    const cdf* q1 = q + types[slot].q1 * kQ + 3 * al * 12;
    const cdf* d = dq + slot * kDq;
    MIXED::A a;
    MIXED::acc_zero(a);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        MIXED::fma(a, d[c * 144 + s3 * 12 + s2], q1[c * 12 + s1]);
        MIXED::fms(a, d[c * 144 + s1 * 12 + s2], q1[c * 12 + s3]);
    }
    return MIXED::get(a);
}

// unit = (slice, tile, entry chunk); part [slice][tile][n_f] in complex double
__global__ void __launch_bounds__(kThreads) block_project_df_kernel(BlockDev b, const double* __restrict__ U,
                                                                     const double* __restrict__ D, int64_t V3, int L,
                                                                     int px, int py, int pz, int tiles, int f_chunk,
                                                                     int n_fc, cd* __restrict__ part) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ BlockTypeDev ty[6];
    __shared__ unsigned red[64];
    __shared__ int eref[2];
    __shared__ cdf ph_s;
    cdf* q = reinterpret_cast<cdf*>(smem_raw);
    cdf* dq = q + 2 * kQ;
    cdf* acc = dq + b.n_types * kDq;
    load_types(b, ty);
    const int64_t unit = blockIdx.x;
    const int fc = (int)(unit % n_fc);
    const int tile = (int)((unit / n_fc) % tiles);
    const int64_t slice = unit / ((int64_t)n_fc * tiles);
    const int f0 = fc * f_chunk;
    const int nf = min(f_chunk, b.n_f - f0);
    for (int f = threadIdx.x; f < nf; f += blockDim.x) acc[f] = MIXED::zero();
    const int64_t x0 = V3 * tile / tiles, x1 = V3 * (tile + 1) / tiles;
    // largest 2 e_q1 + e_q2 over the tile's sites, for q1 = u and q1 = d (one warp per site)
    {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
        int r0 = -(1 << 30), r1 = -(1 << 30);
        for (int64_t x = x0 + warp; x < x1; x += nw) {
            const double2* u = reinterpret_cast<const double2*>(U + (slice * V3 + x) * 288);
            const double2* d = reinterpret_cast<const double2*>(D + (slice * V3 + x) * 288);
            unsigned mu = 0u, md = 0u;
            for (int i = lane; i < 144; i += 32) {
                const double2 a = __ldg(u + i), c = __ldg(d + i);
                mu = max(mu, max(abs_hiword(a.x), abs_hiword(a.y)));
                md = max(md, max(abs_hiword(c.x), abs_hiword(c.y)));
            }
            mu = __reduce_max_sync(0xffffffffu, mu);
            md = __reduce_max_sync(0xffffffffu, md);
            const int eu = exponent_of(mu), ed = exponent_of(md);
            r0 = max(r0, 2 * eu + ed);
            r1 = max(r1, 2 * ed + eu);
        }
        if (lane == 0) { red[warp] = (unsigned)(r0 + (1 << 30)); red[32 + warp] = (unsigned)(r1 + (1 << 30)); }
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned m0 = 0u, m1 = 0u;
            for (int w = 0; w < nw; ++w) { m0 = max(m0, red[w]); m1 = max(m1, red[32 + w]); }
            eref[0] = (int)m0 - (1 << 30);
            eref[1] = (int)m1 - (1 << 30);
        }
        __syncthreads();
    }
    const bool mom = (px | py | pz) != 0;
    for (int64_t x = x0; x < x1; ++x) {
        __syncthreads();
        int eU, eD;
        stage_site_df(U, D, slice * V3 + x, q, red, eU, eD);
        if (mom && threadIdx.x == 0) {
            const int64_t cx = x % L, cy = (x / L) % L, cz = x / ((int64_t)L * L);
            int64_t k = ((int64_t)px * cx + (int64_t)py * cy + (int64_t)pz * cz) % L;
            if (k < 0) k += L;
            double sn, cs;
            sincospi(-2.0 * (double)k / (double)L, &sn, &cs);
            ph_s.re = df_from_double(cs);
            ph_s.im = df_from_double(sn);
        }
        __syncthreads();
        diquarks_df(b.n_types, ty, q, dq);
        __syncthreads();
        const float sc0 = pow2f_le0(2 * eU + eD - eref[0]), sc1 = pow2f_le0(2 * eD + eU - eref[1]);
        const cdf ph = ph_s;
        for (int f = threadIdx.x; f < nf; f += blockDim.x) {
            const uint32_t code = entry_code(b, f0 + f);
            cdf v = block_entry_df(ty, code, q, dq);
            if (mom) v = MIXED::mul(v, ph);
            const float sc = ty[code >> 16].q1 ? sc1 : sc0;
            v.re.hi *= sc; v.re.lo *= sc; v.im.hi *= sc; v.im.lo *= sc;
            acc[f] = MIXED::vadd(acc[f], v);
        }
    }
    cd* o = part + (slice * tiles + tile) * (int64_t)b.n_f + f0;
    const double s0 = pow2d(max(min(eref[0], 1000), -1000)), s1 = pow2d(max(min(eref[1], 1000), -1000));
    for (int f = threadIdx.x; f < nf; f += blockDim.x) {
        const cdf v = acc[f];
        const double sc = ty[entry_code(b, f0 + f) >> 16].q1 ? s1 : s0;
        o[f] = cd_make(df_to_double(v.re) * sc, df_to_double(v.im) * sc);
    }
}

// F[slice][f] = sum over tiles in order (compensated)
__global__ void block_tile_reduce_kernel(const cd* __restrict__ part, int64_t n_slices, int tiles, int n_f,
                                         cd* __restrict__ F) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_slices * n_f) return;
    const int64_t slice = i / n_f, f = i % n_f;
    kacc re = {0.0, 0.0}, im = {0.0, 0.0};
    for (int t = 0; t < tiles; ++t) {
        const cd v = part[(slice * tiles + t) * n_f + f];
        kacc_add(re, v.re);
        kacc_add(im, v.im);
    }
    F[i] = cd_make(re.hi + re.lo, im.hi + im.lo);
}

// unit = (chunk, slice), chunk-major so that the blocks working on one chunk of the tree
// run together and share its arrays in L2
template <bool SMEM>
__global__ void __launch_bounds__(kTreeThreads) block_tree_kernel(BlockTreeDev t, const cd* __restrict__ F,
                                                                   int64_t n_slices, d4* __restrict__ part) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[4 * (kTreeThreads / 32)];
    const int64_t chunk = blockIdx.x / n_slices, slice = blockIdx.x % n_slices;
    const cd* Fs = F + slice * t.n_f;
    if (SMEM) {
        cd* fs = reinterpret_cast<cd*>(smem_raw);
        for (int i = threadIdx.x; i < t.n_f; i += blockDim.x) fs[i] = Fs[i];
        __syncthreads();
        Fs = fs;
    }
    const int np = t.A - 1;
    kacc re = {0.0, 0.0}, im = {0.0, 0.0};
    // units are added in groups of four in plain double, each group's sum compensated
    cd grp = cd_make(0.0, 0.0);
    int in_grp = 0;
    for (int64_t u = t.chunk_unit[chunk] + threadIdx.x; u < t.chunk_unit[chunk + 1]; u += blockDim.x) {
        cd pre = cd_make(1.0, 0.0);
        for (int k = 0; k < np; ++k) pre = cmul(pre, Fs[__ldg(t.unit_pre + u * np + k)]);
        cd s = cd_make(0.0, 0.0);
        const int32_t l1 = __ldg(t.unit_leaf + u + 1);
        for (int32_t l = __ldg(t.unit_leaf + u); l < l1; ++l) {
            const double2 w = __ldg(t.leaf_wd + l);
            cfma(s, cd_make(w.x, w.y), Fs[__ldg(t.leaf_f + l)]);
        }
        cfma(grp, pre, s);
        if (++in_grp == 4) {
            kacc_add(re, grp.re);
            kacc_add(im, grp.im);
            grp = cd_make(0.0, 0.0);
            in_grp = 0;
        }
    }
    kacc_add(re, grp.re);
    kacc_add(im, grp.im);
    kacc ore, oim;
    block_sum(cd_make(re.hi + re.lo, im.hi + im.lo), ore, oim, red);
    if (threadIdx.x == 0) part[slice * t.n_chunks + chunk] = make_d4(ore.hi, ore.lo, oim.hi, oim.lo);
}

// The same walk in double-float arithmetic: the slice's projected blocks are scaled by an
// exact power of two 2^-e (e from the largest |re|, |im| among them) into (hi, lo) float
// pairs in shared memory; a term of A factors then carries 2^(A e), restored in double
// on the block's partial sum.
__global__ void __launch_bounds__(kTreeThreads) block_tree_df_kernel(BlockTreeDev t, const cd* __restrict__ F,
                                                                      int64_t n_slices, d4* __restrict__ part) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[4 * (kTreeThreads / 32)];
    __shared__ unsigned redu[64];
    const int64_t chunk = blockIdx.x / n_slices, slice = blockIdx.x % n_slices;
    const cd* Fg = F + slice * t.n_f;
    cdf* fs = reinterpret_cast<cdf*>(smem_raw);
    unsigned m = 0u, m2 = 0u;
    for (int i = threadIdx.x; i < t.n_f; i += blockDim.x) {
        const cd v = Fg[i];
        m = max(m, max(abs_hiword(v.re), abs_hiword(v.im)));
    }
    block_max_u2(m, m2, redu);
    const int e = exponent_of(m);
    const double sc = pow2d(-max(min(e, 1000), -1000));
    for (int i = threadIdx.x; i < t.n_f; i += blockDim.x) {
        const cd v = Fg[i];
        cdf z;
        z.re = df_from_double(v.re * sc);
        z.im = df_from_double(v.im * sc);
        fs[i] = z;
    }
    __syncthreads();
    const int np = t.A - 1;
    MIXED::A tot;
    MIXED::acc_zero(tot);
    for (int64_t u = t.chunk_unit[chunk] + threadIdx.x; u < t.chunk_unit[chunk + 1]; u += blockDim.x) {
        cdf pre = MIXED::one();
        for (int k = 0; k < np; ++k) pre = MIXED::mul(pre, fs[__ldg(t.unit_pre + u * np + k)]);
        MIXED::A a;
        MIXED::acc_zero(a);
        const int32_t l1 = __ldg(t.unit_leaf + u + 1);
        for (int32_t l = __ldg(t.unit_leaf + u); l < l1; ++l) {
            const float2 w = __ldg(t.leaf_w + l);
            const cdf f = fs[__ldg(t.leaf_f + l)];
            // (w.x + i w.y) f with float weights (exact products by error-free transformation)
            dacc_fma_f(a.r0, w.x, f.re);
            dacc_fma_f(a.r1, -w.y, f.im);
            dacc_fma_f(a.i0, w.x, f.im);
            dacc_fma_f(a.i1, w.y, f.re);
        }
        MIXED::add(tot, MIXED::mul(pre, MIXED::get(a)));
    }
    const cd v = MIXED::to_cd(MIXED::get(tot));
    kacc ore, oim;
    block_sum(v, ore, oim, red);
    if (threadIdx.x == 0) {
        const double back = pow2d(max(min(t.A * e, 1000), -1000));
        part[slice * t.n_chunks + chunk] = make_d4(ore.hi * back, ore.lo * back, oim.hi * back, oim.lo * back);
    }
}

// The block form of the local-sink correlator (every baryon at the same sink site x):
//     C_x = sum_k w_k prod_i f^{h_ik}(x; eta_ik),
// which is the quark-level correlator of the same operator.  One block per site at a
// time: the site's block entries are built in shared memory (diquark tables, then the
// entries the plan uses), and the whole block factor tree is walked over them; the
// site's compensated sum goes to its partial.  Complex double.
__global__ void __launch_bounds__(kThreads) block_local_kernel(BlockDev b, BlockTreeDev t,
                                                                const double* __restrict__ U,
                                                                const double* __restrict__ D, int64_t n_sites,
                                                                d4* __restrict__ part) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ BlockTypeDev ty[6];
    __shared__ double red[4 * (kThreads / 32)];
    cd* q = reinterpret_cast<cd*>(smem_raw);
    cd* dq = q + 2 * kQ;
    cd* fs = dq + b.n_types * kDq;
    load_types(b, ty);
    const int np = t.A - 1;
    for (int64_t site = blockIdx.x; site < n_sites; site += gridDim.x) {
        __syncthreads();
        stage_site(U, D, site, q);
        __syncthreads();
        diquarks(b.n_types, ty, q, dq);
        __syncthreads();
        for (int f = threadIdx.x; f < b.n_f; f += blockDim.x) fs[f] = block_entry(ty, entry_code(b, f), q, dq);
        __syncthreads();
        kacc re = {0.0, 0.0}, im = {0.0, 0.0};
        cd grp = cd_make(0.0, 0.0);
        int in_grp = 0;
        for (int64_t u = threadIdx.x; u < t.n_units; u += blockDim.x) {
            cd pre = cd_make(1.0, 0.0);
            for (int k = 0; k < np; ++k) pre = cmul(pre, fs[__ldg(t.unit_pre + u * np + k)]);
            cd s = cd_make(0.0, 0.0);
            const int32_t l1 = __ldg(t.unit_leaf + u + 1);
            for (int32_t l = __ldg(t.unit_leaf + u); l < l1; ++l) {
                const double2 w = __ldg(t.leaf_wd + l);
                cfma(s, cd_make(w.x, w.y), fs[__ldg(t.leaf_f + l)]);
            }
            cfma(grp, pre, s);
            if (++in_grp == 4) {
                kacc_add(re, grp.re);
                kacc_add(im, grp.im);
                grp = cd_make(0.0, 0.0);
                in_grp = 0;
            }
        }
        kacc_add(re, grp.re);
        kacc_add(im, grp.im);
        kacc ore, oim;
        block_sum(cd_make(re.hi + re.lo, im.hi + im.lo), ore, oim, red);
        if (threadIdx.x == 0) part[site] = make_d4(ore.hi, ore.lo, oim.hi, oim.lo);
    }
}

}  // namespace

int block_entries_per_cta(int n_types) { return (int)(kSmemBudget / 16) - 2 * kQ - n_types * kDq; }

size_t block_kernel_smem(int n_f, int n_types, bool projected) {
    return (size_t)(2 * kQ + n_types * kDq + (projected ? n_f : 0)) * 16;
}

namespace {
void project_shape(int n_f, int n_types, int64_t n_slices, int64_t V3, int sms, int& f_chunk, int& n_fc, int& tiles) {
    const int per_cta = block_entries_per_cta(n_types);
    n_fc = (n_f + per_cta - 1) / per_cta;
    f_chunk = (n_f + n_fc - 1) / n_fc;
    // at least four waves of one resident block per SM, tiles of at least 32 sites, and
    // among up to four times that many tiles the count whose last wave is fullest
    const int64_t base = n_slices * n_fc;
    const int64_t lo = (4LL * std::max(sms, 1) + base - 1) / base, cap = std::max<int64_t>(1, V3 / 32);
    tiles = (int)std::max<int64_t>(1, std::min(lo, cap));
    double best = 0.0;
    for (int64_t t = std::min(lo, cap); t <= std::min(4 * lo, cap); ++t) {
        const int64_t u = base * t;
        const double eff = (double)u / (double)(((u + sms - 1) / sms) * sms);
        if (eff > best + 1e-9) { best = eff; tiles = (int)t; }
        if (eff >= 0.999) break;
    }
}
}  // namespace

int64_t block_project_scratch(int n_f, int n_types, int64_t n_slices, int64_t V3, int sms) {
    int f_chunk, n_fc, tiles;
    project_shape(n_f, n_types, n_slices, V3, sms, f_chunk, n_fc, tiles);
    return n_slices * tiles * (int64_t)n_f;
}

cudaError_t launch_blocks_site(const BlockDev& b, const double* U, const double* D, int64_t n_sites, cd* out,
                               int sms, cudaStream_t s, int64_t* launches) {
    if (n_sites <= 0 || b.n_f <= 0) return cudaSuccess;
    const size_t smem = block_kernel_smem(b.n_f, b.n_types, false);
    const int64_t grid = std::min<int64_t>(n_sites, 4LL * sms);
    block_site_kernel<<<(unsigned)grid, kThreads, smem, s>>>(b, U, D, n_sites, out);
    ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_blocks_projected(const BlockDev& b, int prec, const double* U, const double* D, int64_t n_slices,
                                    int64_t V3, int L, const int* p, cd* part, cd* F, int sms, cudaStream_t s,
                                    int64_t* launches) {
    if (n_slices <= 0 || b.n_f <= 0) return cudaSuccess;
    if (V3 <= 0) return cudaMemsetAsync(F, 0, sizeof(cd) * (size_t)n_slices * b.n_f, s);
    int f_chunk, n_fc, tiles;
    project_shape(b.n_f, b.n_types, n_slices, V3, sms, f_chunk, n_fc, tiles);
    const size_t smem = block_kernel_smem(f_chunk, b.n_types, true);
    const int64_t units = n_slices * tiles * n_fc;
    const int px = p ? p[0] : 0, py = p ? p[1] : 0, pz = p ? p[2] : 0;
    if (prec == 0) {
        cudaError_t e = cudaFuncSetAttribute(block_project_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        block_project_kernel<<<(unsigned)units, kThreads, smem, s>>>(b, U, D, V3, L, px, py, pz, tiles, f_chunk, n_fc,
                                                                     part);
    } else {
        cudaError_t e = cudaFuncSetAttribute(block_project_df_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        block_project_df_kernel<<<(unsigned)units, kThreads, smem, s>>>(b, U, D, V3, L, px, py, pz, tiles, f_chunk,
                                                                        n_fc, part);
    }
    ++*launches;
    const int64_t n = n_slices * b.n_f;
    block_tile_reduce_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(part, n_slices, tiles, b.n_f, F);
    ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_block_tree(const BlockTreeDev& t, int prec, const cd* F, int64_t n_slices, d4* part,
                              cudaStream_t s, int64_t* launches) {
    if (n_slices <= 0 || t.n_chunks <= 0) return cudaSuccess;
    const size_t smem = (size_t)t.n_f * 16;
    const int64_t grid = (int64_t)t.n_chunks * n_slices;
    if (prec == 1 && smem <= kSmemBudget) {
        cudaError_t e = cudaFuncSetAttribute(block_tree_df_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        block_tree_df_kernel<<<(unsigned)grid, kTreeThreads, smem, s>>>(t, F, n_slices, part);
    } else if (smem <= kSmemBudget) {
        cudaError_t e = cudaFuncSetAttribute(block_tree_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        block_tree_kernel<true><<<(unsigned)grid, kTreeThreads, smem, s>>>(t, F, n_slices, part);
    } else {
        block_tree_kernel<false><<<(unsigned)grid, kTreeThreads, 0, s>>>(t, F, n_slices, part);
    }
    ++*launches;
    return cudaGetLastError();
}

}  // namespace mbc

namespace mbc {

cudaError_t launch_block_local(const BlockDev& b, const BlockTreeDev& t, const double* U, const double* D,
                               int64_t n_sites, d4* part, int sms, cudaStream_t s, int64_t* launches) {
    if (n_sites <= 0) return cudaSuccess;
    const size_t smem = block_kernel_smem(b.n_f, b.n_types, true);
    if (smem > kSmemBudget) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(block_local_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int per_sm = std::max(1, (int)((227 * 1024) / (smem + 2 * 1024)));
    const int64_t grid = std::min<int64_t>(n_sites, (int64_t)sms * std::min(per_sm, 2048 / kThreads));
    block_local_kernel<<<(unsigned)grid, kThreads, smem, s>>>(b, t, U, D, n_sites, part);
    ++*launches;
    return cudaGetLastError();
}

}  // namespace mbc
