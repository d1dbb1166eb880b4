// gen.cu - the seeded synthetic propagator recipe of mbc_inputs (see __init__.py) on the
// GPU, for workloads too large to generate on the host (the batched workload holds about
// 117 GB of fields).  Input generation only: no correlator arithmetic lives here.
//
// Entry (s, t, x, i, j) of flavour f is exp(-kappa t) G (or exp(-kappa t) (B_t + eps G)
// with the shared base B_t of site 2^40), G complex standard normal from outputs 2n+1
// and 2n+2 (n = x * 144 + 12 i + j) of the SplitMix64 sequence started at
//   stream = mix(mix(mix(seed + golden) ^ set) ^ (flavour << 32 | t)),
// u1 = ((z1 >> 11) + 1) 2^-53, u2 = (z2 >> 11) 2^-53, G = sqrt(-ln u1) e^{2 pi i u2}
// (Box-Muller).  SplitMix64 is the generator of Steele, Lea and Flood (OOPSLA 2014).
// The transcendental functions are CUDA's, so an entry can differ from the host recipe
// in the last bits; consumers compare results within their tolerances.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

constexpr uint64_t kGolden = 0x9E3779B97F4A7C15ull;

__host__ __device__ __forceinline__ uint64_t mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ double2 gaussian(uint64_t stream, uint64_t n) {
    const uint64_t k1 = 2 * n + 1;
    const uint64_t z1 = mix(stream + k1 * kGolden);
    const uint64_t z2 = mix(stream + (k1 + 1) * kGolden);
    const double u1 = ((double)(z1 >> 11) + 1.0) * 0x1p-53;
    const double u2 = (double)(z2 >> 11) * 0x1p-53;
    const double r = sqrt(-log(u1));
    double sn, cs;
    sincos(2.0 * 3.141592653589793 * u2, &sn, &cs);
    return make_double2(r * cs, r * sn);
}

// out [n_t][V3][144] complex double for the time slices t_list[0..n_t)
__global__ void fill_kernel(double2* __restrict__ out, const uint64_t* __restrict__ streams,
                            const int* __restrict__ ts, int n_t, int64_t V3, double kappa, double noise) {
    const int64_t per_t = V3 * 144;
    const int64_t total = per_t * n_t;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(q / per_t);
        const int64_t n = q - (int64_t)k * per_t;             // x * 144 + e
        const uint64_t st = streams[k];
        double2 g = gaussian(st, (uint64_t)n);
        if (noise >= 0.0) {
            const double2 b = gaussian(st, (uint64_t)(1ull << 40) * 144ull + (uint64_t)(n % 144));
            g = make_double2(b.x + noise * g.x, b.y + noise * g.y);
        }
        const double f = exp(-kappa * (double)ts[k]);
        out[q] = make_double2(f * g.x, f * g.y);
    }
}

}  // namespace

extern "C" {

// Fill out (device, complex double [n_t][V3][12][12]) with the fields of time slices
// ts[0..n_t) (host array) of one (seed, set, flavour); noise < 0 means plain fields.
// Returns a cudaError_t value (0 on success); asynchronous on the stream.
int mbcgen_fill(void* out, uint64_t seed, uint64_t set_index, int flavour, const int* ts, int n_t, int64_t V3,
                double kappa, double noise, void* stream) {
    if (n_t <= 0 || V3 <= 0) return 0;
    if (!out || !ts) return (int)cudaErrorInvalidValue;
    cudaStream_t s = (cudaStream_t)stream;
    uint64_t* d_st = nullptr;
    int* d_t = nullptr;
    cudaError_t e = cudaMallocAsync(&d_st, sizeof(uint64_t) * n_t, s);
    if (e == cudaSuccess) e = cudaMallocAsync(&d_t, sizeof(int) * n_t, s);
    if (e != cudaSuccess) return (int)e;
    uint64_t* h_st = new uint64_t[n_t];
    for (int k = 0; k < n_t; ++k) {
        uint64_t h = mix(seed + kGolden);
        h = mix(h ^ set_index);
        h = mix(h ^ (((uint64_t)flavour << 32) | (uint64_t)(uint32_t)ts[k]));
        h_st[k] = h;
    }
    e = cudaMemcpyAsync(d_st, h_st, sizeof(uint64_t) * n_t, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_t, ts, sizeof(int) * n_t, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        fill_kernel<<<152 * 8, 256, 0, s>>>((double2*)out, d_st, d_t, n_t, V3, kappa, noise);
        e = cudaGetLastError();
    }
    cudaStreamSynchronize(s);
    delete[] h_st;
    cudaFreeAsync(d_st, s);
    cudaFreeAsync(d_t, s);
    cudaStreamSynchronize(s);
    return (int)e;
}

}  // extern "C"
