// input_check.cu -- the device scan of checked mode (rt_options.check_inputs): finds
// non-finite emissivities, negative or non-finite opacities, unusable source coordinates and a
// non-finite loss gradient before a call runs.
#include <cuda_runtime.h>

#include "rt_internal.h"

namespace rt {

namespace {

unsigned check_grid(long long n) {
    long long g = (n + 255) / 256;
    if (g > 152LL * 16) g = 152LL * 16;   // grid-stride beyond 16 blocks per SM
    return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace

// Checked mode: flags[0] |= 1 if some j is not finite, flags[1] |= 1 if some kappa is not
// finite or negative, flags[2] |= 1 if some source coordinate is not finite or |x| >= 2^24,
// flags[3] |= 1 if some value of `extra` (the loss gradient of an adjoint call) is not finite.
__global__ void k_check_inputs(const float* __restrict__ j, const float* __restrict__ kappa, long long n,
                               const float* __restrict__ src, int nsrc, const float* __restrict__ extra,
                               int* __restrict__ flags) {
    int bad_j = 0, bad_k = 0, bad_s = 0, bad_x = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float a = __ldg(j + i), b = __ldg(kappa + i);
        bad_j |= !isfinite(a);
        bad_k |= !isfinite(b) || b < 0.0f;
        if (extra) bad_x |= !isfinite(__ldg(extra + i));
    }
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < 3LL * nsrc;
         i += (long long)gridDim.x * blockDim.x) {
        const float s = __ldg(src + i);
        bad_s |= !isfinite(s) || fabsf(s) >= 16777216.0f;
    }
    bad_j = __any_sync(0xffffffffu, bad_j);
    bad_k = __any_sync(0xffffffffu, bad_k);
    bad_s = __any_sync(0xffffffffu, bad_s);
    bad_x = __any_sync(0xffffffffu, bad_x);
    if ((threadIdx.x & 31) == 0) {
        if (bad_j) atomicOr(flags + 0, 1);
        if (bad_k) atomicOr(flags + 1, 1);
        if (bad_s) atomicOr(flags + 2, 1);
        if (bad_x) atomicOr(flags + 3, 1);
    }
}

// Content hash of a march's inputs, for checkpoint reuse: *out = sum over elements of a mixed
// 64-bit word (the SplitMix64 finaliser of Steele, Lea and Flood, 2014) of each (j, kappa) bit
// pair and each source coordinate, salted with its index. The sum is order-independent, so any
// launch shape gives the same value; changing any element changes it except with probability
// about 2^-64.
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

__global__ void k_input_hash(const float* __restrict__ j, const float* __restrict__ kappa, long long n,
                             const float* __restrict__ src, int nsrc, unsigned long long* __restrict__ out) {
    constexpr unsigned long long kGolden = 0x9e3779b97f4a7c15ULL;
    unsigned long long h = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const unsigned long long w = ((unsigned long long)__float_as_uint(__ldg(kappa + i)) << 32) |
                                     __float_as_uint(__ldg(j + i));
        h += mix64(w + (unsigned long long)(i + 1) * kGolden);
    }
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < 3LL * nsrc;
         i += (long long)gridDim.x * blockDim.x)
        h += mix64(((unsigned long long)__float_as_uint(__ldg(src + i)) | (1ULL << 40)) +
                   (unsigned long long)(n + i + 1) * kGolden);
    for (int o = 16; o > 0; o >>= 1) h += __shfl_xor_sync(0xffffffffu, h, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, h);
}

cudaError_t launch_input_hash(const float* j, const float* kappa, long long n, const float* src, int nsrc,
                              unsigned long long* out, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    k_input_hash<<<check_grid(n), 256, 0, st>>>(j, kappa, n, src, nsrc, out);
    return cudaGetLastError();
}

cudaError_t launch_check_inputs(const float* j, const float* kappa, long long n, const float* src, int nsrc,
                                const float* extra, int* flags, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(flags, 0, 4 * sizeof(int), st);
    if (e != cudaSuccess) return e;
    k_check_inputs<<<check_grid(n), 256, 0, st>>>(j, kappa, n, src, nsrc, extra, flags);
    return cudaGetLastError();
}

}  // namespace rt
