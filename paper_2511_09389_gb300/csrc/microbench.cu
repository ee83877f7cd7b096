// microbench.cu -- peaks of the memory operations the march is made of, measured on the GPU it
// runs on: L2 reductions (`red.global.add`) and read-only gathers on an L2-resident array, with
// random, warp-coherent and 8-corner-stencil addresses, 4 or 16 bytes per operation. The march's
// roofline fractions are reported against these (the paper has no counterpart).
//
// Addresses come from a per-thread linear congruential generator (the Numerical Recipes
// constants 1664525, 1013904223) mapped onto [0, n) by a 32 x 32 -> 64-bit multiply, so every
// access is in bounds by construction.
#include <cuda_runtime.h>
#include <stdint.h>

#include "march_common.cuh"
#include "rt_internal.h"

namespace rt {

// The march's attenuation factor exp(-x) (neg_exp), element by element, so its accuracy can be
// checked against a reference exponential.
__global__ void k_neg_exp(const float* __restrict__ x, float* __restrict__ y, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = neg_exp(x[i]);
}

namespace {

__device__ __forceinline__ uint32_t lcg(uint32_t& s) {
    s = s * 1664525u + 1013904223u;
    return s;
}

__device__ __forceinline__ uint32_t below(uint32_t r, uint32_t n) {
    return (uint32_t)(((uint64_t)r * n) >> 32);
}

template <int V>
__device__ __forceinline__ void red_v(float* p, float a) {
    if (V == 4) {
        asm volatile("red.global.add.v4.f32 [%0], {%1, %1, %1, %1};" ::"l"(p), "f"(a) : "memory");
    } else {
        asm volatile("red.global.add.f32 [%0], %1;" ::"l"(p), "f"(a) : "memory");
    }
}

template <int V>
__device__ __forceinline__ float ld_v(const float* p) {
    if (V == 4) {
        const float4 q = __ldg(reinterpret_cast<const float4*>(p));
        return (q.x + q.y) + (q.z + q.w);
    }
    return __ldg(p);
}

// kind 0: each thread reduces into uniformly random V-vectors of the array
template <int V>
__global__ void k_red_random(float* buf, uint32_t nvec, int iters) {
    uint32_t s = 0x9e3779b9u ^ (blockIdx.x * blockDim.x + threadIdx.x);
    for (int i = 0; i < iters; ++i) red_v<V>(buf + (size_t)below(lcg(s), nvec) * V, 1.0f);
}

// kind 1: a warp reduces into 32 consecutive V-vectors at a random warp-aligned position
template <int V>
__global__ void k_red_coherent(float* buf, uint32_t nvec, int iters) {
    const int lane = threadIdx.x & 31;
    uint32_t s = 0x9e3779b9u ^ ((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const uint32_t nwarp = nvec / 32;
    for (int i = 0; i < iters; ++i)
        red_v<V>(buf + ((size_t)below(lcg(s), nwarp) * 32 + lane) * V, 1.0f);
}

// kind 2: each thread reduces into the 8 corners of a random cell of an edge^3 grid of
// V-vectors (cell-major, the march's packed accumulator layout)
template <int V>
__global__ void k_red_stencil(float* buf, int edge, int iters) {
    uint32_t s = 0x9e3779b9u ^ (blockIdx.x * blockDim.x + threadIdx.x);
    const uint32_t m = (uint32_t)(edge - 1);
    for (int i = 0; i < iters; ++i) {
        const uint32_t x = below(lcg(s), m), y = below(lcg(s), m), z = below(lcg(s), m);
        const size_t c = ((size_t)x * edge + y) * edge + z;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const size_t cell = c + (size_t)((k >> 2) & 1) * edge * edge + (size_t)((k >> 1) & 1) * edge + (k & 1);
            red_v<V>(buf + cell * V, 0.125f);
        }
    }
}

// kind 3: each thread loads uniformly random V-vectors
template <int V>
__global__ void k_gather_random(float* buf, uint32_t nvec, int iters) {
    uint32_t s = 0x9e3779b9u ^ (blockIdx.x * blockDim.x + threadIdx.x);
    float acc = 0.0f;
    for (int i = 0; i < iters; ++i) acc += ld_v<V>(buf + (size_t)below(lcg(s), nvec) * V);
    if (acc == -1.0f) buf[0] = acc;   // keeps the loads; the array holds no such sum
}

// kind 4: each thread loads the 8 corners of a random cell of an edge^3 grid of V-vectors
template <int V>
__global__ void k_gather_stencil(float* buf, int edge, int iters) {
    uint32_t s = 0x9e3779b9u ^ (blockIdx.x * blockDim.x + threadIdx.x);
    const uint32_t m = (uint32_t)(edge - 1);
    float acc = 0.0f;
    for (int i = 0; i < iters; ++i) {
        const uint32_t x = below(lcg(s), m), y = below(lcg(s), m), z = below(lcg(s), m);
        const size_t c = ((size_t)x * edge + y) * edge + z;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const size_t cell = c + (size_t)((k >> 2) & 1) * edge * edge + (size_t)((k >> 1) & 1) * edge + (k & 1);
            acc += ld_v<V>(buf + cell * V);
        }
    }
    if (acc == -1.0f) buf[0] = acc;
}

// kinds 5 / 6: the 8-corner stencil of kind 2 with 64-bit reductions, red.global.add.u64 (the
// fixed-point deposit) or red.global.add.f64, into an edge^3 grid of 8-byte cells
template <bool F64>
__global__ void k_red_stencil64(unsigned long long* buf, int edge, int iters) {
    uint32_t s = 0x9e3779b9u ^ (blockIdx.x * blockDim.x + threadIdx.x);
    const uint32_t m = (uint32_t)(edge - 1);
    for (int i = 0; i < iters; ++i) {
        const uint32_t x = below(lcg(s), m), y = below(lcg(s), m), z = below(lcg(s), m);
        const size_t c = ((size_t)x * edge + y) * edge + z;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const size_t cell = c + (size_t)((k >> 2) & 1) * edge * edge + (size_t)((k >> 1) & 1) * edge + (k & 1);
            if (F64)
                asm volatile("red.global.add.f64 [%0], %1;" ::"l"(buf + cell), "d"(0.125) : "memory");
            else
                asm volatile("red.global.add.u64 [%0], %1;" ::"l"(buf + cell), "l"(1ull) : "memory");
        }
    }
}

template <int V>
cudaError_t launch_kind(int kind, float* buf, uint32_t nvec, int edge, int iters, int grid, int block,
                        cudaStream_t st) {
    switch (kind) {
        case 0: k_red_random<V><<<grid, block, 0, st>>>(buf, nvec, iters); break;
        case 1: k_red_coherent<V><<<grid, block, 0, st>>>(buf, nvec, iters); break;
        case 2: k_red_stencil<V><<<grid, block, 0, st>>>(buf, edge, iters); break;
        case 3: k_gather_random<V><<<grid, block, 0, st>>>(buf, nvec, iters); break;
        case 4: k_gather_stencil<V><<<grid, block, 0, st>>>(buf, edge, iters); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_microbench(int kind, int vec, float* buf, long long nvec, int edge, int iters, int grid,
                              int block, cudaStream_t st) {
    if (nvec < 32 || nvec > 0xffffffffLL) return cudaErrorInvalidValue;
    if (kind == 5 || kind == 6) {
        if (kind == 5) k_red_stencil64<false><<<grid, block, 0, st>>>((unsigned long long*)buf, edge, iters);
        else k_red_stencil64<true><<<grid, block, 0, st>>>((unsigned long long*)buf, edge, iters);
        return cudaGetLastError();
    }
    return vec == 4 ? launch_kind<4>(kind, buf, (uint32_t)nvec, edge, iters, grid, block, st)
                    : launch_kind<1>(kind, buf, (uint32_t)nvec, edge, iters, grid, block, st);
}

}  // namespace rt

extern "C" rt_status rt_microbench(int kind, int vec, void* buf, long long buf_bytes, int edge, int iters, float* ms,
                                   double* ops) {
    if (kind < 0 || kind > 6 || (vec != 1 && vec != 4) || (kind >= 5 && vec != 1) || !buf || !ms || !ops ||
        iters < 1 || iters > (1 << 20))
        return rt::set_error(RT_ERR_INVALID_ARG,
                             "rt_microbench: need kind 0-6, vec 1 or 4 (1 for kinds 5, 6), 1 <= iters <= 2^20");
    const long long nvec = buf_bytes / (kind >= 5 ? 8LL : 4LL * vec);
    const bool stencil = kind == 2 || kind == 4 || kind >= 5;
    if (stencil) {
        if (edge < 2 || edge > 2048 || (long long)edge * edge * edge > nvec)
            return rt::set_error(RT_ERR_INVALID_ARG, "rt_microbench: edge^3 vectors must fit in the buffer");
    } else if (nvec < 32 || nvec > 0xffffffffLL) {
        return rt::set_error(RT_ERR_INVALID_ARG, "rt_microbench: the buffer must hold 32 .. 2^32-1 vectors");
    }
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = 8 * (sms > 0 ? sms : 1), block = 256;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return rt::set_error(RT_ERR_CUDA, "rt_microbench: cudaEventCreate");
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return rt::set_error(RT_ERR_CUDA, "rt_microbench: cudaEventCreate");
    }
    cudaError_t e = cudaEventRecord(e0, 0);
    if (e == cudaSuccess) e = rt::launch_microbench(kind, vec, (float*)buf, nvec, edge, iters, grid, block, 0);
    if (e == cudaSuccess) e = cudaEventRecord(e1, 0);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return rt::set_error(RT_ERR_CUDA, cudaGetErrorString(e));
    *ops = (double)grid * block * iters * (stencil ? 8.0 : 1.0);
    return RT_OK;
}

extern "C" rt_status rt_neg_exp(const float* x, float* y, long long n, void* stream) {
    if (n < 0 || (n > 0 && (!x || !y))) return rt::set_error(RT_ERR_INVALID_ARG, "rt_neg_exp: need n >= 0 and device x, y");
    if (n == 0) return RT_OK;
    const long long blocks = (n + 255) / 256;
    rt::k_neg_exp<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, (cudaStream_t)stream>>>(x, y, n);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? RT_OK : rt::set_error(RT_ERR_CUDA, cudaGetErrorString(e));
}
