// surrogate_ops.cu -- element-wise and reduction kernels of the convolutional surrogate.
//
// Layout changes between plain FP32 NCDHW tensors and the C32 bf16 layout of the tensor-core
// convolution ([B][D][H][W][32]), weight packing ([C_out][C_in][27] FP32 -> [27][32][32] bf16,
// also flipped and transposed for the data gradient), per-channel sums (bias gradient, channel
// means), the surrogate's input features and loss, and an Adam step.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "rt_internal.h"

namespace rt {

namespace {

unsigned grid1d(long long n, int block) {
    long long g = (n + block - 1) / block;
    if (g > 152LL * 32) g = 152LL * 32;
    return (unsigned)(g < 1 ? 1 : g);
}

// One thread per (sample, 8-channel quarter, voxel), voxel fastest: coalesced FP32 reads.
__global__ void k_to_c32(const float* __restrict__ src, int C, long long vox, int B, __nv_bfloat16* __restrict__ dst) {
    const long long total = (long long)B * 4 * vox;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long b = i / (4 * vox), r = i - b * 4 * vox;
        const int q = (int)(r / vox);
        const long long v = r - (long long)q * vox;
        __align__(16) __nv_bfloat16 o[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int c = q * 8 + e;
            o[e] = __float2bfloat16_rn(c < C ? __ldg(src + ((long long)b * C + c) * vox + v) : 0.0f);
        }
        reinterpret_cast<uint4*>(dst)[((long long)b * vox + v) * 4 + q] = *reinterpret_cast<uint4*>(o);
    }
}

__global__ void k_from_c32(const __nv_bfloat16* __restrict__ src, int C, long long vox, int B,
                           float* __restrict__ dst) {
    const long long total = (long long)B * C * vox;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long b = i / (C * vox), r = i - b * C * vox;
        const int c = (int)(r / vox);
        const long long v = r - (long long)c * vox;
        dst[i] = __bfloat162float(src[((long long)b * vox + v) * 32 + c]);
    }
}

// packed[tap][n][k]: forward (transpose = 0): w[n][k][tap];
// data gradient (transpose = 1): w[k][n][26 - tap] (input = the forward's outputs).
__global__ void k_pack_weights(const float* __restrict__ w, int c_in, int c_out, int transpose,
                               __nv_bfloat16* __restrict__ packed) {
    const int total = 27 * 32 * 32;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const int k = i & 31, n = (i >> 5) & 31, tap = i >> 10;
        float v = 0.0f;
        if (!transpose) {
            if (n < c_out && k < c_in) v = w[((long long)n * c_in + k) * 27 + tap];
        } else {
            // the transposed convolution maps c_out (its input, index k) to c_in (its output, index n)
            if (k < c_out && n < c_in) v = w[((long long)k * c_in + n) * 27 + (26 - tap)];
        }
        packed[i] = __float2bfloat16_rn(v);
    }
}

// out[b * per_sample][c] += scale * sum over voxels of channel c (c < C) of a C32 tensor. Thread t
// owns channel quarter t & 3 of voxels t >> 2, t >> 2 + blockDim / 4, ... (coalesced 16-byte
// loads); lanes with the same quarter are then summed. Grid: (blocks, B).
__global__ void k_channel_sum(const __nv_bfloat16* __restrict__ x, long long vox, int C, float scale, int per_sample,
                              float* __restrict__ out) {
    const int b = blockIdx.y, q = threadIdx.x & 3;
    const uint4* p = reinterpret_cast<const uint4*>(x) + (long long)b * vox * 4;
    float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const long long step = (long long)gridDim.x * (blockDim.x >> 2);
    for (long long v = blockIdx.x * (long long)(blockDim.x >> 2) + (threadIdx.x >> 2); v < vox; v += step) {
        const uint4 u = __ldg(p + v * 4 + q);
        const __nv_bfloat16* e = reinterpret_cast<const __nv_bfloat16*>(&u);
#pragma unroll
        for (int i = 0; i < 8; ++i) acc[i] += __bfloat162float(e[i]);
    }
    __shared__ float red[32][33];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        float t = acc[i];
        for (int o = 16; o >= 4; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if ((threadIdx.x & 31) < 4) red[q * 8 + i][threadIdx.x >> 5] = t;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        float t = 0.0f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[threadIdx.x][w];
        if ((int)threadIdx.x < C) atomicAdd(out + (per_sample ? (long long)b * C : 0) + threadIdx.x, t * scale);
    }
}

// Surrogate inputs: channel 0 = log(kappa / 0.05), channel 1 = log(1 + j); C32, other channels 0.
__global__ void k_features(const float* __restrict__ kappa, const float* __restrict__ j, long long vox, int B,
                           __nv_bfloat16* __restrict__ x) {
    const long long total = (long long)B * vox;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long b = i / vox, v = i - b * vox;
        const float k = fmaxf(__ldg(kappa + i), 1e-30f);
        __align__(16) __nv_bfloat16 o[8];
        o[0] = __float2bfloat16_rn(logf(k * 20.0f));
        o[1] = __float2bfloat16_rn(log1pf(fmaxf(__ldg(j + i), 0.0f)));
#pragma unroll
        for (int e = 2; e < 8; ++e) o[e] = __float2bfloat16_rn(0.0f);
        uint4* X = reinterpret_cast<uint4*>(x) + (b * vox + v) * 4;
        X[0] = *reinterpret_cast<uint4*>(o);
        X[1] = X[2] = X[3] = make_uint4(0, 0, 0, 0);
    }
}

__device__ __forceinline__ float block_sum(float x, float* red) {
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = x;
    __syncthreads();
    float t = 0.0f;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    __syncthreads();
    return t;
}

// Per-sample maximum of a non-negative field (grid: blocks x B).
__global__ void k_field_max(const float* __restrict__ f, long long vox, float* __restrict__ out) {
    const int b = blockIdx.y;
    float m = 0.0f;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < vox; v += (long long)gridDim.x * blockDim.x)
        m = fmaxf(m, __ldg(f + (long long)b * vox + v));
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(reinterpret_cast<int*>(out + b), __float_as_int(m));
}

// Loss sum_{b,v} (pred - T)^2 / (B vox) with T = (log(F + eps_b) - mu) / sigma,
// eps_b = eps_rel * max_b F; its gradient 2 (pred - T) / (B vox) goes to channel 0 of a C32
// tensor (the other channels zero).
__global__ void k_log_loss(const float* __restrict__ pred, const float* __restrict__ field, long long vox, int B,
                           const float* __restrict__ fmax, float eps_rel, float mu, float inv_sigma,
                           __nv_bfloat16* __restrict__ grad, float* __restrict__ loss) {
    __shared__ float red[32];
    const long long total = (long long)B * vox;
    const float norm = 1.0f / (float)total;
    float acc = 0.0f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long b = i / vox, v = i - b * vox;
        const float eps = eps_rel * __ldg(fmax + b);
        const float T = (logf(__ldg(field + i) + eps) - mu) * inv_sigma;
        const float d = __ldg(pred + i) - T;
        acc += d * d;
        if (grad) {
            __align__(16) __nv_bfloat16 o[8];
            o[0] = __float2bfloat16_rn(2.0f * d * norm);
#pragma unroll
            for (int e = 1; e < 8; ++e) o[e] = __float2bfloat16_rn(0.0f);
            uint4* G = reinterpret_cast<uint4*>(grad) + (b * vox + v) * 4;
            G[0] = *reinterpret_cast<uint4*>(o);
            G[1] = G[2] = G[3] = make_uint4(0, 0, 0, 0);
        }
    }
    const float t = block_sum(acc, red);
    if (threadIdx.x == 0) atomicAdd(loss, t * norm);
}

// Per-sample sums for the relative L2 error of the predicted field F' = exp(pred sigma + mu) - eps:
// out[b] = (sum (F' - F)^2, sum F^2).
__global__ void k_field_error(const float* __restrict__ pred, const float* __restrict__ field, long long vox,
                              const float* __restrict__ fmax, float eps_rel, float mu, float sigma,
                              float* __restrict__ out) {
    __shared__ float red[32];
    const int b = blockIdx.y;
    const float eps = eps_rel * __ldg(fmax + b);
    float e2 = 0.0f, f2 = 0.0f;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < vox; v += (long long)gridDim.x * blockDim.x) {
        const long long i = (long long)b * vox + v;
        const float F = __ldg(field + i);
        const float Fp = expf(__ldg(pred + i) * sigma + mu) - eps;
        e2 += (Fp - F) * (Fp - F);
        f2 += F * F;
    }
    const float a = block_sum(e2, red);
    const float c = block_sum(f2, red);
    if (threadIdx.x == 0) { atomicAdd(out + 2 * b, a); atomicAdd(out + 2 * b + 1, c); }
}

// Adam (bias-corrected), FP32 master parameters.
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, long long n, float lr, float b1, float b2, float eps, float c1, float c2) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    }
}

}  // namespace

cudaError_t launch_features(const float* kappa, const float* j, int B, long long vox, void* x, cudaStream_t st) {
    k_features<<<grid1d((long long)B * vox, 256), 256, 0, st>>>(kappa, j, vox, B, reinterpret_cast<__nv_bfloat16*>(x));
    return cudaGetLastError();
}

cudaError_t launch_field_max(const float* f, int B, long long vox, float* out, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(float) * B, st);
    if (e != cudaSuccess) return e;
    k_field_max<<<dim3(64, B), 256, 0, st>>>(f, vox, out);
    return cudaGetLastError();
}

cudaError_t launch_log_loss(const float* pred, const float* field, int B, long long vox, const float* fmax,
                            float eps_rel, float mu, float sigma, void* grad, float* loss, cudaStream_t st) {
    k_log_loss<<<grid1d((long long)B * vox, 256), 256, 0, st>>>(pred, field, vox, B, fmax, eps_rel, mu, 1.0f / sigma,
                                                                 reinterpret_cast<__nv_bfloat16*>(grad), loss);
    return cudaGetLastError();
}

cudaError_t launch_field_error(const float* pred, const float* field, int B, long long vox, const float* fmax,
                               float eps_rel, float mu, float sigma, float* out, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(float) * 2 * B, st);
    if (e != cudaSuccess) return e;
    k_field_error<<<dim3(64, B), 256, 0, st>>>(pred, field, vox, fmax, eps_rel, mu, sigma, out);
    return cudaGetLastError();
}

cudaError_t launch_channel_mean(const void* x, int B, int C, long long vox, float* out, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(float) * B * C, st);
    if (e != cudaSuccess) return e;
    k_channel_sum<<<dim3(32, B), 256, 0, st>>>(reinterpret_cast<const __nv_bfloat16*>(x), vox, C, 1.0f / (float)vox, 1,
                                               out);
    return cudaGetLastError();
}

cudaError_t launch_adam(float* p, const float* g, float* m, float* v, long long n, float lr, float b1, float b2,
                        float eps, int step, cudaStream_t st) {
    const float c1 = 1.0f / (1.0f - powf(b1, (float)step)), c2 = 1.0f / (1.0f - powf(b2, (float)step));
    k_adam<<<grid1d(n, 256), 256, 0, st>>>(p, g, m, v, n, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError();
}

cudaError_t launch_bias_grad(const void* dz, int B, long long vox, int c_out, float* db, cudaStream_t st) {
    k_channel_sum<<<dim3(32, B), 256, 0, st>>>(reinterpret_cast<const __nv_bfloat16*>(dz), vox, c_out, 1.0f, 0, db);
    return cudaGetLastError();
}

cudaError_t launch_to_c32(const float* src, int B, int C, long long vox, void* dst, cudaStream_t st) {
    k_to_c32<<<grid1d((long long)B * 4 * vox, 256), 256, 0, st>>>(src, C, vox, B, reinterpret_cast<__nv_bfloat16*>(dst));
    return cudaGetLastError();
}

cudaError_t launch_from_c32(const void* src, int B, int C, long long vox, float* dst, cudaStream_t st) {
    k_from_c32<<<grid1d((long long)B * C * vox, 256), 256, 0, st>>>(reinterpret_cast<const __nv_bfloat16*>(src), C, vox,
                                                                     B, dst);
    return cudaGetLastError();
}

cudaError_t launch_pack_weights(const float* w, int c_in, int c_out, int transpose, void* packed, cudaStream_t st) {
    k_pack_weights<<<grid1d(27LL * 32 * 32, 256), 256, 0, st>>>(w, c_in, c_out, transpose,
                                                                 reinterpret_cast<__nv_bfloat16*>(packed));
    return cudaGetLastError();
}

}  // namespace rt
