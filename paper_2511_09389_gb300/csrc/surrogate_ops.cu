// surrogate_ops.cu -- element-wise and reduction kernels of the convolutional surrogate.
//
// Layout changes between plain FP32 NCDHW tensors and the CP8 bf16 layout of the tensor-core
// convolution ([B][C/8][D][H][W][8]), weight packing ([C_out][C_in][27] FP32 -> [27][C_in/8]
// [N][8] bf16, also flipped and transposed for the data gradient), the weight / bias gradient
// of a convolution (a reduction over voxels), the surrogate's input features and loss, and an
// Adam step.
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

__global__ void k_to_cp8(const float* __restrict__ src, int C, int kc, long long vox, int B,
                         __nv_bfloat16* __restrict__ dst) {
    const long long total = (long long)B * kc * vox;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long b = i / (kc * vox), r = i - b * kc * vox;
        const int k = (int)(r / vox);
        const long long v = r - (long long)k * vox;
        __align__(16) __nv_bfloat16 o[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int c = k * 8 + e;
            o[e] = __float2bfloat16_rn(c < C ? __ldg(src + ((long long)b * C + c) * vox + v) : 0.0f);
        }
        reinterpret_cast<uint4*>(dst)[i] = *reinterpret_cast<uint4*>(o);
    }
}

__global__ void k_from_cp8(const __nv_bfloat16* __restrict__ src, int C, int kc, long long vox, int B,
                           float* __restrict__ dst) {
    const long long total = (long long)B * C * vox;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long b = i / (C * vox), r = i - b * C * vox;
        const int c = (int)(r / vox);
        const long long v = r - (long long)c * vox;
        dst[i] = __bfloat162float(src[(((long long)b * kc + c / 8) * vox + v) * 8 + (c & 7)]);
    }
}

// packed[tap][k][n][e]: forward (transpose = 0): w[n][8k+e][tap];
// data gradient (transpose = 1): w[8k+e][n][26 - tap] (input = the forward's outputs).
__global__ void k_pack_weights(const float* __restrict__ w, int c_in, int c_out, int kc, int nco, int transpose,
                               __nv_bfloat16* __restrict__ packed) {
    const int total = 27 * kc * nco * 8;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const int e = i & 7, n = (i >> 3) % nco, k = (i / (8 * nco)) % kc, tap = i / (8 * nco * kc);
        const int c = k * 8 + e;
        float v = 0.0f;
        if (!transpose) {
            if (n < c_out && c < c_in) v = w[((long long)n * c_in + c) * 27 + tap];
        } else {
            // the transposed convolution maps c_out (its input, index c) to c_in (its output, index n)
            if (c < c_out && n < c_in) v = w[((long long)c * c_in + n) * 27 + (26 - tap)];
        }
        packed[i] = __float2bfloat16_rn(v);
    }
}

// db[co] += sum_v dz[b][co/8][v][co%8]: one block per (sample, plane) reduces 8 channels.
__global__ void k_bias_grad(const __nv_bfloat16* __restrict__ dz, int kc, long long vox, int c_out,
                            float* __restrict__ db) {
    const int b = blockIdx.y, k = blockIdx.x;
    const uint4* p = reinterpret_cast<const uint4*>(dz) + ((long long)b * kc + k) * vox;
    float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (long long v = threadIdx.x; v < vox; v += blockDim.x) {
        const uint4 q = __ldg(p + v);
        const __nv_bfloat16* e = reinterpret_cast<const __nv_bfloat16*>(&q);
#pragma unroll
        for (int i = 0; i < 8; ++i) acc[i] += __bfloat162float(e[i]);
    }
    __shared__ float red[8][33];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        float x = acc[i];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if ((threadIdx.x & 31) == 0) red[i][threadIdx.x >> 5] = x;
    }
    __syncthreads();
    if (threadIdx.x < 8) {
        float x = 0.0f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) x += red[threadIdx.x][w];
        const int co = k * 8 + threadIdx.x;
        if (co < c_out) atomicAdd(db + co, x);
    }
}

}  // namespace

cudaError_t launch_bias_grad(const void* dz, int B, int kc, long long vox, int c_out, float* db, cudaStream_t st) {
    k_bias_grad<<<dim3(kc, B), 1024, 0, st>>>(reinterpret_cast<const __nv_bfloat16*>(dz), kc, vox, c_out, db);
    return cudaGetLastError();
}

cudaError_t launch_to_cp8(const float* src, int B, int C, int kc, long long vox, void* dst, cudaStream_t st) {
    k_to_cp8<<<grid1d((long long)B * kc * vox, 256), 256, 0, st>>>(src, C, kc, vox, B,
                                                                    reinterpret_cast<__nv_bfloat16*>(dst));
    return cudaGetLastError();
}

cudaError_t launch_from_cp8(const void* src, int B, int C, int kc, long long vox, float* dst, cudaStream_t st) {
    k_from_cp8<<<grid1d((long long)B * C * vox, 256), 256, 0, st>>>(
        reinterpret_cast<const __nv_bfloat16*>(src), C, kc, vox, B, dst);
    return cudaGetLastError();
}

cudaError_t launch_pack_weights(const float* w, int c_in, int c_out, int kc, int nco, int transpose, void* packed,
                                cudaStream_t st) {
    k_pack_weights<<<grid1d(27LL * kc * nco * 8, 256), 256, 0, st>>>(w, c_in, c_out, kc, nco, transpose,
                                                                      reinterpret_cast<__nv_bfloat16*>(packed));
    return cudaGetLastError();
}

}  // namespace rt
