// inversion.cu -- the element-wise kernels of the emissivity inversion (paper Sec. 4,
// "Gradient-based inversion", generalised from one amplitude to every voxel of j): the log of
// the target field, the log-field misfit with its gradient, and a projected Adam step. The
// march and its adjoint are the library's own (rt_advance, rt_backward); rt_invert_emissivity
// (rt_api.cu) strings them together on one stream.
//
// Loss: L(j) = mean_v (log(F(j)_v + eps) - log(F_target_v + eps))^2, eps = eps_rel max F_target.
#include <cuda_runtime.h>

#include <cmath>

#include "rt_internal.h"

namespace rt {

namespace {

constexpr int kThreads = 256;

int blocks_for(long long n) {
    const long long b = (n + kThreads - 1) / kThreads;
    return (int)(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

// log_t[v] = log(target[v] + eps_rel * fmax[0])
__global__ void k_log_target(const float* __restrict__ target, long long n, const float* __restrict__ fmax,
                             float eps_rel, float* __restrict__ log_t) {
    const float eps = eps_rel * __ldg(fmax);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        log_t[i] = logf(target[i] + eps);
}

// r = log(F + eps) - log_t; grad = dL/dF = 2 r / (n (F + eps)) (grad may be NULL);
// *loss += sum r^2 / n (one atomic per block after a block reduction)
__global__ void k_log_misfit(const float* __restrict__ F, const float* __restrict__ log_t, long long n,
                             const float* __restrict__ fmax, float eps_rel, float* __restrict__ grad,
                             float* __restrict__ loss) {
    __shared__ float part[kThreads / 32];
    const float eps = eps_rel * __ldg(fmax);
    const float inv_n = 1.0f / (float)n;
    float acc = 0.0f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float fe = F[i] + eps;
        const float r = logf(fe) - log_t[i];
        acc = fmaf(r, r, acc);
        if (grad) grad[i] = 2.0f * r * inv_n / fe;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        float s = threadIdx.x < kThreads / 32 ? part[threadIdx.x] : 0.0f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) atomicAdd(loss, s * inv_n);
    }
}

// Bias-corrected Adam (c1 = 1 / (1 - b1^t), c2 = 1 / (1 - b2^t)), then p = max(p, lower)
__global__ void k_adam_projected(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                                 float* __restrict__ v, long long n, float lr, float b1, float b2, float eps,
                                 float c1, float c2, float lower) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] = fmaxf(p[i] - lr * (mi * c1) / (sqrtf(vi * c2) + eps), lower);
    }
}

}  // namespace

cudaError_t launch_log_target(const float* target, long long n, const float* fmax, float eps_rel, float* log_t,
                              cudaStream_t st) {
    k_log_target<<<blocks_for(n), kThreads, 0, st>>>(target, n, fmax, eps_rel, log_t);
    return cudaGetLastError();
}

cudaError_t launch_log_misfit(const float* F, const float* log_t, long long n, const float* fmax, float eps_rel,
                              float* grad, float* loss, cudaStream_t st) {
    k_log_misfit<<<blocks_for(n), kThreads, 0, st>>>(F, log_t, n, fmax, eps_rel, grad, loss);
    return cudaGetLastError();
}

cudaError_t launch_adam_projected(float* p, const float* g, float* m, float* v, long long n, float lr, float b1,
                                  float b2, float eps, int step, float lower, cudaStream_t st) {
    // the bias corrections as rt_adam_step computes them
    const float c1 = 1.0f / (1.0f - std::pow(b1, (float)step)), c2 = 1.0f / (1.0f - std::pow(b2, (float)step));
    k_adam_projected<<<blocks_for(n), kThreads, 0, st>>>(p, g, m, v, n, lr, b1, b2, eps, c1, c2, lower);
    return cudaGetLastError();
}

}  // namespace rt
