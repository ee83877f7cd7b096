// march_batch.cu -- many independent march problems in one persistent launch (sm_103a).
//
// Instances differ in grid shape, source count, lattice size and bin count. The host flattens
// them into work items of 32 rays (instance, source, bin group, first ray), longest first; a
// persistent grid of warps pulls items from a device counter (one atomicAdd per item, no
// waiting on other warps), so small instances fill the gaps that large ones leave and no SM
// idles until the queue is empty. Each lane runs the same march as the single-problem kernel
// (march_lane.cuh). Items are split by bin-group width W, one persistent kernel per width.
// Batched pack / unpack kernels take one grid row (blockIdx.y) per instance.
#include "march_lane.cuh"
#include "rt_internal.h"

namespace rt {

// Persistent march over the items of one bin-group width W (each width has its own kernel so
// that its register count, and hence its occupancy, is that of the W-wide lane alone). The
// launch bound caps registers at 128 per thread: the march is latency-bound and needs the
// warps (measured: 150 registers, 12 warps per SM, 20 % slower than the capped kernel).
template <int W>
__global__ void __launch_bounds__(256, 2) k_march_batch(const BatchInst* __restrict__ insts,
                                                     const int4* __restrict__ items, int n_items,
                                                     int* __restrict__ counter) {
    const int lane = threadIdx.x & 31;
    for (;;) {
        int it = 0;
        if (lane == 0) it = atomicAdd(counter, 1);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= n_items) return;
        const int4 item = items[it];              // instance, source, bin group, first ray
        const BatchInst& B = insts[item.x];
        const int r = item.w + lane;
        if (r < B.ray_count) {
            const long long ncell = (long long)B.n0 * B.n1 * B.n2;
            const size_t off = (size_t)item.z * ncell * W;
            Lane L;
            L.jg = B.jp + off;
            L.kg = B.kp + off;
            L.og = B.acc + off;
            L.pol = red_policy(4LL * B.groups * ncell * W);
            L.n = B.dirs[r];
            L.sx = B.src[3 * item.y + 0]; L.sy = B.src[3 * item.y + 1]; L.sz = B.src[3 * item.y + 2];
            L.n0 = B.n0; L.n1 = B.n1; L.n2 = B.n2;
            L.ns = B.ns;
            L.ds = B.ds;
            L.scale = 1.0f;
            L.kappa_mode = B.kappa_mode;
            RayState<W> rs;
            rs.x = L.sx; rs.y = L.sy; rs.z = L.sz;
#pragma unroll
            for (int b = 0; b < W; ++b) { rs.I[b] = 0.0f; rs.tau[b] = 0.0f; }
            // corner slots with the entering corners gathered a substep ahead (gathers mode 4)
            // where the lane fits the 128-register cap; the four-bin lane needs ~160 registers
            // for that and keeps the slots of mode 0
            march_lane<W, W == 4 ? 0 : 4>(L, rs);
        }
        __syncwarp();
    }
}

// which = 0: pack j, 1: pack kappa (instances with W = 1 read the caller's arrays directly).
__global__ void k_pack_batch(const BatchInst* __restrict__ insts, int which) {
    const BatchInst& B = insts[blockIdx.y];
    if (B.W == 1) return;
    const long long ncell = (long long)B.n0 * B.n1 * B.n2;
    const long long total = (long long)B.groups * ncell;
    const float* __restrict__ in = which == 0 ? B.j : B.kappa;
    float* __restrict__ out = which == 0 ? B.jp_w : B.kp_w;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long g = i / ncell, c = i - g * ncell;
        float v[4];
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            const long long b = g * B.W + w;
            v[w] = (w < B.W && b < B.n_freq) ? __ldg(in + b * ncell + c) : 0.0f;
        }
        if (B.W == 4) reinterpret_cast<float4*>(out)[i] = make_float4(v[0], v[1], v[2], v[3]);
        else reinterpret_cast<float2*>(out)[i] = make_float2(v[0], v[1]);
    }
}

// out[b][c] = scale * acc[b / W][c][b % W]
__global__ void k_unpack_batch(const BatchInst* __restrict__ insts) {
    const BatchInst& B = insts[blockIdx.y];
    const long long ncell = (long long)B.n0 * B.n1 * B.n2;
    const long long total = (long long)B.groups * ncell;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long g = i / ncell, c = i - g * ncell;
        for (int w = 0; w < B.W; ++w) {
            const long long b = g * B.W + w;
            if (b < B.n_freq) B.out[b * ncell + c] = B.scale * B.acc[i * B.W + w];
        }
    }
}

int march_batch_blocks_per_sm(int W, int block) {
    int nb = 0;
    cudaError_t e = cudaErrorInvalidValue;
    if (W == 4) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_march_batch<4>, block, 0);
    else if (W == 2) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_march_batch<2>, block, 0);
    else if (W == 1) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_march_batch<1>, block, 0);
    if (e != cudaSuccess) return 1;
    return nb > 0 ? nb : 1;
}

cudaError_t launch_march_batch(int W, const BatchInst* insts, const int4* items, int n_items, int* counter,
                               int grid, int block, cudaStream_t st) {
    if (n_items <= 0) return cudaSuccess;
    switch (W) {
        case 4: k_march_batch<4><<<grid, block, 0, st>>>(insts, items, n_items, counter); break;
        case 2: k_march_batch<2><<<grid, block, 0, st>>>(insts, items, n_items, counter); break;
        case 1: k_march_batch<1><<<grid, block, 0, st>>>(insts, items, n_items, counter); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// Blocks per instance row: enough for the largest instance to stream at full bandwidth (about
// eight elements per thread); rows of smaller instances finish early.
static unsigned layout_blocks(long long max_elems) {
    long long b = (max_elems + 256 * 8 - 1) / (256 * 8);
    return (unsigned)(b < 1 ? 1 : (b > 4096 ? 4096 : b));
}

cudaError_t launch_pack_batch(const BatchInst* insts, int n_inst, long long max_elems, int which, cudaStream_t st) {
    if (n_inst <= 0) return cudaSuccess;
    k_pack_batch<<<dim3(layout_blocks(max_elems), n_inst), 256, 0, st>>>(insts, which);
    return cudaGetLastError();
}

cudaError_t launch_unpack_batch(const BatchInst* insts, int n_inst, long long max_elems, cudaStream_t st) {
    if (n_inst <= 0) return cudaSuccess;
    k_unpack_batch<<<dim3(layout_blocks(max_elems), n_inst), 256, 0, st>>>(insts);
    return cudaGetLastError();
}

}  // namespace rt
