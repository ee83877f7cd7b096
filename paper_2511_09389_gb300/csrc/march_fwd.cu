// march_fwd.cu -- forward march (paper Sec. 2, Eq. 2) and its layout kernels, sm_103a.
//
// One thread marches one (ray, source, bin-group) lane through all N_s substeps. The W bins
// of a group share the ray geometry (bins are a batch axis, Sec. 2 "Frequency-bin
// agnosticism"), so j and kappa are read as W-wide vectors from a cell-major packed copy and
// each of the 8 deposits is a single W-wide `red.global.add.v{W}.f32`. Rays of a block are
// angular neighbours (the host sorts the lattice), so their gathers and deposits share
// cache lines near the source.
//
// Consecutive substeps of a ray often fall in the same cell (ds < 1), and once a ray has left
// the box its clamped corners stay fixed for long stretches. The deposits of such runs are
// summed in registers and sent to memory once, when the corner set changes: fewer L2 atomics,
// and far fewer tiny FP32 additions into the large sums that pile up on boundary voxels.
#include "march_common.cuh"
#include "rt_internal.h"

namespace rt {

// Gathers of one substep: the 8 j corners and the kappa cell, W bins each.
template <int W>
struct Gathered {
    Vec<W> j[8];
    Vec<W> k;
};

template <int W>
__device__ __forceinline__ void gather(const float* __restrict__ jg, const float* __restrict__ kg,
                                       const Sample& sm, Gathered<W>& gd) {
#pragma unroll
    for (int c = 0; c < 8; ++c) gd.j[c] = ldg_vec<W>(jg, sm.cell[c]);
    gd.k = ldg_vec<W>(kg, sm.nn);
}

// PF = 1: the gathers of substep k+1 are issued before the update of substep k (positions do
// not depend on I, so they can run ahead), which doubles the loads in flight per thread.
// PF = 0: gathers are issued only when the corner set (or the kappa cell) changes; otherwise
// the values from the previous substep, still in registers, are reused.
template <int W, int PF>
__global__ void __launch_bounds__(256) k_march_fwd(MarchArgs a) {
    const int rblocks = (a.ray_count + blockDim.x - 1) / blockDim.x;
    const int rb = blockIdx.x % rblocks;
    const int sg = blockIdx.x / rblocks;
    const int s = sg % a.nsrc;
    const int g = sg / a.nsrc;
    const int r = rb * blockDim.x + threadIdx.x;
    if (r >= a.ray_count) return;

    const long long ncell = (long long)a.n0 * a.n1 * a.n2;
    const float* __restrict__ jg = a.jp + (size_t)g * ncell * W;
    const float* __restrict__ kg = a.kp + (size_t)g * ncell * W;
    float* __restrict__ og = a.acc + (size_t)g * ncell * W;

    const float4 n = a.dirs[r];
    const float dx = __fmul_rn(n.x, a.ds), dy = __fmul_rn(n.y, a.ds), dz = __fmul_rn(n.z, a.ds);
    float x = a.src[3 * s + 0], y = a.src[3 * s + 1], z = a.src[3 * s + 2];

    float I[W], tau[W];
#pragma unroll
    for (int b = 0; b < W; ++b) { I[b] = 0.0f; tau[b] = 0.0f; }
    const float ds = a.ds, scale = a.dep_scale;

    // pending deposit of the current run of substeps with an unchanged corner set
    int pc[8];
    float pend[8][W];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        pc[c] = -1;
#pragma unroll
        for (int b = 0; b < W; ++b) pend[c][b] = 0.0f;
    }

    Sample sm;
    Gathered<W> gd;
    int gnn = -1;   // kappa cell of the gathered values (PF = 0)
    make_sample(x, y, z, a.n0, a.n1, a.n2, a.kappa_mode, sm);
    if (PF) gather<W>(jg, kg, sm, gd);

#pragma unroll 1
    for (int k = 0; k < a.ns; ++k) {
        x = __fadd_rn(x, dx);                             // Eq. 2: x_{k+1}
        y = __fadd_rn(y, dy);
        z = __fadd_rn(z, dz);
        Sample nx;
        Gathered<W> ng;
        // same 8 corners as the previous substep: the registers already hold their j values
        const bool same_cells = sm.cell[0] == pc[0] && sm.cell[7] == pc[7];
        if (PF) {
            make_sample(x, y, z, a.n0, a.n1, a.n2, a.kappa_mode, nx);
            if (k + 1 < a.ns) gather<W>(jg, kg, nx, ng);
        } else {
            if (!same_cells) {
#pragma unroll
                for (int c = 0; c < 8; ++c) gd.j[c] = ldg_vec<W>(jg, sm.cell[c]);
            }
            if (sm.nn != gnn) {
                gd.k = ldg_vec<W>(kg, sm.nn);
                gnn = sm.nn;
            }
        }
        float dep[W];
#pragma unroll
        for (int b = 0; b < W; ++b) {
            float jk = 0.0f;
#pragma unroll
            for (int c = 0; c < 8; ++c) jk = fmaf(sm.w[c], gd.j[c].v[b], jk);
            const float kds = gd.k.v[b] * ds;
            const float att = expf(-kds);                 // exp(-kappa(x_k) ds)
            const float em = expf(-tau[b]);               // exp(-tau_k)
            I[b] = fmaf(I[b], att, jk * em * ds);         // Eq. 2: I_{k+1}
            tau[b] += kds;                                // Eq. 2: tau_{k+1}
            dep[b] = I[b] * scale;
        }
        // the corner set is fixed by its lowest and highest corner
        if (!same_cells) {
            if (pc[0] >= 0) {
#pragma unroll
                for (int c = 0; c < 8; ++c) red_vec<W>(og, pc[c], pend[c]);
            }
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                pc[c] = sm.cell[c];
#pragma unroll
                for (int b = 0; b < W; ++b) pend[c][b] = sm.w[c] * dep[b];
            }
        } else {
#pragma unroll
            for (int c = 0; c < 8; ++c) {
#pragma unroll
                for (int b = 0; b < W; ++b) pend[c][b] = fmaf(sm.w[c], dep[b], pend[c][b]);
            }
        }
        if (PF) {
            sm = nx;
            gd = ng;
        } else {
            make_sample(x, y, z, a.n0, a.n1, a.n2, a.kappa_mode, sm);
        }
    }
    if (pc[0] >= 0) {
#pragma unroll
        for (int c = 0; c < 8; ++c) red_vec<W>(og, pc[c], pend[c]);
    }
}

cudaError_t launch_march_fwd(int W, const MarchArgs& a, cudaStream_t st) {
    const int block = a.block > 0 ? a.block : 128;
    const long long rblocks = (a.ray_count + block - 1) / block;
    const long long nblk = rblocks * a.nsrc * a.groups;
    if (nblk <= 0) return cudaSuccess;
    if (nblk > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    const int pf = a.prefetch ? 1 : 0;
    switch (W * 2 + pf) {
        case 2: k_march_fwd<1, 0><<<(unsigned)nblk, block, 0, st>>>(a); break;
        case 3: k_march_fwd<1, 1><<<(unsigned)nblk, block, 0, st>>>(a); break;
        case 4: k_march_fwd<2, 0><<<(unsigned)nblk, block, 0, st>>>(a); break;
        case 5: k_march_fwd<2, 1><<<(unsigned)nblk, block, 0, st>>>(a); break;
        case 8: k_march_fwd<4, 0><<<(unsigned)nblk, block, 0, st>>>(a); break;
        case 9: k_march_fwd<4, 1><<<(unsigned)nblk, block, 0, st>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// ---- layout kernels ----------------------------------------------------------------------
template <int W>
__global__ void k_pack(const float* __restrict__ in, float* __restrict__ out, int n_freq,
                       long long ncell, long long total) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long g = i / ncell, c = i - g * ncell;
        float v[W];
#pragma unroll
        for (int w = 0; w < W; ++w) {
            const long long b = g * W + w;
            v[w] = b < n_freq ? __ldg(in + b * ncell + c) : 0.0f;
        }
        if (W == 4) {
            reinterpret_cast<float4*>(out)[i] = make_float4(v[0], v[1], v[2], v[3]);
        } else if (W == 2) {
            reinterpret_cast<float2*>(out)[i] = make_float2(v[0], v[1 % W]);
        } else {
            out[i] = v[0];
        }
    }
}

template <int W>
__global__ void k_unpack(const float* __restrict__ acc, float* __restrict__ out, int n_freq,
                         long long ncell, long long total, float scale, int accumulate) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long g = i / ncell, c = i - g * ncell;
        float v[W];
        if (W == 4) {
            const float4 q = __ldg(reinterpret_cast<const float4*>(acc) + i);
            v[0] = q.x; v[1 % W] = q.y; v[2 % W] = q.z; v[3 % W] = q.w;
        } else if (W == 2) {
            const float2 q = __ldg(reinterpret_cast<const float2*>(acc) + i);
            v[0] = q.x; v[1 % W] = q.y;
        } else {
            v[0] = __ldg(acc + i);
        }
#pragma unroll
        for (int w = 0; w < W; ++w) {
            const long long b = g * W + w;
            if (b < n_freq) {
                float* o = out + b * ncell + c;
                const float val = scale * v[w];
                *o = accumulate ? *o + val : val;
            }
        }
    }
}

static unsigned grid_for(long long total, int block) {
    long long g = (total + block - 1) / block;
    const long long cap = 152LL * 16;   // 16 blocks per SM on 152 SMs, grid-stride beyond
    if (g > cap) g = cap;
    return (unsigned)(g < 1 ? 1 : g);
}

cudaError_t launch_pack(const float* in, float* out, int n_freq, int W, int groups, long long ncell,
                        cudaStream_t st) {
    const long long total = (long long)groups * ncell;
    const unsigned grid = grid_for(total, 256);
    switch (W) {
        case 1: k_pack<1><<<grid, 256, 0, st>>>(in, out, n_freq, ncell, total); break;
        case 2: k_pack<2><<<grid, 256, 0, st>>>(in, out, n_freq, ncell, total); break;
        case 4: k_pack<4><<<grid, 256, 0, st>>>(in, out, n_freq, ncell, total); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_unpack(const float* acc, float* out, int n_freq, int W, long long ncell, float scale,
                          int accumulate, cudaStream_t st) {
    const long long groups = (n_freq + W - 1) / W;
    const long long total = groups * ncell;
    const unsigned grid = grid_for(total, 256);
    switch (W) {
        case 1: k_unpack<1><<<grid, 256, 0, st>>>(acc, out, n_freq, ncell, total, scale, accumulate); break;
        case 2: k_unpack<2><<<grid, 256, 0, st>>>(acc, out, n_freq, ncell, total, scale, accumulate); break;
        case 4: k_unpack<4><<<grid, 256, 0, st>>>(acc, out, n_freq, ncell, total, scale, accumulate); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// ---- geometry trace (test hook) ------------------------------------------------------------
__global__ void k_trace(float sx, float sy, float sz, float nx, float ny, float nz, float ds, int ns,
                        int n0, int n1, int n2, int kappa_mode, long long* base, long long* nn) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    const float dx = __fmul_rn(nx, ds), dy = __fmul_rn(ny, ds), dz = __fmul_rn(nz, ds);
    float x = sx, y = sy, z = sz;
    for (int k = 0; k < ns; ++k) {
        Sample sm;
        make_sample(x, y, z, n0, n1, n2, kappa_mode, sm);
        base[k] = sm.cell[0];
        nn[k] = sm.nn;
        x = __fadd_rn(x, dx);
        y = __fadd_rn(y, dy);
        z = __fadd_rn(z, dz);
    }
}

cudaError_t launch_trace(float sx, float sy, float sz, float nx, float ny, float nz, float ds, int ns,
                         int n0, int n1, int n2, int kappa_mode, long long* base, long long* nn,
                         cudaStream_t st) {
    k_trace<<<1, 32, 0, st>>>(sx, sy, sz, nx, ny, nz, ds, ns, n0, n1, n2, kappa_mode, base, nn);
    return cudaGetLastError();
}

}  // namespace rt
