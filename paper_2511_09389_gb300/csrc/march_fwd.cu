// march_fwd.cu -- forward march of one problem (paper Sec. 2, Eq. 2) and its layout kernels.
//
// One thread (or, with two lanes per ray, a pair of adjacent threads) marches one (ray, source,
// bin-group) lane through all N_s substeps (march_lane.cuh). Rays of a block are angular
// neighbours (the host sorts the lattice), so their gathers and deposits share cache lines near
// the source.
#include "march_lane.cuh"
#include "rt_internal.h"

namespace rt {

// Tile origin along one axis: the kTile cells starting kTile/2 - 1 below the source's cell,
// moved inside [0, n - kTile].
__device__ __forceinline__ int tile_origin(float src, int n) {
    const int f = (int)floorf(fminf(fmaxf(src, -4.0e6f), 4.0e6f));
    return min(max(f - (kTile / 2 - 1), 0), n - kTile);
}

// TILE: every block (one source, one bin group) keeps the kTile^3 cells around its source in
// shared memory; its lanes' deposits there are summed with shared-memory atomics and added to
// the field once per block. The cells next to a source receive a deposit from every ray of it,
// so this takes the most contended L2 atomics off the march and sums them in shorter chains.
// REC: also write the reverse march's checkpoints (march_lane).
// Gathers mode 4 with four bins keeps a second set of slot values in registers: it launches with
// 32-thread blocks only, bounded so that 11 of them fit on an SM (a 128^3 problem with 16 sources
// and 3072 rays has 10.1 warps per SM of the 152).
template <int W, int PF>
constexpr int fwd_max_threads() { return PF == 4 && W == 4 ? 32 : 256; }
template <int W, int PF>
constexpr int fwd_min_blocks() { return PF == 4 && W == 4 ? 11 : 1; }

template <int W, int PF, int DET, bool TILE, bool REC = false>
__global__ void __launch_bounds__(fwd_max_threads<W, PF>(), fwd_min_blocks<W, PF>()) k_march_fwd(MarchArgs a) {
    constexpr int TCELLS = kTile * kTile * kTile;
    __shared__ float tile[TILE ? TCELLS * W : 1];
    const int rblocks = (a.ray_count + blockDim.x - 1) / blockDim.x;
    const int rb = blockIdx.x % rblocks;
    const int sg = blockIdx.x / rblocks;
    const int s = sg % a.nsrc;
    const int g = sg / a.nsrc;
    const int r = rb * blockDim.x + threadIdx.x;
    const long long ncell = (long long)a.n0 * a.n1 * a.n2;
    float* og = a.acc + (size_t)g * ncell * W;
    int to0 = 0, to1 = 0, to2 = 0;
    // the launcher uses TILE only when every grid extent is at least kTile
    if (TILE) {
        to0 = tile_origin(a.src[3 * s + 0], a.n0);
        to1 = tile_origin(a.src[3 * s + 1], a.n1);
        to2 = tile_origin(a.src[3 * s + 2], a.n2);
        for (int i = threadIdx.x; i < TCELLS * W; i += blockDim.x) tile[i] = 0.0f;
        __syncthreads();
    }
    if (r < a.ray_count) {
    Lane L;
    L.jg = a.jp + (size_t)g * ncell * W;
    L.kg = a.kp + (size_t)g * ncell * W;
    L.og = og;
    L.pol = red_policy((DET ? 8LL : 4LL) * a.groups * ncell * W);   // bytes of the accumulator
    L.n = a.dirs[r];
    L.sx = a.src[3 * s + 0]; L.sy = a.src[3 * s + 1]; L.sz = a.src[3 * s + 2];
    L.n0 = a.n0; L.n1 = a.n1; L.n2 = a.n2;
    L.ns = a.ns;
    L.ds = a.ds;
    L.scale = a.dep_scale;
    L.kappa_mode = a.kappa_mode;
    L.og64 = a.acc64 ? a.acc64 + (size_t)g * ncell * W : nullptr;
    L.ncell = ncell;
    L.nbins = min(W, a.n_freq - g * W);
    if (DET == 1) L.fix = __ldg(a.fix);   // the fixed-point unit, read once per lane
    L.tile = TILE ? tile : nullptr;
    L.to0 = to0; L.to1 = to1; L.to2 = to2;
    // start at the source with I = tau = 0, or (stateful advance) where the previous call left
    // the ray: per-(source, ray) position, per-(bin, source, ray) I and tau
    RayState<W> rs;
    rs.x = L.sx; rs.y = L.sy; rs.z = L.sz;
#pragma unroll
    for (int b = 0; b < W; ++b) { rs.I[b] = 0.0f; rs.tau[b] = 0.0f; }
    const long long lanes = (long long)a.nsrc * a.ray_count;
    const long long lane = (long long)s * a.ray_count + r;
    if (a.st_I && a.st_read) {
        rs.x = a.st_pos_in[3 * lane + 0]; rs.y = a.st_pos_in[3 * lane + 1]; rs.z = a.st_pos_in[3 * lane + 2];
#pragma unroll
        for (int b = 0; b < W; ++b)
            if (b < L.nbins) {
                rs.I[b] = a.st_I[(long long)(g * W + b) * lanes + lane];
                rs.tau[b] = a.st_tau[(long long)(g * W + b) * lanes + lane];
            }
    }
    if (REC) {
        L.ck_lanes = (long long)a.ray_count * a.nsrc * a.groups;
        L.ck = a.ckpt + ((long long)g * a.nsrc + s) * a.ray_count + r;
        L.ck_stride = a.ck_stride;
    }
    march_lane<W, PF, DET, TILE, REC>(L, rs);
    if (a.st_I) {
#pragma unroll
        for (int b = 0; b < W; ++b)
            if (b < L.nbins) {
                a.st_I[(long long)(g * W + b) * lanes + lane] = rs.I[b];
                a.st_tau[(long long)(g * W + b) * lanes + lane] = rs.tau[b];
            }
        if (g == 0) {   // every bin group of the ray reads the old position: written to the other buffer
            a.st_pos_out[3 * lane + 0] = rs.x; a.st_pos_out[3 * lane + 1] = rs.y; a.st_pos_out[3 * lane + 2] = rs.z;
        }
    }
    }
    if (TILE) {
        __syncthreads();
        for (int i = threadIdx.x; i < TCELLS; i += blockDim.x) {
            float v[W];
            bool any = false;
#pragma unroll
            for (int b = 0; b < W; ++b) {
                v[b] = tile[i * W + b];
                any = any || v[b] != 0.0f;
            }
            if (any) {
                const int u0 = i / (kTile * kTile), u1 = (i / kTile) % kTile, u2 = i % kTile;
                const int cell = ((to0 + u0) * a.n1 + (to1 + u1)) * a.n2 + (to2 + u2);
                red_vec<W>(og, cell, v, red_policy(4LL * a.groups * a.n0 * a.n1 * a.n2 * W));
            }
        }
    }
}

// Lanes per ray = 2: adjacent lanes (sub = threadIdx.x & 1) share one (ray, source, bin group),
// each with half of its corner slots (march_lane_pair; gathers mode PF = 4: march_lane_pair_ahead).
// REC: also the reverse march's checkpoints. DET: the accumulation (flush() in march_lane.cuh).
template <int W, bool REC = false, int DET = 0, int PF = 0>
__global__ void __launch_bounds__(256) k_march_fwd_pair(MarchArgs a) {
    const int rays_per_block = blockDim.x / 2;
    const int rblocks = (a.ray_count + rays_per_block - 1) / rays_per_block;
    const int rb = blockIdx.x % rblocks;
    const int sg = blockIdx.x / rblocks;
    const int s = sg % a.nsrc;
    const int g = sg / a.nsrc;
    const int sub = threadIdx.x & 1;
    const int r = rb * rays_per_block + (threadIdx.x >> 1);
    if (r >= a.ray_count) return;   // both lanes of a pair leave together
    const unsigned pmask = 3u << (threadIdx.x & 30);
    const long long ncell = (long long)a.n0 * a.n1 * a.n2;
    Lane L;
    L.jg = a.jp + (size_t)g * ncell * W;
    L.kg = a.kp + (size_t)g * ncell * W;
    L.og = a.acc + (size_t)g * ncell * W;
    L.pol = red_policy((DET ? 8LL : 4LL) * a.groups * ncell * W);   // bytes of the accumulator
    L.n = a.dirs[r];
    L.sx = a.src[3 * s + 0]; L.sy = a.src[3 * s + 1]; L.sz = a.src[3 * s + 2];
    L.n0 = a.n0; L.n1 = a.n1; L.n2 = a.n2;
    L.ns = a.ns;
    L.ds = a.ds;
    L.scale = a.dep_scale;
    L.kappa_mode = a.kappa_mode;
    L.og64 = a.acc64 ? a.acc64 + (size_t)g * ncell * W : nullptr;
    L.ncell = ncell;
    L.nbins = min(W, a.n_freq - g * W);
    if (DET == 1) L.fix = __ldg(a.fix);   // the fixed-point unit, read once per lane
    if (REC) {
        L.ck_lanes = (long long)a.ray_count * a.nsrc * a.groups;
        L.ck = a.ckpt + ((long long)g * a.nsrc + s) * a.ray_count + r;
        L.ck_stride = a.ck_stride;
    }
    if constexpr (PF == 4)
        march_lane_pair_ahead<W, REC, DET>(L, sub, pmask);
    else
        march_lane_pair<W, REC, DET>(L, sub, pmask);
}

// ---- kernel table ------------------------------------------------------------------------
// The compiled (W, gathers mode, accumulation, tiles, checkpoints, lanes per ray) combinations:
//   FP32: every W and gathers mode with and without tiles (mode 4: without); recording with
//         gathers modes 0 and 4 (and 1 or 3 for one bin); two lanes per ray for every W with
//         gathers mode 0 or 4, recording or not.
//   fixed point: corner slots and gathers mode 4 for every W; for one bin also recording and two
//         lanes per ray; two lanes per ray with gathers mode 4 for one and four bins.
//   FP64: corner slots for every W, with and without recording; two lanes per ray for one bin.
using MarchKernel = void (*)(MarchArgs);

template <int W>
MarchKernel pick_one_lane(int pf, int acc, bool tile, bool rec) {
    if (pf == 4) {   // corner slots with the gathers one substep ahead: no tiles
        if (tile) return nullptr;
        if (rec) return acc == 0 ? k_march_fwd<W, 4, 0, false, true> : nullptr;
        if (acc == 0) return k_march_fwd<W, 4, 0, false>;
        if (acc == 1) return k_march_fwd<W, 4, 1, false>;
        return nullptr;
    }
    if (acc == 0 && !rec) {
        switch (pf * 2 + (tile ? 1 : 0)) {
            case 0: return k_march_fwd<W, 0, 0, false>;
            case 1: return k_march_fwd<W, 0, 0, true>;
            case 2: return k_march_fwd<W, 1, 0, false>;
            case 3: return k_march_fwd<W, 1, 0, true>;
            case 4: return k_march_fwd<W, 2, 0, false>;
            case 5: return k_march_fwd<W, 2, 0, true>;
            case 6: return k_march_fwd<W, 3, 0, false>;
            case 7: return k_march_fwd<W, 3, 0, true>;
        }
        return nullptr;
    }
    if (acc == 0) {   // recording
        if (pf == 0) return tile ? k_march_fwd<W, 0, 0, true, true> : k_march_fwd<W, 0, 0, false, true>;
        if (W == 1 && pf == 1) return tile ? k_march_fwd<1, 1, 0, true, true> : k_march_fwd<1, 1, 0, false, true>;
        if (W == 1 && pf == 3) return tile ? k_march_fwd<1, 3, 0, true, true> : k_march_fwd<1, 3, 0, false, true>;
        return nullptr;
    }
    if (tile || pf != 0) return nullptr;
    if (acc == 1) {
        if (!rec) return k_march_fwd<W, 0, 1, false>;
        return W == 1 ? k_march_fwd<1, 0, 1, false, true> : nullptr;
    }
    return rec ? k_march_fwd<W, 0, 2, false, true> : k_march_fwd<W, 0, 2, false>;
}

MarchKernel pick_pair(int W, int pf, int acc, bool rec) {
    if (pf == 4) {   // gathers one substep ahead: FP32 (recording for one bin) and fixed point
        if (acc == 0 && !rec)
            return W == 1 ? k_march_fwd_pair<1, false, 0, 4> : (W == 2 ? k_march_fwd_pair<2, false, 0, 4>
                                                                     : k_march_fwd_pair<4, false, 0, 4>);
        if (acc == 0)   // recording
            return W == 1 ? k_march_fwd_pair<1, true, 0, 4> : (W == 2 ? k_march_fwd_pair<2, true, 0, 4>
                                                                  : k_march_fwd_pair<4, true, 0, 4>);
        if (acc == 1 && !rec && (W == 1 || W == 4))
            return W == 1 ? k_march_fwd_pair<1, false, 1, 4> : k_march_fwd_pair<4, false, 1, 4>;
        return nullptr;
    }
    if (pf != 0) return nullptr;
    if (acc == 0) {
        switch (W * 2 + (rec ? 1 : 0)) {
            case 2: return k_march_fwd_pair<1>;
            case 3: return k_march_fwd_pair<1, true>;
            case 4: return k_march_fwd_pair<2>;
            case 5: return k_march_fwd_pair<2, true>;
            case 8: return k_march_fwd_pair<4>;
            case 9: return k_march_fwd_pair<4, true>;
        }
        return nullptr;
    }
    if (W != 1) return nullptr;
    if (acc == 1) return rec ? k_march_fwd_pair<1, true, 1> : k_march_fwd_pair<1, false, 1>;
    return rec ? k_march_fwd_pair<1, true, 2> : k_march_fwd_pair<1, false, 2>;
}

MarchKernel pick_march(int W, int pf, int acc, bool tile, bool rec, int lpr) {
    if (pf < 0 || pf > 4 || acc < 0 || acc > 2) return nullptr;
    if (lpr == 2) return !tile && (W == 1 || W == 2 || W == 4) ? pick_pair(W, pf, acc, rec) : nullptr;
    if (lpr != 1) return nullptr;
    switch (W) {
        case 1: return pick_one_lane<1>(pf, acc, tile, rec);
        case 2: return pick_one_lane<2>(pf, acc, tile, rec);
        case 4: return pick_one_lane<4>(pf, acc, tile, rec);
    }
    return nullptr;
}

int max_block(int W, int pf, int lpr) { return lpr == 1 && pf == 4 && W == 4 ? fwd_max_threads<4, 4>() : 256; }

bool march_fwd_available(int W, int prefetch, int acc_mode, int tile, int record, int lanes_per_ray, int block) {
    const int lpr = lanes_per_ray <= 1 ? 1 : lanes_per_ray;
    if (block > max_block(W, prefetch, lpr)) return false;
    return pick_march(W, prefetch, acc_mode, tile != 0 && lpr == 1, record != 0, lpr) != nullptr;
}

cudaError_t launch_march_fwd(int W, const MarchArgs& a, cudaStream_t st) {
    if (a.acc_mode < 0 || a.acc_mode > 2 || ((a.acc_mode != 0) != (a.acc64 != nullptr))) return cudaErrorInvalidValue;
    if (a.acc_mode == 1 && !a.fix) return cudaErrorInvalidValue;
    if (a.ckpt && a.ck_stride < 1) return cudaErrorInvalidValue;
    const int lpr = a.lanes_per_ray <= 1 ? 1 : a.lanes_per_ray;   // 0: one lane per ray
    const bool pair = lpr == 2;
    if (pair && a.st_I) return cudaErrorInvalidValue;   // the stateful march runs one lane per ray
    // tiles only when every grid extent is at least kTile (and never with two lanes per ray)
    const bool tile = !pair && a.tile && a.n0 >= kTile && a.n1 >= kTile && a.n2 >= kTile;
    const MarchKernel k = pick_march(W, a.prefetch, a.acc_mode, tile, a.ckpt != nullptr, lpr);
    if (!k) return cudaErrorInvalidValue;
    // two lanes per ray: block counts threads (a multiple of 32), block / 2 rays per block
    const int block = a.block > 0 ? a.block : (pair ? 64 : (a.prefetch == 4 && W == 4 ? 32 : 128));
    if (block % 32 || block > max_block(W, a.prefetch, lpr)) return cudaErrorInvalidValue;
    const int rays_per_block = pair ? block / 2 : block;
    const long long rblocks = (a.ray_count + rays_per_block - 1) / rays_per_block;
    const long long nblk = rblocks * a.nsrc * a.groups;
    if (nblk <= 0) return cudaSuccess;
    if (nblk > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    k<<<(unsigned)nblk, block, 0, st>>>(a);
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

// j and kappa in one pass, and the packed accumulator cleared (acc != NULL): one launch instead
// of three before a march.
template <int W>
__global__ void k_pack_pair(const float* __restrict__ j, const float* __restrict__ kap, float* __restrict__ jp,
                            float* __restrict__ kp, float* __restrict__ acc, int n_freq, long long ncell,
                            long long total) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long g = i / ncell, c = i - g * ncell;
        float vj[W], vk[W];
#pragma unroll
        for (int w = 0; w < W; ++w) {
            const long long b = g * W + w;
            vj[w] = b < n_freq ? __ldg(j + b * ncell + c) : 0.0f;
            vk[w] = b < n_freq ? __ldg(kap + b * ncell + c) : 0.0f;
        }
        if (W == 4) {
            reinterpret_cast<float4*>(jp)[i] = make_float4(vj[0], vj[1 % W], vj[2 % W], vj[3 % W]);
            reinterpret_cast<float4*>(kp)[i] = make_float4(vk[0], vk[1 % W], vk[2 % W], vk[3 % W]);
            if (acc) reinterpret_cast<float4*>(acc)[i] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        } else if (W == 2) {
            reinterpret_cast<float2*>(jp)[i] = make_float2(vj[0], vj[1 % W]);
            reinterpret_cast<float2*>(kp)[i] = make_float2(vk[0], vk[1 % W]);
            if (acc) reinterpret_cast<float2*>(acc)[i] = make_float2(0.0f, 0.0f);
        } else {
            jp[i] = vj[0];
            kp[i] = vk[0];
            if (acc) acc[i] = 0.0f;
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

cudaError_t launch_pack_pair(const float* j, const float* kappa, float* jp, float* kp, float* acc, int n_freq, int W,
                             int groups, long long ncell, cudaStream_t st) {
    const long long total = (long long)groups * ncell;
    const unsigned grid = grid_for(total, 256);
    switch (W) {
        case 1: k_pack_pair<1><<<grid, 256, 0, st>>>(j, kappa, jp, kp, acc, n_freq, ncell, total); break;
        case 2: k_pack_pair<2><<<grid, 256, 0, st>>>(j, kappa, jp, kp, acc, n_freq, ncell, total); break;
        case 4: k_pack_pair<4><<<grid, 256, 0, st>>>(j, kappa, jp, kp, acc, n_freq, ncell, total); break;
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

// ---- fixed-point accumulation: unit and conversion ----------------------------------------
// One launch clears the 8-byte accumulator and finds max|j|; the last block to finish turns it
// into the unit fix = the largest power of two with fix * per_jmax * max|j| <= 2^62, by integer
// operations on the encodings (no FP64 arithmetic beyond the one product), and resets the
// reduction words for the next call. work[0]: max|j| as float bits; work[1]: finished blocks
// (both zero before the first call).
__global__ void k_fix_prepare(const float* __restrict__ j, long long nj, unsigned long long* __restrict__ acc,
                              long long nacc, double per_jmax, unsigned* __restrict__ work, float* __restrict__ fix) {
    float m = 0.0f;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nj || i < nacc; i += stride) {
        if (i < nj) m = fmaxf(m, fabsf(__ldg(j + i)));
        if (i < nacc) acc[i] = 0ull;
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    __shared__ bool last;
    if ((threadIdx.x & 31) == 0) atomicMax(work, __float_as_uint(m));   // m >= 0: bit order = value order
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(work + 1, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last || threadIdx.x != 0) return;
    __threadfence();
    const float jmax = __uint_as_float(atomicExch(work, 0u));
    atomicExch(work + 1, 0u);
    const double bound = per_jmax * (double)jmax;
    int e = 0;   // a zero field needs no particular unit
    if (bound > 0.0) {
        // bound = 2^E (1 + f): ceil(log2 bound) = E, or E + 1 when f > 0; e = 62 - ceil(log2 bound)
        const unsigned long long bits = (unsigned long long)__double_as_longlong(bound);
        const int E = (int)((bits >> 52) & 0x7FF) - 1023;
        e = 62 - E - ((bits & 0xFFFFFFFFFFFFFull) != 0ull ? 1 : 0);
    }
    e = max(-126, min(127, e));
    *fix = __uint_as_float((unsigned)(e + 127) << 23);
}

// out[b][c] (+)= acc[b][c] / fix (the accumulator is bin-major, groups of W bins padded at the
// end): the integer is rounded once to FP32 and scaled by the power of two 1 / fix (exact)
__global__ void k_fixed_to_float(const unsigned long long* __restrict__ acc, int n_freq, long long ncell,
                                 const float* __restrict__ fix, float* __restrict__ out, int accumulate) {
    const float inv = 1.0f / *fix;
    const long long n = (long long)n_freq * ncell;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float v = __ll2float_rn((long long)acc[i]) * inv;
        out[i] = accumulate ? out[i] + v : v;
    }
}

// out[b][c] (+)= (float) (scale * acc[b][c]) (the FP64 accumulator, bin-major like the fixed-point one)
__global__ void k_f64_to_float(const double* __restrict__ acc, int n_freq, long long ncell, double scale,
                               float* __restrict__ out, int accumulate) {
    const long long n = (long long)n_freq * ncell;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float v = (float)(scale * __ldg(acc + i));
        out[i] = accumulate ? out[i] + v : v;
    }
}

cudaError_t launch_f64_to_float(const double* acc, int n_freq, long long ncell, double scale, float* out,
                                int accumulate, cudaStream_t st) {
    k_f64_to_float<<<grid_for((long long)n_freq * ncell, 256), 256, 0, st>>>(acc, n_freq, ncell, scale, out, accumulate);
    return cudaGetLastError();
}

cudaError_t launch_fix_prepare(const float* j, long long nj, unsigned long long* acc, long long nacc,
                               double per_jmax, unsigned* work, float* fix, cudaStream_t st) {
    k_fix_prepare<<<grid_for(nj > nacc ? nj : nacc, 256), 256, 0, st>>>(j, nj, acc, nacc, per_jmax, work, fix);
    return cudaGetLastError();
}

cudaError_t launch_fixed_to_float(const unsigned long long* acc, int n_freq, long long ncell, const float* fix,
                                  float* out, int accumulate, cudaStream_t st) {
    k_fixed_to_float<<<grid_for((long long)n_freq * ncell, 256), 256, 0, st>>>(acc, n_freq, ncell, fix, out, accumulate);
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
