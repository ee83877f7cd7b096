// conv3d_tc.cu -- 3x3x3 convolution ("same" zero padding, dilation d) as an implicit GEMM on the
// 5th-generation tensor cores (tcgen05.mma, BF16 operands, FP32 accumulator in tensor memory).
//
// Activations use the chunk-planar layout CP8: bf16 [batch][C/8][D][H][W][8], i.e. planes of
// 8 channels in which consecutive voxels are consecutive 16-byte rows. For one output tile of
// M = 128 voxels (two x-rows of 64 at fixed batch, z, y0) and one kernel tap (dz, dy, dx), the
// input rows the tap needs form a box (8 ch, 64 x, 2 y, 1 z, C/8 planes) of that tensor,
// shifted by (dx, dy, dz) * d. One TMA tensor load fetches it; out-of-range coordinates read
// zeros, which is exactly the convolution's zero padding. In shared memory the box is, per
// plane, 128 consecutive 16-byte rows: the canonical no-swizzle K-major operand layout (core
// matrices of 8 rows x 16 B; 128 B between row groups, one plane between K halves). So A is
// read by the tensor core straight from the TMA destination, and the 27 taps are 27 boxes.
//
// B (weights) sits in shared memory for the whole kernel as [tap][C_in/8][C_out][8] (same
// layout, N = C_out rows). Per tap: C_in/16 MMAs of M=128, N=C_out(16 or 32), K=16 into one
// TMEM accumulator of 32 columns. Roles: thread 0 of warp 0 issues TMA loads into a 4-stage
// ring, thread 0 of warp 1 issues MMAs and commits each stage back to its "empty" barrier, and
// all four warps read the accumulator (32 TMEM lanes each) for the epilogue: bias, optional
// sign mask from another activation (the LeakyReLU derivative in the backward pass), LeakyReLU,
// bf16 store in CP8 and/or an FP32 copy of channel 0.
//
// Every wait is bounded (about one second of global time): on timeout the kernel records an
// error word, stops issuing work, frees its tensor memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "rt_internal.h"

namespace rt {

namespace {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Wait until the phase with the given parity has completed; false after ~1 s.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    const uint64_t t0 = global_ns();
    for (uint32_t i = 0;; ++i) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (done) return true;
        if ((i & 63) == 63 && global_ns() - t0 > 1000000000ull) return false;
    }
}

__device__ __forceinline__ void tma_load_5d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1,
                                            int c2, int c3, int c4) {
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, "
        "%4, %5, %6}], [%7];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor, no swizzle: start address, leading (K-direction) and stride
// (M/N-direction) byte offsets between 8x16-byte core matrices; bits 46-48 hold 0b001.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both K-major (or, with
// mn_major = 1, both MN-major).
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N, int mn_major = 0) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)mn_major << 15) | ((uint32_t)mn_major << 16) |
           ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

template <int N>
__device__ __forceinline__ void tmem_load(uint32_t taddr, float* v);

template <>
__device__ __forceinline__ void tmem_load<32>(uint32_t taddr, float* v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

template <>
__device__ __forceinline__ void tmem_load<16>(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

constexpr int kStages = 4;
constexpr int kTmemCols = 32;

struct WgradArgs {
    float* dw;                        // [c_out][c_in][27], accumulated
    int B, D, H, W, c_in, c_out, dil;
    int n_tiles;
    int* err;
};

struct ConvArgs {
    const uint4* w_packed;            // [27][KC][NCO][8] bf16 in 16-byte units
    const float* bias;                // [c_out] or NULL
    const __nv_bfloat16* mask_src;    // CP8 [B][NCO/8][D][H][W][8] or NULL
    __nv_bfloat16* y;                 // CP8 [B][NCO/8][D][H][W][8] or NULL
    float* y_f32;                     // [B][D][H][W] (channel 0) or NULL
    int B, D, H, W, c_out, dil, act;
    float slope;
    int n_tiles;
    int* err;
};

constexpr int kConvThreads = 192;     // warp 0: TMA, warp 1: MMA, warps 2-5: epilogue

// The ring is as deep as shared memory allows (about 200 KB with the weights): the tap boxes
// come from L2 with microsecond latency, so the bytes in flight set the throughput.
template <int KC, int NCO>
struct ConvSmem {
    static constexpr int kWBytes = 27 * KC * NCO * 16;
    static constexpr int kWAligned = (kWBytes + 1023) / 1024 * 1024;
    static constexpr int kAStage = KC * 2048;               // KC planes x 128 rows x 16 B
    static constexpr int kStages = (200 * 1024 - kWAligned) / kAStage > 32 ? 32 : (200 * 1024 - kWAligned) / kAStage;
    static constexpr int kBarOff = kWAligned + kStages * kAStage;
    // full[S], empty[S], acc_full[2], acc_empty[2], tmem slot, abort flag
    static constexpr int kBytes = kBarOff + (2 * kStages + 4) * 8 + 16;
};

}  // namespace

// Persistent, warp-specialised: warp 0 streams the 27 tap boxes of every tile through a deep
// ring, warp 1 issues the MMAs into one of two TMEM accumulators (64 columns), and
// warps 2-5 drain the other accumulator (epilogue) meanwhile, so loads, MMAs and stores of
// consecutive tiles overlap.
template <int KC, int NCO>
__global__ void __launch_bounds__(kConvThreads, 1) k_conv3d_tc(const __grid_constant__ CUtensorMap tmap, ConvArgs a) {
    using L = ConvSmem<KC, NCO>;
    constexpr int S = L::kStages;
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* sw = smem;
    unsigned char* sa = smem + L::kWAligned;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + L::kBarOff);
    uint64_t* empty = full + S;
    uint64_t* acc_full = empty + S;
    uint64_t* acc_empty = acc_full + 2;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_empty + 2);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    // weights -> shared memory with ordinary stores, made visible to the tensor core below
    for (int i = tid; i < L::kWBytes / 16; i += kConvThreads)
        reinterpret_cast<uint4*>(sw)[i] = __ldg(a.w_packed + i);
    if (tid == 0) {
        for (int q = 0; q < S; ++q) {
            mbar_init(&full[q], 1);
            mbar_init(&empty[q], 1);
        }
        for (int q = 0; q < 2; ++q) {
            mbar_init(&acc_full[q], 1);
            mbar_init(&acc_empty[q], 128);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(2 * kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    constexpr uint32_t idesc = idesc_bf16(128, NCO);
    constexpr int KCO = NCO / 8;
    const int half_h = a.H >> 1;
    const int tiles_per_b = a.D * half_h;

    if (warp == 0) {
        if (lane == 0) {
            // producer: one TMA box per (tile, tap)
            int q = 0;
            for (int tile = blockIdx.x; tile < a.n_tiles && !*abort_flag; tile += gridDim.x) {
                const int b = tile / tiles_per_b, rem = tile - b * tiles_per_b;
                const int z = rem / half_h, y0 = 2 * (rem - (rem / half_h) * half_h);
                for (int tap = 0; tap < 27; ++tap, ++q) {
                    const int st = q % S;
                    if (!mbar_wait(&empty[st], ((uint32_t)(q / S) & 1u) ^ 1u)) {
                        *abort_flag = 1;
                        atomicExch(a.err, 1);
                        break;
                    }
                    mbar_expect_tx(&full[st], L::kAStage);
                    const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
                    tma_load_5d(sa + st * L::kAStage, &tmap, &full[st], 0, dx * a.dil, y0 + dy * a.dil,
                                z + dz * a.dil, b * KC);
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // MMA issuer: KC/2 MMAs (K = 16) per tap into accumulator t & 1
            int q = 0, t = 0;
            for (int tile = blockIdx.x; tile < a.n_tiles && !*abort_flag; tile += gridDim.x, ++t) {
                const int acc = t & 1;
                if (!mbar_wait(&acc_empty[acc], ((uint32_t)(t >> 1) & 1u) ^ 1u)) {
                    *abort_flag = 1;
                    atomicExch(a.err, 3);
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(acc * kTmemCols);
                bool ok = true;
                for (int tap = 0; tap < 27; ++tap, ++q) {
                    const int st = q % S;
                    if (!mbar_wait(&full[st], (uint32_t)(q / S) & 1u)) {
                        *abort_flag = 1;
                        atomicExch(a.err, 2);
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t abase = smem_u32(sa + st * L::kAStage);
                    const uint32_t bbase = smem_u32(sw) + (uint32_t)(tap * KC * NCO * 16);
#pragma unroll
                    for (int k = 0; k < KC / 2; ++k) {
                        const uint64_t ad = sdesc(abase + (uint32_t)(k * 2 * 2048), 2048, 128);
                        const uint64_t bd = sdesc(bbase + (uint32_t)(k * 2 * NCO * 16), NCO * 16, 128);
                        mma_bf16(d, ad, bd, idesc, (tap | k) != 0 ? 1u : 0u);
                    }
                    mma_commit(&empty[st]);
                }
                if (!ok) break;
                mma_commit(&acc_full[acc]);
            }
        }
    } else {
        // epilogue warps 2-5: warp w reads TMEM lanes 32 (w % 4) .. +31 = accumulator rows
        const int quad = warp & 3;
        const int row = quad * 32 + lane;
        const size_t plane = (size_t)a.D * a.H * a.W;
        int t = 0;
        for (int tile = blockIdx.x; tile < a.n_tiles; tile += gridDim.x, ++t) {
            const int acc = t & 1;
            const bool ready = mbar_wait(&acc_full[acc], (uint32_t)(t >> 1) & 1u);
            if (!ready || *abort_flag) {
                if (!ready) { *abort_flag = 1; atomicExch(a.err, 4); }
                break;
            }
            __syncwarp();
            tc_fence_after();
            float v[NCO];
            tmem_load<NCO>(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(acc * kTmemCols), v);
            tc_fence_before();
            mbar_arrive(&acc_empty[acc]);
            const int b = tile / tiles_per_b, rem = tile - b * tiles_per_b;
            const int z = rem / half_h, y0 = 2 * (rem - (rem / half_h) * half_h);
            const int yy = y0 + (row >> 6), xx = row & 63;
            const size_t vox = ((size_t)z * a.H + yy) * a.W + xx;
#pragma unroll
            for (int c = 0; c < NCO; ++c) {
                float x = v[c];
                if (c < a.c_out) {
                    if (a.bias) x += __ldg(a.bias + c);
                } else {
                    x = 0.0f;
                }
                v[c] = x;
            }
            if (a.mask_src) {
#pragma unroll
                for (int kc = 0; kc < KCO; ++kc) {
                    const uint4 m = __ldg(reinterpret_cast<const uint4*>(a.mask_src) +
                                          ((size_t)(b * KCO + kc) * plane + vox));
                    const __nv_bfloat16* mb = reinterpret_cast<const __nv_bfloat16*>(&m);
#pragma unroll
                    for (int e = 0; e < 8; ++e)
                        if (!(__bfloat162float(mb[e]) > 0.0f)) v[kc * 8 + e] *= a.slope;
                }
            }
            if (a.act == 1) {
#pragma unroll
                for (int c = 0; c < NCO; ++c) v[c] = v[c] > 0.0f ? v[c] : a.slope * v[c];
            }
            if (a.y) {
#pragma unroll
                for (int kc = 0; kc < KCO; ++kc) {
                    uint4 o;
                    __nv_bfloat162* ob = reinterpret_cast<__nv_bfloat162*>(&o);
#pragma unroll
                    for (int e = 0; e < 4; ++e) ob[e] = __floats2bfloat162_rn(v[kc * 8 + 2 * e], v[kc * 8 + 2 * e + 1]);
                    reinterpret_cast<uint4*>(a.y)[(size_t)(b * KCO + kc) * plane + vox] = o;
                }
            }
            if (a.y_f32) a.y_f32[(size_t)b * plane + vox] = v[0];
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * kTmemCols)
                     : "memory");
    }
}

// ---- weight gradient ------------------------------------------------------------------------
// dW[co][ci][tap] = sum over voxels v of dZ[v][co] * X[v + off(tap)][ci] (zero outside). As a
// GEMM: M = (tap, ci) rows, N = co, K = voxels. Both operands are the CP8 boxes the forward
// kernel loads, read MN-major (for a fixed voxel, 8 consecutive channels are one 16-byte row):
// A = G taps' input boxes stored back to back, so the 8-channel core matrices of all G * 8 * KC
// rows are uniformly 2048 bytes apart (G = 128 / (8 KC)); B = the dZ box of the tile. Each CTA
// accumulates its share of tiles in tensor memory (one 128 x NCO accumulator per tap group) and
// adds the result to dW once, with FP32 atomics.

namespace {
template <int KC>
struct WgradSmem {
    static constexpr int kBox = KC * 2048;                  // one tap box (128 voxels, KC planes)
    static constexpr int kG = 128 / (8 * KC);               // taps per group
    static constexpr int kGroups = (27 + kG - 1) / kG;
    static constexpr int kGroupBytes = kG * kBox;           // 32 KB
    static constexpr int kZBytes = 4 * 2048;                // dZ box (up to 4 planes)
    static constexpr int kBarOff = 2 * kGroupBytes + kZBytes;
    static constexpr int kBytes = kBarOff + 6 * 8 + 16;
};
}  // namespace

template <int KC, int NCO>
__global__ void __launch_bounds__(128, 1) k_conv3d_wgrad(const __grid_constant__ CUtensorMap tmap_x,
                                                         const __grid_constant__ CUtensorMap tmap_dz, WgradArgs a) {
    using L = WgradSmem<KC>;
    constexpr int KCO = NCO / 8;
    constexpr int kCols = (L::kGroups * NCO) <= 128 ? 128 : 256;
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* sg = smem;                                   // two group buffers
    unsigned char* sz = smem + 2 * L::kGroupBytes;              // dZ box
    uint64_t* gfull = reinterpret_cast<uint64_t*>(smem + L::kBarOff);   // [2]
    uint64_t* gempty = gfull + 2;                                       // [2]
    uint64_t* zfull = gempty + 2;
    uint64_t* zempty = zfull + 1;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(zempty + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (tid == 0) {
        for (int i = 0; i < 2; ++i) { mbar_init(&gfull[i], 1); mbar_init(&gempty[i], 1); }
        mbar_init(zfull, 1);
        mbar_init(zempty, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    constexpr uint32_t idesc = idesc_bf16(128, NCO, 1);

    const int half_h = a.H >> 1;
    const int tiles_per_b = a.D * half_h;
    const int t_begin = (int)((long long)a.n_tiles * blockIdx.x / gridDim.x);
    const int t_end = (int)((long long)a.n_tiles * (blockIdx.x + 1) / gridDim.x);
    int done_tiles = 0;
    if (warp == 0 && lane == 0) {
        // producer: per tile, the dZ box, then the tap groups through two group buffers
        int gq = 0;
        for (int tile = t_begin; tile < t_end && !*abort_flag; ++tile, ++done_tiles) {
            const int b = tile / tiles_per_b, rem = tile - b * tiles_per_b;
            const int z = rem / half_h, y0 = 2 * (rem - (rem / half_h) * half_h);
            if (!mbar_wait(zempty, ((uint32_t)done_tiles & 1u) ^ 1u)) { *abort_flag = 1; atomicExch(a.err, 4); break; }
            mbar_expect_tx(zfull, KCO * 2048);
            tma_load_5d(sz, &tmap_dz, zfull, 0, 0, y0, z, b * KCO);
            for (int g = 0; g < L::kGroups; ++g, ++gq) {
                const int buf = gq & 1;
                if (!mbar_wait(&gempty[buf], ((uint32_t)(gq >> 1) & 1u) ^ 1u)) { *abort_flag = 1; atomicExch(a.err, 5); break; }
                const int ntap = min(L::kG, 27 - g * L::kG);
                mbar_expect_tx(&gfull[buf], ntap * L::kBox);
                for (int t = 0; t < ntap; ++t) {
                    const int tap = g * L::kG + t;
                    const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
                    tma_load_5d(sg + buf * L::kGroupBytes + t * L::kBox, &tmap_x, &gfull[buf], 0, dx * a.dil,
                                y0 + dy * a.dil, z + dz * a.dil, b * KC);
                }
            }
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer: 8 MMAs (K = 16 voxels each) per tap group and tile
        int gq = 0;
        for (int tile = t_begin; tile < t_end && !*abort_flag; ++tile, ++done_tiles) {
            if (!mbar_wait(zfull, (uint32_t)done_tiles & 1u)) { *abort_flag = 1; atomicExch(a.err, 6); break; }
            const uint32_t zb = smem_u32(sz);
            for (int g = 0; g < L::kGroups; ++g, ++gq) {
                const int buf = gq & 1;
                if (!mbar_wait(&gfull[buf], (uint32_t)(gq >> 1) & 1u)) { *abort_flag = 1; atomicExch(a.err, 7); break; }
                tc_fence_after();
                const uint32_t ab = smem_u32(sg + buf * L::kGroupBytes);
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    // MN-major: leading (K) offset 128 B = 8 voxels, stride (MN) offset 2048 B = 8 channels
                    const uint64_t ad = sdesc(ab + (uint32_t)(k * 256), 128, 2048);
                    const uint64_t bd = sdesc(zb + (uint32_t)(k * 256), 128, 2048);
                    mma_bf16(tmem + (uint32_t)(g * NCO), ad, bd, idesc, (tile != t_begin || k != 0) ? 1u : 0u);
                }
                mma_commit(&gempty[buf]);
            }
            mma_commit(zempty);
        }
    }
    __syncthreads();
    // Wait for the last MMAs: the dZ-box barrier's phase of the last tile completes only when
    // every earlier MMA has. It lags by at most one phase here (the producer waited on the one
    // before), so the parity test is unambiguous.
    const int ntile = t_end - t_begin;
    bool ok = !*abort_flag;
    if (ok && ntile > 0) ok = mbar_wait(zempty, (uint32_t)(ntile - 1) & 1u);
    if (!ok) { *abort_flag = 1; atomicExch(a.err, 8); }
    tc_fence_after();
    if (ok && ntile > 0) {
        // row m = warp * 32 + lane -> (tap within group, input channel)
        const int m = warp * 32 + lane;
        const int tl = m / (8 * KC), ci = m % (8 * KC);
        for (int g = 0; g < L::kGroups; ++g) {
            float v[NCO];
            tmem_load<NCO>(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(g * NCO), v);
            const int tap = g * L::kG + tl;
            if (tap < 27 && ci < a.c_in) {
#pragma unroll
                for (int co = 0; co < NCO; ++co)
                    if (co < a.c_out) atomicAdd(a.dw + ((size_t)co * a.c_in + ci) * 27 + tap, v[co]);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols) : "memory");
    }
}

// ---- host side -----------------------------------------------------------------------------

namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

template <int KC, int NCO>
cudaError_t launch_one(const ConvLaunch& c, cudaStream_t st) {
    using L = ConvSmem<KC, NCO>;
    auto fn = encode_fn();
    if (!fn) return cudaErrorNotSupported;
    CUtensorMap map;
    const cuuint64_t dims[5] = {8, (cuuint64_t)c.W, (cuuint64_t)c.H, (cuuint64_t)c.D, (cuuint64_t)c.B * KC};
    const cuuint64_t strides[4] = {16, 16ull * c.W, 16ull * c.W * c.H, 16ull * c.W * c.H * c.D};
    const cuuint32_t box[5] = {8, 64, 2, 1, (cuuint32_t)KC};
    const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    if (fn(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void*>(c.x), dims, strides, box, estr,
           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_conv3d_tc<KC, NCO>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             L::kBytes);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    ConvArgs a{};
    a.w_packed = reinterpret_cast<const uint4*>(c.w_packed);
    a.bias = c.bias;
    a.mask_src = reinterpret_cast<const __nv_bfloat16*>(c.mask_src);
    a.y = reinterpret_cast<__nv_bfloat16*>(c.y);
    a.y_f32 = c.y_f32;
    a.B = c.B; a.D = c.D; a.H = c.H; a.W = c.W;
    a.c_out = c.c_out;
    a.dil = c.dil;
    a.act = c.act;
    a.slope = c.slope;
    a.n_tiles = c.B * c.D * (c.H / 2);
    a.err = c.err;
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int grid = sms;
    if (grid > a.n_tiles) grid = a.n_tiles;
    if (grid < 1) return cudaSuccess;
    k_conv3d_tc<KC, NCO><<<grid, kConvThreads, L::kBytes, st>>>(map, a);
    return cudaGetLastError();
}

bool make_map(CUtensorMap* map, const void* base, int B, int planes, int D, int H, int W) {
    auto fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[5] = {8, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)D, (cuuint64_t)B * planes};
    const cuuint64_t strides[4] = {16, 16ull * W, 16ull * W * H, 16ull * W * H * D};
    const cuuint32_t box[5] = {8, 64, 2, 1, (cuuint32_t)planes};
    const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void*>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int KC, int NCO>
cudaError_t launch_wgrad_one(const WgradLaunch& c, cudaStream_t st) {
    using L = WgradSmem<KC>;
    CUtensorMap mx, mz;
    if (!make_map(&mx, c.x, c.B, KC, c.D, c.H, c.W) || !make_map(&mz, c.dz, c.B, NCO / 8, c.D, c.H, c.W))
        return cudaErrorInvalidValue;
    // at most two CTAs per SM: each holds up to 256 tensor-memory columns of the SM's 512
    const int bytes = L::kBytes < 100 * 1024 ? 100 * 1024 : L::kBytes;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_conv3d_wgrad<KC, NCO>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    WgradArgs a{};
    a.dw = c.dw;
    a.B = c.B; a.D = c.D; a.H = c.H; a.W = c.W;
    a.c_in = c.c_in; a.c_out = c.c_out; a.dil = c.dil;
    a.n_tiles = c.B * c.D * (c.H / 2);
    a.err = c.err;
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int grid = 2 * sms;
    if (grid > a.n_tiles) grid = a.n_tiles;
    if (grid < 1) return cudaSuccess;
    k_conv3d_wgrad<KC, NCO><<<grid, 128, bytes, st>>>(mx, mz, a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_conv3d_wgrad(const WgradLaunch& c, cudaStream_t st) {
    if (c.W != 64 || c.H % 2 != 0 || c.B < 1 || c.D < 1 || c.H < 2) return cudaErrorInvalidValue;
    if (c.kc_in == 4 && c.nco == 32) return launch_wgrad_one<4, 32>(c, st);
    if (c.kc_in == 2 && c.nco == 32) return launch_wgrad_one<2, 32>(c, st);
    if (c.kc_in == 4 && c.nco == 16) return launch_wgrad_one<4, 16>(c, st);
    if (c.kc_in == 2 && c.nco == 16) return launch_wgrad_one<2, 16>(c, st);
    return cudaErrorInvalidValue;
}

cudaError_t launch_conv3d_tc(const ConvLaunch& c, cudaStream_t st) {
    if (c.W != 64 || c.H % 2 != 0 || c.B < 1 || c.D < 1 || c.H < 2) return cudaErrorInvalidValue;
    if (c.kc_in == 2 && c.nco == 32) return launch_one<2, 32>(c, st);
    if (c.kc_in == 4 && c.nco == 32) return launch_one<4, 32>(c, st);
    if (c.kc_in == 4 && c.nco == 16) return launch_one<4, 16>(c, st);
    if (c.kc_in == 2 && c.nco == 16) return launch_one<2, 16>(c, st);
    return cudaErrorInvalidValue;
}

}  // namespace rt
