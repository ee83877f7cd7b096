// conv3d_tc.cu -- 3x3x3 convolution ("same" zero padding, dilation d) as an implicit GEMM on the
// 5th-generation tensor cores (tcgen05.mma, BF16 operands, FP32 accumulator in tensor memory).
//
// Activations use the C32 layout: bf16 [batch][D][H][W][32] -- 32 channels (64 bytes) per voxel,
// unused channels zero. For one output tile of M = 128 voxels (two x-rows of 64 at fixed batch,
// z, y0) and one kernel tap (dz, dy, dx), the input rows the tap needs form a box (32 ch, 64 x,
// 2 y, 1 z, 1 batch) shifted by (dx, dy, dz) * d. One TMA tensor load fetches it; out-of-range
// coordinates read zeros, which is exactly the convolution's zero padding, and the TMA's 64-byte
// swizzle lays the box out as the canonical SW64 K-major operand (8-row atoms of 512 bytes): the
// tensor core reads A straight from the TMA destination, K = 32 channels = two MMAs of K = 16.
// B (weights) sits in shared memory for the whole kernel as [tap][32 out][32 in] in the same
// swizzled layout. The forward kernel walks chains of output slices along z so that each box
// serves the three outputs that need it; the weight gradient reads the same boxes MN-major.
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

// Bring a box into L2 ahead of its load (no shared memory, no completion to wait for).
__device__ __forceinline__ void tma_prefetch_5d(const CUtensorMap* map, int c0, int c1, int c2, int c3, int c4) {
    asm volatile("cp.async.bulk.prefetch.tensor.5d.L2.global.tile [%0, {%1, %2, %3, %4, %5}];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4)
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor with 64-byte swizzling (layout type 4 in bits 61-63): start
// address, leading and stride byte offsets; bits 46-48 hold 0b001. K-major: SBO = 512 bytes
// between 8-row atoms (LBO unused). MN-major: LBO between 32-element MN blocks, SBO between
// 8-row K blocks.
__device__ __forceinline__ uint64_t sdesc_sw64(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)4 << 61;
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

// Write zeros to 32 columns of the warp's 32 tensor-memory lanes starting at taddr.
__device__ __forceinline__ void tmem_zero32(uint32_t taddr) {
    const uint32_t z = 0u;
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, "
        "%1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1};" ::"r"(taddr),
        "r"(z)
        : "memory");
}

constexpr int kTmemCols = 32;
constexpr int kBox = 128 * 64;             // one tap box: 128 voxels x 32 channels x 2 bytes
constexpr int kWBytes = 27 * 32 * 64;      // weights: 27 taps x 32 outputs x 64-byte rows
constexpr int kConvThreads = 192;          // warp 0: TMA, warp 1: MMA, warps 2-5: epilogue
struct ConvArgs {
    const uint4* w_packed;            // [27][32][32] bf16 (tap, out, in) in 16-byte units
    const float* bias;                // [c_out] or NULL
    const __nv_bfloat16* mask_src;    // C32 [B][D][H][W][32] or NULL
    __nv_bfloat16* y;                 // C32 or NULL
    float* y_f32;                     // [B][D][H][W] (channel 0) or NULL
    int B, D, H, W, c_out, dil, act;
    float slope;
    int* err;
};

struct WgradArgs {
    float* dw;                        // [c_out][c_in][27], accumulated
    int B, D, H, W, c_in, c_out, dil;
    int* err;
};

// byte offset of 16-byte chunk c of row r in a 64-byte-swizzled block (atoms of 8 rows)
__device__ __forceinline__ int sw64(int r, int c) { return r * 64 + ((c ^ ((r >> 1) & 3)) << 4); }

}  // namespace

// ---- forward, chained along z ------------------------------------------------------------
// An output slice z takes the input slices z - d, z, z + d. Along a chain of outputs r, r + d,
// r + 2d, ... (fixed batch, y-pair and residue r = z mod d) consecutive outputs share input
// slices, so each input box (slice z', dy, dx) is loaded once and feeds the three outputs it
// belongs to (dz = -1, 0, +1, with the weights of tap (dz, dy, dx)). A work item is a chain
// segment of at most kChainMax outputs; its inputs are the segment's slices plus one on each
// side (those outside the volume are zero padding and skipped). A ring stage carries the three
// dx boxes of one (input slice, dy). The weights sit in shared memory with the three dz taps of
// each (dy, dx) back to back in the order dz = +1, 0, -1, and each output of the segment has its
// own 32-column TMEM accumulator at its position in the segment, so the outputs an input feeds
// (positions i - 1, i, i + 1 for dz = +1, 0, -1) are adjacent columns and adjacent weight rows:
// one MMA of N = 96 (64 or 32 at the ends of the segment) per dx box and K half, 6 per stage,
// reads the box once for all three outputs. Since such an MMA accumulates into two outputs that
// are under way and one that is fresh, the accumulators are zero beforehand: the epilogue warps
// clear each accumulator when they drain it (and all of them at the start). Per output tile ~11
// boxes are loaded instead of 27.
namespace {
#ifndef RT_CHAIN_MAX
#define RT_CHAIN_MAX 8
#endif
constexpr int kChainMax = RT_CHAIN_MAX;   // outputs per work item
constexpr int kChainSlots = kChainMax;   // one accumulator per output position of a segment
#ifndef RT_CHAIN_CTAS
#define RT_CHAIN_CTAS 2
#endif
constexpr int kChainCtas = RT_CHAIN_CTAS;
constexpr int kChainStageBytes = 3 * kBox;
constexpr int kChainStages = ((228 * 1024) / kChainCtas - 1024 - kWBytes - 512) / kChainStageBytes;
static_assert(kChainStages >= 2, "chain ring");
constexpr int kChainBarOff = kWBytes + kChainStages * kChainStageBytes;
constexpr int kChainBytes = kChainBarOff + (2 * kChainStages + 2 * kChainSlots + 1) * 8 + 16;

struct ChainItem {
    int b, y0, r, n0, n1;   // outputs z = r + n * dil for n in [n0, n1)
};

// Items ordered (batch, segment, residue, y-pair), y-pair fastest: neighbouring items share halo rows.
__device__ __forceinline__ bool chain_item(int H, int D, int dil, int item, int Q, ChainItem& it) {
    const int half_h = H >> 1;
    int t = item;
    const int p = t % half_h;
    t /= half_h;
    const int r = t % dil;
    t /= dil;
    const int q = t % Q;
    it.b = t / Q;
    it.y0 = 2 * p;
    it.r = r;
    const int lc = (D - r + dil - 1) / dil;   // outputs of residue r (0 when r >= D)
    it.n0 = q * kChainMax;
    it.n1 = min(lc, it.n0 + kChainMax);
    return it.n0 < it.n1;
}
__device__ __forceinline__ bool chain_item(const ConvArgs& a, int item, int Q, ChainItem& it) {
    return chain_item(a.H, a.D, a.dil, item, Q, it);
}
}  // namespace

__global__ void __launch_bounds__(kConvThreads, kChainCtas) k_conv3d_chain(const __grid_constant__ CUtensorMap tmap,
                                                                           ConvArgs a, int n_items, int Q) {
    constexpr int S = kChainStages;
    constexpr int NS = kChainSlots;
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* sw = smem;
    unsigned char* sa = smem + kWBytes;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + kChainBarOff);
    uint64_t* empty = full + S;
    uint64_t* acc_full = empty + S;
    uint64_t* acc_empty = acc_full + NS;
    uint64_t* mma_done = acc_empty + NS;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mma_done + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (smem_u32(smem) & 1023u) {
        if (tid == 0) atomicExch(a.err, 10);
        return;
    }
    for (int i = tid; i < kWBytes / 16; i += kConvThreads) {
        // packed tap (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1) goes to block ((dy + 1) * 3 + dx + 1) * 3 + (1 - dz)
        const int c = i & 3, r = (i >> 2) & 31, tap = i >> 7;
        const int pos = (tap % 9) * 3 + (2 - tap / 9);
        *reinterpret_cast<uint4*>(sw + pos * 2048 + sw64(r, c)) = __ldg(a.w_packed + i);
    }
    if (tid == 0) {
        for (int q = 0; q < S; ++q) {
            mbar_init(&full[q], 1);
            mbar_init(&empty[q], 1);
        }
        for (int q = 0; q < NS; ++q) {
            mbar_init(&acc_full[q], 1);
            mbar_init(&acc_empty[q], 128);
        }
        mbar_init(mma_done, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(NS * kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    if (warp >= 2) {   // the MMAs accumulate from the start: clear every accumulator first
        const uint32_t lanes = (uint32_t)((warp & 3) * 32) << 16;
#pragma unroll
        for (int j = 0; j < NS; ++j) tmem_zero32(tmem + lanes + (uint32_t)(j * kTmemCols));
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();

    if (warp == 0) {
        if (lane == 0) {
            int q = 0;
            for (int item = blockIdx.x; item < n_items && !*abort_flag; item += gridDim.x) {
                ChainItem it;
                if (!chain_item(a, item, Q, it)) continue;
                for (int i = it.n0 - 1; i <= it.n1 && !*abort_flag; ++i) {
                    const int zi = it.r + i * a.dil;
                    if (zi < 0 || zi >= a.D) continue;
                    for (int dy = -1; dy <= 1; ++dy, ++q) {
                        const int st = q % S;
                        if (!mbar_wait(&empty[st], ((uint32_t)(q / S) & 1u) ^ 1u)) {
                            *abort_flag = 1;
                            atomicExch(a.err, 1);
                            break;
                        }
                        mbar_expect_tx(&full[st], kChainStageBytes);
#pragma unroll
                        for (int u = 0; u < 3; ++u)
                            tma_load_5d(sa + st * kChainStageBytes + u * kBox, &tmap, &full[st], 0, (u - 1) * a.dil,
                                        it.y0 + dy * a.dil, zi, it.b);
                    }
                }
            }
            for (int p = q > S ? q - S : 0; p < q; ++p) mbar_wait(&full[p % S], (uint32_t)(p / S) & 1u);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            int q = 0;
            uint32_t phase = 0;   // bit j: parity of accumulator j's next acc_empty wait, flipped per use
            bool ok = true;
            for (int item = blockIdx.x; item < n_items && ok && !*abort_flag; item += gridDim.x) {
                ChainItem it;
                if (!chain_item(a, item, Q, it)) continue;
                int started = it.n0;   // outputs [n0, started) have their accumulators
                for (int i = it.n0 - 1; i <= it.n1 && ok; ++i) {
                    const int zi = it.r + i * a.dil;
                    if (zi >= 0 && zi < a.D) {
                        // outputs fed by this input: i - 1 (dz = +1), i (dz = 0), i + 1 (dz = -1)
                        const int lo = max(i - 1, it.n0), hi = min(i + 1, it.n1 - 1);
                        for (; started <= hi && ok; ++started) {
                            const int j = started - it.n0;
                            if (!mbar_wait(&acc_empty[j], ((phase >> j) & 1u) ^ 1u)) {
                                *abort_flag = 1;
                                atomicExch(a.err, 3);
                                ok = false;
                            }
                            phase ^= 1u << j;
                        }
                        if (!ok) break;
                        tc_fence_after();
                        const int cnt = hi - lo + 1;
                        const uint32_t idesc = cnt == 3 ? idesc_bf16(128, 96)
                                               : (cnt == 2 ? idesc_bf16(128, 64) : idesc_bf16(128, 32));
                        const uint32_t d = tmem + (uint32_t)((lo - it.n0) * kTmemCols);
                        const int block0 = 1 - (i - lo);   // weight block of output lo: dz = i - lo
                        for (int dy = -1; dy <= 1; ++dy, ++q) {
                            const int st = q % S;
                            if (!mbar_wait(&full[st], (uint32_t)(q / S) & 1u)) {
                                *abort_flag = 1;
                                atomicExch(a.err, 2);
                                ok = false;
                                break;
                            }
                            tc_fence_after();
                            const uint32_t sbase = smem_u32(sa + st * kChainStageBytes);
#pragma unroll
                            for (int u = 0; u < 3; ++u) {
                                const int pos = ((dy + 1) * 3 + u) * 3 + block0;
                                const uint32_t abase = sbase + (uint32_t)(u * kBox);
                                const uint32_t bbase = smem_u32(sw) + (uint32_t)(pos * 2048);
#pragma unroll
                                for (int k = 0; k < 2; ++k) {
                                    const uint64_t ad = sdesc_sw64(abase + (uint32_t)(k * 32), 16, 512);
                                    const uint64_t bd = sdesc_sw64(bbase + (uint32_t)(k * 32), 16, 512);
                                    mma_bf16(d, ad, bd, idesc, 1u);
                                }
                            }
                            mma_commit(&empty[st]);
                        }
                        if (!ok) break;
                    }
                    // after input i, output i - 1 has all its contributions
                    if (i - 1 >= it.n0 && i - 1 < it.n1) mma_commit(&acc_full[i - 1 - it.n0]);
                }
            }
            mma_commit(mma_done);
        }
    } else {
        const int quad = warp & 3;
        const int row = quad * 32 + lane;
        uint32_t phase = 0;   // bit j: parity of accumulator j's next acc_full wait
        bool live = true;
        for (int item = blockIdx.x; item < n_items && live; item += gridDim.x) {
            ChainItem it;
            if (!chain_item(a, item, Q, it)) continue;
            for (int n = it.n0; n < it.n1; ++n) {
                const int slot = n - it.n0;
                const bool ready = mbar_wait(&acc_full[slot], (phase >> slot) & 1u);
                phase ^= 1u << slot;
                if (!ready || *abort_flag) {
                    if (!ready) { *abort_flag = 1; atomicExch(a.err, 4); }
                    live = false;
                    break;
                }
                __syncwarp();
                tc_fence_after();
                float v[32];
                const uint32_t taddr = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(slot * kTmemCols);
                tmem_load<32>(taddr, v);
                tmem_zero32(taddr);   // the next segment's MMAs accumulate onto zero
                asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                tc_fence_before();
                mbar_arrive(&acc_empty[slot]);
                const int z = it.r + n * a.dil;
                const int yy = it.y0 + (row >> 6), xx = row & 63;
                const size_t vox = (((size_t)it.b * a.D + z) * a.H + yy) * a.W + xx;
#pragma unroll
                for (int c = 0; c < 32; ++c) {
                    float x = v[c];
                    if (c < a.c_out) {
                        if (a.bias) x += __ldg(a.bias + c);
                    } else {
                        x = 0.0f;
                    }
                    v[c] = x;
                }
                if (a.mask_src) {
                    const uint4* mp = reinterpret_cast<const uint4*>(a.mask_src) + vox * 4;
#pragma unroll
                    for (int q4 = 0; q4 < 4; ++q4) {
                        const uint4 m = __ldg(mp + q4);
                        const __nv_bfloat16* mb = reinterpret_cast<const __nv_bfloat16*>(&m);
#pragma unroll
                        for (int e = 0; e < 8; ++e)
                            if (!(__bfloat162float(mb[e]) > 0.0f)) v[q4 * 8 + e] *= a.slope;
                    }
                }
                if (a.act == 1) {
#pragma unroll
                    for (int c = 0; c < 32; ++c) v[c] = v[c] > 0.0f ? v[c] : a.slope * v[c];
                }
                if (a.y) {
                    uint4* yp = reinterpret_cast<uint4*>(a.y) + vox * 4;
#pragma unroll
                    for (int q4 = 0; q4 < 4; ++q4) {
                        uint4 o;
                        __nv_bfloat162* ob = reinterpret_cast<__nv_bfloat162*>(&o);
#pragma unroll
                        for (int e = 0; e < 4; ++e) ob[e] = __floats2bfloat162_rn(v[q4 * 8 + 2 * e], v[q4 * 8 + 2 * e + 1]);
                        yp[q4] = o;
                    }
                }
                if (a.y_f32) a.y_f32[vox] = v[0];
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        if (!mbar_wait(mma_done, 0) && lane == 0) atomicExch(a.err, 11);
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NS * kTmemCols)
                     : "memory");
    }
}

// ---- weight gradient, chained along z -------------------------------------------------------
// dW[co][ci][tap] = sum over voxels v of dZ[v][co] * X[v + off(tap)][ci] (zero outside). As a
// GEMM: M = (tap, ci) rows, N = co, K = voxels, both operands read MN-major from the boxes the
// forward loads (for a fixed voxel the 32 channels are one 64-byte swizzled row). The work items
// are the forward's chain segments: outputs z = r + n d (n in [n0, n1)) at a fixed batch and
// y-pair. The input box of slice z' = r + i d and offset (dy, dx) pairs voxel for voxel with the
// dZ box of output n = i - 1 + j for j = 0, 1, 2 (tap dz = 1 - j), so it is loaded once per
// slice for the three outputs instead of once per (output, tap). A ring stage holds one group of
// four input boxes (the nine (dy, dx) offsets make groups of 4, 4 and 1; the last group's other
// three box slots hold stale data whose accumulator rows are never read); the segment's dZ boxes
// pass through a ring of four slots, the boxes of slots 0 and 1 also written to mirror slots 4
// and 5, so the (up to) three boxes a slice pairs with, starting at any slot, are consecutive in
// shared memory: one MMA of N = 96 (64 or
// 32 at the ends of a segment) per group and K step reads them all. Per (group, j) one 128 x 32
// accumulator in tensor memory (9 of them, adjacent in j) sums over every item of the CTA; the
// CTA adds them to dW once, with FP32 atomics. Per output tile ~12 boxes are loaded instead of 28.

namespace {
constexpr int kWcStageBytes = 4 * kBox;    // one group of four input boxes, 32 KB
constexpr int kWcStages = 5;
constexpr int kWcZSlots = 4;               // ring positions, plus mirrors of slots 0 and 1
constexpr int kWcZOff = kWcStages * kWcStageBytes;
constexpr int kWcBarOff = kWcZOff + (kWcZSlots + 2) * kBox;
constexpr int kWcBytes = kWcBarOff + (2 * kWcStages + 2 * kWcZSlots + 1) * 8 + 16;
constexpr int kWcCols = 512;               // 9 accumulators x 32 columns, rounded up to a power of two
static_assert(kWcBytes <= 227 * 1024, "weight-gradient shared memory");
}  // namespace

__global__ void __launch_bounds__(128, 1) k_conv3d_wgrad(const __grid_constant__ CUtensorMap tmap_x,
                                                         const __grid_constant__ CUtensorMap tmap_dz, WgradArgs a,
                                                         int n_items, int Q) {
    constexpr int S = kWcStages, ZS = kWcZSlots;
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* sa = smem;                                   // input stages
    unsigned char* sz = smem + kWcZOff;                         // dZ slots and their mirrors
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + kWcBarOff);
    uint64_t* empty = full + S;
    uint64_t* zfull = empty + S;
    uint64_t* zempty = zfull + ZS;
    uint64_t* mma_done = zempty + ZS;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mma_done + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (smem_u32(smem) & 1023u) {
        if (tid == 0) atomicExch(a.err, 10);
        return;
    }
    if (tid == 0) {
        for (int i = 0; i < S; ++i) { mbar_init(&full[i], 1); mbar_init(&empty[i], 1); }
        for (int i = 0; i < ZS; ++i) { mbar_init(&zfull[i], 1); mbar_init(&zempty[i], 1); }
        mbar_init(mma_done, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kWcCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    {   // every MMA accumulates: clear the nine accumulators (each warp its 32 lanes)
        const uint32_t lanes = (uint32_t)(warp * 32) << 16;
#pragma unroll
        for (int c = 0; c < 9; ++c) tmem_zero32(tmem + lanes + (uint32_t)(c * 32));
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();

    if (warp == 0 && lane == 0) {
        // producer: per input slice i, the dZ box of output i + 1 (its first use), then the
        // slice's three groups of input boxes
        int q = 0, zt = 0;
        for (int item = blockIdx.x; item < n_items && !*abort_flag; item += gridDim.x) {
            ChainItem it;
            if (!chain_item(a.H, a.D, a.dil, item, Q, it)) continue;
            for (int i = it.n0 - 1; i <= it.n1 && !*abort_flag; ++i) {
                if (i + 1 >= it.n0 && i + 1 < it.n1) {
                    const int slot = zt % ZS;
                    if (!mbar_wait(&zempty[slot], ((uint32_t)(zt / ZS) & 1u) ^ 1u)) {
                        *abort_flag = 1;
                        atomicExch(a.err, 5);
                        break;
                    }
                    mbar_expect_tx(&zfull[slot], (slot < 2 ? 2 : 1) * kBox);
                    const int zo = it.r + (i + 1) * a.dil;
                    tma_load_5d(sz + slot * kBox, &tmap_dz, &zfull[slot], 0, 0, it.y0, zo, it.b);
                    if (slot < 2) tma_load_5d(sz + (slot + ZS) * kBox, &tmap_dz, &zfull[slot], 0, 0, it.y0, zo, it.b);
                    ++zt;
                }
                // L2 prefetch two slices ahead (the three dy rows; dx only shifts x) and of the dZ
                // box loaded then: their loads find them in L2 instead of waiting on DRAM
                const int zp = it.r + (i + 2) * a.dil;
                if (i + 2 <= it.n1 && zp < a.D) {
                    for (int dy = -1; dy <= 1; ++dy) {
                        const int yp = it.y0 + dy * a.dil;   // whole boxes inside the volume only
                        if (yp >= 0 && yp + 2 <= a.H) tma_prefetch_5d(&tmap_x, 0, 0, yp, zp, it.b);
                    }
                    if (i + 3 < it.n1) tma_prefetch_5d(&tmap_dz, 0, 0, it.y0, it.r + (i + 3) * a.dil, it.b);
                }
                const int zi = it.r + i * a.dil;
                if (zi < 0 || zi >= a.D) continue;
                for (int g = 0; g < 3; ++g, ++q) {
                    const int st = q % S;
                    if (!mbar_wait(&empty[st], ((uint32_t)(q / S) & 1u) ^ 1u)) {
                        *abort_flag = 1;
                        atomicExch(a.err, 6);
                        break;
                    }
                    const int nb = g < 2 ? 4 : 1;
                    mbar_expect_tx(&full[st], nb * kBox);
                    for (int u = 0; u < nb; ++u) {
                        const int p = 4 * g + u, dy = p / 3 - 1, dx = p % 3 - 1;
                        tma_load_5d(sa + st * kWcStageBytes + u * kBox, &tmap_x, &full[st], 0, dx * a.dil,
                                    it.y0 + dy * a.dil, zi, it.b);
                    }
                }
            }
        }
        // let the last loads land before the block can exit
        for (int p = q > S ? q - S : 0; p < q; ++p) mbar_wait(&full[p % S], (uint32_t)(p / S) & 1u);
        for (int p = zt > ZS ? zt - ZS : 0; p < zt; ++p) mbar_wait(&zfull[p % ZS], (uint32_t)(p / ZS) & 1u);
    } else if (warp == 1 && lane == 0) {
        // MMA issuer: for input slice i and group g, the outputs i - 1 + j (j = 0, 1, 2) of the
        // segment, each into accumulator g * 3 + j; the dZ box of output n is released after
        // slice n + 1, its last use
        int q = 0, zt = 0;
        bool ok = true;
        for (int item = blockIdx.x; item < n_items && ok && !*abort_flag; item += gridDim.x) {
            ChainItem it;
            if (!chain_item(a.H, a.D, a.dil, item, Q, it)) continue;
            const int t0 = zt;   // ring index of output n0's dZ box
            for (int i = it.n0 - 1; i <= it.n1 && ok; ++i) {
                if (i + 1 >= it.n0 && i + 1 < it.n1) {
                    const int t = t0 + (i + 1 - it.n0);
                    if (!mbar_wait(&zfull[t % ZS], (uint32_t)(t / ZS) & 1u)) {
                        *abort_flag = 1;
                        atomicExch(a.err, 7);
                        ok = false;
                        break;
                    }
                }
                const int zi = it.r + i * a.dil;
                if (zi >= 0 && zi < a.D) {
                    for (int g = 0; g < 3; ++g, ++q) {
                        const int st = q % S;
                        if (!mbar_wait(&full[st], (uint32_t)(q / S) & 1u)) {
                            *abort_flag = 1;
                            atomicExch(a.err, 8);
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t ab = smem_u32(sa + st * kWcStageBytes);
                        // outputs i - 1 + j, j in [jl, jh], within the segment
                        const int jl = max(0, it.n0 - (i - 1)), jh = min(2, it.n1 - 1 - (i - 1));
                        const int cnt = jh - jl + 1;
                        const uint32_t idesc = cnt == 3 ? idesc_bf16(128, 96, 1)
                                               : (cnt == 2 ? idesc_bf16(128, 64, 1) : idesc_bf16(128, 32, 1));
                        const uint32_t zb = smem_u32(sz + ((t0 + (i - 1 + jl) - it.n0) % ZS) * kBox);
                        const uint32_t d = tmem + (uint32_t)((g * 3 + jl) * 32);
#pragma unroll
                        for (int k = 0; k < 8; ++k) {
                            // MN-major SW64: K = 16 voxels = two 8-row blocks (1 KB); MN blocks 8 KB apart
                            const uint64_t ad = sdesc_sw64(ab + (uint32_t)(k * 1024), kBox, 512);
                            const uint64_t bd = sdesc_sw64(zb + (uint32_t)(k * 1024), kBox, 512);
                            mma_bf16(d, ad, bd, idesc, 1u);
                        }
                        mma_commit(&empty[st]);
                    }
                    if (!ok) break;
                }
                if (i - 1 >= it.n0 && i - 1 < it.n1) mma_commit(&zempty[(t0 + i - 1 - it.n0) % ZS]);
            }
            zt = t0 + (it.n1 - it.n0);
        }
        mma_commit(mma_done);   // arrives once every MMA issued above has completed
    }
    __syncthreads();
    const bool mma_ok = mbar_wait(mma_done, 0);
    const bool ok = mma_ok && !*abort_flag;
    if (!mma_ok && tid == 0) atomicExch(a.err, 9);
    tc_fence_after();
    if (ok && blockIdx.x < n_items) {
        // lane m = warp * 32 + lane of group g's accumulators: input box 4 g + warp, channel lane
        const int ci = lane;
        for (int g = 0; g < 3; ++g) {
            const int p = 4 * g + warp;
            if (p >= 9) continue;   // warp-uniform: stale box slots of the last group
            const int dy = p / 3 - 1, dx = p % 3 - 1;
            for (int j = 0; j < 3; ++j) {
                float v[32];
                tmem_load<32>(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)((g * 3 + j) * 32), v);
                const int tap = (2 - j) * 9 + (dy + 1) * 3 + (dx + 1);   // dz = 1 - j
                if (ci < a.c_in) {
#pragma unroll
                    for (int co = 0; co < 32; ++co)
                        if (co < a.c_out) atomicAdd(a.dw + ((size_t)co * a.c_in + ci) * 27 + tap, v[co]);
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kWcCols) : "memory");
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

// C32 tensor [B][D][H][W][32] bf16 as a 5-D map with boxes (32 ch, 64 x, 2 y, 1 z, 1 batch),
// 64-byte swizzle, zero fill outside.
bool make_map(CUtensorMap* map, const void* base, int B, int D, int H, int W) {
    auto fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[5] = {32, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)D, (cuuint64_t)B};
    const cuuint64_t strides[4] = {64, 64ull * W, 64ull * W * H, 64ull * W * H * D};
    const cuuint32_t box[5] = {32, 64, 2, 1, 1};
    const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void*>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int sm_count() {
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

}  // namespace

cudaError_t launch_conv3d_tc(const ConvLaunch& c, cudaStream_t st) {
    if (c.W != 64 || c.H % 2 != 0 || c.B < 1 || c.D < 1 || c.H < 2) return cudaErrorInvalidValue;
    CUtensorMap map;
    if (!make_map(&map, c.x, c.B, c.D, c.H, c.W)) return cudaErrorInvalidValue;
    // per launch: the attribute belongs to the current device's context (a few microseconds)
    cudaError_t ea = cudaFuncSetAttribute(k_conv3d_chain, cudaFuncAttributeMaxDynamicSharedMemorySize, kChainBytes);
    if (ea != cudaSuccess) return ea;
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
    a.err = c.err;
    const int Q = ((c.D + c.dil - 1) / c.dil + kChainMax - 1) / kChainMax;
    const long long items = (long long)c.B * Q * c.dil * (c.H / 2);
    if (items > 0x7fffffffLL) return cudaErrorInvalidValue;
    int grid = kChainCtas * sm_count();
    if (grid > items) grid = (int)items;
    if (grid < 1) return cudaSuccess;
    k_conv3d_chain<<<grid, kConvThreads, kChainBytes, st>>>(map, a, (int)items, Q);
    return cudaGetLastError();
}

cudaError_t launch_conv3d_wgrad(const WgradLaunch& c, cudaStream_t st) {
    if (c.W != 64 || c.H % 2 != 0 || c.B < 1 || c.D < 1 || c.H < 2 || c.dil < 1) return cudaErrorInvalidValue;
    CUtensorMap mx, mz;
    if (!make_map(&mx, c.x, c.B, c.D, c.H, c.W) || !make_map(&mz, c.dz, c.B, c.D, c.H, c.W))
        return cudaErrorInvalidValue;
    // one CTA per SM: it holds 512 tensor-memory columns and 192 KB of rings
    cudaError_t ea = cudaFuncSetAttribute(k_conv3d_wgrad, cudaFuncAttributeMaxDynamicSharedMemorySize, kWcBytes);
    if (ea != cudaSuccess) return ea;
    WgradArgs a{};
    a.dw = c.dw;
    a.B = c.B; a.D = c.D; a.H = c.H; a.W = c.W;
    a.c_in = c.c_in; a.c_out = c.c_out; a.dil = c.dil;
    a.err = c.err;
    const int Q = ((c.D + c.dil - 1) / c.dil + kChainMax - 1) / kChainMax;
    const long long items = (long long)c.B * Q * c.dil * (c.H / 2);
    if (items > 0x7fffffffLL) return cudaErrorInvalidValue;
    int grid = sm_count();
    if (grid > items) grid = (int)items;
    if (grid < 1) return cudaSuccess;
    k_conv3d_wgrad<<<grid, 128, kWcBytes, st>>>(mx, mz, a, (int)items, Q);
    return cudaGetLastError();
}

}  // namespace rt
