// march_common.cuh -- device building blocks of the emission-absorption march (sm_103a).
//
// Geometry (paper Sec. 2): node-centred grid, per axis f = floor(x), corners
// clamp(f, 0, n-1) / clamp(f+1, 0, n-1), fraction t = x - f; kappa at the nearest cell of the
// previous position x_k. All geometry uses explicit round-to-nearest FP32 intrinsics so the
// compiler cannot contract or reorder it: the cell sequence of a ray is a pure function of
// (source, direction, ds) and identical in every kernel of this library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace rt {

constexpr float kFourPi = 12.566370614359172f;

// Clamped corner pair and fraction along one axis.
struct Axis {
    int lo, hi;   // clamped floor corner and clamped floor+1 corner
    float t;      // x - floor(x), not clamped
    int f;        // floor(x), limited to [-1, n-1] (lo = max(f, 0), hi = min(f + 1, n - 1))
};

__device__ __forceinline__ Axis axis_sample(float x, int n) {
    Axis a;
    const float f = floorf(x);
    a.t = __fsub_rn(x, f);
    // clamp in float first so the conversion never leaves the int range
    const int fi = __float2int_rz(fminf(fmaxf(f, -1.0f), (float)(n - 1)));
    a.lo = max(fi, 0);
    a.hi = min(fi + 1, n - 1);
    a.f = fi;
    return a;
}

__device__ __forceinline__ int nearest_round(float x, int n) {
    const float f = floorf(__fadd_rn(x, 0.5f));
    return __float2int_rz(fminf(fmaxf(f, 0.0f), (float)(n - 1)));
}

// The eight trilinear corners of x_k and its kappa cell. Corner c has bits (b0 b1 b2) =
// (c >> 2, c >> 1, c) & 1 selecting hi along axes 0, 1, 2.
struct Sample {
    int cell[8];
    float w[8];
    int nn;
    int tl;       // with a deposit tile: tile-local index of corner 0, or -1 (see below)
};

// Edge of the shared-memory deposit tile a block keeps around its source (cells per axis).
constexpr int kTile = 8;

// TILE: also locate the 8 corners in a kTile^3 tile with origin (o0, o1, o2) lying inside the
// grid: s.tl = local index of corner 0 when floor(x) - o is in [0, kTile - 2] on every axis
// (then no corner is clamped and corner c sits at s.tl + tile_offset(c)), else -1.
template <bool TILE = false>
__device__ __forceinline__ void make_sample(float x0, float x1, float x2, int n0, int n1, int n2,
                                            int kappa_mode, Sample& s, int o0 = 0, int o1 = 0, int o2 = 0) {
    const Axis a0 = axis_sample(x0, n0), a1 = axis_sample(x1, n1), a2 = axis_sample(x2, n2);
    if (TILE) {
        const unsigned u0 = (unsigned)(a0.f - o0), u1 = (unsigned)(a1.f - o1), u2 = (unsigned)(a2.f - o2);
        const unsigned lim = kTile - 2;
        s.tl = (u0 <= lim && u1 <= lim && u2 <= lim) ? (int)((u0 * kTile + u1) * kTile + u2) : -1;
    }
    const int r00 = (a0.lo * n1 + a1.lo) * n2, r01 = (a0.lo * n1 + a1.hi) * n2;
    const int r10 = (a0.hi * n1 + a1.lo) * n2, r11 = (a0.hi * n1 + a1.hi) * n2;
    s.cell[0] = r00 + a2.lo; s.cell[1] = r00 + a2.hi;
    s.cell[2] = r01 + a2.lo; s.cell[3] = r01 + a2.hi;
    s.cell[4] = r10 + a2.lo; s.cell[5] = r10 + a2.hi;
    s.cell[6] = r11 + a2.lo; s.cell[7] = r11 + a2.hi;
    const float u0 = 1.0f - a0.t, u1 = 1.0f - a1.t, u2 = 1.0f - a2.t;
    const float w00 = u0 * u1, w01 = u0 * a1.t, w10 = a0.t * u1, w11 = a0.t * a1.t;
    s.w[0] = w00 * u2; s.w[1] = w00 * a2.t;
    s.w[2] = w01 * u2; s.w[3] = w01 * a2.t;
    s.w[4] = w10 * u2; s.w[5] = w10 * a2.t;
    s.w[6] = w11 * u2; s.w[7] = w11 * a2.t;
    if (kappa_mode == 0) {
        s.nn = s.cell[0];
    } else {
        s.nn = (nearest_round(x0, n0) * n1 + nearest_round(x1, n1)) * n2 + nearest_round(x2, n2);
    }
}

__device__ __forceinline__ constexpr int tile_offset(int c) {
    return ((c >> 2) & 1) * kTile * kTile + ((c >> 1) & 1) * kTile + (c & 1);
}

// exp(-x) for the march's attenuation factors (x = kappa ds >= 0, or tau >= 0), from the
// identity exp(-x) = 2^(-x log2(e)): one FP32 multiply by the constant log2(e) and the PTX
// base-2 exponential ex2.approx.ftz.f32 (results below the smallest normal FP32 number, i.e.
// x > 87.3, flush to zero, far below any deposit that matters). Its relative error is a few
// ulp plus the rounding of the product, which grows with x: about |x| log2(e) ln(2) 2^-24 --
// checked against FP64 exp in the tests through rt_neg_exp, and far inside the relative 1e-5
// the march is held to against the FP64 oracle. Every kernel of the library (forward, adjoint
// replay, batch) uses this one function, so a replayed march repeats the forward's intensities
// exactly.
__device__ __forceinline__ float neg_exp(float x) {
    constexpr float kLog2e = 1.4426950408889634f;   // log2(e)
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x * -kLog2e));
    return r;
}

// ---- W-wide bin vectors -----------------------------------------------------------------
template <int W> struct Vec;
template <> struct Vec<1> { float v[1]; };
template <> struct Vec<2> { float v[2]; };
template <> struct Vec<4> { float v[4]; };

template <int W>
__device__ __forceinline__ Vec<W> ldg_vec(const float* __restrict__ p, int cell);

template <>
__device__ __forceinline__ Vec<1> ldg_vec<1>(const float* __restrict__ p, int cell) {
    Vec<1> r; r.v[0] = __ldg(p + cell); return r;
}
template <>
__device__ __forceinline__ Vec<2> ldg_vec<2>(const float* __restrict__ p, int cell) {
    const float2 q = __ldg(reinterpret_cast<const float2*>(p) + cell);
    Vec<2> r; r.v[0] = q.x; r.v[1] = q.y; return r;
}
template <>
__device__ __forceinline__ Vec<4> ldg_vec<4>(const float* __restrict__ p, int cell) {
    const float4 q = __ldg(reinterpret_cast<const float4*>(p) + cell);
    Vec<4> r; r.v[0] = q.x; r.v[1] = q.y; r.v[2] = q.z; r.v[3] = q.w; return r;
}

// Predicated gather (no branch): v is loaded from cell when p is true and left as it was
// otherwise. The inputs are read-only for the whole kernel, so the load may be scheduled freely
// (non-volatile asm); the index must be a valid cell either way (callers clamp it).
template <int W>
__device__ __forceinline__ void ldg_vec_if(bool p, const float* __restrict__ base, int cell, Vec<W>& v);
template <>
__device__ __forceinline__ void ldg_vec_if<1>(bool p, const float* __restrict__ base, int cell, Vec<1>& v) {
    asm("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %1, 0;\n\t@q ld.global.nc.f32 %0, [%2];\n\t}"
        : "+f"(v.v[0])
        : "r"((int)p), "l"(base + cell));
}
template <>
__device__ __forceinline__ void ldg_vec_if<2>(bool p, const float* __restrict__ base, int cell, Vec<2>& v) {
    asm("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %2, 0;\n\t@q ld.global.nc.v2.f32 {%0, %1}, [%3];\n\t}"
        : "+f"(v.v[0]), "+f"(v.v[1])
        : "r"((int)p), "l"(base + 2 * (size_t)cell));
}
template <>
__device__ __forceinline__ void ldg_vec_if<4>(bool p, const float* __restrict__ base, int cell, Vec<4>& v) {
    asm("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %4, 0;\n\t@q ld.global.nc.v4.f32 {%0, %1, %2, %3}, [%5];\n\t}"
        : "+f"(v.v[0]), "+f"(v.v[1]), "+f"(v.v[2]), "+f"(v.v[3])
        : "r"((int)p), "l"(base + 4 * (size_t)cell));
}

// Fire-and-forget global reductions (no return value): one L2 atomic per W-vector. They carry
// no "memory" clobber: the accumulators they target are never read by the kernels that issue
// them, so loads of the read-only inputs may be scheduled across them; kernel completion
// orders them before any later reader. Each carries an L2 eviction policy (red_policy).
//
// An accumulator that fits in L2 with room for the packed inputs beside it (at most 64 MiB of
// the 126 MB L2) is marked evict-last, so the reductions keep finding its lines there while the
// gathers stream the inputs through; a larger one is marked evict-normal (measured on GB300, 4
// bins on 128^3 with 16 sources, a 32 MiB accumulator: 3 % less march time with evict-last).
constexpr long long kL2KeepBytes = 64ll << 20;
__device__ __forceinline__ unsigned long long red_policy(long long acc_bytes) {
    unsigned long long p;
    if (acc_bytes <= kL2KeepBytes)
        asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    else
        asm("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ void red_add(float* p, float a, unsigned long long pol) {
    asm volatile("red.global.add.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(p), "f"(a), "l"(pol));
}
__device__ __forceinline__ void red_add2(float* p, float a, float b, unsigned long long pol) {
    asm volatile("red.global.add.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;" ::"l"(p), "f"(a), "f"(b), "l"(pol));
}
__device__ __forceinline__ void red_add4(float* p, float a, float b, float c, float d, unsigned long long pol) {
    asm volatile("red.global.add.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p), "f"(a), "f"(b),
                 "f"(c), "f"(d), "l"(pol));
}

template <int W>
__device__ __forceinline__ void red_vec(float* __restrict__ base, int cell, const float* v, unsigned long long pol);
template <>
__device__ __forceinline__ void red_vec<1>(float* __restrict__ base, int cell, const float* v, unsigned long long pol) {
    red_add(base + cell, v[0], pol);
}
template <>
__device__ __forceinline__ void red_vec<2>(float* __restrict__ base, int cell, const float* v, unsigned long long pol) {
    red_add2(base + 2 * (size_t)cell, v[0], v[1], pol);
}
template <>
__device__ __forceinline__ void red_vec<4>(float* __restrict__ base, int cell, const float* v, unsigned long long pol) {
    red_add4(base + 4 * (size_t)cell, v[0], v[1], v[2], v[3], pol);
}

// Predicated form: the reduction happens only when p is true; the index must be a valid cell
// either way (callers clamp it), so no address outside the grid is formed. (The compiler still
// places each predicated reduction in a short branch of its own.)
template <int W>
__device__ __forceinline__ void red_vec_if(bool p, float* __restrict__ base, int cell, const float* v,
                                           unsigned long long pol);
template <>
__device__ __forceinline__ void red_vec_if<1>(bool p, float* __restrict__ base, int cell, const float* v,
                                              unsigned long long pol) {
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %0, 0;\n\t@q red.global.add.L2::cache_hint.f32 [%1], %2, %3;\n\t}"
                 ::"r"((int)p), "l"(base + cell), "f"(v[0]), "l"(pol));
}
template <>
__device__ __forceinline__ void red_vec_if<2>(bool p, float* __restrict__ base, int cell, const float* v,
                                              unsigned long long pol) {
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %0, 0;\n\t@q red.global.add.L2::cache_hint.v2.f32 [%1], {%2, %3}, %4;\n\t}"
                 ::"r"((int)p), "l"(base + 2 * (size_t)cell), "f"(v[0]), "f"(v[1]), "l"(pol));
}
template <>
__device__ __forceinline__ void red_vec_if<4>(bool p, float* __restrict__ base, int cell, const float* v,
                                              unsigned long long pol) {
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %0, 0;\n\t@q red.global.add.L2::cache_hint.v4.f32 [%1], {%2, %3, %4, %5}, %6;\n\t}"
                 ::"r"((int)p), "l"(base + 4 * (size_t)cell), "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]), "l"(pol));
}

// FP64 reductions for the wide accumulation mode. The deposit is an FP32 number; it is widened
// to FP64 exactly by integer operations on the IEEE-754 encodings (binary32: sign, 8 exponent
// bits with bias 127, 23 fraction bits; binary64: sign, 11 exponent bits with bias 1023, 52
// fraction bits): a normal number keeps its sign and fraction and has its exponent rebiased by
// 1023 - 127 = 896; zeros and subnormals give a signed zero (the FP32 reductions flush
// subnormals too); infinities and NaNs stay infinities and NaNs. No FP64 arithmetic runs on the
// SM: the L2 performs the addition.
__device__ __forceinline__ double widen_f32(float v) {
    const unsigned b = __float_as_uint(v);
    const unsigned e = (b >> 23) & 0xFFu;
    const unsigned long long sign = (unsigned long long)(b >> 31) << 63;
    const unsigned long long frac = e == 0u ? 0ull : (unsigned long long)(b & 0x7FFFFFu) << 29;
    const unsigned long long e64 = e == 0u ? 0ull : (e == 0xFFu ? 0x7FFull : (unsigned long long)(e + 896u));
    return __longlong_as_double((long long)(sign | (e64 << 52) | frac));
}
__device__ __forceinline__ void red_add_f64(double* p, float v) {
    asm volatile("red.global.add.f64 [%0], %1;" ::"l"(p), "d"(widen_f32(v)));
}

// 64-bit integer reduction for the deterministic (fixed-point) accumulation mode, with the L2
// policy of red_policy().
__device__ __forceinline__ void red_add_u64(unsigned long long* p, unsigned long long a, unsigned long long pol) {
    asm volatile("red.global.add.L2::cache_hint.u64 [%0], %1, %2;" ::"l"(p), "l"(a), "l"(pol));
}

}  // namespace rt
