// march_lane.cuh -- the march of one (ray, source, bin group) lane (paper Sec. 2, Eq. 2).
//
// Shared by the single-problem kernel (march_fwd.cu) and the batched persistent kernel
// (march_batch.cu). The W bins of a group share the ray geometry (bins are a batch axis, Sec. 2
// "Frequency-bin agnosticism"), so j and kappa are read as W-wide vectors from a cell-major
// packed copy and each deposit is one W-wide `red.global.add.v{W}.f32`.
//
// Consecutive substeps of a ray often fall in the same cell (ds < 1), and once a ray has left
// the box its clamped corners stay fixed for long stretches. The deposits a corner receives are
// summed in registers and sent to memory once: in gathers mode 0 (march_lane_slots, the
// default) for as long as the ray keeps that corner, across face crossings; in modes 1 and 3
// (march_lane_runs) until the corner set changes. Fewer L2 atomics, and far fewer tiny FP32
// additions into the large sums that pile up on boundary voxels. One thread marches a lane, or
// two adjacent threads share it (march_lane_pair).
#pragma once

#include "march_common.cuh"

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

// Geometry and data of one lane. jg / kg / og point at the lane's bin group.
struct Lane {
    const float* __restrict__ jg;
    const float* __restrict__ kg;
    float* __restrict__ og;
    unsigned long long* __restrict__ og64;   // 8-byte accumulator of the group, bin-major
                                              //   ([W][cell]): fixed point (deterministic mode) or
                                              //   FP64 (the wide accumulation), see flush()
    long long ncell;
    int nbins;                                //   real bins in this group (the rest are padding)
    float fix = 0.0f;                         //   fixed point: units per unit deposit, a power of two
    float4 n;                 // direction
    float sx, sy, sz;         // source position
    int n0, n1, n2;
    int ns;
    float ds;
    float scale;              // factor of every deposit
    int kappa_mode;
    unsigned long long pol = 0;   // L2 policy of the FP32 field reductions (red_policy)
    float* tile = nullptr;    // the block's shared-memory deposit tile ([kTile^3][W]) or NULL
    int to0 = 0, to1 = 0, to2 = 0;   // its origin cell
    // REC: adjoint checkpoints written during the march, in the reverse march's layout: the
    // lane's fields f of checkpoint c at ck[(c * (3 + 2W) + f) * ck_lanes]
    float* ck = nullptr;
    long long ck_lanes = 0;
    int ck_stride = 0;
};

// The state a lane carries through its march, in and out: position, and I and tau of its bins.
// A fresh lane starts at its source with I = tau = 0; a continued lane (stateful advance) with
// the values its previous call left.
template <int W>
struct RayState {
    float x, y, z;
    float I[W], tau[W];
};

// Send one merged deposit (the sums for one corner) to memory. DET (the accumulation):
//   0: one W-wide FP32 reduction;
//   1: deterministic mode, one 64-bit fixed-point reduction per bin (integer addition is
//      associative, so the result does not depend on the order of the deposits);
//   2: one FP64 reduction per bin (the sums keep 53 bits however many small deposits a
//      large cell sum takes; same L2 rate per operation as the W-wide FP32 one).
// Modes 1 and 2 use the 8-byte accumulator og64, bin-major ([W][cell]): the W reductions of one
// corner go to W different sectors (L2 slices) instead of queueing on one, which matters on the
// crowded cells next to the sources. The padding bins of a group (past nbins) have
// j = kappa = 0, so they deposit exact zeros into their own rows and need no test.
template <int W, int DET>
__device__ __forceinline__ void flush(const Lane& L, int cell, const float* v) {
    if (DET == 2) {
        double* o = reinterpret_cast<double*>(L.og64) + cell;
#pragma unroll
        for (int b = 0; b < W; ++b) red_add_f64(o + b * L.ncell, v[b]);
    } else if (DET) {
        // v * 2^k is exact in FP32; its rounding to an integer is the fixed-point quantisation
        unsigned long long* o = L.og64 + cell;
#pragma unroll
        for (int b = 0; b < W; ++b)
            red_add_u64(o + b * L.ncell, (unsigned long long)__float2ll_rn(v[b] * L.fix), L.pol);
    } else {
        red_vec<W>(L.og, cell, v, L.pol);
    }
}

// flush() when p is true (callers pass a valid cell either way). FP32: one predicated vector
// reduction. 8-byte sums: the W reductions of a corner under one branch, not one each.
template <int W, int DET>
__device__ __forceinline__ void flush_if(bool p, const Lane& L, int cell, const float* v) {
    if (DET) {
        if (p) flush<W, DET>(L, cell, v);
    } else {
        red_vec_if<W>(p, L.og, cell, v, L.pol);
    }
}

// Send the merged deposits of one run (8 corners) to memory. Runs whose corners lie in the
// block's tile (tl >= 0) go to shared memory: the rays of a block all start at its source, so
// these are the most contended cells of the march; the block adds the tile to the field once.
template <int W, int DET, bool TILE>
__device__ __forceinline__ void flush_run(const Lane& L, const int* pc, const float (*pend)[W], int tl) {
    if (TILE && tl >= 0) {
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            float* t = L.tile + (tl + tile_offset(c)) * W;
#pragma unroll
            for (int b = 0; b < W; ++b) atomicAdd(t + b, pend[c][b]);
        }
    } else {
#pragma unroll
        for (int c = 0; c < 8; ++c) flush<W, DET>(L, pc[c], pend[c]);
    }
}

// PF = 2: prefetch and reuse combined. The corner set of substep k+1 is computed one step
// ahead; its gathers are issued (only if it differs from the current set, else the registers
// are carried over) before the update of substep k, so their latency overlaps that update.
template <int W, int DET, bool TILE = false>
__device__ __forceinline__ void march_lane_ahead(const Lane& L, RayState<W>& R) {
    const float* __restrict__ jg = L.jg;
    const float* __restrict__ kg = L.kg;
    const float dx = __fmul_rn(L.n.x, L.ds), dy = __fmul_rn(L.n.y, L.ds), dz = __fmul_rn(L.n.z, L.ds);
    float x = R.x, y = R.y, z = R.z;
    float I[W], tau[W];
#pragma unroll
    for (int b = 0; b < W; ++b) { I[b] = R.I[b]; tau[b] = R.tau[b]; }
    const float ds = L.ds, scale = L.scale;
    int pc[8];
    float pend[8][W];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        pc[c] = -1;
#pragma unroll
        for (int b = 0; b < W; ++b) pend[c][b] = 0.0f;
    }
    int ptl = -1;
    Sample sm;
    Gathered<W> gd;
    make_sample<TILE>(x, y, z, L.n0, L.n1, L.n2, L.kappa_mode, sm, L.to0, L.to1, L.to2);
    gather<W>(jg, kg, sm, gd);
#pragma unroll 1
    for (int k = 0; k < L.ns; ++k) {
        x = __fadd_rn(x, dx);                             // Eq. 2: x_{k+1}
        y = __fadd_rn(y, dy);
        z = __fadd_rn(z, dz);
        Sample nx;
        make_sample<TILE>(x, y, z, L.n0, L.n1, L.n2, L.kappa_mode, nx, L.to0, L.to1, L.to2);
        Gathered<W> ng = gd;
        if (k + 1 < L.ns) {
            if (nx.cell[0] != sm.cell[0] || nx.cell[7] != sm.cell[7]) {
#pragma unroll
                for (int c = 0; c < 8; ++c) ng.j[c] = ldg_vec<W>(jg, nx.cell[c]);
            }
            if (nx.nn != sm.nn) ng.k = ldg_vec<W>(kg, nx.nn);
        }
        float dep[W];
#pragma unroll
        for (int b = 0; b < W; ++b) {
            float jk = 0.0f;
#pragma unroll
            for (int c = 0; c < 8; ++c) jk = fmaf(sm.w[c], gd.j[c].v[b], jk);
            const float kds = gd.k.v[b] * ds;
            const float att = neg_exp(kds);               // exp(-kappa(x_k) ds)
            const float em = neg_exp(tau[b]);             // exp(-tau_k)
            I[b] = fmaf(I[b], att, jk * em * ds);         // Eq. 2: I_{k+1}
            tau[b] += kds;                                // Eq. 2: tau_{k+1}
            dep[b] = I[b] * scale;
        }
        if (sm.cell[0] != pc[0] || sm.cell[7] != pc[7]) {
            if (pc[0] >= 0) flush_run<W, DET, TILE>(L, pc, pend, ptl);
            ptl = TILE ? sm.tl : -1;
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
        sm = nx;
        gd = ng;
    }
    if (pc[0] >= 0) flush_run<W, DET, TILE>(L, pc, pend, ptl);
    R.x = x; R.y = y; R.z = z;
#pragma unroll
    for (int b = 0; b < W; ++b) { R.I[b] = I[b]; R.tau[b] = tau[b]; }
}

// Gathers mode 0: the corner slots. A lane keeps the 8 corners of its current corner set in 8
// slots, each holding the corner's cell, its gathered j (W bins) and the sum of the deposits it
// has received since it was filled. Slot s holds the corner whose bit along axis a is
// bit_a(s) ^ P_a. Per axis the set is the clamped pair (lo, hi) of the current position. When
// the pair moves up by one cell (the new lo is the old hi), the old hi face is shared by both
// sets: its four slots keep their cells, j values and sums and only flip role (P_a ^= 1), while
// the four slots of the old lo face are flushed (one reduction each) and refilled (one gather
// each) as the new hi face; moving down is the mirror image, an unchanged pair changes nothing,
// and any other change (a jump of more than one cell) flushes and refills every slot. A ray
// crosses a face about every other substep at ds = 0.5, so against flushing and re-gathering
// all eight corners at every change of the set this halves both the reductions and the gathers.
// The deposits a cell receives are summed in its slot for as long as the ray keeps it, which
// also means fewer FP32 additions into the large sums of the field.
// REC: store (x_k, I_k, tau_k) every ck_stride substeps, the forward sweep the reverse march
// would otherwise repeat.
template <int W, int DET, bool TILE, bool REC>
__device__ __forceinline__ void march_lane_slots(const Lane& L, RayState<W>& R) {
    const float* __restrict__ jg = L.jg;
    const float* __restrict__ kg = L.kg;
    const float dx = __fmul_rn(L.n.x, L.ds), dy = __fmul_rn(L.n.y, L.ds), dz = __fmul_rn(L.n.z, L.ds);
    float x = R.x, y = R.y, z = R.z;
    float I[W], tau[W];
#pragma unroll
    for (int b = 0; b < W; ++b) { I[b] = R.I[b]; tau[b] = R.tau[b]; }
    const float ds = L.ds, scale = L.scale;

    int pc[8];           // cell of each slot, -1 while empty
    int tl[8];           // TILE: its index in the block's shared-memory tile, or -1
    float pend[8][W];    // deposits summed in the slot
    Vec<W> gj[8];        // j at the slot's cell
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        pc[c] = -1;
        tl[c] = -1;
#pragma unroll
        for (int b = 0; b < W; ++b) { pend[c][b] = 0.0f; gj[c].v[b] = 0.0f; }
    }
    // per axis: the (lo, hi) pair of the current set (-2: none yet) and the role flip P_a
    int rl0 = -2, rh0 = -2, rl1 = -2, rh1 = -2, rl2 = -2, rh2 = -2;
    int P0 = 0, P1 = 0, P2 = 0;
    Vec<W> gk;
#pragma unroll
    for (int b = 0; b < W; ++b) gk.v[b] = 0.0f;
    int gnn = -1;

    int ck_left = 0;     // REC: substeps until the next checkpoint
    float* ckp = L.ck;   // REC: this lane's next checkpoint
#pragma unroll 1
    for (int k = 0; k < L.ns; ++k) {
        if (REC) {
            if (ck_left == 0) {
                ckp[0] = x; ckp[L.ck_lanes] = y; ckp[2 * L.ck_lanes] = z;
#pragma unroll
                for (int b = 0; b < W; ++b) {
                    ckp[(3 + b) * L.ck_lanes] = I[b];
                    ckp[(3 + W + b) * L.ck_lanes] = tau[b];
                }
                ckp += (3 + 2 * W) * L.ck_lanes;
                ck_left = L.ck_stride;
            }
            --ck_left;
        }
        const Axis a0 = axis_sample(x, L.n0), a1 = axis_sample(y, L.n1), a2 = axis_sample(z, L.n2);
        // transition of each axis pair: same, up (new lo = old hi), down (new hi = old lo), other
        const int key0 = a0.lo | (a0.hi << 16), key1 = a1.lo | (a1.hi << 16), key2 = a2.lo | (a2.hi << 16);
        const bool same0 = key0 == (rl0 | (rh0 << 16)), same1 = key1 == (rl1 | (rh1 << 16)),
                   same2 = key2 == (rl2 | (rh2 << 16));
        const bool up0 = !same0 && a0.lo == rh0, up1 = !same1 && a1.lo == rh1, up2 = !same2 && a2.lo == rh2;
        const bool dn0 = !same0 && !up0 && a0.hi == rl0, dn1 = !same1 && !up1 && a1.hi == rl1,
                   dn2 = !same2 && !up2 && a2.hi == rl2;
        const bool change = !(same0 && same1 && same2);
        bool flag[8];
        if (change) {
            const bool other = !(same0 || up0 || dn0) || !(same1 || up1 || dn1) || !(same2 || up2 || dn2);
            // the leaving face: slots whose axis bit equals P_a ^ (1 if moving down)
            const bool sh0 = up0 || dn0, sh1 = up1 || dn1, sh2 = up2 || dn2;
            const int q0 = P0 ^ (dn0 ? 1 : 0), q1 = P1 ^ (dn1 ? 1 : 0), q2 = P2 ^ (dn2 ? 1 : 0);
            // leaving slots as a bit mask: the bit-0 / bit-1 face of axis 0 is 0x0F / 0xF0, of axis
            // 1 0x33 / 0xCC, of axis 2 0x55 / 0xAA
            unsigned mask = other ? 0xFFu : 0u;
            mask |= sh0 ? (q0 ? 0xF0u : 0x0Fu) : 0u;
            mask |= sh1 ? (q1 ? 0xCCu : 0x33u) : 0u;
            mask |= sh2 ? (q2 ? 0xAAu : 0x55u) : 0u;
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                flag[c] = (mask >> c) & 1u;
                const bool send = flag[c] && pc[c] >= 0;
                if (TILE) {
                    if (send) {
                        if (tl[c] >= 0) {
                            float* t = L.tile + tl[c] * W;
#pragma unroll
                            for (int b = 0; b < W; ++b) atomicAdd(t + b, pend[c][b]);
                        } else {
                            flush<W, DET>(L, pc[c], pend[c]);
                        }
                    }
                } else {
                    flush_if<W, DET>(send, L, max(pc[c], 0), pend[c]);
                }
                if constexpr (W % 2 == 0) {   // a flushed slot starts again from zero
                    const float keep = flag[c] ? 0.0f : 1.0f;
#pragma unroll
                    for (int h = 0; h < W; h += 2) {
                        const float2 v = __fmul2_rn(make_float2(pend[c][h], pend[c][h + 1]), make_float2(keep, keep));
                        pend[c][h] = v.x; pend[c][h + 1] = v.y;
                    }
                } else {
#pragma unroll
                    for (int b = 0; b < W; ++b) pend[c][b] = flag[c] ? 0.0f : pend[c][b];
                }
            }
            P0 ^= sh0 ? 1 : 0; P1 ^= sh1 ? 1 : 0; P2 ^= sh2 ? 1 : 0;
            rl0 = a0.lo; rh0 = a0.hi; rl1 = a1.lo; rh1 = a1.hi; rl2 = a2.lo; rh2 = a2.hi;
        }
        // slot geometry: coordinate and weight factor of slot bit 0 / 1 along each axis
        const int c00 = P0 ? a0.hi : a0.lo, c01 = P0 ? a0.lo : a0.hi;
        const int c10 = P1 ? a1.hi : a1.lo, c11 = P1 ? a1.lo : a1.hi;
        const int c20 = P2 ? a2.hi : a2.lo, c21 = P2 ? a2.lo : a2.hi;
        const float u0 = 1.0f - a0.t, u1 = 1.0f - a1.t, u2 = 1.0f - a2.t;
        const float f00 = P0 ? a0.t : u0, f01 = P0 ? u0 : a0.t;
        const float f10 = P1 ? a1.t : u1, f11 = P1 ? u1 : a1.t;
        const float f20 = P2 ? a2.t : u2, f21 = P2 ? u2 : a2.t;
        float w[8];
        {
            const float w00 = f00 * f10, w01 = f00 * f11, w10 = f01 * f10, w11 = f01 * f11;
            w[0] = w00 * f20; w[1] = w00 * f21; w[2] = w01 * f20; w[3] = w01 * f21;
            w[4] = w10 * f20; w[5] = w10 * f21; w[6] = w11 * f20; w[7] = w11 * f21;
        }
        if (change) {
            const int r00 = (c00 * L.n1 + c10) * L.n2, r01 = (c00 * L.n1 + c11) * L.n2;
            const int r10 = (c01 * L.n1 + c10) * L.n2, r11 = (c01 * L.n1 + c11) * L.n2;
            const int cell[8] = {r00 + c20, r00 + c21, r01 + c20, r01 + c21,
                                 r10 + c20, r10 + c21, r11 + c20, r11 + c21};
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                if (flag[c]) {
                    gj[c] = ldg_vec<W>(jg, cell[c]);
                    pc[c] = cell[c];
                }
                if (TILE && flag[c]) {
                    const unsigned v0 = (unsigned)((((c >> 2) & 1) ? c01 : c00) - L.to0);
                    const unsigned v1 = (unsigned)((((c >> 1) & 1) ? c11 : c10) - L.to1);
                    const unsigned v2 = (unsigned)(((c & 1) ? c21 : c20) - L.to2);
                    tl[c] = (v0 < (unsigned)kTile && v1 < (unsigned)kTile && v2 < (unsigned)kTile)
                                ? (int)((v0 * kTile + v1) * kTile + v2) : -1;
                }
            }
        }
        // kappa at the nearest cell of x_k (the floor corner, or the rounded position)
        const int nn = L.kappa_mode == 0 ? (a0.lo * L.n1 + a1.lo) * L.n2 + a2.lo
                                         : (nearest_round(x, L.n0) * L.n1 + nearest_round(y, L.n1)) * L.n2 +
                                               nearest_round(z, L.n2);
        if (nn != gnn) {
            gk = ldg_vec<W>(kg, nn);
            gnn = nn;
        }
        float dep[W];
        if constexpr (W % 2 == 0) {
            // bins in pairs: the paired FP32 instructions compute two round-to-nearest results
            // each, the same numbers as the scalar code below
#pragma unroll
            for (int h = 0; h < W; h += 2) {
                float2 jk = make_float2(0.0f, 0.0f);
#pragma unroll
                for (int c = 0; c < 8; ++c)
                    jk = __ffma2_rn(make_float2(w[c], w[c]), make_float2(gj[c].v[h], gj[c].v[h + 1]), jk);
                const float2 kds = __fmul2_rn(make_float2(gk.v[h], gk.v[h + 1]), make_float2(ds, ds));
                const float2 att = make_float2(neg_exp(kds.x), neg_exp(kds.y));       // exp(-kappa(x_k) ds)
                const float2 em = make_float2(neg_exp(tau[h]), neg_exp(tau[h + 1]));  // exp(-tau_k)
                const float2 e = __fmul2_rn(__fmul2_rn(jk, em), make_float2(ds, ds));
                const float2 In = __ffma2_rn(make_float2(I[h], I[h + 1]), att, e);    // Eq. 2: I_{k+1}
                const float2 tn = __fadd2_rn(make_float2(tau[h], tau[h + 1]), kds);   // Eq. 2: tau_{k+1}
                const float2 d = __fmul2_rn(In, make_float2(scale, scale));
                I[h] = In.x; I[h + 1] = In.y;
                tau[h] = tn.x; tau[h + 1] = tn.y;
                dep[h] = d.x; dep[h + 1] = d.y;
            }
#pragma unroll
            for (int c = 0; c < 8; ++c) {
#pragma unroll
                for (int h = 0; h < W; h += 2) {
                    const float2 v = __ffma2_rn(make_float2(w[c], w[c]), make_float2(dep[h], dep[h + 1]),
                                                make_float2(pend[c][h], pend[c][h + 1]));
                    pend[c][h] = v.x; pend[c][h + 1] = v.y;
                }
            }
        } else {
#pragma unroll
            for (int b = 0; b < W; ++b) {
                float jk = 0.0f;
#pragma unroll
                for (int c = 0; c < 8; ++c) jk = fmaf(w[c], gj[c].v[b], jk);
                const float kds = gk.v[b] * ds;
                const float att = neg_exp(kds);               // exp(-kappa(x_k) ds)
                const float em = neg_exp(tau[b]);             // exp(-tau_k)
                I[b] = fmaf(I[b], att, jk * em * ds);         // Eq. 2: I_{k+1}
                tau[b] += kds;                                // Eq. 2: tau_{k+1}
                dep[b] = I[b] * scale;
            }
#pragma unroll
            for (int c = 0; c < 8; ++c) {
#pragma unroll
                for (int b = 0; b < W; ++b) pend[c][b] = fmaf(w[c], dep[b], pend[c][b]);
            }
        }
        x = __fadd_rn(x, dx);                             // Eq. 2: x_{k+1}
        y = __fadd_rn(y, dy);
        z = __fadd_rn(z, dz);
    }
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        if (pc[c] >= 0) {
            if (TILE && tl[c] >= 0) {
                float* t = L.tile + tl[c] * W;
#pragma unroll
                for (int b = 0; b < W; ++b) atomicAdd(t + b, pend[c][b]);
            } else {
                flush<W, DET>(L, pc[c], pend[c]);
            }
        }
    }
    R.x = x; R.y = y; R.z = z;
#pragma unroll
    for (int b = 0; b < W; ++b) { R.I[b] = I[b]; R.tau[b] = tau[b]; }
}

// Gathers mode 4: the corner slots of mode 0 with the gathers of each substep issued one substep
// early. Positions do not depend on the intensity, so while substep k is updated, the slot
// transition k -> k+1 is already known: as soon as the trilinear sum of substep k has read the
// slots, the j values of the corners that enter at k+1 are loaded into the slots that they replace
// (and, once kappa(x_k) has been used, kappa(x_{k+1}) into its register). Their latency overlaps
// the rest of substep k and the geometry of k+1 instead of stalling the trilinear sum that needs
// them. Flushes happen at the same points and the deposits are summed in the same order as in
// mode 0, so the two modes produce the same sums. REC: checkpoints as in mode 0.
template <int W, int DET, bool REC>
__device__ __forceinline__ void march_lane_slots_ahead(const Lane& L, RayState<W>& R) {
    const float* __restrict__ jg = L.jg;
    const float* __restrict__ kg = L.kg;
    const float dx = __fmul_rn(L.n.x, L.ds), dy = __fmul_rn(L.n.y, L.ds), dz = __fmul_rn(L.n.z, L.ds);
    float x = R.x, y = R.y, z = R.z;
    float I[W], tau[W];
#pragma unroll
    for (int b = 0; b < W; ++b) { I[b] = R.I[b]; tau[b] = R.tau[b]; }
    const float ds = L.ds, scale = L.scale;
    const int n1 = L.n1, n2 = L.n2;
    auto kappa_cell = [&](const Axis& a0, const Axis& a1, const Axis& a2, float px, float py, float pz) {
        return L.kappa_mode == 0 ? (a0.lo * n1 + a1.lo) * n2 + a2.lo
                                 : (nearest_round(px, L.n0) * n1 + nearest_round(py, n1)) * n2 + nearest_round(pz, n2);
    };

    // the current corner set (x_k): per-axis samples, slot roles P_a, slot cells, j and sums
    Axis a0 = axis_sample(x, L.n0), a1 = axis_sample(y, n1), a2 = axis_sample(z, n2);
    int P0 = 0, P1 = 0, P2 = 0;
    int pc[8];
    float pend[8][W];
    Vec<W> gj[8];
    {
        const int r00 = (a0.lo * n1 + a1.lo) * n2, r01 = (a0.lo * n1 + a1.hi) * n2;
        const int r10 = (a0.hi * n1 + a1.lo) * n2, r11 = (a0.hi * n1 + a1.hi) * n2;
        const int cell[8] = {r00 + a2.lo, r00 + a2.hi, r01 + a2.lo, r01 + a2.hi,
                             r10 + a2.lo, r10 + a2.hi, r11 + a2.lo, r11 + a2.hi};
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            pc[c] = cell[c];
            gj[c] = ldg_vec<W>(jg, cell[c]);
#pragma unroll
            for (int b = 0; b < W; ++b) pend[c][b] = 0.0f;
        }
    }
    int gnn = kappa_cell(a0, a1, a2, x, y, z);
    Vec<W> gk = ldg_vec<W>(kg, gnn);

    int ck_left = 0;     // REC: substeps until the next checkpoint
    float* ckp = L.ck;   // REC: this lane's next checkpoint
#pragma unroll 1
    for (int k = 0; k < L.ns; ++k) {
        if (REC) {
            if (ck_left == 0) {
                ckp[0] = x; ckp[L.ck_lanes] = y; ckp[2 * L.ck_lanes] = z;
#pragma unroll
                for (int b = 0; b < W; ++b) {
                    ckp[(3 + b) * L.ck_lanes] = I[b];
                    ckp[(3 + W + b) * L.ck_lanes] = tau[b];
                }
                ckp += (3 + 2 * W) * L.ck_lanes;
                ck_left = L.ck_stride;
            }
            --ck_left;
        }
        // ---- x_{k+1}, its corner set and the slots that change (nothing changes after the last) ----
        const float xn = __fadd_rn(x, dx), yn = __fadd_rn(y, dy), zn = __fadd_rn(z, dz);   // Eq. 2: x_{k+1}
        const Axis b0 = axis_sample(xn, L.n0), b1 = axis_sample(yn, n1), b2 = axis_sample(zn, n2);
        const bool more = k + 1 < L.ns;
        // The pair (lo, hi) = (max(f, 0), min(f + 1, n - 1)) of an axis with n >= 2 cells is a
        // one-to-one function of the clamped floor f in [-1, n - 1], and f -> f + 1 makes the old hi
        // the new lo (up), f -> f - 1 the old lo the new hi (down); a single-cell axis keeps (0, 0).
        // So the change of f classifies each axis as march_lane_slots does from the pairs.
        const int d0 = L.n0 > 1 ? b0.f - a0.f : 0, d1 = n1 > 1 ? b1.f - a1.f : 0, d2 = n2 > 1 ? b2.f - a2.f : 0;
        const bool up0 = d0 == 1, up1 = d1 == 1, up2 = d2 == 1;
        const bool dn0 = d0 == -1, dn1 = d1 == -1, dn2 = d2 == -1;
        const bool other = (unsigned)(d0 + 1) > 2u || (unsigned)(d1 + 1) > 2u || (unsigned)(d2 + 1) > 2u;
        const bool sh0 = up0 || dn0, sh1 = up1 || dn1, sh2 = up2 || dn2;
        const int q0 = P0 ^ (dn0 ? 1 : 0), q1 = P1 ^ (dn1 ? 1 : 0), q2 = P2 ^ (dn2 ? 1 : 0);
        unsigned mask = other ? 0xFFu : 0u;   // leaving slots, as in march_lane_slots
        mask |= sh0 ? (q0 ? 0xF0u : 0x0Fu) : 0u;
        mask |= sh1 ? (q1 ? 0xCCu : 0x33u) : 0u;
        mask |= sh2 ? (q2 ? 0xAAu : 0x55u) : 0u;
        if (!more) mask = 0u;
        const int Q0 = P0 ^ (sh0 ? 1 : 0), Q1 = P1 ^ (sh1 ? 1 : 0), Q2 = P2 ^ (sh2 ? 1 : 0);   // roles at k+1

        // ---- substep k with the current slots (weights of x_k in slot order) ----
        const float u0 = 1.0f - a0.t, u1 = 1.0f - a1.t, u2 = 1.0f - a2.t;
        const float f00 = P0 ? a0.t : u0, f01 = P0 ? u0 : a0.t;
        const float f10 = P1 ? a1.t : u1, f11 = P1 ? u1 : a1.t;
        const float f20 = P2 ? a2.t : u2, f21 = P2 ? u2 : a2.t;
        float w[8];
        {
            const float w00 = f00 * f10, w01 = f00 * f11, w10 = f01 * f10, w11 = f01 * f11;
            w[0] = w00 * f20; w[1] = w00 * f21; w[2] = w01 * f20; w[3] = w01 * f21;
            w[4] = w10 * f20; w[5] = w10 * f21; w[6] = w11 * f20; w[7] = w11 * f21;
        }
        // trilinear sum of j(x_k) over the current slots
        float jk[W];
#pragma unroll
        for (int b = 0; b < W; ++b) jk[b] = 0.0f;
        if constexpr (W % 2 == 0) {
#pragma unroll
            for (int h = 0; h < W; h += 2) {
                float2 acc = make_float2(0.0f, 0.0f);
#pragma unroll
                for (int c = 0; c < 8; ++c)
                    acc = __ffma2_rn(make_float2(w[c], w[c]), make_float2(gj[c].v[h], gj[c].v[h + 1]), acc);
                jk[h] = acc.x; jk[h + 1] = acc.y;
            }
        } else {
#pragma unroll
            for (int b = 0; b < W; ++b) {
#pragma unroll
                for (int c = 0; c < 8; ++c) jk[b] = fmaf(w[c], gj[c].v[b], jk[b]);
            }
        }
        // the slots are read: gather the corners that enter at k+1 into the slots they replace
        // (slot bit 0 along axis a is Q_a ? hi : lo at k+1)
        const int e00 = Q0 ? b0.hi : b0.lo, e01 = Q0 ? b0.lo : b0.hi;
        const int e10 = Q1 ? b1.hi : b1.lo, e11 = Q1 ? b1.lo : b1.hi;
        const int e20 = Q2 ? b2.hi : b2.lo, e21 = Q2 ? b2.lo : b2.hi;
        const int s00 = (e00 * n1 + e10) * n2, s01 = (e00 * n1 + e11) * n2;
        const int s10 = (e01 * n1 + e10) * n2, s11 = (e01 * n1 + e11) * n2;
        const int ncell[8] = {s00 + e20, s00 + e21, s01 + e20, s01 + e21, s10 + e20, s10 + e21, s11 + e20, s11 + e21};
#pragma unroll
        for (int c = 0; c < 8; ++c) ldg_vec_if<W>((mask >> c) & 1u, jg, ncell[c], gj[c]);
        // Eq. 2 with kappa(x_k); then kappa(x_{k+1}) is gathered
        float dep[W];
        if constexpr (W % 2 == 0) {
#pragma unroll
            for (int h = 0; h < W; h += 2) {
                const float2 kds = __fmul2_rn(make_float2(gk.v[h], gk.v[h + 1]), make_float2(ds, ds));
                const float2 att = make_float2(neg_exp(kds.x), neg_exp(kds.y));       // exp(-kappa(x_k) ds)
                const float2 em = make_float2(neg_exp(tau[h]), neg_exp(tau[h + 1]));  // exp(-tau_k)
                const float2 e = __fmul2_rn(__fmul2_rn(make_float2(jk[h], jk[h + 1]), em), make_float2(ds, ds));
                const float2 In = __ffma2_rn(make_float2(I[h], I[h + 1]), att, e);    // Eq. 2: I_{k+1}
                const float2 tn = __fadd2_rn(make_float2(tau[h], tau[h + 1]), kds);   // Eq. 2: tau_{k+1}
                const float2 d = __fmul2_rn(In, make_float2(scale, scale));
                I[h] = In.x; I[h + 1] = In.y;
                tau[h] = tn.x; tau[h + 1] = tn.y;
                dep[h] = d.x; dep[h + 1] = d.y;
            }
        } else {
#pragma unroll
            for (int b = 0; b < W; ++b) {
                const float kds = gk.v[b] * ds;
                const float att = neg_exp(kds);               // exp(-kappa(x_k) ds)
                const float em = neg_exp(tau[b]);             // exp(-tau_k)
                I[b] = fmaf(I[b], att, jk[b] * em * ds);      // Eq. 2: I_{k+1}
                tau[b] += kds;                                // Eq. 2: tau_{k+1}
                dep[b] = I[b] * scale;
            }
        }
        const int nnn = kappa_cell(b0, b1, b2, xn, yn, zn);
        ldg_vec_if<W>(more && nnn != gnn, kg, nnn, gk);
        gnn = nnn;
        // deposits of substep k into the current slots
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            if constexpr (W % 2 == 0) {
#pragma unroll
                for (int h = 0; h < W; h += 2) {
                    const float2 v = __ffma2_rn(make_float2(w[c], w[c]), make_float2(dep[h], dep[h + 1]),
                                                make_float2(pend[c][h], pend[c][h + 1]));
                    pend[c][h] = v.x; pend[c][h + 1] = v.y;
                }
            } else {
#pragma unroll
                for (int b = 0; b < W; ++b) pend[c][b] = fmaf(w[c], dep[b], pend[c][b]);
            }
        }

        // ---- the slots that leave at k+1: flush their sums (this substep included) and start the
        // entering corners' sums from zero (predicated, no branch: some lane of a warp almost
        // always has a slot to change) ----
        {
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const bool f = (mask >> c) & 1u;
                flush_if<W, DET>(f, L, pc[c], pend[c]);
                if constexpr (W % 2 == 0) {
                    const float keep = f ? 0.0f : 1.0f;
#pragma unroll
                    for (int h = 0; h < W; h += 2) {
                        const float2 v = __fmul2_rn(make_float2(pend[c][h], pend[c][h + 1]), make_float2(keep, keep));
                        pend[c][h] = v.x; pend[c][h + 1] = v.y;
                    }
                } else {
#pragma unroll
                    for (int b = 0; b < W; ++b) pend[c][b] = f ? 0.0f : pend[c][b];
                }
                pc[c] = f ? ncell[c] : pc[c];
            }
        }
        P0 = Q0; P1 = Q1; P2 = Q2;
        a0 = b0; a1 = b1; a2 = b2;
        x = xn; y = yn; z = zn;
    }
#pragma unroll
    for (int c = 0; c < 8; ++c) flush<W, DET>(L, pc[c], pend[c]);
    R.x = x; R.y = y; R.z = z;
#pragma unroll
    for (int b = 0; b < W; ++b) { R.I[b] = I[b]; R.tau[b] = tau[b]; }
}

// Two lanes per ray with gathers mode 4: the slots of march_lane_pair (lane `sub` keeps the four
// slots whose axis-2 bit is `sub`) updated as in march_lane_slots_ahead -- the transition
// k -> k+1 is classified during substep k, the corners that enter at k+1 are gathered into the
// slots they replace right after substep k's partial trilinear sum has read them, kappa(x_{k+1})
// right after kappa(x_k) is used -- and every gather, flush and slot change is predicated, so the
// loop has no branch. Both lanes compute the same geometry, transitions and radiometry (the two
// partial sums are exchanged with one shuffle per bin; a + b and b + a are the same FP32
// number). REC: lane 0 of the pair stores the checkpoints (x_k, I_k, tau_k).
template <int W, bool REC, int DET>
__device__ __forceinline__ void march_lane_pair_ahead(const Lane& L, int sub, unsigned pmask) {
    const float* __restrict__ jg = L.jg;
    const float* __restrict__ kg = L.kg;
    const float dx = __fmul_rn(L.n.x, L.ds), dy = __fmul_rn(L.n.y, L.ds), dz = __fmul_rn(L.n.z, L.ds);
    float x = L.sx, y = L.sy, z = L.sz;
    float I[W], tau[W];
#pragma unroll
    for (int b = 0; b < W; ++b) { I[b] = 0.0f; tau[b] = 0.0f; }
    const float ds = L.ds, scale = L.scale;
    const int n1 = L.n1, n2 = L.n2;
    auto kappa_cell = [&](const Axis& a0, const Axis& a1, const Axis& a2, float px, float py, float pz) {
        return L.kappa_mode == 0 ? (a0.lo * n1 + a1.lo) * n2 + a2.lo
                                 : (nearest_round(px, L.n0) * n1 + nearest_round(py, n1)) * n2 + nearest_round(pz, n2);
    };

    // slot i of this lane is slot c = 2 i + sub of the ray: bits (c >> 2, c >> 1, c) & 1 =
    // (i >> 1, i & 1, sub) along axes 0, 1, 2; with roles P_a the bit selects lo (bit == P_a) or hi
    Axis a0 = axis_sample(x, L.n0), a1 = axis_sample(y, n1), a2 = axis_sample(z, n2);
    int P0 = 0, P1 = 0, P2 = 0;
    int pc[4];
    float pend[4][W];
    Vec<W> gj[4];
    {
        const int c2 = sub ? a2.hi : a2.lo;
        const int r0 = a0.lo * n1, r1 = a0.hi * n1;
        const int cell[4] = {(r0 + a1.lo) * n2 + c2, (r0 + a1.hi) * n2 + c2, (r1 + a1.lo) * n2 + c2,
                             (r1 + a1.hi) * n2 + c2};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            pc[i] = cell[i];
            gj[i] = ldg_vec<W>(jg, cell[i]);
#pragma unroll
            for (int b = 0; b < W; ++b) pend[i][b] = 0.0f;
        }
    }
    int gnn = kappa_cell(a0, a1, a2, x, y, z);
    Vec<W> gk = ldg_vec<W>(kg, gnn);

    int ck_left = 0;     // REC: substeps until the next checkpoint
    float* ckp = L.ck;   // REC: this lane's next checkpoint
#pragma unroll 1
    for (int k = 0; k < L.ns; ++k) {
        if (REC) {
            if (ck_left == 0) {
                if (sub == 0) {
                    ckp[0] = x; ckp[L.ck_lanes] = y; ckp[2 * L.ck_lanes] = z;
#pragma unroll
                    for (int b = 0; b < W; ++b) {
                        ckp[(3 + b) * L.ck_lanes] = I[b];
                        ckp[(3 + W + b) * L.ck_lanes] = tau[b];
                    }
                }
                ckp += (3 + 2 * W) * L.ck_lanes;
                ck_left = L.ck_stride;
            }
            --ck_left;
        }
        // ---- x_{k+1} and the slots that change (classification as in march_lane_slots_ahead) ----
        const float xn = __fadd_rn(x, dx), yn = __fadd_rn(y, dy), zn = __fadd_rn(z, dz);   // Eq. 2: x_{k+1}
        const Axis b0 = axis_sample(xn, L.n0), b1 = axis_sample(yn, n1), b2 = axis_sample(zn, n2);
        const bool more = k + 1 < L.ns;
        const int d0 = L.n0 > 1 ? b0.f - a0.f : 0, d1 = n1 > 1 ? b1.f - a1.f : 0, d2 = n2 > 1 ? b2.f - a2.f : 0;
        const bool up0 = d0 == 1, up1 = d1 == 1, up2 = d2 == 1;
        const bool dn0 = d0 == -1, dn1 = d1 == -1, dn2 = d2 == -1;
        const bool other = (unsigned)(d0 + 1) > 2u || (unsigned)(d1 + 1) > 2u || (unsigned)(d2 + 1) > 2u;
        const bool sh0 = up0 || dn0, sh1 = up1 || dn1, sh2 = up2 || dn2;
        const int q0 = P0 ^ (dn0 ? 1 : 0), q1 = P1 ^ (dn1 ? 1 : 0), q2 = P2 ^ (dn2 ? 1 : 0);
        // leaving slots of this lane, bit i = slot i: axis 0 bit is i >> 1, axis 1 bit is i & 1
        unsigned mask = other ? 0xFu : 0u;
        mask |= sh0 ? (q0 ? 0xCu : 0x3u) : 0u;
        mask |= sh1 ? (q1 ? 0xAu : 0x5u) : 0u;
        mask |= (sh2 && q2 == sub) ? 0xFu : 0u;
        if (!more) mask = 0u;
        const int Q0 = P0 ^ (sh0 ? 1 : 0), Q1 = P1 ^ (sh1 ? 1 : 0), Q2 = P2 ^ (sh2 ? 1 : 0);   // roles at k+1

        // ---- substep k: weights of x_k in this lane's slot order ----
        const float u0 = 1.0f - a0.t, u1 = 1.0f - a1.t, u2 = 1.0f - a2.t;
        const float f00 = P0 ? a0.t : u0, f01 = P0 ? u0 : a0.t;
        const float f10 = P1 ? a1.t : u1, f11 = P1 ? u1 : a1.t;
        const float f2 = (P2 ^ sub) ? a2.t : u2;
        float w[4];
        w[0] = (f00 * f10) * f2; w[1] = (f00 * f11) * f2; w[2] = (f01 * f10) * f2; w[3] = (f01 * f11) * f2;
        float part[W];
#pragma unroll
        for (int b = 0; b < W; ++b) part[b] = 0.0f;
        if constexpr (W % 2 == 0) {
#pragma unroll
            for (int h = 0; h < W; h += 2) {
                float2 acc = make_float2(0.0f, 0.0f);
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    acc = __ffma2_rn(make_float2(w[i], w[i]), make_float2(gj[i].v[h], gj[i].v[h + 1]), acc);
                part[h] = acc.x; part[h + 1] = acc.y;
            }
        } else {
#pragma unroll
            for (int b = 0; b < W; ++b) {
#pragma unroll
                for (int i = 0; i < 4; ++i) part[b] = fmaf(w[i], gj[i].v[b], part[b]);
            }
        }
        // the slots are read: gather the corners entering at k+1 into the slots they replace
        const int e00 = Q0 ? b0.hi : b0.lo, e01 = Q0 ? b0.lo : b0.hi;
        const int e10 = Q1 ? b1.hi : b1.lo, e11 = Q1 ? b1.lo : b1.hi;
        const int e2 = (Q2 ^ sub) ? b2.hi : b2.lo;
        const int s0 = e00 * n1, s1 = e01 * n1;
        const int ncell[4] = {(s0 + e10) * n2 + e2, (s0 + e11) * n2 + e2, (s1 + e10) * n2 + e2, (s1 + e11) * n2 + e2};
#pragma unroll
        for (int i = 0; i < 4; ++i) ldg_vec_if<W>((mask >> i) & 1u, jg, ncell[i], gj[i]);
        // Eq. 2 with kappa(x_k) and the whole trilinear sum of j(x_k)
        float dep[W];
#pragma unroll
        for (int b = 0; b < W; ++b) {
            const float jk = part[b] + __shfl_xor_sync(pmask, part[b], 1);
            const float kds = gk.v[b] * ds;
            const float att = neg_exp(kds);               // exp(-kappa(x_k) ds)
            const float em = neg_exp(tau[b]);             // exp(-tau_k)
            I[b] = fmaf(I[b], att, jk * em * ds);         // Eq. 2: I_{k+1}
            tau[b] += kds;                                // Eq. 2: tau_{k+1}
            dep[b] = I[b] * scale;
        }
        const int nnn = kappa_cell(b0, b1, b2, xn, yn, zn);
        ldg_vec_if<W>(more && nnn != gnn, kg, nnn, gk);
        gnn = nnn;
        // deposits of substep k into this lane's slots
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            if constexpr (W % 2 == 0) {
#pragma unroll
                for (int h = 0; h < W; h += 2) {
                    const float2 v = __ffma2_rn(make_float2(w[i], w[i]), make_float2(dep[h], dep[h + 1]),
                                                make_float2(pend[i][h], pend[i][h + 1]));
                    pend[i][h] = v.x; pend[i][h + 1] = v.y;
                }
            } else {
#pragma unroll
                for (int b = 0; b < W; ++b) pend[i][b] = fmaf(w[i], dep[b], pend[i][b]);
            }
        }
        // the leaving slots: flush their sums (this substep included), start the entering ones
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const bool f = (mask >> i) & 1u;
            flush_if<W, DET>(f, L, pc[i], pend[i]);
            if constexpr (W % 2 == 0) {
                const float keep = f ? 0.0f : 1.0f;
#pragma unroll
                for (int h = 0; h < W; h += 2) {
                    const float2 v = __fmul2_rn(make_float2(pend[i][h], pend[i][h + 1]), make_float2(keep, keep));
                    pend[i][h] = v.x; pend[i][h + 1] = v.y;
                }
            } else {
#pragma unroll
                for (int b = 0; b < W; ++b) pend[i][b] = f ? 0.0f : pend[i][b];
            }
            pc[i] = f ? ncell[i] : pc[i];
        }
        P0 = Q0; P1 = Q1; P2 = Q2;
        a0 = b0; a1 = b1; a2 = b2;
        x = xn; y = yn; z = zn;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) flush<W, DET>(L, pc[i], pend[i]);
}

// Gathers modes 1 and 3, the corner set as one unit: deposits are merged in registers while the
// set is unchanged and all eight corners are flushed when it changes. AHEAD (mode 1): the gathers
// of substep k+1 are issued before the update of substep k, every substep. Otherwise (mode 3)
// the gathers are issued only when the set (or the kappa cell) changes and reused in between;
// with few lanes per SM and one bin per thread this is faster than the slots of mode 0, whose
// bookkeeping is paid per lane.
// REC: store (x_k, I_k, tau_k) every ck_stride substeps, the forward sweep the reverse march
// would otherwise repeat.
template <int W, bool AHEAD, int DET, bool TILE, bool REC>
__device__ __forceinline__ void march_lane_runs(const Lane& L, RayState<W>& R) {
    constexpr int PF = AHEAD ? 1 : 0;
    const float* __restrict__ jg = L.jg;
    const float* __restrict__ kg = L.kg;
    float* __restrict__ og = L.og;
    const float dx = __fmul_rn(L.n.x, L.ds), dy = __fmul_rn(L.n.y, L.ds), dz = __fmul_rn(L.n.z, L.ds);
    float x = R.x, y = R.y, z = R.z;

    float I[W], tau[W];
#pragma unroll
    for (int b = 0; b < W; ++b) { I[b] = R.I[b]; tau[b] = R.tau[b]; }
    const float ds = L.ds, scale = L.scale;
    // pending deposit of the current run of substeps with an unchanged corner set
    int pc[8];
    float pend[8][W];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        pc[c] = -1;
#pragma unroll
        for (int b = 0; b < W; ++b) pend[c][b] = 0.0f;
    }

    int ptl = -1;   // tile index of the pending run (TILE)
    Sample sm;
    Gathered<W> gd;
    int gnn = -1;   // kappa cell of the gathered values (PF = 0)
    make_sample<TILE>(x, y, z, L.n0, L.n1, L.n2, L.kappa_mode, sm, L.to0, L.to1, L.to2);
    if (PF) gather<W>(jg, kg, sm, gd);

    int ck_left = 0;     // REC: substeps until the next checkpoint
    float* ckp = L.ck;   // REC: this lane's next checkpoint
#pragma unroll 1
    for (int k = 0; k < L.ns; ++k) {
        if (REC) {
            if (ck_left == 0) {
                ckp[0] = x; ckp[L.ck_lanes] = y; ckp[2 * L.ck_lanes] = z;
#pragma unroll
                for (int b = 0; b < W; ++b) {
                    ckp[(3 + b) * L.ck_lanes] = I[b];
                    ckp[(3 + W + b) * L.ck_lanes] = tau[b];
                }
                ckp += (3 + 2 * W) * L.ck_lanes;
                ck_left = L.ck_stride;
            }
            --ck_left;
        }
        x = __fadd_rn(x, dx);                             // Eq. 2: x_{k+1}
        y = __fadd_rn(y, dy);
        z = __fadd_rn(z, dz);
        Sample nx;
        Gathered<W> ng;
        // same 8 corners as the previous substep: the registers already hold their j values
        const bool same_cells = sm.cell[0] == pc[0] && sm.cell[7] == pc[7];
        if (PF) {
            make_sample<TILE>(x, y, z, L.n0, L.n1, L.n2, L.kappa_mode, nx, L.to0, L.to1, L.to2);
            if (k + 1 < L.ns) gather<W>(jg, kg, nx, ng);
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
            const float att = neg_exp(kds);               // exp(-kappa(x_k) ds)
            const float em = neg_exp(tau[b]);             // exp(-tau_k)
            I[b] = fmaf(I[b], att, jk * em * ds);         // Eq. 2: I_{k+1}
            tau[b] += kds;                                // Eq. 2: tau_{k+1}
            dep[b] = I[b] * scale;
        }
        // the corner set is fixed by its lowest and highest corner
        if (!same_cells) {
            if (pc[0] >= 0) flush_run<W, DET, TILE>(L, pc, pend, ptl);
            ptl = TILE ? sm.tl : -1;
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
            make_sample<TILE>(x, y, z, L.n0, L.n1, L.n2, L.kappa_mode, sm, L.to0, L.to1, L.to2);
        }
    }
    if (pc[0] >= 0) flush_run<W, DET, TILE>(L, pc, pend, ptl);
    R.x = x; R.y = y; R.z = z;
#pragma unroll
    for (int b = 0; b < W; ++b) { R.I[b] = I[b]; R.tau[b] = tau[b]; }
    (void)og;
}

// Two adjacent lanes march one ray with corner slots (lanes per ray = 2): lane `sub` keeps the
// four slots whose axis-2 bit is `sub`, so each lane gathers, merges and flushes half of the
// corners, and the workload has twice the warps. Both lanes compute the geometry and the
// radiometry of Eq. 2 alike; the two halves of the trilinear sum of j are exchanged with one
// shuffle per bin (a + b and b + a are the same FP32 number, so both lanes carry identical I
// and tau). pmask holds the pair's two lanes. REC: lane 0 of the pair stores the reverse march's
// checkpoints (x_k, I_k, tau_k) every ck_stride substeps (both lanes hold the same values).
template <int W, bool REC = false, int DET = 0>
__device__ __forceinline__ void march_lane_pair(const Lane& L, int sub, unsigned pmask) {
    const float* __restrict__ jg = L.jg;
    const float* __restrict__ kg = L.kg;
    const float dx = __fmul_rn(L.n.x, L.ds), dy = __fmul_rn(L.n.y, L.ds), dz = __fmul_rn(L.n.z, L.ds);
    float x = L.sx, y = L.sy, z = L.sz;
    float I[W], tau[W];
#pragma unroll
    for (int b = 0; b < W; ++b) { I[b] = 0.0f; tau[b] = 0.0f; }
    const float ds = L.ds, scale = L.scale;
    int pc[4];           // slot i of this lane is slot 2 i + sub of the ray: its cell, -1 while empty
    float pend[4][W];
    Vec<W> gj[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        pc[i] = -1;
#pragma unroll
        for (int b = 0; b < W; ++b) { pend[i][b] = 0.0f; gj[i].v[b] = 0.0f; }
    }
    int rl0 = -2, rh0 = -2, rl1 = -2, rh1 = -2, rl2 = -2, rh2 = -2;
    int P0 = 0, P1 = 0, P2 = 0;
    Vec<W> gk;
#pragma unroll
    for (int b = 0; b < W; ++b) gk.v[b] = 0.0f;
    int gnn = -1;
    int ck_left = 0;     // REC: substeps until the next checkpoint
    float* ckp = L.ck;   // REC: this lane's next checkpoint
#pragma unroll 1
    for (int k = 0; k < L.ns; ++k) {
        if (REC) {
            if (ck_left == 0) {
                if (sub == 0) {
                    ckp[0] = x; ckp[L.ck_lanes] = y; ckp[2 * L.ck_lanes] = z;
#pragma unroll
                    for (int b = 0; b < W; ++b) {
                        ckp[(3 + b) * L.ck_lanes] = I[b];
                        ckp[(3 + W + b) * L.ck_lanes] = tau[b];
                    }
                }
                ckp += (3 + 2 * W) * L.ck_lanes;
                ck_left = L.ck_stride;
            }
            --ck_left;
        }
        const Axis a0 = axis_sample(x, L.n0), a1 = axis_sample(y, L.n1), a2 = axis_sample(z, L.n2);
        const int key0 = a0.lo | (a0.hi << 16), key1 = a1.lo | (a1.hi << 16), key2 = a2.lo | (a2.hi << 16);
        const bool same0 = key0 == (rl0 | (rh0 << 16)), same1 = key1 == (rl1 | (rh1 << 16)),
                   same2 = key2 == (rl2 | (rh2 << 16));
        const bool up0 = !same0 && a0.lo == rh0, up1 = !same1 && a1.lo == rh1, up2 = !same2 && a2.lo == rh2;
        const bool dn0 = !same0 && !up0 && a0.hi == rl0, dn1 = !same1 && !up1 && a1.hi == rl1,
                   dn2 = !same2 && !up2 && a2.hi == rl2;
        const bool change = !(same0 && same1 && same2);
        bool flag[4];
        if (change) {
            const bool other = !(same0 || up0 || dn0) || !(same1 || up1 || dn1) || !(same2 || up2 || dn2);
            const bool sh0 = up0 || dn0, sh1 = up1 || dn1, sh2 = up2 || dn2;
            const int q0 = P0 ^ (dn0 ? 1 : 0), q1 = P1 ^ (dn1 ? 1 : 0), q2 = P2 ^ (dn2 ? 1 : 0);
            unsigned mask = other ? 0xFFu : 0u;   // leaving slots of the ray, as in march_lane_slots
            mask |= sh0 ? (q0 ? 0xF0u : 0x0Fu) : 0u;
            mask |= sh1 ? (q1 ? 0xCCu : 0x33u) : 0u;
            mask |= sh2 ? (q2 ? 0xAAu : 0x55u) : 0u;
            mask >>= sub;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                flag[i] = (mask >> (2 * i)) & 1u;
                flush_if<W, DET>(flag[i] && pc[i] >= 0, L, max(pc[i], 0), pend[i]);
#pragma unroll
                for (int b = 0; b < W; ++b) pend[i][b] = flag[i] ? 0.0f : pend[i][b];
            }
            P0 ^= sh0 ? 1 : 0; P1 ^= sh1 ? 1 : 0; P2 ^= sh2 ? 1 : 0;
            rl0 = a0.lo; rh0 = a0.hi; rl1 = a1.lo; rh1 = a1.hi; rl2 = a2.lo; rh2 = a2.hi;
        }
        const int c00 = P0 ? a0.hi : a0.lo, c01 = P0 ? a0.lo : a0.hi;
        const int c10 = P1 ? a1.hi : a1.lo, c11 = P1 ? a1.lo : a1.hi;
        const int c2 = (P2 ^ sub) ? a2.hi : a2.lo;   // this lane's axis-2 coordinate
        const float u0 = 1.0f - a0.t, u1 = 1.0f - a1.t, u2 = 1.0f - a2.t;
        const float f00 = P0 ? a0.t : u0, f01 = P0 ? u0 : a0.t;
        const float f10 = P1 ? a1.t : u1, f11 = P1 ? u1 : a1.t;
        const float f2 = (P2 ^ sub) ? a2.t : u2;
        float w[4];
        w[0] = (f00 * f10) * f2; w[1] = (f00 * f11) * f2; w[2] = (f01 * f10) * f2; w[3] = (f01 * f11) * f2;
        if (change) {
            const int cell[4] = {(c00 * L.n1 + c10) * L.n2 + c2, (c00 * L.n1 + c11) * L.n2 + c2,
                                 (c01 * L.n1 + c10) * L.n2 + c2, (c01 * L.n1 + c11) * L.n2 + c2};
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                if (flag[i]) {
                    gj[i] = ldg_vec<W>(jg, cell[i]);
                    pc[i] = cell[i];
                }
            }
        }
        const int nn = L.kappa_mode == 0 ? (a0.lo * L.n1 + a1.lo) * L.n2 + a2.lo
                                         : (nearest_round(x, L.n0) * L.n1 + nearest_round(y, L.n1)) * L.n2 +
                                               nearest_round(z, L.n2);
        if (nn != gnn) {
            gk = ldg_vec<W>(kg, nn);
            gnn = nn;
        }
        float dep[W];
#pragma unroll
        for (int b = 0; b < W; ++b) {
            float part = 0.0f;
#pragma unroll
            for (int i = 0; i < 4; ++i) part = fmaf(w[i], gj[i].v[b], part);
            const float jk = part + __shfl_xor_sync(pmask, part, 1);
            const float kds = gk.v[b] * ds;
            const float att = neg_exp(kds);               // exp(-kappa(x_k) ds)
            const float em = neg_exp(tau[b]);             // exp(-tau_k)
            I[b] = fmaf(I[b], att, jk * em * ds);           // Eq. 2: I_{k+1}
            tau[b] += kds;                                  // Eq. 2: tau_{k+1}
            dep[b] = I[b] * scale;
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
#pragma unroll
            for (int b = 0; b < W; ++b) pend[i][b] = fmaf(w[i], dep[b], pend[i][b]);
        }
        x = __fadd_rn(x, dx);                               // Eq. 2: x_{k+1}
        y = __fadd_rn(y, dy);
        z = __fadd_rn(z, dz);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
        if (pc[i] >= 0) flush<W, DET>(L, pc[i], pend[i]);
}

// Gathers modes: PF = 0 march_lane_slots, 1 and 3 march_lane_runs, 2 march_lane_ahead, 4
// march_lane_slots_ahead (no tiles). REC (checkpoints) is available with modes 0, 1, 3 and 4.
template <int W, int PF, int DET = 0, bool TILE = false, bool REC = false>
__device__ __forceinline__ void march_lane(const Lane& L, RayState<W>& R) {
    if (PF == 4) march_lane_slots_ahead<W, DET, REC>(L, R);
    else if (PF == 2) march_lane_ahead<W, DET, TILE>(L, R);
    else if (PF == 0) march_lane_slots<W, DET, TILE, REC>(L, R);
    else march_lane_runs<W, PF == 1, DET, TILE, REC>(L, R);
}

}  // namespace rt
