// march_bwd.cu -- reverse-mode adjoint of the forward march (sm_103a).
//
// For a loss L with G = dL/d(field), differentiating Eq. 2 along one ray and bin gives, with
// a_k = exp(-kappa_k ds), E_k = exp(-tau_k), e_k = j_k E_k ds and s = 4 pi / N_Omega:
//     g_k       = s * sum_c w_{k,c} G[c_{k,c}]          (adjoint of the deposit of I_{k+1})
//     lam_{k+1} = g_k + a_{k+1} lam_{k+2},   lam_{N_s+1} = 0
//     dj[c_{k,c}]  += lam_{k+1} E_k ds w_{k,c}            (adjoint of the trilinear gather)
//     dkap[cell_k] += -ds (lam_{k+1} I_k a_k + mu_{k+1}),  (nearest-cell kappa)
//     mu_k = mu_{k+1} + lam_{k+1} e_k,  mu_{N_s} = 0.
// One thread per (ray, source, bin group). A forward sweep stores (x_k, I_k, tau_k) every K
// substeps; the reverse sweep replays each K-substep segment from its checkpoint into a
// per-thread record (x_k, I_k, E_k, a_k, e_k) and then walks it backwards, so the forward state
// is recomputed exactly and never reconstructed by dividing out exp(-kappa ds). Scatters into
// dj / dkappa are merged in registers while the corner set (or kappa cell) is unchanged, and
// gathers are skipped while it is unchanged (the registers still hold those corner values). With
// one bin and K = 4 a segment's four samples are formed from its checkpoint first and all their
// gathers (j, kappa, G) issued together, so the replay and the walk run on registers.
#include "march_common.cuh"
#include "rt_internal.h"

namespace rt {

// SG: also dL/d(source position). Each position of the ray is x_k = src + k n ds, so the source
// gradient sums dL/dx_k over substeps with everything else fixed. x_k enters through trilinear
// weights twice: the deposit of I_{k+1} and the gather of j (adjoint lam_{k+1} E_k ds). With the
// corner values V_c = s I_{k+1} G[c] + lam_{k+1} E_k ds j[c] (summed over the lane's bins),
// dL/dx_k is the gradient of the trilinear interpolant of V at x_k; the nearest-cell kappa is
// piecewise constant and contributes nothing, and on a clamped axis the two corners are one
// cell, so that component vanishes. The lanes of a block share the source: a warp reduction,
// then one atomic per warp and axis.
template <int W, int K, bool SG>
__global__ void __launch_bounds__(256) k_march_bwd(BackArgs a) {
    const int rblocks = (a.ray_count + blockDim.x - 1) / blockDim.x;
    const int rb = blockIdx.x % rblocks;
    const int sg = blockIdx.x / rblocks;
    const int s = sg % a.nsrc;
    const int g = sg / a.nsrc;
    const int r = rb * blockDim.x + threadIdx.x;
    float gsx = 0.0f, gsy = 0.0f, gsz = 0.0f;   // SG: this lane's dL/d(source position)
    if (!SG && r >= a.ray_count) return;
    if (r < a.ray_count) {
    const long long lanes = (long long)a.ray_count * a.nsrc * ((a.n_freq + W - 1) / W);
    const long long lane = ((long long)g * a.nsrc + s) * a.ray_count + r;

    const long long ncell = (long long)a.n0 * a.n1 * a.n2;
    const float* __restrict__ jg = a.j + (size_t)g * ncell * W;
    const float* __restrict__ kg = a.kappa + (size_t)g * ncell * W;
    const float* __restrict__ Gg = a.grad + (size_t)g * ncell * W;
    float* __restrict__ djg = a.dj ? a.dj + (size_t)g * ncell * W : nullptr;
    float* __restrict__ dkg = a.dk ? a.dk + (size_t)g * ncell * W : nullptr;
    // dL/dj and dL/dkappa together: kept in L2 while they fit (red_policy)
    const int bwd_groups = (a.n_freq + W - 1) / W;
    const unsigned long long pol = red_policy(8LL * bwd_groups * ncell * W);

    const float4 n = a.dirs[r];
    const float ds = a.ds;
    const float dx = __fmul_rn(n.x, ds), dy = __fmul_rn(n.y, ds), dz = __fmul_rn(n.z, ds);
    constexpr int F = 3 + 2 * W;   // checkpoint fields: x, y, z, I[W], tau[W]
    float* __restrict__ ck = a.ckpt;
    auto ck_at = [&](int c, int f) -> float& { return ck[((size_t)c * F + f) * lanes + lane]; };

    // ---- forward sweep: Eq. 2, checkpoint every K substeps (skipped when the forward march
    // recorded them for these very inputs: same pointers and scalars, checked on the host, and
    // the same content hash of j, kappa and the sources, checked here) ----
    const bool have = a.have_ckpt && (!a.hash_rec || *a.hash_rec == *a.hash_now);
    if (!have) {
        float x = a.src[3 * s + 0], y = a.src[3 * s + 1], z = a.src[3 * s + 2];
        float I[W], tau[W];
#pragma unroll
        for (int b = 0; b < W; ++b) { I[b] = 0.0f; tau[b] = 0.0f; }
        Vec<W> jc[8], kc;
        int c0 = -1, c7 = -1, cn = -1;   // cells of the values held in jc / kc
#pragma unroll 1
        for (int k = 0; k < a.ns; ++k) {
            if (k % K == 0) {
                const int c = k / K;
                ck_at(c, 0) = x; ck_at(c, 1) = y; ck_at(c, 2) = z;
#pragma unroll
                for (int b = 0; b < W; ++b) { ck_at(c, 3 + b) = I[b]; ck_at(c, 3 + W + b) = tau[b]; }
            }
            Sample sm;
            make_sample(x, y, z, a.n0, a.n1, a.n2, a.kappa_mode, sm);
            if (sm.cell[0] != c0 || sm.cell[7] != c7) {
#pragma unroll
                for (int c = 0; c < 8; ++c) jc[c] = ldg_vec<W>(jg, sm.cell[c]);
                c0 = sm.cell[0]; c7 = sm.cell[7];
            }
            if (sm.nn != cn) { kc = ldg_vec<W>(kg, sm.nn); cn = sm.nn; }
#pragma unroll
            for (int b = 0; b < W; ++b) {
                float jk = 0.0f;
#pragma unroll
                for (int c = 0; c < 8; ++c) jk = fmaf(sm.w[c], jc[c].v[b], jk);
                const float kds = kc.v[b] * ds;
                I[b] = fmaf(I[b], neg_exp(kds), jk * neg_exp(tau[b]) * ds);
                tau[b] += kds;
            }
            x = __fadd_rn(x, dx);
            y = __fadd_rn(y, dy);
            z = __fadd_rn(z, dz);
        }
    }

    // ---- reverse sweep ----
    float lam_next[W], a_next[W], mu[W];
#pragma unroll
    for (int b = 0; b < W; ++b) { lam_next[b] = 0.0f; a_next[b] = 0.0f; mu[b] = 0.0f; }
    int pc[8];
    float pdj[8][W];
    int pnn = -1;
    float pdk[W];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        pc[c] = -1;
#pragma unroll
        for (int b = 0; b < W; ++b) pdj[c][b] = 0.0f;
    }
#pragma unroll
    for (int b = 0; b < W; ++b) pdk[b] = 0.0f;

    Vec<W> gc[8];                     // G at the corners of pc (the pending dj corner set)
    int g0 = -1, g7 = -1;
    Vec<W> jr[8];                     // SG: j at the corners of the current substep
    int jr0 = -1, jr7 = -1;
    // per-thread segment record: x, I_k, E_k, a_k, e_k. For strides up to 8 the segment loops
    // are unrolled with constant indices, so the record lives in registers; longer records go
    // to local memory
    float rx[K], ry[K], rz[K], rI[K][W], rE[K][W], ra[K][W], re[K][W];
    // one bin with K = 4: the segment's gathers are issued together (below)
    constexpr bool kBatch = K == 4 && W == 1;
    const int nseg = (a.ns + K - 1) / K;
#pragma unroll 1
    for (int seg = nseg - 1; seg >= 0; --seg) {
        const int k0 = seg * K;
        const int len = min(K, a.ns - k0);
        float x = ck_at(seg, 0), y = ck_at(seg, 1), z = ck_at(seg, 2);
        float I[W], tau[W];
#pragma unroll
        for (int b = 0; b < W; ++b) { I[b] = ck_at(seg, 3 + b); tau[b] = ck_at(seg, 3 + W + b); }
        // One replay step (the forward sweep's Eq. 2 exactly as it ran it) for sample sm with the j
        // values jv of its corners and kappa kv at its cell: fills the record at q, advances I, tau.
        auto replay_step = [&](const int q, const Sample& sm, const Vec<W>* jv, const Vec<W>& kv, float px,
                               float py, float pz) {
            rx[q] = px; ry[q] = py; rz[q] = pz;
#pragma unroll
            for (int b = 0; b < W; ++b) {
                float jk = 0.0f;
#pragma unroll
                for (int c = 0; c < 8; ++c) jk = fmaf(sm.w[c], jv[c].v[b], jk);
                const float kds = kv.v[b] * ds;
                const float att = neg_exp(kds), em = neg_exp(tau[b]);
                const float emis = jk * em * ds;
                rI[q][b] = I[b]; rE[q][b] = em; ra[q][b] = att; re[q][b] = emis;
                I[b] = fmaf(I[b], att, emis);
                tau[b] += kds;
            }
        };
        // One reverse step at record q for sample sm, with G (gv) and, for the source gradient,
        // j (jv) at its corners: lam, mu, the dj / dkappa contributions (merged while the corner
        // set / kappa cell is unchanged) and dL/dx_q.
        auto walk_step = [&](const int q, const Sample& sm, const Vec<W>* gv, const Vec<W>* jv) {
            float ddj[W], ddk[W];
#pragma unroll
            for (int b = 0; b < W; ++b) {
                float gk = 0.0f;
#pragma unroll
                for (int c = 0; c < 8; ++c) gk = fmaf(sm.w[c], gv[c].v[b], gk);
                const float lam = fmaf(a_next[b], lam_next[b], gk * a.scale);      // lam_{k+1}
                ddj[b] = lam * rE[q][b] * ds;
                ddk[b] = -ds * fmaf(lam * rI[q][b], ra[q][b], mu[b]);              // uses mu_{k+1}
                mu[b] = fmaf(lam, re[q][b], mu[b]);                                // mu_k
                lam_next[b] = lam;
                a_next[b] = ra[q][b];
            }
            if (SG) {
                float V[8];
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    float v = 0.0f;
#pragma unroll
                    for (int b = 0; b < W; ++b) {
                        const float In = fmaf(rI[q][b], ra[q][b], re[q][b]);     // I_{k+1}
                        v = fmaf(a.scale * In, gv[c].v[b], v);
                        v = fmaf(ddj[b], jv[c].v[b], v);
                    }
                    V[c] = v;
                }
                const float t0 = __fsub_rn(rx[q], floorf(rx[q]));
                const float t1 = __fsub_rn(ry[q], floorf(ry[q]));
                const float t2 = __fsub_rn(rz[q], floorf(rz[q]));
                const float u0 = 1.0f - t0, u1 = 1.0f - t1, u2 = 1.0f - t2;
                // corner c = (bit axis 0, bit axis 1, bit axis 2) = (c >> 2, c >> 1, c) & 1
                gsx += ((V[4] - V[0]) * u1 * u2 + (V[5] - V[1]) * u1 * t2 + (V[6] - V[2]) * t1 * u2 +
                        (V[7] - V[3]) * t1 * t2);
                gsy += ((V[2] - V[0]) * u0 * u2 + (V[3] - V[1]) * u0 * t2 + (V[6] - V[4]) * t0 * u2 +
                        (V[7] - V[5]) * t0 * t2);
                gsz += ((V[1] - V[0]) * u0 * u1 + (V[3] - V[2]) * u0 * t1 + (V[5] - V[4]) * t0 * u1 +
                        (V[7] - V[6]) * t0 * t1);
            }
            if (djg) {
                if (sm.cell[0] != pc[0] || sm.cell[7] != pc[7]) {
                    if (pc[0] >= 0) {
#pragma unroll
                        for (int c = 0; c < 8; ++c) red_vec<W>(djg, pc[c], pdj[c], pol);
                    }
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        pc[c] = sm.cell[c];
#pragma unroll
                        for (int b = 0; b < W; ++b) pdj[c][b] = sm.w[c] * ddj[b];
                    }
                } else {
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
#pragma unroll
                        for (int b = 0; b < W; ++b) pdj[c][b] = fmaf(sm.w[c], ddj[b], pdj[c][b]);
                    }
                }
            }
            if (dkg) {
                if (sm.nn != pnn) {
                    if (pnn >= 0) red_vec<W>(dkg, pnn, pdk, pol);
                    pnn = sm.nn;
#pragma unroll
                    for (int b = 0; b < W; ++b) pdk[b] = ddk[b];
                } else {
#pragma unroll
                    for (int b = 0; b < W; ++b) pdk[b] += ddk[b];
                }
            }
        };
        if constexpr (!kBatch) {
            // replay the segment exactly as the forward sweep ran it, gathering the corner set
            // when it changes; then walk it backwards, gathering G (and j) likewise
            Vec<W> jc[8], kc;
            int c0 = -1, c7 = -1, cn = -1;
            auto replay = [&](const int q) {
                Sample sm;
                make_sample(x, y, z, a.n0, a.n1, a.n2, a.kappa_mode, sm);
                if (sm.cell[0] != c0 || sm.cell[7] != c7) {
#pragma unroll
                    for (int c = 0; c < 8; ++c) jc[c] = ldg_vec<W>(jg, sm.cell[c]);
                    c0 = sm.cell[0]; c7 = sm.cell[7];
                }
                if (sm.nn != cn) { kc = ldg_vec<W>(kg, sm.nn); cn = sm.nn; }
                replay_step(q, sm, jc, kc, x, y, z);
                x = __fadd_rn(x, dx);
                y = __fadd_rn(y, dy);
                z = __fadd_rn(z, dz);
            };
            if constexpr (K <= 8) {   // constant indices: the record stays in registers
#pragma unroll
                for (int q = 0; q < K; ++q)
                    if (q < len) replay(q);
            } else {
#pragma unroll 1
                for (int q = 0; q < len; ++q) replay(q);
            }
            auto walk = [&](const int q) {
                Sample sm;
                make_sample(rx[q], ry[q], rz[q], a.n0, a.n1, a.n2, a.kappa_mode, sm);
                if (sm.cell[0] != g0 || sm.cell[7] != g7) {
#pragma unroll
                    for (int c = 0; c < 8; ++c) gc[c] = ldg_vec<W>(Gg, sm.cell[c]);
                    g0 = sm.cell[0]; g7 = sm.cell[7];
                }
                if (SG && (sm.cell[0] != jr0 || sm.cell[7] != jr7)) {
#pragma unroll
                    for (int c = 0; c < 8; ++c) jr[c] = ldg_vec<W>(jg, sm.cell[c]);
                    jr0 = sm.cell[0]; jr7 = sm.cell[7];
                }
                walk_step(q, sm, gc, jr);
            };
            if constexpr (K <= 8) {
#pragma unroll
                for (int q = K - 1; q >= 0; --q)
                    if (q < len) walk(q);
            } else {
#pragma unroll 1
                for (int q = len - 1; q >= 0; --q) walk(q);
            }
        } else {
            // one bin, K = 4: every position of the segment follows from its checkpoint, so its
            // samples are formed first and all their gathers (j and kappa for the replay, G for
            // the walk) are issued together -- one L2 round trip per segment instead of one per
            // corner-set change -- and both passes then run on registers
            Sample smq[K];
            float px[K], py[K], pz[K];
            Vec<W> jq[K][8], kq[K], gq[K][8];
#pragma unroll
            for (int q = 0; q < K; ++q) {
                px[q] = x; py[q] = y; pz[q] = z;
                make_sample(x, y, z, a.n0, a.n1, a.n2, a.kappa_mode, smq[q]);
                x = __fadd_rn(x, dx);
                y = __fadd_rn(y, dy);
                z = __fadd_rn(z, dz);
            }
#pragma unroll
            for (int q = 0; q < K; ++q) {
                if (q < len) {
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        jq[q][c] = ldg_vec<W>(jg, smq[q].cell[c]);
                        gq[q][c] = ldg_vec<W>(Gg, smq[q].cell[c]);
                    }
                    kq[q] = ldg_vec<W>(kg, smq[q].nn);
                }
            }
#pragma unroll
            for (int q = 0; q < K; ++q)
                if (q < len) replay_step(q, smq[q], jq[q], kq[q], px[q], py[q], pz[q]);
#pragma unroll
            for (int q = K - 1; q >= 0; --q)
                if (q < len) walk_step(q, smq[q], gq[q], jq[q]);
        }
    }
    if (djg && pc[0] >= 0) {
#pragma unroll
        for (int c = 0; c < 8; ++c) red_vec<W>(djg, pc[c], pdj[c], pol);
    }
    if (dkg && pnn >= 0) red_vec<W>(dkg, pnn, pdk, pol);
    }   // r < ray_count
    if (SG) {
        // every thread of the block reaches here (blocks are whole warps; lanes past the last ray
        // contribute zero)
        for (int o = 16; o > 0; o >>= 1) {
            gsx += __shfl_xor_sync(0xffffffffu, gsx, o);
            gsy += __shfl_xor_sync(0xffffffffu, gsy, o);
            gsz += __shfl_xor_sync(0xffffffffu, gsz, o);
        }
        if ((threadIdx.x & 31) == 0) {
            atomicAdd(a.dsrc + 3 * s + 0, gsx);
            atomicAdd(a.dsrc + 3 * s + 1, gsy);
            atomicAdd(a.dsrc + 3 * s + 2, gsz);
        }
    }
}

size_t backward_ckpt_floats(const BackArgs& a, int W) {
    const int K = a.stride;
    const long long lanes = (long long)a.ray_count * a.nsrc * ((a.n_freq + W - 1) / W);
    const long long nck = (a.ns + K - 1) / K;
    return (size_t)(nck * (3 + 2 * W) * lanes);
}

cudaError_t launch_march_bwd(int W, const BackArgs& a, cudaStream_t st) {
    const int block = a.block > 0 ? a.block : 32;
    const long long rblocks = (a.ray_count + block - 1) / block;
    const long long groups = (a.n_freq + W - 1) / W;
    const long long nblk = rblocks * a.nsrc * groups;
    if (nblk <= 0) return cudaSuccess;
    if (nblk > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    const unsigned grid = (unsigned)nblk;
    if (block % 32) return cudaErrorInvalidValue;
    const int key = (W * 100 + a.stride) * 2 + (a.dsrc ? 1 : 0);
    switch (key) {
#define RT_BWD_CASE(W_, K_)                                                                        \
        case (W_ * 100 + K_) * 2: k_march_bwd<W_, K_, false><<<grid, block, 0, st>>>(a); break;    \
        case (W_ * 100 + K_) * 2 + 1: k_march_bwd<W_, K_, true><<<grid, block, 0, st>>>(a); break;
        RT_BWD_CASE(1, 4) RT_BWD_CASE(1, 8) RT_BWD_CASE(1, 16) RT_BWD_CASE(1, 32)
        RT_BWD_CASE(2, 4) RT_BWD_CASE(2, 8) RT_BWD_CASE(2, 16) RT_BWD_CASE(2, 32)
        RT_BWD_CASE(4, 4) RT_BWD_CASE(4, 8) RT_BWD_CASE(4, 16) RT_BWD_CASE(4, 32)
#undef RT_BWD_CASE
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace rt
