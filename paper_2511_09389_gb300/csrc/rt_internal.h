// rt_internal.h -- launchers shared between the C-ABI host code and the kernel files.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "raytrax.h"

namespace rt {

// Fibonacci lattice rays [begin, end) of an n-ray lattice, FP64 -> FP32, sorted into angular
// patches; writes end-begin float4 entries to out. key/order: caller buffers of end-begin
// entries (the function allocates nothing).
void sorted_lattice(int n, int begin, int end, float4* out, uint32_t* key, int* order);

// N_s = ceil(c dt / ds) in FP64 with a 1e-9 relative guard, capped when cap > 0; -1 if the
// arguments are invalid or N_s does not fit in an int (paper Sec. 2 after Eq. 2).
int substeps(float ds, float c, float dt, int cap);

// Record a message for rt_last_error() on this thread and return st.
rt_status set_error(rt_status st, const char* msg);

// One forward march launch over a set of (source, bin-group, ray) lanes.
struct MarchArgs {
    const float* jp;        // packed j    [groups][ncell][W]   (W = 1: plain [n_freq][ncell])
    const float* kp;        // packed kappa, same layout
    float* acc;             // FP32 accumulator, same layout (W = 1: may be the output itself)
    int acc_mode;               // 0: FP32 reductions into acc; 1: 64-bit fixed point into acc64
                                // (deterministic mode); 2: FP64 reductions into acc64 (as double)
    unsigned long long* acc64;  // 8-byte accumulator [groups][W][ncell] (modes 1 and 2) or NULL
    const float* fix;           // fixed-point units per unit deposit, a power of two (device scalar)
    const float4* dirs;     // ray directions (xyz, w unused), ray_count entries
    const float* src;       // device [nsrc][3]
    int n0, n1, n2;
    int ns;                 // substeps N_s
    float ds;               // step length
    float dep_scale;        // factor applied to every deposit (4 pi / N_Omega, or 1)
    int ray_count;
    int nsrc;
    int groups;             // bin groups of width W
    int n_freq;             // real bins (deterministic mode writes only these)
    int kappa_mode;
    int block;              // threads per block
    int prefetch;           // gathers mode. 0: corner slots (a face shared by consecutive corner
                            // sets keeps its gathers and sums); 1: the next substep's gathers
                            // issued before the current update; 2: both; 3: the whole corner set
                            // reused while unchanged, flushed and re-gathered when it changes;
                            // 4: corner slots with the entering corners gathered a substep early
    int lanes_per_ray;      // 1, or 2 adjacent lanes sharing a ray (each with half of its corner slots)
    int tile;               // 1: source deposit tiles in shared memory (FP32 mode, one lane per ray)
    // stateful advance (NULL st_I: none): st_I / st_tau [n_freq][nsrc][ray_count], positions
    // [nsrc][ray_count][3] read from st_pos_in when st_read and written to st_pos_out (a
    // different buffer: every bin group of a ray reads the position)
    const float* st_pos_in;
    float* st_pos_out;
    float* st_I;
    float* st_tau;
    int st_read;
    // adjoint checkpoints recorded during the march (NULL: none), layout of BackArgs::ckpt
    float* ckpt;
    int ck_stride;
};

cudaError_t launch_march_fwd(int W, const MarchArgs& a, cudaStream_t st);
// Whether a forward kernel is compiled for this plan and accumulation (acc_mode as in MarchArgs;
// record: with adjoint checkpoints) and accepts this block size. launch_march_fwd returns
// cudaErrorInvalidValue otherwise.
bool march_fwd_available(int W, int prefetch, int acc_mode, int tile, int record, int lanes_per_ray, int block);

// A forward launch plan: bins per thread W, threads per block, gather mode (MarchArgs::prefetch),
// lanes per ray, source tiles.
struct MarchPlan {
    int W, block, prefetch, lpr, tile;
};
// The plans the autotuners time for n_freq bins (rt_api.cu for single calls, rt_batch.cu for the
// batch's dedicated instances), at most kMaxMarchPlans; returns how many were written to out.
constexpr int kMaxMarchPlans = 132;
int march_plan_candidates(int n_freq, MarchPlan* out);

// [n_freq][ncell] -> [groups][ncell][W] (bins >= n_freq padded with zero).
cudaError_t launch_pack(const float* in, float* out, int n_freq, int W, int groups, long long ncell,
                        cudaStream_t st);
// j and kappa packed in one launch, and acc (if not NULL) set to zero, all [groups][ncell][W].
cudaError_t launch_pack_pair(const float* j, const float* kappa, float* jp, float* kp, float* acc, int n_freq, int W,
                             int groups, long long ncell, cudaStream_t st);
// out[b][c] (+)= scale * acc[b / W][c][b % W]
cudaError_t launch_unpack(const float* acc, float* out, int n_freq, int W, long long ncell,
                          float scale, int accumulate, cudaStream_t st);
// Fixed-point accumulation: acc (nacc words) set to zero and *fix = the largest power of two with
// fix * per_jmax * max|j| <= 2^62 (j: nj floats), in one launch; work: 2 device words, zero before
// the first call and left zero by every call.
cudaError_t launch_fix_prepare(const float* j, long long nj, unsigned long long* acc, long long nacc,
                               double per_jmax, unsigned* work, float* fix, cudaStream_t st);
// out[b][c] (+)= acc[b / W][c][b % W] / *fix.
// Checked mode: flags (4 device ints, cleared first) mark non-finite j / negative or non-finite
// kappa / non-finite or too large source coordinates / non-finite extra (a loss gradient, may be NULL).
cudaError_t launch_check_inputs(const float* j, const float* kappa, long long n, const float* src, int nsrc,
                                const float* extra, int* flags, cudaStream_t st);
// *out = a 64-bit content hash of j and kappa (n floats each) and the source coordinates
// (order-independent; equal inputs give equal hashes); checkpoint reuse compares two of them.
cudaError_t launch_input_hash(const float* j, const float* kappa, long long n, const float* src, int nsrc,
                              unsigned long long* out, cudaStream_t st);
// FP64 accumulation: out[b][c] (+)= (float) (scale * acc[b / W][c][b % W]), the product in FP64.
cudaError_t launch_f64_to_float(const double* acc, int n_freq, long long ncell, double scale, float* out,
                                int accumulate, cudaStream_t st);
cudaError_t launch_fixed_to_float(const unsigned long long* acc, int n_freq, long long ncell, const float* fix,
                                  float* out, int accumulate, cudaStream_t st);

// Geometry trace of one ray (test hook).
cudaError_t launch_trace(float sx, float sy, float sz, float nx, float ny, float nz, float ds,
                         int ns, int n0, int n1, int n2, int kappa_mode, long long* base,
                         long long* nn, cudaStream_t st);

// Reverse-mode adjoint.
struct BackArgs {
    const float* grad;      // G, packed like j
    const float* j;         // packed [groups][ncell][W] (W = 1: plain [n_freq][ncell])
    const float* kappa;     // packed like j
    float* dj;              // accumulator packed like j, or NULL (not wanted)
    float* dk;              // accumulator packed like j, or NULL (not wanted)
    float* dsrc;            // dL/d(source positions) [nsrc][3], accumulated, or NULL (not wanted)
    int have_ckpt;          // 1: ckpt may hold this problem's checkpoints (skip the forward sweep when
                            // the hashes below agree, or when they are NULL)
    const unsigned long long* hash_rec;   // input hash taken when the checkpoints were recorded
    const unsigned long long* hash_now;   // input hash of this call
    float* ckpt;            // checkpoint scratch
    const float4* dirs;
    const float* src;
    int n0, n1, n2;
    int ns;
    int stride;             // checkpoint stride K
    float ds;
    float scale;            // 4 pi / N_Omega
    int ray_count;
    int nsrc;
    int n_freq;
    int kappa_mode;
    int block;
};
// Checkpoint scratch (floats) for bin-group width W and stride a.stride.
size_t backward_ckpt_floats(const BackArgs& a, int W);
// W in {1, 2, 4}, a.stride in {4, 8, 16, 32}.
cudaError_t launch_march_bwd(int W, const BackArgs& a, cudaStream_t st);

// One instance of a batched launch (device-resident table entry).
struct BatchInst {
    const float* j;         // caller's j   [n_freq][ncell]
    const float* kappa;     // caller's kappa
    float* out;             // caller's field (overwritten)
    const float* jp;        // march inputs: packed copies (W > 1) or the caller's arrays (W = 1)
    const float* kp;
    float* jp_w;            // writable packed copies (W > 1), else NULL
    float* kp_w;
    float* acc;             // packed accumulator [groups][ncell][W]
    const float4* dirs;     // sorted lattice of ray_count rays
    const float* src;       // device [nsrc][3]
    int n0, n1, n2, n_freq, W, groups, ns, nsrc, ray_count, kappa_mode;
    float ds, scale;
};

int march_batch_blocks_per_sm(int W, int block);
// items of width-W instances: (instance, source, bin group, first ray) x n_items;
// counter: device int, zero at launch
cudaError_t launch_march_batch(int W, const BatchInst* insts, const int4* items, int n_items, int* counter,
                               int grid, int block, cudaStream_t st);
// max_elems: the largest groups * ncell over the instances (sizes the grid)
cudaError_t launch_pack_batch(const BatchInst* insts, int n_inst, long long max_elems, int which, cudaStream_t st);
cudaError_t launch_unpack_batch(const BatchInst* insts, int n_inst, long long max_elems, cudaStream_t st);

// One 3x3x3 convolution layer on the tensor cores (conv3d_tc.cu). Activations in the C32
// layout: bf16 [B][D][H][W][32], channels beyond the real count zero; W must be 64, H even.
struct ConvLaunch {
    const void* x;            // C32 input
    const void* w_packed;     // bf16 [27][32 out][32 in] (tap = (dz+1)*9 + (dy+1)*3 + (dx+1))
    const float* bias;        // [c_out] or NULL
    const void* mask_src;     // C32 or NULL: outputs where it is <= 0 are scaled by slope
    void* y;                  // C32 output, or NULL
    float* y_f32;             // [B][D][H][W] FP32 copy of output channel 0, or NULL
    int B, D, H, W;
    int c_out;                // real output channels (the rest are written as 0)
    int dil;                  // dilation
    int act;                  // 0: identity, 1: LeakyReLU(slope)
    float slope;
    int* err;                 // device error word (timeouts)
};
cudaError_t launch_conv3d_tc(const ConvLaunch& c, cudaStream_t st);

// Weight gradient of one layer on the tensor cores: dw[co][ci][27] += sum over voxels of
// dz[v][co] * x[v + off(tap)][ci]. x, dz: C32.
struct WgradLaunch {
    const void* x;
    const void* dz;
    float* dw;
    int B, D, H, W, c_in, c_out, dil;
    int* err;
};
cudaError_t launch_conv3d_wgrad(const WgradLaunch& c, cudaStream_t st);
// db[co] += sum over voxels of dz[v][co] (dz: C32).
cudaError_t launch_bias_grad(const void* dz, int B, long long vox, int c_out, float* db, cudaStream_t st);

// Surrogate element-wise and reduction kernels (surrogate_ops.cu).
cudaError_t launch_features(const float* kappa, const float* j, int B, long long vox, void* x, cudaStream_t st);
cudaError_t launch_field_max(const float* f, int B, long long vox, float* out, cudaStream_t st);
cudaError_t launch_log_loss(const float* pred, const float* field, int B, long long vox, const float* fmax,
                            float eps_rel, float mu, float sigma, void* grad, float* loss, cudaStream_t st);
cudaError_t launch_field_error(const float* pred, const float* field, int B, long long vox, const float* fmax,
                               float eps_rel, float mu, float sigma, float* out, cudaStream_t st);
cudaError_t launch_channel_mean(const void* x, int B, int C, long long vox, float* out, cudaStream_t st);
cudaError_t launch_adam(float* p, const float* g, float* m, float* v, long long n, float lr, float b1, float b2,
                        float eps, int step, cudaStream_t st);

// Emissivity inversion (inversion.cu). fmax: device scalar, the target's maximum; eps =
// eps_rel * fmax. log_t = log(target + eps); the misfit writes dL/dF to grad (if non-NULL) and
// adds mean (log(F + eps) - log_t)^2 to *loss; the Adam step (bias corrections as launch_adam)
// is followed by p = max(p, lower).
cudaError_t launch_log_target(const float* target, long long n, const float* fmax, float eps_rel, float* log_t,
                              cudaStream_t st);
cudaError_t launch_log_misfit(const float* F, const float* log_t, long long n, const float* fmax, float eps_rel,
                              float* grad, float* loss, cudaStream_t st);
cudaError_t launch_adam_projected(float* p, const float* g, float* m, float* v, long long n, float lr, float b1,
                                  float b2, float eps, int step, float lower, cudaStream_t st);

// FP32 [B][C][vox] <-> C32 bf16 [B][vox][32] (channels >= C are zero), C <= 32.
cudaError_t launch_to_c32(const float* src, int B, int C, long long vox, void* dst, cudaStream_t st);
cudaError_t launch_from_c32(const void* src, int B, int C, long long vox, float* dst, cudaStream_t st);
// FP32 [c_out][c_in][27] -> bf16 [27][32][32] (tap, n, k); forward: n = output, k = input
// channel; transpose = 1 (data gradient): flipped taps, n = input, k = output channel.
cudaError_t launch_pack_weights(const float* w, int c_in, int c_out, int transpose, void* packed, cudaStream_t st);

// Microbenchmarks of L2 reductions and gathers (microbench.cu): kind 0-4, vec 1 or 4 floats.
cudaError_t launch_microbench(int kind, int vec, float* buf, long long nvec, int edge, int iters, int grid,
                              int block, cudaStream_t st);

}  // namespace rt
