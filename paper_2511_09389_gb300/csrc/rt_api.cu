// rt_api.cu -- host side of the C ABI declared in include/raytrax.h.
//
// Validation, the substep rule, the Fibonacci lattice (built in FP64 on the host, rounded to
// FP32 and sorted into angular patches), handle-owned scratch, and the dispatch of the march
// kernels on the caller's stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "raytrax.h"
#include "rt_internal.h"

namespace {

thread_local std::string g_last_error;

rt_status fail(rt_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

rt_status cuda_fail(cudaError_t e, const char* what) {
    if (e == cudaErrorMemoryAllocation)
        return fail(RT_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
    return fail(RT_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define RT_CUDA(call, what)                             \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

// ---- Fibonacci lattice (Sec. 2) ------------------------------------------------------------
// n_i = (rho cos phi, rho sin phi, z), z = 1 - (2i+1)/N, rho = sqrt(1 - z^2),
// phi = i * pi (3 - sqrt 5) mod 2 pi, in FP64, each component rounded once to FP32.
void lattice_entry(int i, int n, float out[3]) {
    const double pi = 3.14159265358979323846;
    const double golden = pi * (3.0 - std::sqrt(5.0));
    const double z = 1.0 - (2.0 * i + 1.0) / (double)n;
    const double rho = std::sqrt(std::fmax(0.0, 1.0 - z * z));
    const double phi = std::fmod((double)i * golden, 2.0 * pi);
    out[0] = (float)(rho * std::cos(phi));
    out[1] = (float)(rho * std::sin(phi));
    out[2] = (float)z;
}

// Sort key grouping angular neighbours: cube face of the direction, then a Morton code of the
// two minor components over that face. Consecutive keys form compact patches on the sphere,
// so a warp's rays start out sharing cells near the source.
uint32_t spread10(uint32_t v) {
    v &= 0x3ff;
    v = (v | (v << 16)) & 0x030000ff;
    v = (v | (v << 8)) & 0x0300f00f;
    v = (v | (v << 4)) & 0x030c30c3;
    v = (v | (v << 2)) & 0x09249249;
    return v;
}

uint32_t angular_key(const float d[3]) {
    const float ax = std::fabs(d[0]), ay = std::fabs(d[1]), az = std::fabs(d[2]);
    int major;
    if (ax >= ay && ax >= az) major = 0;
    else if (ay >= az) major = 1;
    else major = 2;
    const float m = std::fmax(std::fabs(d[major]), 1e-30f);
    const int u_ax = (major + 1) % 3, v_ax = (major + 2) % 3;
    const float u = d[u_ax] / m, v = d[v_ax] / m;
    auto q = [](float s) {
        int k = (int)std::floor((s + 1.0f) * 512.0f);
        return (uint32_t)std::min(std::max(k, 0), 1023);
    };
    const uint32_t face = (uint32_t)(2 * major + (d[major] < 0.0f ? 1 : 0));
    return (face << 20) | (spread10(q(u)) << 1) | spread10(q(v));
}

}  // namespace

namespace rt {

void sorted_lattice(int n, int begin, int end, float4* out, uint32_t* key, int* order) {
    const int cnt = end - begin;
    for (int i = 0; i < cnt; ++i) {
        float d[3];
        lattice_entry(begin + i, n, d);
        key[i] = angular_key(d);
        order[i] = i;
    }
    // (key, index) order: the same permutation a stable sort by key gives, without a buffer
    std::sort(order, order + cnt, [&](int a, int b) { return key[a] < key[b] || (key[a] == key[b] && a < b); });
    for (int i = 0; i < cnt; ++i) {
        float d[3];
        lattice_entry(begin + order[i], n, d);
        out[i] = make_float4(d[0], d[1], d[2], 0.0f);
    }
}

rt_status set_error(rt_status st, const char* msg) { return fail(st, "%s", msg); }

}  // namespace rt

namespace {

struct DirTable {
    int n = 0, begin = 0, end = 0;
    float4* d = nullptr;
};

// Launch plan of the forward march: bin-group width, threads per block, gather prefetch, and
// lanes per ray (2 or 4 adjacent lanes share the ray of a 4-bin group).
struct Plan {
    int W = 1, block = 64, prefetch = 1, lpr = 1, tile = 1;
};

}  // namespace

struct rt_grid {
    int n0 = 0, n1 = 0, n2 = 0, max_freq = 0;
    rt_options opt{};
    int device = 0;
    std::vector<DirTable> dirs;
    // scratch slots
    enum Slot { JP, KP, ACC, ACC64, HJ, HK, HOUT, HSRC, TRACE, CKPT, GP, DJ, DK, DETS, STPOS, STI, STTAU, CHK,
                AJ0, AK0, AOUT0, ASRC0, AJ1, AK1, AOUT1, ASRC1, HASH, INV, NSLOT };
    void* buf[NSLOT] = {};
    size_t cap[NSLOT] = {};
    // profiling events around the last march kernel
    cudaEvent_t ev[2] = {nullptr, nullptr};
    bool ev_valid = false;
    // autotuning cache: shape class -> fastest launch plan
    struct TuneKey {
        int n_freq, nsrc, rays, ns;
        int rec = 0;   // forward plans: tuned for a recording call (checkpoint stores included)
        bool operator==(const TuneKey& o) const {
            return n_freq == o.n_freq && nsrc == o.nsrc && rays == o.rays && ns == o.ns && rec == o.rec;
        }
    };
    std::vector<std::pair<TuneKey, std::pair<Plan, float>>> tuned;
    // checkpoint strides picked by the reverse-march tuner: shape class -> (K, adjoint ms)
    std::vector<std::pair<TuneKey, std::pair<int, float>>> tuned_k;
    int last_k = 0;            // stride of the last reverse march
    float last_k_ms = -1.0f;   // its tuned adjoint time (-1: not tuned)
    Plan last_plan;
    int last_acc = 0;          // accumulation of the last forward call (MarchArgs::acc_mode)
    bool dets_zeroed = false;  // the fixed-point reduction words of the DETS slot are zero
    float last_plan_ms = -1.0f;
    std::string tune_report;   // candidates timed by the last autotuning pass
    // state of the stateful advance (rt_advance_continue): which problem it belongs to, which of
    // the two position buffers holds the current positions, substeps marched since the restart
    // checkpoints recorded by the last recording rt_advance (record_checkpoints): the call they
    // belong to; valid until a reverse march or another recording overwrites the CKPT slot
    struct Recording {
        bool valid = false;
        const float *j = nullptr, *kappa = nullptr, *src = nullptr;
        int nsrc = 0, rays = 0, ns = 0, n_freq = 0, stride = 0, W = 0, kappa_mode = 0;
        float ds = 0.0f;
    } rec;
    // pipelined host calls (rt_advance_host_async): a copy-in and a copy-out stream, and per
    // buffer set the events that order its reuse
    struct HostPipe {
        cudaStream_t h2d = nullptr, d2h = nullptr;
        cudaEvent_t in_ready[2] = {}, done[2] = {}, out_done[2] = {};
        long long calls = 0;
    } pipe;
    struct ContinueState {
        bool valid = false;
        int nsrc = 0, rays = 0, n_freq = 0, parity = 0;
        float ds = 0.0f;
        long long steps = 0;
    } cont;

    rt_status mark(int which, cudaStream_t st) {
        if (!opt.profile) return RT_OK;
        if (!ev[which]) RT_CUDA(cudaEventCreate(&ev[which]), "cudaEventCreate");
        RT_CUDA(cudaEventRecord(ev[which], st), "cudaEventRecord");
        ev_valid = which == 1;
        return RT_OK;
    }

    long long ncell() const { return (long long)n0 * n1 * n2; }

    rt_status ensure(Slot s, size_t bytes, void** out) {
        *out = nullptr;
        if (bytes == 0) bytes = 16;
        if (cap[s] < bytes) {
            if (buf[s]) {
                cudaError_t e = cudaFree(buf[s]);
                buf[s] = nullptr;
                cap[s] = 0;
                if (e != cudaSuccess) return cuda_fail(e, "cudaFree(scratch)");
            }
            cudaError_t e = cudaMalloc(&buf[s], bytes);
            if (e != cudaSuccess) {
                buf[s] = nullptr;
                return cuda_fail(e, "cudaMalloc(scratch)");
            }
            cap[s] = bytes;
        }
        *out = buf[s];
        return RT_OK;
    }

    // Direction table of lattice rays [begin, end) of an N-ray lattice, sorted by angular_key.
    rt_status table(int n, int begin, int end, const float4** out) {
        for (auto& t : dirs)
            if (t.n == n && t.begin == begin && t.end == end) { *out = t.d; return RT_OK; }
        const int cnt = end - begin;
        std::vector<uint32_t> key(cnt);
        std::vector<int> order(cnt);
        std::vector<float4> host(cnt);
        rt::sorted_lattice(n, begin, end, host.data(), key.data(), order.data());
        DirTable t;
        t.n = n; t.begin = begin; t.end = end;
        RT_CUDA(cudaMalloc(&t.d, sizeof(float4) * (size_t)std::max(cnt, 1)), "cudaMalloc(directions)");
        cudaError_t e = cudaMemcpy(t.d, host.data(), sizeof(float4) * (size_t)cnt, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) { cudaFree(t.d); return cuda_fail(e, "cudaMemcpy(directions)"); }
        if (dirs.size() >= 16) {
            cudaFree(dirs.front().d);
            dirs.erase(dirs.begin());
        }
        dirs.push_back(t);
        *out = t.d;
        return RT_OK;
    }

    void release() {
        cudaDeviceSynchronize();
        for (auto& e : ev)
            if (e) cudaEventDestroy(e);
        for (int i = 0; i < 2; ++i) {
            if (pipe.in_ready[i]) cudaEventDestroy(pipe.in_ready[i]);
            if (pipe.done[i]) cudaEventDestroy(pipe.done[i]);
            if (pipe.out_done[i]) cudaEventDestroy(pipe.out_done[i]);
        }
        if (pipe.h2d) cudaStreamDestroy(pipe.h2d);
        if (pipe.d2h) cudaStreamDestroy(pipe.d2h);
        pipe = HostPipe{};
        for (auto& t : dirs) cudaFree(t.d);
        dirs.clear();
        for (int s = 0; s < NSLOT; ++s) {
            if (buf[s]) cudaFree(buf[s]);
            buf[s] = nullptr;
            cap[s] = 0;
        }
        dets_zeroed = false;
    }
};

namespace {

int num_substeps(float ds, float c, float dt, int cap) { return rt::substeps(ds, c, dt, cap); }

}  // namespace

// Widths W in {the default, 2, 1} that fit n_freq; 32, 64, 128, 256 threads per block; gather
// modes 0, 1, 2, 3 with and without source tiles, mode 4, and modes 0 and 4 with two lanes per ray.
int rt::march_plan_candidates(int n_freq, MarchPlan* out) {
    int widths[3], nw = 0;
    widths[nw++] = n_freq == 1 ? 1 : (n_freq == 2 ? 2 : 4);
    if (n_freq >= 3) widths[nw++] = 2;
    if (n_freq >= 2) widths[nw++] = 1;
    int n = 0;
    for (int wi = 0; wi < nw; ++wi)
        for (int b : {32, 64, 128, 256})
            for (int cand = 0; cand < 11; ++cand) {
                MarchPlan p;
                p.W = widths[wi];
                p.block = b;
                p.prefetch = cand < 8 ? cand >> 1 : (cand == 8 ? 0 : 4);
                p.tile = cand < 8 ? (cand & 1) : 0;
                p.lpr = cand == 8 || cand == 10 ? 2 : 1;
                out[n++] = p;
            }
    return n;
}

int rt::substeps(float ds, float c, float dt, int cap) {
    if (!std::isfinite(ds) || !std::isfinite(c) || !std::isfinite(dt)) return -1;
    if (!(ds > 0.0f) || !(c > 0.0f) || !(dt >= 0.0f)) return -1;
    const double q = (double)c * (double)dt / (double)ds;
    const double n = std::ceil(q - 1e-9 * q);
    if (!(n <= 2147483647.0)) return -1;
    int ns = n < 0.0 ? 0 : (int)n;
    if (cap > 0 && ns > cap) ns = cap;
    return ns;
}

namespace {

rt_status check_device(rt_grid* g) {
    int dev = -1;
    RT_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev != g->device)
        return fail(RT_ERR_INVALID_ARG, "current device %d differs from the handle's device %d", dev, g->device);
    return RT_OK;
}

struct Call {
    const float* j; const float* kappa; const float* src;
    int nsrc, num_rays, ray_begin, ray_end;
    float ds, c, dt;
    int n_freq;
    float* out;
    int accumulate;
    cudaStream_t st;
    // stateful advance (rt_advance_continue); see MarchArgs
    const float* st_pos_in = nullptr;
    float* st_pos_out = nullptr;
    float* st_I = nullptr;
    float* st_tau = nullptr;
    int st_read = 0;
};

rt_status validate(rt_grid* g, const Call& a, int* ns_out) {
    if (!g) return fail(RT_ERR_INVALID_ARG, "grid handle is NULL");
    if (a.n_freq < 1 || a.n_freq > g->max_freq)
        return fail(RT_ERR_INVALID_ARG, "n_freq = %d outside [1, max_freq = %d]", a.n_freq, g->max_freq);
    if (a.num_rays < 1) return fail(RT_ERR_INVALID_ARG, "num_rays = %d must be >= 1", a.num_rays);
    if (a.nsrc < 0) return fail(RT_ERR_INVALID_ARG, "num_sources = %d must be >= 0", a.nsrc);
    if (a.ray_begin < 0 || a.ray_end > a.num_rays || a.ray_begin > a.ray_end)
        return fail(RT_ERR_INVALID_ARG, "ray range [%d, %d) not inside [0, %d)", a.ray_begin, a.ray_end,
                    a.num_rays);
    if (!(a.ds > 0.0f) || !std::isfinite(a.ds))
        return fail(RT_ERR_INVALID_ARG, "step_size must be finite and > 0");
    if (!(a.c > 0.0f) || !std::isfinite(a.c))
        return fail(RT_ERR_INVALID_ARG, "radiation_velocity must be finite and > 0");
    if (!(a.dt >= 0.0f) || !std::isfinite(a.dt))
        return fail(RT_ERR_INVALID_ARG, "time_step must be finite and >= 0");
    const int ns = num_substeps(a.ds, a.c, a.dt, g->opt.ns_cap);
    if (ns < 0) return fail(RT_ERR_INVALID_ARG, "substep count c*dt/ds does not fit in an int");
    if ((double)ns * a.ds > 1.6e7)
        return fail(RT_ERR_INVALID_ARG, "ray length N_s*ds = %g exceeds 1.6e7 cells", (double)ns * a.ds);
    if (!a.j || !a.kappa || !a.out) return fail(RT_ERR_INVALID_ARG, "j_map, kappa_map and out_field must be non-NULL");
    if (a.nsrc > 0 && !a.src) return fail(RT_ERR_INVALID_ARG, "source_pos is NULL");
    if (a.out == a.j || a.out == a.kappa) return fail(RT_ERR_INVALID_ARG, "out_field aliases an input");
    *ns_out = ns;
    return RT_OK;
}

// Default bin-group width W: one bin needs no repacking; wider groups share the geometry.
int pick_width(int n_freq) {
    if (n_freq == 1) return 1;
    if (n_freq == 2) return 2;
    return 4;
}

// Accumulation of a launch plan (MarchArgs::acc_mode: 0 FP32, 1 fixed point, 2 FP64).
// deterministic = 1 or rt_options.accumulation 3: 64-bit fixed point; 1: FP32; 2: FP64;
// 0 (automatic): FP32 unless the call deposits at least kDenseUpdates updates per cell and bin on
// average (N_src N_Omega N_s >= kDenseUpdates n0 n1 n2), where crowded cells -- around clustered
// sources, on the clamped corners of the box -- take so many small deposits on top of large sums
// that FP32 rounds a measurable part of them away (rel-L2 ~1e-4 against the oracle on 2,097
// clustered sources, ~1,000 updates per cell); such calls sum in 64-bit fixed point (measured on
// GB300: the same one-bin march time as FP32 there), or in FP64 where the fixed-point unit would
// be coarse (fixed_point_fits) or a continued march carries intensities past its bound. Source
// tiles sum in FP32 shared memory: a plan that pins them keeps FP32.
constexpr double kDenseUpdates = 32.0;

bool fixed_point_fits(const Call& a, int ns) {
    // the fixed-point unit is the bound 4 pi N_src ds max|j| N_s (N_s + 1) / 2 over 2^62; with
    // N_src N_s (N_s + 1) / 2 <= 2^32 it is at most 2^-30 of 4 pi ds max|j|, the scale of one
    // ray's first deposit
    return (double)a.nsrc * (double)ns * ((double)ns + 1.0) * 0.5 <= 4294967296.0;
}

// The automatic choice for the call, before any plan: 0 FP32, 1 fixed point, 2 FP64.
int auto_accumulation(const rt_grid* g, const Call& a, int ns) {
    const double updates = (double)a.nsrc * (double)(a.ray_end - a.ray_begin) * (double)ns;
    if (updates < kDenseUpdates * (double)g->ncell()) return 0;
    return fixed_point_fits(a, ns) && !a.st_I ? 1 : 2;
}

int acc_mode_for(const rt_grid* g, const Plan& p, const Call& a, int ns) {
    // (carried intensities of a continued march void the fixed-point bound: FP64 then)
    if (g->opt.deterministic || g->opt.accumulation == 3) return a.st_I ? 2 : 1;
    if (g->opt.accumulation == 1) return 0;
    if (g->opt.accumulation == 2) return 2;
    if (p.lpr == 1 && p.tile) return 0;
    return auto_accumulation(g, a, ns);
}

// Set up the accumulator of acc_mode on the call's stream (after prepare()): mode 1 computes the
// fixed-point unit from max|j| and clears the 8-byte accumulator, mode 2 clears it; mode 0 was
// set up by prepare() (packing cleared the packed FP32 accumulator; for W = 1 the caller clears
// out_field unless accumulating). Fills m->acc_mode, acc64, fix and dep_scale.
rt_status setup_accumulator(rt_grid* g, const Call& a, int ns, const Plan& plan, int acc, float scale,
                            rt::MarchArgs* m) {
    m->acc_mode = acc;
    if (acc == 0) return RT_OK;
    const int groups = (a.n_freq + plan.W - 1) / plan.W;
    const long long ncell = g->ncell();
    const size_t bytes = 8 * (size_t)groups * plan.W * ncell;
    void* p = nullptr;
    rt_status st = g->ensure(rt_grid::ACC64, bytes, &p);
    if (st != RT_OK) return st;
    m->acc64 = (unsigned long long*)p;
    if (acc == 1) {
        // 64-bit fixed point: every flushed deposit s * w * I is rounded to a multiple of 1 / fix
        // and added as an integer, so the sums are independent of the order of the deposits. With
        // kappa >= 0 each I_{k+1} <= (k+1) ds max|j|, so a cell sums to at most
        // 4 pi N_src ds max|j| N_s (N_s + 1) / 2 per bin; fix keeps that below 2^62. One launch
        // clears the accumulator and computes fix.
        void* dets = nullptr;
        if ((st = g->ensure(rt_grid::DETS, 16, &dets)) != RT_OK) return st;
        if (!g->dets_zeroed) {   // the reduction words start at zero; each call leaves them so
            RT_CUDA(cudaMemsetAsync(dets, 0, 16, a.st), "cudaMemsetAsync(fixed-point words)");
            g->dets_zeroed = true;
        }
        float* fix = (float*)dets;
        unsigned* work = (unsigned*)((char*)dets + 8);
        const double per_jmax = 4.0 * 3.14159265358979323846 * (double)a.nsrc * (double)a.ds * (double)ns *
                                ((double)ns + 1.0) * 0.5;
        RT_CUDA(rt::launch_fix_prepare(a.j, (long long)a.n_freq * ncell, (unsigned long long*)p,
                                       (long long)(bytes / 8), per_jmax, work, fix, a.st),
                "fixed-point set-up");
        m->fix = fix;
        m->dep_scale = scale;
        return RT_OK;
    }
    m->dep_scale = 1.0f;   // 4 pi / N_Omega is applied in FP64 by the conversion
    RT_CUDA(cudaMemsetAsync(p, 0, bytes, a.st), "cudaMemsetAsync(8-byte accumulator)");
    return RT_OK;
}

// After the march: the 8-byte accumulators are converted into out_field (scaled, unpacked,
// added when accumulating); the packed FP32 one is unpacked for W > 1.
rt_status finish_accumulator(rt_grid* g, const Call& a, const Plan& plan, float scale, const rt::MarchArgs& m) {
    const long long ncell = g->ncell();
    if (m.acc_mode == 1)
        RT_CUDA(rt::launch_fixed_to_float(m.acc64, a.n_freq, ncell, m.fix, a.out, a.accumulate, a.st),
                "fixed-point conversion");
    else if (m.acc_mode == 2)
        RT_CUDA(rt::launch_f64_to_float((const double*)m.acc64, a.n_freq, ncell, (double)scale, a.out,
                                        a.accumulate, a.st),
                "FP64 conversion launch");
    else if (plan.W > 1)
        RT_CUDA(rt::launch_unpack(m.acc, a.out, a.n_freq, plan.W, ncell, scale, a.accumulate, a.st), "unpack launch");
    return RT_OK;
}

// Lay out the inputs for bin-group width W (packing for W > 1) and fill the march arguments.
// The accumulator is `out` itself for W = 1 with an output, else the handle's scratch; with
// clear_acc, packing for W > 1 also zeroes the packed accumulator (same launch).
rt_status prepare(rt_grid* g, const Call& a, int ns, const Plan& plan, const float4* dirs, float scale,
                  float* out, rt::MarchArgs* m, bool clear_acc = false) {
    rt_status st;
    const long long ncell = g->ncell();
    *m = rt::MarchArgs{};
    m->dirs = dirs;
    m->src = a.src;
    m->n0 = g->n0; m->n1 = g->n1; m->n2 = g->n2;
    m->ns = ns;
    m->ds = a.ds;
    m->ray_count = a.ray_end - a.ray_begin;
    m->nsrc = a.nsrc;
    m->n_freq = a.n_freq;
    m->kappa_mode = g->opt.kappa_mode;
    m->block = plan.block;
    m->prefetch = plan.prefetch;
    m->lanes_per_ray = plan.lpr;
    m->tile = plan.lpr == 1 ? plan.tile : 0;
    if (plan.W == 1) {
        float* acc = out;
        if (!acc) {
            void* p;
            if ((st = g->ensure(rt_grid::ACC, sizeof(float) * (size_t)a.n_freq * ncell, &p)) != RT_OK) return st;
            acc = (float*)p;
        }
        m->jp = a.j; m->kp = a.kappa; m->acc = acc;
        m->groups = a.n_freq;
        m->dep_scale = scale;
        return RT_OK;
    }
    const int W = plan.W, groups = (a.n_freq + W - 1) / W;
    const size_t packed = sizeof(float) * (size_t)groups * ncell * W;
    void *jp = nullptr, *kp = nullptr, *acc = nullptr;
    if ((st = g->ensure(rt_grid::JP, packed, &jp)) != RT_OK) return st;
    if ((st = g->ensure(rt_grid::KP, packed, &kp)) != RT_OK) return st;
    if ((st = g->ensure(rt_grid::ACC, packed, &acc)) != RT_OK) return st;
    RT_CUDA(rt::launch_pack_pair(a.j, a.kappa, (float*)jp, (float*)kp, clear_acc ? (float*)acc : nullptr, a.n_freq,
                                 W, groups, ncell, a.st),
            "pack launch");
    m->jp = (const float*)jp; m->kp = (const float*)kp; m->acc = (float*)acc;
    m->groups = groups;
    m->dep_scale = 1.0f;
    return RT_OK;
}

// Adjoint checkpoint stride K in {4, 8, 16, 32}: the option rounded to the nearest supported
// value; automatic: the stride the reverse-march tuner picked for this shape class (n_freq,
// sources, rays, N_s) when the handle autotunes and has tuned it, else 16.
int ckpt_stride(const rt_grid* g, int n_freq = 0, int nsrc = 0, int rays = 0, int ns = 0) {
    if (g->opt.ckpt_stride <= 0) {
        const rt_grid::TuneKey key{n_freq, nsrc, rays, ns};
        for (const auto& e : g->tuned_k)
            if (e.first == key) return e.second.first;
        return 16;
    }
    const int want = g->opt.ckpt_stride;
    return want <= 5 ? 4 : (want <= 11 ? 8 : (want <= 23 ? 16 : 32));
}

size_t acc_bytes(const rt_grid* g, const Call& a, const Plan& plan) {
    const int groups = (a.n_freq + plan.W - 1) / plan.W;
    return sizeof(float) * (size_t)groups * g->ncell() * plan.W;
}

// Autotuner: on the first call of a shape class, time every candidate plan's march kernel on
// the call's own inputs (into scratch; best of two runs each) and keep the fastest. A call that
// records the reverse march's checkpoints is tuned apart, over the plans with a recording kernel
// at the adjoint's bin grouping, each timed with its checkpoint stores.
rt_status tune(rt_grid* g, const Call& a, int ns, const float4* dirs, float scale, Plan* best, bool record) {
    rt_grid::TuneKey key{a.n_freq, a.nsrc, a.ray_end - a.ray_begin, ns};
    key.rec = record ? 1 : 0;
    for (const auto& e : g->tuned)
        if (e.first == key) {
            *best = e.second.first;
            g->last_plan_ms = e.second.second;
            return RT_OK;
        }
    rt::MarchPlan cands[rt::kMaxMarchPlans];
    const int n_cand = rt::march_plan_candidates(a.n_freq, cands);
    cudaEvent_t e[2] = {nullptr, nullptr};
    float best_ms = 3.0e38f;
    Plan bp;
    bp.W = cands[0].W;
    g->tune_report.clear();
    rt_status st = RT_OK;
    cudaError_t ce = cudaEventCreate(&e[0]);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e[1]);
    if (ce != cudaSuccess) st = cuda_fail(ce, "cudaEventCreate");
    for (int ci = 0; ci < n_cand && st == RT_OK; ++ci) {
        Plan p;
        p.W = cands[ci].W; p.block = cands[ci].block; p.prefetch = cands[ci].prefetch;
        p.lpr = cands[ci].lpr; p.tile = cands[ci].tile;
        const int W = p.W, b = p.block;
        // tiles sum in FP32: not a plan of an 8-byte accumulation, nor of the automatic mode for one
        // bin (whose other plans sum in 8-byte words)
        if (p.lpr == 1 && p.tile && g->opt.accumulation == 0 && auto_accumulation(g, a, ns) != 0) continue;
        const int acc = acc_mode_for(g, p, a, ns);
        if (acc != 0 && p.lpr == 1 && p.tile) continue;
        if (record && W != pick_width(a.n_freq)) continue;
        if (!rt::march_fwd_available(W, p.prefetch, acc, p.tile, record, p.lpr, p.block)) continue;
        rt::MarchArgs m;
        if ((st = prepare(g, a, ns, p, dirs, scale, nullptr, &m)) != RT_OK) break;
        if (record) {   // the checkpoint stores into the CKPT slot (the call then records anew)
            rt::BackArgs sz{};
            sz.ray_count = a.num_rays; sz.nsrc = a.nsrc; sz.n_freq = a.n_freq; sz.ns = ns;
            sz.stride = ckpt_stride(g, a.n_freq, a.nsrc, a.num_rays, ns);
            void* ck;
            g->rec.valid = false;
            if ((st = g->ensure(rt_grid::CKPT, sizeof(float) * rt::backward_ckpt_floats(sz, W), &ck)) != RT_OK) break;
            m.ckpt = (float*)ck;
            m.ck_stride = sz.stride;
        }
        float cand_ms = 3.0e38f;
        for (int rep = 0; rep < 2; ++rep) {
            if (acc != 0) {
                if ((st = setup_accumulator(g, a, ns, p, acc, scale, &m)) != RT_OK) break;
                ce = cudaSuccess;
            } else {
                ce = cudaMemsetAsync(m.acc, 0, acc_bytes(g, a, p), a.st);
            }
            if (ce == cudaSuccess) ce = cudaEventRecord(e[0], a.st);
            if (ce == cudaSuccess) ce = rt::launch_march_fwd(W, m, a.st);
            if (ce == cudaSuccess) ce = cudaEventRecord(e[1], a.st);
            if (ce == cudaSuccess) ce = cudaEventSynchronize(e[1]);
            float ms = 0.0f;
            if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e[0], e[1]);
            if (ce != cudaSuccess) { st = cuda_fail(ce, "autotune run"); break; }
            if (ms < cand_ms) cand_ms = ms;
            if (ms < best_ms) { best_ms = ms; bp = p; }
        }
        if (st == RT_OK) {
            char line[128];
            snprintf(line, sizeof line, "W=%d block=%d prefetch=%d lanes=%d tile=%d acc=%s%s %.4f ms\n", W, b,
                     p.prefetch, p.lpr, p.tile, acc == 2 ? "fp64" : (acc == 1 ? "fixed" : "fp32"),
                     record ? " recording" : "", cand_ms);
            g->tune_report += line;
        }
    }
    for (auto ev : e)
        if (ev) cudaEventDestroy(ev);
    if (st != RT_OK) return st;
    if (g->tuned.size() >= 64) g->tuned.erase(g->tuned.begin());
    g->tuned.push_back({key, {bp, best_ms}});
    *best = bp;
    g->last_plan_ms = best_ms;
    return RT_OK;
}

// Checked mode (rt_options.check_inputs): scan the call's inputs on the device, synchronise,
// and name the first offending array.
rt_status check_inputs(rt_grid* g, const Call& a, const float* grad) {
    if (!g->opt.check_inputs) return RT_OK;
    void* f;
    rt_status st = g->ensure(rt_grid::CHK, 4 * sizeof(int), &f);
    if (st != RT_OK) return st;
    const long long n = (long long)a.n_freq * g->ncell();
    RT_CUDA(rt::launch_check_inputs(a.j, a.kappa, n, a.src, a.nsrc, grad, (int*)f, a.st), "input check launch");
    int h[4] = {0, 0, 0, 0};
    RT_CUDA(cudaMemcpyAsync(h, f, sizeof h, cudaMemcpyDeviceToHost, a.st), "input check copy");
    RT_CUDA(cudaStreamSynchronize(a.st), "input check synchronise");
    if (h[0]) return fail(RT_ERR_INVALID_ARG, "checked mode: j_map holds a value that is not finite");
    if (h[1]) return fail(RT_ERR_INVALID_ARG, "checked mode: kappa_map holds a negative or non-finite value");
    if (h[2]) return fail(RT_ERR_INVALID_ARG, "checked mode: source_pos holds a non-finite coordinate or |x| >= 2^24");
    if (h[3]) return fail(RT_ERR_INVALID_ARG, "checked mode: grad_out holds a value that is not finite");
    return RT_OK;
}

rt_status advance_impl(rt_grid* g, const Call& a) {
    int ns = 0;
    rt_status st = validate(g, a, &ns);
    if (st != RT_OK) return st;
    if ((st = check_device(g)) != RT_OK) return st;
    if ((st = check_inputs(g, a, nullptr)) != RT_OK) return st;
    const long long ncell = g->ncell();
    const size_t field_bytes = sizeof(float) * (size_t)a.n_freq * ncell;
    const int count = a.ray_end - a.ray_begin;
    if (ns == 0 || a.nsrc == 0 || count == 0) {
        if (!a.accumulate) RT_CUDA(cudaMemsetAsync(a.out, 0, field_bytes, a.st), "cudaMemsetAsync(out)");
        return RT_OK;
    }
    const float4* dirs = nullptr;
    if ((st = g->table(a.num_rays, a.ray_begin, a.ray_end, &dirs)) != RT_OK) return st;
    const float scale = (float)(4.0 * 3.14159265358979323846 / (double)a.num_rays);

    // default plan (measured on GB300): 32-thread blocks, corner slots with the gathers a substep
    // ahead (gathers mode 4). One bin per thread: two lanes per ray while the call has too few
    // lanes to fill the GPU (64^3, 8 sources, 3,072 rays: 0.09 ms against 0.15 ms for tiles with
    // prefetch); otherwise, summing in FP32, gather prefetch with source deposit tiles. Wider
    // groups: one lane per ray (four bins on 128^3 with 16 sources: 0.25 ms against 0.37 ms with
    // two lanes, which repeat the geometry; a tiled 4-bin deposit is 32 shared-memory atomics).
    // Summing in 8-byte words (no tiles): gathers mode 4.
    const bool det = g->opt.deterministic != 0;
    Plan plan;
    plan.W = pick_width(a.n_freq);
    plan.block = 32;
    if (g->opt.plan_width) plan.W = g->opt.plan_width;
    {
        const double lanes = (double)a.nsrc * (a.ray_end - a.ray_begin) * ((a.n_freq + plan.W - 1) / plan.W);
        plan.prefetch = 4;
        plan.tile = 0;
        if (plan.W == 1 && lanes < 152.0 * 1024.0) {
            plan.lpr = 2;
        } else if (plan.W == 1 && acc_mode_for(g, plan, a, ns) == 0) {   // FP32 sums: tiles
            plan.prefetch = 1;
            plan.tile = 1;
        }
    }
    if (det) {   // deterministic mode: corner slots, one lane per ray (validated at creation)
        plan.prefetch = 4;
        plan.tile = 0;
        plan.lpr = 1;
        plan.block = 32;
    }
    if (g->opt.plan_block) plan.block = g->opt.plan_block;
    if (g->opt.plan_prefetch) plan.prefetch = g->opt.plan_prefetch - 1;
    if (g->opt.plan_lanes) plan.lpr = g->opt.plan_lanes;
    if (g->opt.plan_tile) plan.tile = g->opt.plan_tile - 1;
    // a pinned gathers mode or tile that two lanes per ray do not have: one lane (unless pinned)
    if (!g->opt.plan_lanes && plan.lpr == 2 && ((plan.prefetch != 0 && plan.prefetch != 4) || plan.tile))
        plan.lpr = 1;
    if (plan.lpr != 1 && (plan.lpr != 2 || (plan.prefetch != 0 && plan.prefetch != 4)))
        return fail(RT_ERR_INVALID_ARG, "plan_lanes must be 1, or 2 with gathers mode 0 or 4");
    g->last_plan_ms = -1.0f;
    bool record = g->opt.record_checkpoints && !a.st_I && a.ray_begin == 0 && a.ray_end == a.num_rays;
    if (g->opt.autotune && !det && (st = tune(g, a, ns, dirs, scale, &plan, record)) != RT_OK) return st;
    if (a.st_I && plan.lpr > 1) {   // the stateful march runs one lane per (ray, source, bin group)
        plan.lpr = 1;
        plan.prefetch = 0;
    }
    // record the reverse march's checkpoints with the adjoint's bin grouping and gathers mode 4:
    // two lanes per ray for one bin per thread, one lane for wider groups (measured on GB300, 64^3
    // with 8 sources and 3,072 rays: one bin 0.087 ms against 0.12 for two lanes with mode 0,
    // 0.155 for mode 3 and 0.17 for mode 1 with one lane; four bins 0.094 ms against 0.124 for two
    // lanes and 0.131 for one lane with mode 0), unless a plan was pinned or tuned
    if (record) {
        const int w = pick_width(a.n_freq);
        const bool keep = plan.W == w && (g->opt.plan_prefetch || g->opt.plan_lanes || g->opt.autotune);
        if (!keep) {
            plan.block = 32;
            plan.tile = 0;
            plan.lpr = w == 1 && !det ? 2 : 1;
            if (plan.lpr == 2) plan.prefetch = 4;
        }
        plan.W = w;
        if (plan.prefetch != 4) {
            if (w != 1 || plan.lpr == 2) plan.prefetch = 0;          // corner slots
            else if (plan.prefetch == 2) plan.prefetch = 3;          // (recording has no gathers mode 2)
        }
    }
    const int acc = acc_mode_for(g, plan, a, ns);
    if (acc != 0) plan.tile = 0;
    // a default tile that the (pinned) gathers mode has no kernel for is dropped
    if (plan.tile && !g->opt.plan_tile && !rt::march_fwd_available(plan.W, plan.prefetch, acc, 1, record, plan.lpr, plan.block))
        plan.tile = 0;
    // a plan that this accumulation has no kernel for falls back to corner slots (every mode has
    // them); recording stays off where no recording kernel exists (the reverse march then makes
    // its own forward sweep)
    if (!rt::march_fwd_available(plan.W, plan.prefetch, acc, plan.tile, record, plan.lpr, plan.block)) {
        plan.prefetch = 0;
        if (!rt::march_fwd_available(plan.W, 0, acc, plan.tile, record, plan.lpr, plan.block)) plan.lpr = 1;
        if (record && !rt::march_fwd_available(plan.W, 0, acc, plan.tile, 1, plan.lpr, plan.block)) record = false;
    }
    g->last_plan = plan;
    g->last_acc = acc;

    rt::MarchArgs m;
    if ((st = prepare(g, a, ns, plan, dirs, scale, plan.W == 1 ? a.out : nullptr, &m, acc == 0)) != RT_OK) return st;
    m.st_pos_in = a.st_pos_in;
    m.st_pos_out = a.st_pos_out;
    m.st_I = a.st_I;
    m.st_tau = a.st_tau;
    m.st_read = a.st_read;
    if (!record && g->opt.record_checkpoints) g->rec.valid = false;
    if (record) {
        rt::BackArgs sz{};
        sz.ray_count = a.num_rays; sz.nsrc = a.nsrc; sz.n_freq = a.n_freq; sz.ns = ns;
        sz.stride = ckpt_stride(g, a.n_freq, a.nsrc, a.num_rays, ns);
        void* ck;
        g->rec.valid = false;
        if ((st = g->ensure(rt_grid::CKPT, sizeof(float) * rt::backward_ckpt_floats(sz, plan.W), &ck)) != RT_OK)
            return st;
        m.ckpt = (float*)ck;
        m.ck_stride = sz.stride;
        // content hash of the recorded inputs: the reverse march reuses the checkpoints only if
        // its own inputs hash alike (buffers rewritten in place in between do not)
        void* h;
        if ((st = g->ensure(rt_grid::HASH, 2 * sizeof(unsigned long long), &h)) != RT_OK) return st;
        RT_CUDA(rt::launch_input_hash(a.j, a.kappa, (long long)a.n_freq * ncell, a.src, a.nsrc,
                                      (unsigned long long*)h, a.st),
                "input hash launch");
        g->rec = rt_grid::Recording{true, a.j, a.kappa, a.src, a.nsrc, a.num_rays, ns, a.n_freq, sz.stride,
                                    plan.W, g->opt.kappa_mode, a.ds};
    }
    if (acc != 0) {
        if ((st = setup_accumulator(g, a, ns, plan, acc, scale, &m)) != RT_OK) return st;
    } else if (plan.W == 1 && !a.accumulate) {   // (for W > 1 the packing launch cleared the accumulator)
        RT_CUDA(cudaMemsetAsync(m.acc, 0, field_bytes, a.st), "cudaMemsetAsync(accumulator)");
    }
    if ((st = g->mark(0, a.st)) != RT_OK) return st;
    RT_CUDA(rt::launch_march_fwd(plan.W, m, a.st), "march kernel launch");
    if ((st = g->mark(1, a.st)) != RT_OK) return st;
    return finish_accumulator(g, a, plan, scale, m);
}

}  // namespace

extern "C" {

void rt_default_options(rt_options* opt) {
    if (opt) std::memset(opt, 0, sizeof(*opt));
}

rt_status rt_create_grid(rt_grid** out, int n0, int n1, int n2, int max_freq, const rt_options* opt) {
    if (!out) return fail(RT_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n0 < 1 || n1 < 1 || n2 < 1) return fail(RT_ERR_INVALID_ARG, "grid extents must be >= 1");
    if (max_freq < 1) return fail(RT_ERR_INVALID_ARG, "max_freq must be >= 1");
    const long long cells = (long long)n0 * n1 * n2;
    // packed groups of 4 bins may exceed n_freq by 3: keep every flat index below 2^31
    if (cells * (long long)((max_freq + 3) / 4 * 4) >= (1LL << 31))
        return fail(RT_ERR_INVALID_ARG, "grid too large: n_freq * n0 * n1 * n2 must stay below 2^31");
    rt_options o;
    rt_default_options(&o);
    if (opt) o = *opt;
    if (o.kappa_mode != 0 && o.kappa_mode != 1) return fail(RT_ERR_INVALID_ARG, "kappa_mode must be 0 or 1");
    if (o.ns_cap < 0 || o.ckpt_stride < 0) return fail(RT_ERR_INVALID_ARG, "ns_cap and ckpt_stride must be >= 0");
    if (o.plan_width != 0 && o.plan_width != 1 && o.plan_width != 2 && o.plan_width != 4)
        return fail(RT_ERR_INVALID_ARG, "plan_width must be 0, 1, 2 or 4");
    if (o.plan_block != 0 && (o.plan_block < 32 || o.plan_block > 256 || o.plan_block % 32))
        return fail(RT_ERR_INVALID_ARG, "plan_block must be 0 or a multiple of 32 in [32, 256]");
    if (o.plan_prefetch < 0 || o.plan_prefetch > 5) return fail(RT_ERR_INVALID_ARG, "plan_prefetch must be 0 .. 5");
    if (o.plan_lanes != 0 && o.plan_lanes != 1 && o.plan_lanes != 2)
        return fail(RT_ERR_INVALID_ARG, "plan_lanes must be 0, 1 or 2");
    if (o.plan_tile < 0 || o.plan_tile > 2) return fail(RT_ERR_INVALID_ARG, "plan_tile must be 0, 1 or 2");
    if (o.accumulation < 0 || o.accumulation > 3)
        return fail(RT_ERR_INVALID_ARG, "accumulation must be 0, 1, 2 or 3");
    // the fixed-point march runs one lane per ray with corner slots and no tiles: a pinned plan
    // asking for anything else would be accepted here and then silently not used
    if (o.deterministic && (o.plan_lanes == 2 || o.plan_tile == 2 || (o.plan_prefetch > 1 && o.plan_prefetch != 5)))
        return fail(RT_ERR_INVALID_ARG, "deterministic mode marches with plan_lanes 1, plan_tile 1 (off) and "
                                        "plan_prefetch 1 or 5 (corner slots, gathered in time or ahead) only");
    rt_grid* g = new (std::nothrow) rt_grid();
    if (!g) return fail(RT_ERR_OOM, "host allocation failed");
    g->n0 = n0; g->n1 = n1; g->n2 = n2; g->max_freq = max_freq;
    g->opt = o;
    if (cudaGetDevice(&g->device) != cudaSuccess) {
        delete g;
        return fail(RT_ERR_CUDA, "no CUDA device available");
    }
    *out = g;
    return RT_OK;
}

rt_status rt_destroy(rt_grid* g) {
    if (!g) return RT_OK;
    g->release();
    delete g;
    return RT_OK;
}

const char* rt_last_error(void) { return g_last_error.c_str(); }

int rt_num_substeps(float step_size, float radiation_velocity, float time_step, int ns_cap) {
    return num_substeps(step_size, radiation_velocity, time_step, ns_cap);
}

rt_status rt_direction_table(int num_rays, float* out) {
    if (num_rays < 1 || !out) return fail(RT_ERR_INVALID_ARG, "num_rays must be >= 1 and out non-NULL");
    for (int i = 0; i < num_rays; ++i) lattice_entry(i, num_rays, out + 3 * (size_t)i);
    return RT_OK;
}

rt_status rt_advance(rt_grid* grid, const float* j_map, const float* kappa_map, const float* source_pos,
                     int num_sources, int num_rays, float step_size, float radiation_velocity,
                     float time_step, int n_freq, float* out_field, int accumulate, void* cuda_stream) {
    Call a{j_map, kappa_map, source_pos, num_sources, num_rays, 0, num_rays, step_size,
           radiation_velocity, time_step, n_freq, out_field, accumulate ? 1 : 0, (cudaStream_t)cuda_stream};
    return advance_impl(grid, a);
}

rt_status rt_sync_status(void* cuda_stream) {
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)cuda_stream);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return fail(RT_ERR_CUDA, "device error: %s", cudaGetErrorString(e));
    int code = 0;
    return rt_device_status(&code);
}

rt_status rt_advance_batch(rt_grid* g, const rt_instance* inst, int n_inst, void* cuda_stream) {
    if (!g) return fail(RT_ERR_INVALID_ARG, "grid handle is NULL");
    rt_status st = check_device(g);
    if (st != RT_OK) return st;
    rt_batch* b = nullptr;
    if ((st = rt_batch_create(&b, inst, n_inst, &g->opt)) != RT_OK) return st;
    st = rt_batch_run(b, cuda_stream);
    if (st == RT_OK) {
        cudaError_t e = cudaStreamSynchronize((cudaStream_t)cuda_stream);
        if (e != cudaSuccess) st = cuda_fail(e, "rt_advance_batch synchronise");
    }
    rt_batch_destroy(b);
    return st;
}

rt_status rt_advance_continue(rt_grid* g, const float* j_map, const float* kappa_map, const float* source_pos,
                              int num_sources, int num_rays, float step_size, float radiation_velocity,
                              float time_step, int n_freq, float* out_field, int accumulate, int restart,
                              void* cuda_stream) {
    if (!g) return fail(RT_ERR_INVALID_ARG, "grid handle is NULL");
    if (g->opt.deterministic)
        return fail(RT_ERR_UNSUPPORTED, "rt_advance_continue: not available in deterministic mode");
    Call a{j_map, kappa_map, source_pos, num_sources, num_rays, 0, num_rays, step_size,
           radiation_velocity, time_step, n_freq, out_field, accumulate ? 1 : 0, (cudaStream_t)cuda_stream};
    int ns = 0;
    rt_status st = validate(g, a, &ns);
    if (st != RT_OK) return st;
    if ((st = check_device(g)) != RT_OK) return st;
    auto& c = g->cont;
    const bool fresh = restart || !c.valid || c.nsrc != num_sources || c.rays != num_rays || c.n_freq != n_freq ||
                       c.ds != step_size;
    const size_t lanes = (size_t)std::max(num_sources, 1) * (size_t)num_rays;
    void *pos = nullptr, *I = nullptr, *tau = nullptr;
    if ((st = g->ensure(rt_grid::STPOS, 2 * 3 * sizeof(float) * lanes, &pos)) != RT_OK) return st;
    if ((st = g->ensure(rt_grid::STI, sizeof(float) * (size_t)n_freq * lanes, &I)) != RT_OK) return st;
    if ((st = g->ensure(rt_grid::STTAU, sizeof(float) * (size_t)n_freq * lanes, &tau)) != RT_OK) return st;
    if (fresh) {
        c.valid = false;
        c.parity = 0;
        c.steps = 0;
    }
    float* p0 = (float*)pos + (size_t)c.parity * 3 * lanes;
    float* p1 = (float*)pos + (size_t)(c.parity ^ 1) * 3 * lanes;
    a.st_pos_in = p0;
    a.st_pos_out = p1;
    a.st_I = (float*)I;
    a.st_tau = (float*)tau;
    a.st_read = fresh ? 0 : 1;
    if (ns == 0 || num_sources == 0)   // nothing marches: zero (or unchanged) field, state as it was
        return advance_impl(g, a);
    if ((st = advance_impl(g, a)) != RT_OK) {
        c.valid = false;
        return st;
    }
    c.valid = true;
    c.nsrc = num_sources; c.rays = num_rays; c.n_freq = n_freq; c.ds = step_size;
    c.parity ^= 1;
    c.steps += ns;
    return RT_OK;
}

rt_status rt_advance_rays(rt_grid* grid, const float* j_map, const float* kappa_map, const float* source_pos,
                          int num_sources, int num_rays, int ray_begin, int ray_end, float step_size,
                          float radiation_velocity, float time_step, int n_freq, float* out_field,
                          int accumulate, void* cuda_stream) {
    Call a{j_map, kappa_map, source_pos, num_sources, num_rays, ray_begin, ray_end, step_size,
           radiation_velocity, time_step, n_freq, out_field, accumulate ? 1 : 0, (cudaStream_t)cuda_stream};
    return advance_impl(grid, a);
}

rt_status rt_advance_host(rt_grid* g, const float* j_map, const float* kappa_map, const float* source_pos,
                          int num_sources, int num_rays, float step_size, float radiation_velocity,
                          float time_step, int n_freq, float* out_field, void* cuda_stream) {
    if (!g) return fail(RT_ERR_INVALID_ARG, "grid handle is NULL");
    if (n_freq < 1 || n_freq > g->max_freq)
        return fail(RT_ERR_INVALID_ARG, "n_freq = %d outside [1, max_freq = %d]", n_freq, g->max_freq);
    if (num_sources < 0) return fail(RT_ERR_INVALID_ARG, "num_sources must be >= 0");
    if (!j_map || !kappa_map || !out_field || (num_sources > 0 && !source_pos))
        return fail(RT_ERR_INVALID_ARG, "host buffers must be non-NULL");
    rt_status st = check_device(g);
    if (st != RT_OK) return st;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const size_t field = sizeof(float) * (size_t)n_freq * g->ncell();
    const size_t srcb = sizeof(float) * 3 * (size_t)std::max(num_sources, 1);
    void *dj = nullptr, *dk = nullptr, *dout = nullptr, *dsrc = nullptr;
    if ((st = g->ensure(rt_grid::HJ, field, &dj)) != RT_OK) return st;
    if ((st = g->ensure(rt_grid::HK, field, &dk)) != RT_OK) return st;
    if ((st = g->ensure(rt_grid::HOUT, field, &dout)) != RT_OK) return st;
    if ((st = g->ensure(rt_grid::HSRC, srcb, &dsrc)) != RT_OK) return st;
    RT_CUDA(cudaMemcpyAsync(dj, j_map, field, cudaMemcpyHostToDevice, s), "copy j to device");
    RT_CUDA(cudaMemcpyAsync(dk, kappa_map, field, cudaMemcpyHostToDevice, s), "copy kappa to device");
    if (num_sources > 0)
        RT_CUDA(cudaMemcpyAsync(dsrc, source_pos, sizeof(float) * 3 * (size_t)num_sources,
                                cudaMemcpyHostToDevice, s), "copy sources to device");
    Call a{(const float*)dj, (const float*)dk, (const float*)dsrc, num_sources, num_rays, 0, num_rays,
           step_size, radiation_velocity, time_step, n_freq, (float*)dout, 0, s};
    if ((st = advance_impl(g, a)) != RT_OK) return st;
    RT_CUDA(cudaMemcpyAsync(out_field, dout, field, cudaMemcpyDeviceToHost, s), "copy field to host");
    RT_CUDA(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    return RT_OK;
}

rt_status rt_advance_host_async(rt_grid* g, const float* j_map, const float* kappa_map, const float* source_pos,
                                int num_sources, int num_rays, float step_size, float radiation_velocity,
                                float time_step, int n_freq, float* out_field, void* cuda_stream) {
    if (!g) return fail(RT_ERR_INVALID_ARG, "grid handle is NULL");
    if (n_freq < 1 || n_freq > g->max_freq)
        return fail(RT_ERR_INVALID_ARG, "n_freq = %d outside [1, max_freq = %d]", n_freq, g->max_freq);
    if (num_sources < 0) return fail(RT_ERR_INVALID_ARG, "num_sources must be >= 0");
    if (!j_map || !kappa_map || !out_field || (num_sources > 0 && !source_pos))
        return fail(RT_ERR_INVALID_ARG, "host buffers must be non-NULL");
    rt_status st = check_device(g);
    if (st != RT_OK) return st;
    {   // argument errors return before anything is enqueued
        Call probe{j_map, kappa_map, source_pos, num_sources, num_rays, 0, num_rays, step_size, radiation_velocity,
                   time_step, n_freq, out_field, 0, (cudaStream_t)cuda_stream};
        int ns = 0;
        if ((st = validate(g, probe, &ns)) != RT_OK) return st;
    }
    auto& P = g->pipe;
    if (!P.h2d) {   // all or nothing: a failed set-up leaves no half-made pipeline behind
        rt_grid::HostPipe q;
        cudaError_t e = cudaStreamCreateWithFlags(&q.h2d, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&q.d2h, cudaStreamNonBlocking);
        for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
            e = cudaEventCreateWithFlags(&q.in_ready[i], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&q.done[i], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&q.out_done[i], cudaEventDisableTiming);
        }
        if (e != cudaSuccess) {
            for (int i = 0; i < 2; ++i)
                for (cudaEvent_t ev : {q.in_ready[i], q.done[i], q.out_done[i]})
                    if (ev) cudaEventDestroy(ev);
            if (q.h2d) cudaStreamDestroy(q.h2d);
            if (q.d2h) cudaStreamDestroy(q.d2h);
            return cuda_fail(e, "host pipeline set-up");
        }
        P = q;
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int b = (int)(P.calls & 1);
    const rt_grid::Slot sj = b ? rt_grid::AJ1 : rt_grid::AJ0, sk = b ? rt_grid::AK1 : rt_grid::AK0;
    const rt_grid::Slot so = b ? rt_grid::AOUT1 : rt_grid::AOUT0, ss = b ? rt_grid::ASRC1 : rt_grid::ASRC0;
    const size_t field = sizeof(float) * (size_t)n_freq * g->ncell();
    const size_t srcb = sizeof(float) * 3 * (size_t)std::max(num_sources, 1);
    // growing a buffer set frees memory that enqueued copies may still use: drain the pipeline
    if (g->cap[sj] < field || g->cap[sk] < field || g->cap[so] < field || g->cap[ss] < srcb)
        if ((st = rt_host_wait(g)) != RT_OK) return st;
    void *dj = nullptr, *dk = nullptr, *dout = nullptr, *dsrc = nullptr;
    if ((st = g->ensure(sj, field, &dj)) != RT_OK) return st;
    if ((st = g->ensure(sk, field, &dk)) != RT_OK) return st;
    if ((st = g->ensure(so, field, &dout)) != RT_OK) return st;
    if ((st = g->ensure(ss, srcb, &dsrc)) != RT_OK) return st;
    // copy in once the march two calls back has read this set (an unrecorded event is complete)
    RT_CUDA(cudaStreamWaitEvent(P.h2d, P.done[b], 0), "cudaStreamWaitEvent");
    RT_CUDA(cudaMemcpyAsync(dj, j_map, field, cudaMemcpyHostToDevice, P.h2d), "copy j to device");
    RT_CUDA(cudaMemcpyAsync(dk, kappa_map, field, cudaMemcpyHostToDevice, P.h2d), "copy kappa to device");
    if (num_sources > 0)
        RT_CUDA(cudaMemcpyAsync(dsrc, source_pos, sizeof(float) * 3 * (size_t)num_sources,
                                cudaMemcpyHostToDevice, P.h2d), "copy sources to device");
    RT_CUDA(cudaEventRecord(P.in_ready[b], P.h2d), "cudaEventRecord");
    // march once the inputs are in and the field of two calls back has left this set
    RT_CUDA(cudaStreamWaitEvent(s, P.in_ready[b], 0), "cudaStreamWaitEvent");
    RT_CUDA(cudaStreamWaitEvent(s, P.out_done[b], 0), "cudaStreamWaitEvent");
    Call a{(const float*)dj, (const float*)dk, (const float*)dsrc, num_sources, num_rays, 0, num_rays,
           step_size, radiation_velocity, time_step, n_freq, (float*)dout, 0, s};
    if ((st = advance_impl(g, a)) != RT_OK) return st;
    RT_CUDA(cudaEventRecord(P.done[b], s), "cudaEventRecord");
    RT_CUDA(cudaStreamWaitEvent(P.d2h, P.done[b], 0), "cudaStreamWaitEvent");
    RT_CUDA(cudaMemcpyAsync(out_field, dout, field, cudaMemcpyDeviceToHost, P.d2h), "copy field to host");
    RT_CUDA(cudaEventRecord(P.out_done[b], P.d2h), "cudaEventRecord");
    ++P.calls;
    return RT_OK;
}

rt_status rt_host_wait(rt_grid* g) {
    if (!g) return fail(RT_ERR_INVALID_ARG, "grid handle is NULL");
    if (!g->pipe.d2h) return RT_OK;
    // the last copy out waits for every march and copy in before it
    RT_CUDA(cudaStreamSynchronize(g->pipe.h2d), "cudaStreamSynchronize(copy in)");
    RT_CUDA(cudaStreamSynchronize(g->pipe.d2h), "cudaStreamSynchronize(copy out)");
    return RT_OK;
}

rt_status rt_host_join(rt_grid* g, void* cuda_stream) {
    if (!g) return fail(RT_ERR_INVALID_ARG, "grid handle is NULL");
    if (!g->pipe.d2h || g->pipe.calls == 0) return RT_OK;
    const int last = (int)((g->pipe.calls - 1) & 1);
    RT_CUDA(cudaStreamWaitEvent((cudaStream_t)cuda_stream, g->pipe.out_done[last], 0), "cudaStreamWaitEvent");
    return RT_OK;
}

rt_status rt_trace_cells(rt_grid* g, const float* src, int num_rays, int ray, float step_size, int num_steps,
                         long long* base_cell, long long* kappa_cell) {
    if (!g || !src || !base_cell || !kappa_cell) return fail(RT_ERR_INVALID_ARG, "NULL argument");
    if (num_rays < 1 || ray < 0 || ray >= num_rays || num_steps < 0 || !(step_size > 0.0f))
        return fail(RT_ERR_INVALID_ARG, "invalid ray / num_rays / num_steps / step_size");
    rt_status st = check_device(g);
    if (st != RT_OK) return st;
    if (num_steps == 0) return RT_OK;
    float d[3];
    lattice_entry(ray, num_rays, d);
    void* buf;
    if ((st = g->ensure(rt_grid::TRACE, 2 * sizeof(long long) * (size_t)num_steps, &buf)) != RT_OK) return st;
    long long* dbase = (long long*)buf;
    long long* dnn = dbase + num_steps;
    RT_CUDA(rt::launch_trace(src[0], src[1], src[2], d[0], d[1], d[2], step_size, num_steps, g->n0, g->n1,
                             g->n2, g->opt.kappa_mode, dbase, dnn, 0),
            "trace kernel launch");
    RT_CUDA(cudaMemcpy(base_cell, dbase, sizeof(long long) * num_steps, cudaMemcpyDeviceToHost), "copy trace");
    RT_CUDA(cudaMemcpy(kappa_cell, dnn, sizeof(long long) * num_steps, cudaMemcpyDeviceToHost), "copy trace");
    return RT_OK;
}

rt_status rt_kernel_ms(rt_grid* g, float* ms) {
    if (!g || !ms) return fail(RT_ERR_INVALID_ARG, "NULL argument");
    if (!g->opt.profile) return fail(RT_ERR_INVALID_ARG, "the handle was created without rt_options.profile");
    if (!g->ev_valid) return fail(RT_ERR_INVALID_ARG, "no march kernel has been timed on this handle yet");
    RT_CUDA(cudaEventSynchronize(g->ev[1]), "cudaEventSynchronize");
    RT_CUDA(cudaEventElapsedTime(ms, g->ev[0], g->ev[1]), "cudaEventElapsedTime");
    return RT_OK;
}

rt_status rt_last_plan(rt_grid* g, int* width, int* block, int* prefetch, int* lanes_per_ray, int* tile,
                       float* tuned_ms) {
    if (!g) return fail(RT_ERR_INVALID_ARG, "grid handle is NULL");
    if (width) *width = g->last_plan.W;
    if (block) *block = g->last_plan.block;
    if (prefetch) *prefetch = g->last_plan.prefetch;
    if (lanes_per_ray) *lanes_per_ray = g->last_plan.lpr;
    if (tile) *tile = g->last_plan.lpr == 1 ? g->last_plan.tile : 0;
    if (tuned_ms) *tuned_ms = g->last_plan_ms;
    return RT_OK;
}

rt_status rt_shard_plan(int num_sources, int num_rays, int n_shards, int shard, int* pieces, int* n_pieces) {
    if (!pieces || !n_pieces) return fail(RT_ERR_INVALID_ARG, "rt_shard_plan: NULL output");
    *n_pieces = 0;
    if (num_sources < 0 || num_rays < 1 || n_shards < 1 || shard < 0 || shard >= n_shards)
        return fail(RT_ERR_INVALID_ARG, "rt_shard_plan: need num_sources >= 0, num_rays >= 1, 0 <= shard < n_shards");
    // shard s owns pairs [p0, p1) of the source-major (source, ray) order: sizes differ by at most one
    const long long total = (long long)num_sources * num_rays;
    const long long base = total / n_shards, rem = total % n_shards;
    const long long p0 = shard * base + std::min<long long>(shard, rem);
    const long long p1 = p0 + base + (shard < rem ? 1 : 0);
    long long p = p0;
    while (p < p1) {
        const int s0 = (int)(p / num_rays), r0 = (int)(p % num_rays);
        int* q = pieces + 4 * (*n_pieces);
        if (r0 != 0 || p1 - p < num_rays) {   // part of one source's rays
            const long long end = std::min<long long>(p1, (long long)(s0 + 1) * num_rays);
            q[0] = s0; q[1] = s0 + 1; q[2] = r0; q[3] = (int)(end - (long long)s0 * num_rays);
            p = end;
        } else {                               // whole sources
            const int s1 = (int)(p1 / num_rays);
            q[0] = s0; q[1] = s1; q[2] = 0; q[3] = num_rays;
            p = (long long)s1 * num_rays;
        }
        ++*n_pieces;
    }
    return RT_OK;
}

rt_status rt_last_ckpt_stride(rt_grid* g, int* stride, float* tuned_ms) {
    if (!g) return fail(RT_ERR_INVALID_ARG, "grid handle is NULL");
    if (stride) *stride = g->last_k;
    if (tuned_ms) *tuned_ms = g->last_k_ms;
    return RT_OK;
}

rt_status rt_last_accumulation(rt_grid* g, int* mode) {
    if (!g || !mode) return fail(RT_ERR_INVALID_ARG, "NULL argument");
    *mode = g->last_acc == 0 ? 1 : (g->last_acc == 2 ? 2 : 3);
    return RT_OK;
}

rt_status rt_tuning_report(rt_grid* g, char* buf, int len) {
    if (!g || !buf || len < 1) return fail(RT_ERR_INVALID_ARG, "NULL buffer or length < 1");
    const std::string& r = g->tune_report;
    const size_t n = std::min(r.size(), (size_t)len - 1);
    std::memcpy(buf, r.data(), n);
    buf[n] = 0;
    return RT_OK;
}

}  // extern "C"

namespace {

rt_status backward_impl(rt_grid* g, const float* grad_out, const float* j_map, const float* kappa_map,
                        const float* source_pos, int num_sources, int num_rays, float step_size,
                        float radiation_velocity, float time_step, int n_freq, float* grad_j, float* grad_kappa,
                        float* grad_src, void* cuda_stream) {
    // the Call's output pointer only carries validation (non-NULL, no aliasing with the inputs)
    float* any_out = grad_j ? grad_j : (grad_kappa ? grad_kappa : grad_src);
    Call a{j_map, kappa_map, source_pos, num_sources, num_rays, 0, num_rays, step_size, radiation_velocity,
           time_step, n_freq, any_out, 0, (cudaStream_t)cuda_stream};
    int ns = 0;
    if (!g) return fail(RT_ERR_INVALID_ARG, "grid handle is NULL");
    if (!grad_out) return fail(RT_ERR_INVALID_ARG, "grad_out is NULL");
    if (!grad_j && !grad_kappa && !grad_src) return RT_OK;   // nothing requested
    rt_status st = validate(g, a, &ns);
    if (st != RT_OK) return st;
    for (const float* o : {(const float*)grad_j, (const float*)grad_kappa, (const float*)grad_src})
        if (o && (o == grad_out || o == j_map || o == kappa_map || o == source_pos))
            return fail(RT_ERR_INVALID_ARG, "a gradient output aliases an input");
    if (grad_j && grad_j == grad_kappa) return fail(RT_ERR_INVALID_ARG, "grad_j and grad_kappa alias");
    if (grad_src && (grad_src == grad_j || grad_src == grad_kappa))
        return fail(RT_ERR_INVALID_ARG, "grad_src aliases another gradient");
    if ((st = check_device(g)) != RT_OK) return st;
    if ((st = check_inputs(g, a, grad_out)) != RT_OK) return st;
    const long long ncell = g->ncell();
    const size_t field_bytes = sizeof(float) * (size_t)n_freq * ncell;
    if (grad_src && num_sources > 0)
        RT_CUDA(cudaMemsetAsync(grad_src, 0, sizeof(float) * 3 * (size_t)num_sources, a.st), "cudaMemsetAsync(grad_src)");
    if (ns == 0 || num_sources == 0) {
        if (grad_j) RT_CUDA(cudaMemsetAsync(grad_j, 0, field_bytes, a.st), "cudaMemsetAsync(grad_j)");
        if (grad_kappa) RT_CUDA(cudaMemsetAsync(grad_kappa, 0, field_bytes, a.st), "cudaMemsetAsync(grad_kappa)");
        return RT_OK;
    }
    const float4* dirs = nullptr;
    if ((st = g->table(num_rays, 0, num_rays, &dirs)) != RT_OK) return st;

    rt::BackArgs b{};
    b.dirs = dirs;
    b.src = source_pos;
    b.n0 = g->n0; b.n1 = g->n1; b.n2 = g->n2;
    b.ns = ns;
    b.ds = step_size;
    b.scale = (float)(4.0 * 3.14159265358979323846 / (double)num_rays);
    b.ray_count = num_rays;
    b.nsrc = num_sources;
    b.n_freq = n_freq;
    b.kappa_mode = g->opt.kappa_mode;
    b.block = 32;
    b.dsrc = grad_src;
    const int W = pick_width(n_freq);
    const int groups = (n_freq + W - 1) / W;
    // inputs of the reverse march: the caller's arrays for one bin, packed copies otherwise
    const size_t packed = sizeof(float) * (size_t)groups * ncell * W;
    void *djp = nullptr, *dkp = nullptr;
    if (W == 1) {
        b.grad = grad_out; b.j = j_map; b.kappa = kappa_map;
        b.dj = grad_j; b.dk = grad_kappa;
    } else {
        void *jp = nullptr, *kp = nullptr, *gp = nullptr;
        if ((st = g->ensure(rt_grid::JP, packed, &jp)) != RT_OK) return st;
        if ((st = g->ensure(rt_grid::KP, packed, &kp)) != RT_OK) return st;
        if ((st = g->ensure(rt_grid::GP, packed, &gp)) != RT_OK) return st;
        if (grad_j && (st = g->ensure(rt_grid::DJ, packed, &djp)) != RT_OK) return st;
        if (grad_kappa && (st = g->ensure(rt_grid::DK, packed, &dkp)) != RT_OK) return st;
        RT_CUDA(rt::launch_pack(j_map, (float*)jp, n_freq, W, groups, ncell, a.st), "pack(j) launch");
        RT_CUDA(rt::launch_pack(kappa_map, (float*)kp, n_freq, W, groups, ncell, a.st), "pack(kappa) launch");
        RT_CUDA(rt::launch_pack(grad_out, (float*)gp, n_freq, W, groups, ncell, a.st), "pack(grad) launch");
        b.grad = (const float*)gp; b.j = (const float*)jp; b.kappa = (const float*)kp;
        b.dj = (float*)djp; b.dk = (float*)dkp;
    }
    // checkpoint stride: tuned once per shape class when the handle autotunes and leaves the stride
    // automatic -- every K is timed on this call's own inputs (the full reverse march with its own
    // forward sweep, best of two runs; its gradients are discarded) and the fastest kept. The own
    // sweep also stands for what a recording forward pays to write that K's checkpoints (timing
    // the reverse march alone on recorded checkpoints gave a slower forward + adjoint step on the
    // 64^3 inverse workload: 8.5 against 8.9 x 10^9 updates/s, measured on GB300)
    const rt_grid::TuneKey kkey{n_freq, num_sources, num_rays, ns};
    bool tuned_now = false;
    g->last_k_ms = -1.0f;
    for (const auto& e : g->tuned_k)
        if (e.first == kkey) g->last_k_ms = e.second.second;
    if (g->opt.autotune && g->opt.ckpt_stride <= 0 && g->last_k_ms < 0.0f) {
        cudaEvent_t e[2] = {nullptr, nullptr};
        cudaError_t ce = cudaEventCreate(&e[0]);
        if (ce == cudaSuccess) ce = cudaEventCreate(&e[1]);
        int best_k = 16;
        float best_ms = 3.0e38f;
        for (int K : {4, 8, 16, 32}) {
            if (ce != cudaSuccess) break;
            rt::BackArgs t = b;
            t.stride = K;
            t.have_ckpt = 0;
            t.hash_rec = t.hash_now = nullptr;
            void* ck = nullptr;
            if ((st = g->ensure(rt_grid::CKPT, sizeof(float) * rt::backward_ckpt_floats(t, W), &ck)) != RT_OK) break;
            t.ckpt = (float*)ck;
            float kms = 3.0e38f;
            for (int rep = 0; rep < 2 && ce == cudaSuccess; ++rep) {
                ce = cudaEventRecord(e[0], a.st);
                if (ce == cudaSuccess) ce = rt::launch_march_bwd(W, t, a.st);
                if (ce == cudaSuccess) ce = cudaEventRecord(e[1], a.st);
                if (ce == cudaSuccess) ce = cudaEventSynchronize(e[1]);
                float ms = 0.0f;
                if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e[0], e[1]);
                if (ce == cudaSuccess && ms < kms) kms = ms;
            }
            if (ce == cudaSuccess && kms < best_ms) { best_ms = kms; best_k = K; }
        }
        for (auto ev : e)
            if (ev) cudaEventDestroy(ev);
        if (st != RT_OK) return st;
        if (ce != cudaSuccess) return cuda_fail(ce, "checkpoint-stride tuning");
        if (g->tuned_k.size() >= 64) g->tuned_k.erase(g->tuned_k.begin());
        g->tuned_k.push_back({kkey, {best_k, best_ms}});
        g->last_k_ms = best_ms;
        tuned_now = true;
        g->rec.valid = false;   // the tuning runs overwrote the checkpoint slot
    }
    b.stride = ckpt_stride(g, n_freq, num_sources, num_rays, ns);
    g->last_k = b.stride;
    // checkpoints recorded by the forward march of exactly this problem: skip the forward sweep
    const auto& r = g->rec;
    b.have_ckpt = !tuned_now && r.valid && r.j == j_map && r.kappa == kappa_map && r.src == source_pos &&
                  r.nsrc == num_sources && r.rays == num_rays && r.ns == ns && r.n_freq == n_freq &&
                  r.stride == b.stride && r.W == W && r.kappa_mode == g->opt.kappa_mode && r.ds == step_size;
    if (!b.have_ckpt) g->rec.valid = false;   // this reverse march rewrites the checkpoint slot
    if (b.have_ckpt) {
        // the kernel reuses the recording only if the inputs still hash as they did at the forward
        void* h;
        if ((st = g->ensure(rt_grid::HASH, 2 * sizeof(unsigned long long), &h)) != RT_OK) return st;
        b.hash_rec = (const unsigned long long*)h;
        b.hash_now = (const unsigned long long*)h + 1;
        RT_CUDA(rt::launch_input_hash(j_map, kappa_map, (long long)n_freq * ncell, source_pos, num_sources,
                                      (unsigned long long*)h + 1, a.st),
                "input hash launch");
    }
    void* ck;
    if ((st = g->ensure(rt_grid::CKPT, sizeof(float) * rt::backward_ckpt_floats(b, W), &ck)) != RT_OK) return st;
    b.ckpt = (float*)ck;
    // the gradients are sums: clear them (again, after tuning runs) just before the launch
    if (tuned_now && grad_src && num_sources > 0)
        RT_CUDA(cudaMemsetAsync(grad_src, 0, sizeof(float) * 3 * (size_t)num_sources, a.st), "cudaMemsetAsync(grad_src)");
    if (W == 1) {
        if (grad_j) RT_CUDA(cudaMemsetAsync(grad_j, 0, field_bytes, a.st), "cudaMemsetAsync(grad_j)");
        if (grad_kappa) RT_CUDA(cudaMemsetAsync(grad_kappa, 0, field_bytes, a.st), "cudaMemsetAsync(grad_kappa)");
        if ((st = g->mark(0, a.st)) != RT_OK) return st;
        RT_CUDA(rt::launch_march_bwd(1, b, a.st), "adjoint kernel launch");
        return g->mark(1, a.st);
    }
    if (djp) RT_CUDA(cudaMemsetAsync(djp, 0, packed, a.st), "cudaMemsetAsync(dj)");
    if (dkp) RT_CUDA(cudaMemsetAsync(dkp, 0, packed, a.st), "cudaMemsetAsync(dkappa)");
    if ((st = g->mark(0, a.st)) != RT_OK) return st;
    RT_CUDA(rt::launch_march_bwd(W, b, a.st), "adjoint kernel launch");
    if ((st = g->mark(1, a.st)) != RT_OK) return st;
    if (grad_j)
        RT_CUDA(rt::launch_unpack((const float*)djp, grad_j, n_freq, W, ncell, 1.0f, 0, a.st), "unpack(dj) launch");
    if (grad_kappa)
        RT_CUDA(rt::launch_unpack((const float*)dkp, grad_kappa, n_freq, W, ncell, 1.0f, 0, a.st),
                "unpack(dkappa) launch");
    return RT_OK;
}

}  // namespace

extern "C" {

rt_status rt_backward(rt_grid* g, const float* grad_out, const float* j_map, const float* kappa_map,
                      const float* source_pos, int num_sources, int num_rays, float step_size,
                      float radiation_velocity, float time_step, int n_freq, float* grad_j, float* grad_kappa,
                      void* cuda_stream) {
    return backward_impl(g, grad_out, j_map, kappa_map, source_pos, num_sources, num_rays, step_size,
                         radiation_velocity, time_step, n_freq, grad_j, grad_kappa, nullptr, cuda_stream);
}

// Emissivity inversion (Sec. 4): per iteration one recording rt_advance of j, the log-field
// misfit and its gradient dL/dF, one rt_backward for dL/dj, and a projected Adam step, all
// enqueued on the caller's stream. Workspace (INV slot): F, log target, dL/dF, dL/dj, the two
// Adam moments (n floats each) and the target's maximum.
rt_status rt_invert_emissivity(rt_grid* g, const float* target, const float* kappa_map, const float* source_pos,
                               int num_sources, int num_rays, float step_size, float radiation_velocity,
                               float time_step, int n_freq, int iterations, float lr, float eps_rel, float* j_map,
                               float* losses, void* cuda_stream) {
    if (!g) return fail(RT_ERR_INVALID_ARG, "grid handle is NULL");
    if (!target || !kappa_map || !j_map || !losses) return fail(RT_ERR_INVALID_ARG, "a NULL array");
    if (iterations < 0 || !(lr > 0.0f) || !std::isfinite(lr) || !(eps_rel > 0.0f) || !std::isfinite(eps_rel))
        return fail(RT_ERR_INVALID_ARG, "need iterations >= 0, finite lr > 0 and eps_rel > 0");
    if (n_freq < 1 || n_freq > g->max_freq) return fail(RT_ERR_INVALID_ARG, "n_freq must be in [1, max_freq]");
    if (j_map == target || j_map == kappa_map || j_map == source_pos)
        return fail(RT_ERR_INVALID_ARG, "j_map aliases an input");
    const long long n = (long long)n_freq * g->ncell();
    const float* lo = losses;
    for (const float* a : {target, kappa_map, (const float*)j_map})
        if (lo < a + n && a < lo + iterations + 1) return fail(RT_ERR_INVALID_ARG, "losses overlaps an array");
    rt_status st = check_device(g);
    if (st != RT_OK) return st;
    const cudaStream_t cs = (cudaStream_t)cuda_stream;
    void* w = nullptr;
    if ((st = g->ensure(rt_grid::INV, sizeof(float) * (6 * (size_t)n + 4), &w)) != RT_OK) return st;
    float* F = (float*)w;
    float* log_t = F + n;
    float* grad = log_t + n;
    float* dj = grad + n;
    float* m = dj + n;
    float* v = m + n;
    float* fmax = v + n;
    RT_CUDA(cudaMemsetAsync(m, 0, sizeof(float) * 2 * (size_t)n, cs), "cudaMemsetAsync(Adam moments)");
    RT_CUDA(cudaMemsetAsync(losses, 0, sizeof(float) * ((size_t)iterations + 1), cs), "cudaMemsetAsync(losses)");
    RT_CUDA(rt::launch_field_max(target, 1, n, fmax, cs), "target maximum");
    RT_CUDA(rt::launch_log_target(target, n, fmax, eps_rel, log_t, cs), "log target");
    for (int it = 1; it <= iterations; ++it) {
        if ((st = rt_advance(g, j_map, kappa_map, source_pos, num_sources, num_rays, step_size, radiation_velocity,
                             time_step, n_freq, F, 0, cuda_stream)) != RT_OK)
            return st;
        RT_CUDA(rt::launch_log_misfit(F, log_t, n, fmax, eps_rel, grad, losses + it - 1, cs), "log misfit");
        if ((st = rt_backward(g, grad, j_map, kappa_map, source_pos, num_sources, num_rays, step_size,
                              radiation_velocity, time_step, n_freq, dj, nullptr, cuda_stream)) != RT_OK)
            return st;
        RT_CUDA(rt::launch_adam_projected(j_map, dj, m, v, n, lr, 0.9f, 0.999f, 1e-8f, it, 0.0f, cs), "Adam step");
    }
    if ((st = rt_advance(g, j_map, kappa_map, source_pos, num_sources, num_rays, step_size, radiation_velocity,
                         time_step, n_freq, F, 0, cuda_stream)) != RT_OK)
        return st;
    RT_CUDA(rt::launch_log_misfit(F, log_t, n, fmax, eps_rel, nullptr, losses + iterations, cs), "log misfit");
    return RT_OK;
}

rt_status rt_backward_sources(rt_grid* g, const float* grad_out, const float* j_map, const float* kappa_map,
                              const float* source_pos, int num_sources, int num_rays, float step_size,
                              float radiation_velocity, float time_step, int n_freq, float* grad_j,
                              float* grad_kappa, float* grad_src, void* cuda_stream) {
    return backward_impl(g, grad_out, j_map, kappa_map, source_pos, num_sources, num_rays, step_size,
                         radiation_velocity, time_step, n_freq, grad_j, grad_kappa, grad_src, cuda_stream);
}

}  // extern "C"
