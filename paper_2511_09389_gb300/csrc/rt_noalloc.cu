// rt_noalloc.cu -- rt_advance_noalloc: the forward march without any memory allocation.
//
// Some callers cannot allocate memory while they run: a host program whose GPU memory is
// owned by another framework's pool (so a cudaMalloc from this library would fragment or
// overrun a budget it does not control), a real-time loop that must not block in the
// allocator, or an integration that forbids new allocations after start-up. For them this
// entry point runs the same pack / march / unpack kernels as rt_advance, but its scratch
// (sorted direction table, packed j and kappa, packed accumulator) lives in one fixed,
// file-scope device array instead of handle-owned cudaMalloc buffers. It needs no handle.
//
// The array is RT_NOALLOC_SCRATCH_BYTES (16 MiB). Every GPU that loads this library holds it
// until the process exits. All calls share it and it keeps the last call's contents; the
// accumulator part is cleared on the stream at every call. Calls whose work overlaps on the
// GPU (different streams, or different host threads) race on the array.
#include <cuda.h>   // driver types only: the two driver calls below are looked up at run time
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "raytrax.h"
#include "rt_internal.h"

namespace {

constexpr size_t kScratchBytes = RT_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxRays = RT_NOALLOC_MAX_RAYS;
constexpr size_t kDirBytes = sizeof(float4) * (size_t)kMaxRays;
constexpr int kMaxDevices = 64;

// The scratch. Device code could name it directly; host code must use the device address
// returned by cudaGetSymbolAddress (the host-side symbol is only a stand-in).
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

struct DeviceState {
    void* base = nullptr;        // device address of g_scratch on this device
    unsigned long long ctx = 0;  // unique id of the context that address belongs to (0: unknown)
    int dirs_n = 0;              // lattice size whose sorted table is in the scratch (0: none)
};

// Unique id of the calling thread's current context, or 0 if the driver cannot say. The driver
// entry points come through the runtime (no link against the driver library).
unsigned long long current_context_id() {
    using GetCurrent = CUresult (*)(CUcontext*);
    using GetId = CUresult (*)(CUcontext, unsigned long long*);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        looked_up = true;
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = (GetCurrent)f;
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = (GetId)f;
    }
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&c) != CUDA_SUCCESS || !c || get_id(c, &id) != CUDA_SUCCESS) return 0;
    return id;
}

std::mutex g_mutex;
DeviceState g_dev[kMaxDevices];
// host staging for the direction table: static, so building it allocates nothing
float4 g_dirs_host[kMaxRays];
uint32_t g_key[kMaxRays];
int g_order[kMaxRays];

rt_status err(rt_status st, const char* fmt, ...) {
    char buf[384];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    return rt::set_error(st, buf);
}

rt_status cuda_err(cudaError_t e, const char* what) {
    return err(RT_ERR_CUDA, "rt_advance_noalloc: %s: %s", what, cudaGetErrorString(e));
}

}  // namespace

extern "C" rt_status rt_advance_noalloc(const float* j_map, const float* kappa_map, const float* source_pos,
                                        int num_sources, int n0, int n1, int n2, int num_rays, float step_size,
                                        float radiation_velocity, float time_step, int n_freq, float* out_field,
                                        void* cuda_stream) {
    // ---- host-side checks (nothing is enqueued on error) ----
    if (n0 < 1 || n1 < 1 || n2 < 1 || n_freq < 1 || num_sources < 0 || num_rays < 1)
        return err(RT_ERR_INVALID_ARG, "rt_advance_noalloc: extents, n_freq and num_rays must be >= 1, "
                                       "num_sources >= 0");
    if (!j_map || !kappa_map || !out_field || (num_sources > 0 && !source_pos))
        return err(RT_ERR_INVALID_ARG, "rt_advance_noalloc: NULL buffer");
    if (out_field == j_map || out_field == kappa_map)
        return err(RT_ERR_INVALID_ARG, "rt_advance_noalloc: out_field aliases an input");
    if (!(step_size > 0.0f) || !std::isfinite(step_size) || !(radiation_velocity > 0.0f) ||
        !std::isfinite(radiation_velocity) || !(time_step >= 0.0f) || !std::isfinite(time_step))
        return err(RT_ERR_INVALID_ARG, "rt_advance_noalloc: need step_size > 0, radiation_velocity > 0, "
                                       "time_step >= 0, all finite");
    const int ns = rt::substeps(step_size, radiation_velocity, time_step, 0);   // the rule of rt_advance
    if (ns < 0 || (double)ns * step_size > 1.6e7)
        return err(RT_ERR_INVALID_ARG, "rt_advance_noalloc: ray length c*dt too large");
    const long long ncell = (long long)n0 * n1 * n2;
    const int W = n_freq == 1 ? 1 : (n_freq == 2 ? 2 : 4);
    const int groups = (n_freq + W - 1) / W;
    if (ncell * (long long)groups * W >= (1LL << 31))
        return err(RT_ERR_INVALID_ARG, "rt_advance_noalloc: grid too large (n_freq * cells >= 2^31)");
    // packed j, packed kappa and the packed accumulator (W > 1 only) after the direction table
    const size_t packed = W > 1 ? sizeof(float) * (size_t)groups * (size_t)ncell * W : 0;
    if (num_rays > kMaxRays || kDirBytes + 3 * packed > kScratchBytes)
        return err(RT_ERR_INVALID_ARG,
                   "rt_advance_noalloc: needs %zu bytes of scratch for %d rays and %lld cells x %d bins; "
                   "the static scratch holds %zu bytes and %d rays (use rt_advance instead)",
                   kDirBytes + 3 * packed, num_rays, ncell, n_freq, kScratchBytes, kMaxRays);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const size_t field_bytes = sizeof(float) * (size_t)n_freq * (size_t)ncell;

    std::lock_guard<std::mutex> lock(g_mutex);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_err(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return err(RT_ERR_UNSUPPORTED, "rt_advance_noalloc: device index too large");
    DeviceState& ds = g_dev[dev];
    // ---- device address of the static scratch, looked up on every call ----
    // Cheap once the module is loaded. When the device's context has been replaced since the
    // last call (cudaDeviceReset, a new primary context), the module was loaded again: the old
    // address may point at freed memory and the direction table stored there is gone, whether or
    // not the new array landed at the same address. Either change starts the state afresh.
    {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);   // also makes sure the context exists
        if (e != cudaSuccess) return cuda_err(e, "cudaGetSymbolAddress(scratch)");
        const unsigned long long ctx = current_context_id();
        if (p != ds.base || ctx != ds.ctx || ctx == 0) {
            ds.base = p;
            ds.ctx = ctx;
            ds.dirs_n = 0;   // a new array: its direction table must be rebuilt
        }
    }
    unsigned char* base = (unsigned char*)ds.base;
    float4* d_dirs = (float4*)base;
    float* d_jp = (float*)(base + kDirBytes);
    float* d_kp = (float*)(base + kDirBytes + packed);
    float* d_acc = (float*)(base + kDirBytes + 2 * packed);

    if (ns == 0 || num_sources == 0) {
        e = cudaMemsetAsync(out_field, 0, field_bytes, st);
        return e == cudaSuccess ? RT_OK : cuda_err(e, "cudaMemsetAsync(out)");
    }
    // ---- direction table: rebuilt only when the lattice size changes ----
    if (ds.dirs_n != num_rays) {
        // earlier work on this stream may still read the old table: wait for it, copy in stream
        // order, and wait again because the static host staging array is reused next call
        e = cudaStreamSynchronize(st);
        if (e == cudaSuccess) {
            rt::sorted_lattice(num_rays, 0, num_rays, g_dirs_host, g_key, g_order);
            e = cudaMemcpyAsync(d_dirs, g_dirs_host, sizeof(float4) * (size_t)num_rays, cudaMemcpyHostToDevice, st);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            ds.dirs_n = 0;
            return cuda_err(e, "cudaMemcpy(direction table)");
        }
        ds.dirs_n = num_rays;
    }

    rt::MarchArgs m{};
    m.dirs = d_dirs;
    m.src = source_pos;
    m.n0 = n0; m.n1 = n1; m.n2 = n2;
    m.ns = ns;
    m.ds = step_size;
    m.ray_count = num_rays;
    m.nsrc = num_sources;
    m.n_freq = n_freq;
    m.kappa_mode = 0;
    m.block = 32;
    m.prefetch = W == 1 ? 1 : 0;
    m.tile = W == 1 ? 1 : 0;     // source deposit tiles: static shared memory, no allocation
    const float scale = (float)(4.0 * 3.14159265358979323846 / (double)num_rays);
    if (W == 1) {
        // one bin: no packing, the march deposits straight into the (cleared) output
        e = cudaMemsetAsync(out_field, 0, field_bytes, st);
        if (e != cudaSuccess) return cuda_err(e, "cudaMemsetAsync(out)");
        m.jp = j_map; m.kp = kappa_map; m.acc = out_field;
        m.groups = n_freq;
        m.dep_scale = scale;
        e = rt::launch_march_fwd(1, m, st);
        return e == cudaSuccess ? RT_OK : cuda_err(e, "march kernel launch");
    }
    if ((e = rt::launch_pack(j_map, d_jp, n_freq, W, groups, ncell, st)) != cudaSuccess)
        return cuda_err(e, "pack(j) launch");
    if ((e = rt::launch_pack(kappa_map, d_kp, n_freq, W, groups, ncell, st)) != cudaSuccess)
        return cuda_err(e, "pack(kappa) launch");
    // the accumulator keeps the previous call's sums: clear it first
    if ((e = cudaMemsetAsync(d_acc, 0, packed, st)) != cudaSuccess) return cuda_err(e, "cudaMemsetAsync(acc)");
    m.jp = d_jp; m.kp = d_kp; m.acc = d_acc;
    m.groups = groups;
    m.dep_scale = 1.0f;
    if ((e = rt::launch_march_fwd(W, m, st)) != cudaSuccess) return cuda_err(e, "march kernel launch");
    if ((e = rt::launch_unpack(d_acc, out_field, n_freq, W, ncell, scale, 0, st)) != cudaSuccess)
        return cuda_err(e, "unpack launch");
    return RT_OK;
}
