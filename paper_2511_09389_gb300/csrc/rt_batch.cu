// rt_batch.cu -- host side of the batched persistent launch (rt_batch_* in raytrax.h).
//
// At creation the instances are validated, their scratch (packed j / kappa for instances with
// two or more bins, one contiguous accumulator region for all) and lattice tables are
// allocated. Instances with RT_BATCH_DEDICATED_LANES or more (source, ray, bin group) lanes
// fill the GPU alone; they get their own pack / march / unpack launches with a single-call
// plan (autotuned on the first run if asked): on GB300 the persistent kernel ran such
// instances at 0.85x their one-by-one time. The rest are grouped into waves whose working
// sets (packed inputs and accumulator) fit in half the L2 cache, each with its own work queue
// of 32-ray items, longest first. The first run captures the dedicated launches and, per wave,
// batched pack, persistent march and batched unpack into one CUDA graph; every run launches
// it. Packing every instance before marching any (one wave) made the march read its packed
// grids back from DRAM: measured on GB300 with 8 copies of a 128^3, 4-bin problem, 493 MB of
// DRAM reads per instance against 150 MB for a single call.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <map>
#include <new>
#include <vector>

#include "raytrax.h"
#include "rt_internal.h"

namespace {

rt_status err(rt_status st, const char* fmt, ...) {
    char buf[384];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    return rt::set_error(st, buf);
}

rt_status cuda_err(cudaError_t e, const char* what) {
    return err(e == cudaErrorMemoryAllocation ? RT_ERR_OOM : RT_ERR_CUDA, "rt_batch: %s: %s", what,
               cudaGetErrorString(e));
}

#define B_CUDA(call, what)                                   \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return cuda_err(e_, what);    \
    } while (0)

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

struct rt_batch {
    int device = 0;
    rt_options opt{};
    std::vector<rt::BatchInst> host;
    rt::BatchInst* d_insts = nullptr;
    int4* d_items = nullptr;          // per wave: items of width 4, then 2, then 1
    int n_items = 0;
    // a wave: instances [first_inst, first_inst + n_inst) of d_insts and their items
    struct Wave {
        int first_inst = 0, n_inst = 0;
        long long max_elems = 0;      // largest groups * ncell of the wave (sizes the layout kernels)
        int w_first[3] = {0, 0, 0};   // first item of widths 4, 2, 1
        int w_count[3] = {0, 0, 0};
    };
    std::vector<Wave> waves;
    // an instance marched by its own launches: its position in host / d_insts and its plan
    struct Dedicated {
        int inst = 0;
        int W = 1;                    // bin-group width of its march (its scratch fits any width
                                      // up to the instance's own: groups * W never grows)
        int block = 32, prefetch = 0, tile = 0, lpr = 1;
    };
    std::vector<Dedicated> ded;
    // dedicated instances whose working sets together fit in half the L2 cache run as
    // concurrent branches (up to three): [first, first + count) of ded
    struct DedGroup {
        int first = 0, count = 0;
    };
    std::vector<DedGroup> ded_groups;
    std::vector<int> pos;             // caller's instance index -> position in host / d_insts
    int* d_counter = nullptr;         // one counter per wave and width
    cudaStream_t side[2] = {nullptr, nullptr};
    cudaEvent_t fork = nullptr, join[2] = {nullptr, nullptr};
    unsigned char* scratch = nullptr;
    float* acc = nullptr;
    size_t acc_bytes = 0;
    std::map<int, float4*> dirs;
    cudaStream_t cap = nullptr;
    cudaGraphExec_t exec = nullptr;
    int block = 64, sms = 0;
    long long updates = 0;

    static int widx(int W) { return W == 4 ? 0 : (W == 2 ? 1 : 2); }
    int grid_for(int W) const { return sms * rt::march_batch_blocks_per_sm(W, block); }

    void release() {
        cudaDeviceSynchronize();
        if (exec) cudaGraphExecDestroy(exec);
        if (cap) cudaStreamDestroy(cap);
        for (auto s : side)
            if (s) cudaStreamDestroy(s);
        if (fork) cudaEventDestroy(fork);
        for (auto e : join)
            if (e) cudaEventDestroy(e);
        for (auto& d : dirs) cudaFree(d.second);
        cudaFree(d_insts);
        cudaFree(d_items);
        cudaFree(d_counter);
        cudaFree(scratch);
    }

    // The three widths of a wave run as concurrent branches (streams side[0], side[1] fork from
    // st and join back), so the tail of one persistent kernel overlaps the start of the next.
    rt_status march(const Wave& w, int wi, cudaStream_t st) {
        const int widths[3] = {4, 2, 1};
        cudaStream_t on[3] = {st, side[0], side[1]};
        B_CUDA(cudaEventRecord(fork, st), "fork");
        for (int i = 1; i < 3; ++i) B_CUDA(cudaStreamWaitEvent(on[i], fork, 0), "fork wait");
        for (int i = 0; i < 3; ++i)
            B_CUDA(rt::launch_march_batch(widths[i], d_insts, d_items + w.w_first[i], w.w_count[i],
                                          d_counter + 3 * wi + i, grid_for(widths[i]), block, on[i]),
                   "march launch");
        for (int i = 1; i < 3; ++i) {
            B_CUDA(cudaEventRecord(join[i - 1], on[i]), "join");
            B_CUDA(cudaStreamWaitEvent(st, join[i - 1], 0), "join wait");
        }
        return RT_OK;
    }

    rt::MarchArgs dedicated_args(const Dedicated& d) const {
        const rt::BatchInst& b = host[d.inst];
        rt::MarchArgs m{};
        if (d.W == 1) { m.jp = b.j; m.kp = b.kappa; }
        else { m.jp = b.jp_w; m.kp = b.kp_w; }
        m.acc = b.acc;
        m.dirs = b.dirs; m.src = b.src;
        m.n0 = b.n0; m.n1 = b.n1; m.n2 = b.n2;
        m.ns = b.ns; m.ds = b.ds;
        m.dep_scale = 1.0f;           // 4 pi / N_Omega applied by the unpack, as for the waves
        m.ray_count = b.ray_count; m.nsrc = b.nsrc;
        m.groups = (b.n_freq + d.W - 1) / d.W; m.n_freq = b.n_freq; m.kappa_mode = b.kappa_mode;
        m.block = d.block; m.prefetch = d.prefetch; m.lanes_per_ray = d.lpr; m.tile = d.lpr == 1 ? d.tile : 0;
        return m;
    }

    rt_status pack_dedicated(const Dedicated& d, cudaStream_t st) {
        const rt::BatchInst& b = host[d.inst];
        if (d.W == 1) return RT_OK;
        const long long ncell = (long long)b.n0 * b.n1 * b.n2;
        const int groups = (b.n_freq + d.W - 1) / d.W;
        B_CUDA(rt::launch_pack(b.j, b.jp_w, b.n_freq, d.W, groups, ncell, st), "pack(j) launch");
        B_CUDA(rt::launch_pack(b.kappa, b.kp_w, b.n_freq, d.W, groups, ncell, st), "pack(kappa) launch");
        return RT_OK;
    }

    // One bin per thread deposits straight into the caller's field with the 4 pi / N_Omega factor,
    // as a single call does; wider groups go through the packed accumulator and the unpack.
    rt_status run_dedicated(const Dedicated& d, cudaStream_t st) {
        const rt::BatchInst& b = host[d.inst];
        const long long ncell = (long long)b.n0 * b.n1 * b.n2;
        rt_status rs = pack_dedicated(d, st);
        if (rs != RT_OK) return rs;
        rt::MarchArgs m = dedicated_args(d);
        if (d.W == 1) {
            B_CUDA(cudaMemsetAsync(b.out, 0, sizeof(float) * (size_t)b.n_freq * ncell, st), "clear field");
            m.acc = b.out;
            m.dep_scale = b.scale;
        }
        B_CUDA(rt::launch_march_fwd(d.W, m, st), "march launch");
        if (d.W > 1)
            B_CUDA(rt::launch_unpack(b.acc, b.out, b.n_freq, d.W, ncell, b.scale, 0, st), "unpack launch");
        return RT_OK;
    }

    // Time the single-call tuner's candidate plans (rt::march_plan_candidates) for one dedicated
    // instance's march on its own inputs and keep the best. Its scratch, sized for its own
    // width, holds the packed copies of every narrower width.
    rt_status tune_dedicated(Dedicated& d, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1) {
        const rt::BatchInst& b = host[d.inst];
        const size_t accb = sizeof(float) * (size_t)b.groups * b.n0 * b.n1 * b.n2 * b.W;
        rt::MarchPlan cands[rt::kMaxMarchPlans];
        const int n = rt::march_plan_candidates(b.n_freq, cands);
        float best = 3.0e38f;
        Dedicated win = d;
        int packed_w = 0;
        for (int ci = 0; ci < n; ++ci) {
            Dedicated c = d;
            c.W = cands[ci].W; c.block = cands[ci].block; c.prefetch = cands[ci].prefetch;
            c.tile = cands[ci].tile; c.lpr = cands[ci].lpr;
            if (c.W > b.W || !rt::march_fwd_available(c.W, c.prefetch, 0, c.tile, 0, c.lpr, c.block)) continue;
            if (c.W != packed_w) {
                rt_status rs = pack_dedicated(c, st);
                if (rs != RT_OK) return rs;
                packed_w = c.W;
            }
            const rt::MarchArgs m = dedicated_args(c);
            float ms = 3.0e38f;
            for (int rep = 0; rep < 2; ++rep) {   // the first run warms the caches
                B_CUDA(cudaMemsetAsync(b.acc, 0, accb, st), "clear accumulator");
                B_CUDA(cudaEventRecord(e0, st), "cudaEventRecord");
                B_CUDA(rt::launch_march_fwd(c.W, m, st), "march launch");
                B_CUDA(cudaEventRecord(e1, st), "cudaEventRecord");
                B_CUDA(cudaEventSynchronize(e1), "cudaEventSynchronize");
                B_CUDA(cudaEventElapsedTime(&ms, e0, e1), "cudaEventElapsedTime");
            }
            if (ms < best) { best = ms; win = c; }
        }
        d = win;
        return RT_OK;
    }

    rt_status enqueue(cudaStream_t st) {
        B_CUDA(cudaMemsetAsync(d_counter, 0, 3 * std::max<size_t>(waves.size(), 1) * sizeof(int), st),
               "clear work counters");
        B_CUDA(cudaMemsetAsync(acc, 0, acc_bytes, st), "clear accumulators");
        for (const DedGroup& dg : ded_groups) {
            cudaStream_t on[3] = {st, side[0], side[1]};
            if (dg.count > 1) {
                B_CUDA(cudaEventRecord(fork, st), "fork");
                for (int i = 1; i < dg.count; ++i) B_CUDA(cudaStreamWaitEvent(on[i], fork, 0), "fork wait");
            }
            for (int i = 0; i < dg.count; ++i) {
                rt_status rs = run_dedicated(ded[dg.first + i], on[i]);
                if (rs != RT_OK) return rs;
            }
            for (int i = 1; i < dg.count; ++i) {
                B_CUDA(cudaEventRecord(join[i - 1], on[i]), "join");
                B_CUDA(cudaStreamWaitEvent(st, join[i - 1], 0), "join wait");
            }
        }
        for (size_t wi = 0; wi < waves.size(); ++wi) {
            const Wave& w = waves[wi];
            const rt::BatchInst* in = d_insts + w.first_inst;
            B_CUDA(rt::launch_pack_batch(in, w.n_inst, w.max_elems, 0, st), "pack(j) launch");
            B_CUDA(rt::launch_pack_batch(in, w.n_inst, w.max_elems, 1, st), "pack(kappa) launch");
            rt_status rs = march(w, (int)wi, st);
            if (rs != RT_OK) return rs;
            B_CUDA(rt::launch_unpack_batch(in, w.n_inst, w.max_elems, st), "unpack launch");
        }
        return RT_OK;
    }
};

extern "C" {

rt_status rt_batch_create(rt_batch** out, const rt_instance* inst, int n_inst, const rt_options* opt) {
    if (!out) return err(RT_ERR_INVALID_ARG, "rt_batch_create: out is NULL");
    *out = nullptr;
    if (n_inst < 1 || !inst) return err(RT_ERR_INVALID_ARG, "rt_batch_create: need n_inst >= 1 instances");
    rt_options o{};
    if (opt) o = *opt;
    if (o.kappa_mode != 0 && o.kappa_mode != 1) return err(RT_ERR_INVALID_ARG, "rt_batch_create: bad kappa_mode");
    if (o.deterministic) return err(RT_ERR_UNSUPPORTED, "rt_batch_create: deterministic mode is not supported");

    // ---- validate, size the scratch ----
    std::vector<rt::BatchInst> h(n_inst);
    size_t packed_total = 0, acc_total = 0;
    long long updates = 0;
    for (int i = 0; i < n_inst; ++i) {
        const rt_instance& q = inst[i];
        if (q.n0 < 1 || q.n1 < 1 || q.n2 < 1 || q.n_freq < 1 || q.num_sources < 1 || q.num_rays < 1)
            return err(RT_ERR_INVALID_ARG, "rt_batch_create: instance %d: extents, n_freq, num_sources and "
                                           "num_rays must be >= 1", i);
        if (!q.j_map || !q.kappa_map || !q.source_pos || !q.out_field)
            return err(RT_ERR_INVALID_ARG, "rt_batch_create: instance %d: NULL buffer", i);
        if (q.out_field == q.j_map || q.out_field == q.kappa_map)
            return err(RT_ERR_INVALID_ARG, "rt_batch_create: instance %d: out_field aliases an input", i);
        const int ns = rt::substeps(q.step_size, q.radiation_velocity, q.time_step, o.ns_cap);
        if (ns < 0 || !(q.step_size > 0.0f) || !(q.radiation_velocity > 0.0f) || !(q.time_step >= 0.0f) ||
            (double)ns * q.step_size > 1.6e7)
            return err(RT_ERR_INVALID_ARG, "rt_batch_create: instance %d: invalid step_size / "
                                           "radiation_velocity / time_step", i);
        const long long ncell = (long long)q.n0 * q.n1 * q.n2;
        const int W = q.n_freq == 1 ? 1 : (q.n_freq == 2 ? 2 : 4);
        const int groups = (q.n_freq + W - 1) / W;
        if (ncell * groups * W >= (1LL << 31))
            return err(RT_ERR_INVALID_ARG, "rt_batch_create: instance %d: grid too large", i);
        rt::BatchInst& b = h[i];
        b = rt::BatchInst{};
        b.j = q.j_map; b.kappa = q.kappa_map; b.out = q.out_field; b.src = q.source_pos;
        b.n0 = q.n0; b.n1 = q.n1; b.n2 = q.n2; b.n_freq = q.n_freq; b.W = W; b.groups = groups;
        b.ns = ns; b.nsrc = q.num_sources; b.ray_count = q.num_rays; b.kappa_mode = o.kappa_mode;
        b.ds = q.step_size;
        b.scale = (float)(4.0 * 3.14159265358979323846 / (double)q.num_rays);
        const size_t field = sizeof(float) * (size_t)groups * ncell * W;
        if (W > 1) packed_total += 2 * align256(field);
        acc_total += align256(field);
        updates += (long long)ns * q.num_rays * q.num_sources * q.n_freq;
    }

    // ---- waves: working sets (packed j, kappa and accumulator) within half the L2 cache ----
    int l2 = 0, cur_dev = 0;
    if (cudaGetDevice(&cur_dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, cur_dev) != cudaSuccess || l2 <= 0)
        l2 = 64 << 20;
    const double budget = 0.5 * (double)l2;
    std::vector<double> footprint(n_inst);
    for (int i = 0; i < n_inst; ++i) {
        const double field = 4.0 * h[i].groups * (double)h[i].n0 * h[i].n1 * h[i].n2 * h[i].W;
        footprint[i] = 3.0 * field;   // j and kappa (packed, or the caller's arrays) and the accumulator
    }
    // dedicated instances first (largest working set first), then the wave instances
    std::vector<char> dedicated(n_inst);
    int n_ded = 0;
    for (int i = 0; i < n_inst; ++i) {
        const long long lanes = (long long)h[i].nsrc * h[i].ray_count * h[i].groups;
        dedicated[i] = lanes >= RT_BATCH_DEDICATED_LANES;
        n_ded += dedicated[i];
    }
    std::vector<int> order(n_inst);
    for (int i = 0; i < n_inst; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        if (dedicated[a] != dedicated[b]) return dedicated[a] > dedicated[b];
        return footprint[a] > footprint[b];
    });
    std::vector<rt_batch::Wave> waves;
    double wave_bytes = 0.0;
    for (int k = n_ded; k < n_inst; ++k) {
        const int i = order[k];
        if (waves.empty() || (wave_bytes + footprint[i] > budget && waves.back().n_inst > 0)) {
            rt_batch::Wave w;
            w.first_inst = k;
            waves.push_back(w);
            wave_bytes = 0.0;
        }
        waves.back().n_inst++;
        waves.back().max_elems = std::max(waves.back().max_elems, (long long)h[i].groups * h[i].n0 * h[i].n1 * h[i].n2);
        wave_bytes += footprint[i];
    }
    {
        std::vector<rt::BatchInst> hs(n_inst);
        for (int k = 0; k < n_inst; ++k) hs[k] = h[order[k]];
        h.swap(hs);   // waves are contiguous ranges of h from here on
    }

    rt_batch* B = new (std::nothrow) rt_batch();
    if (!B) return err(RT_ERR_OOM, "rt_batch_create: host allocation failed");
    B->opt = o;
    B->updates = updates;
    B->waves = waves;
    B->pos.assign(n_inst, 0);
    for (int k = 0; k < n_inst; ++k) B->pos[order[k]] = k;
    {
        double group_bytes = 0.0;
        for (int k = 0; k < n_ded; ++k) {
            const double fp = footprint[order[k]];
            if (B->ded_groups.empty() || B->ded_groups.back().count == 3 || group_bytes + fp > budget) {
                B->ded_groups.push_back(rt_batch::DedGroup{k, 0});
                group_bytes = 0.0;
            }
            B->ded_groups.back().count++;
            group_bytes += fp;
        }
    }
    for (int k = 0; k < n_ded; ++k) {
        rt_batch::Dedicated d;
        d.inst = k;
        d.W = h[k].W;
        d.prefetch = h[k].W == 1 ? 1 : 0;   // the single-call default plan
        d.tile = h[k].W == 1 ? 1 : 0;
        B->ded.push_back(d);
    }
    auto fail_free = [&](rt_status st) { B->release(); delete B; return st; };
    cudaError_t e = cudaGetDevice(&B->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&B->sms, cudaDevAttrMultiProcessorCount, B->device);
    if (e == cudaSuccess) e = cudaMalloc(&B->scratch, packed_total + acc_total);
    if (e != cudaSuccess) return fail_free(cuda_err(e, "scratch allocation"));

    // ---- lay out scratch, lattice tables ----
    size_t off = 0;
    for (auto& b : h) {
        const size_t field = sizeof(float) * (size_t)b.groups * b.n0 * b.n1 * b.n2 * b.W;
        if (b.W > 1) {
            b.jp_w = (float*)(B->scratch + off); off += align256(field);
            b.kp_w = (float*)(B->scratch + off); off += align256(field);
            b.jp = b.jp_w; b.kp = b.kp_w;
        } else {
            b.jp = b.j; b.kp = b.kappa;
        }
    }
    B->acc = (float*)(B->scratch + off);
    B->acc_bytes = acc_total;
    for (auto& b : h) {
        b.acc = (float*)(B->scratch + off);
        off += align256(sizeof(float) * (size_t)b.groups * b.n0 * b.n1 * b.n2 * b.W);
        auto it = B->dirs.find(b.ray_count);
        if (it == B->dirs.end()) {
            std::vector<float4> t(b.ray_count);
            std::vector<uint32_t> key(b.ray_count);
            std::vector<int> order(b.ray_count);
            rt::sorted_lattice(b.ray_count, 0, b.ray_count, t.data(), key.data(), order.data());
            float4* d = nullptr;
            e = cudaMalloc(&d, sizeof(float4) * t.size());
            if (e == cudaSuccess) e = cudaMemcpy(d, t.data(), sizeof(float4) * t.size(), cudaMemcpyHostToDevice);
            if (e != cudaSuccess) { cudaFree(d); return fail_free(cuda_err(e, "lattice table")); }
            it = B->dirs.emplace(b.ray_count, d).first;
        }
        b.dirs = it->second;
    }

    // ---- work queues: 32-ray items per wave, grouped by width, longest march first ----
    // bin group outside sources: one group's packed j, kappa and accumulator stay L2-resident
    // while all of its sources march
    std::vector<int4> items;
    for (auto& w : B->waves) {
        const size_t begin = items.size();
        for (int i = w.first_inst; i < w.first_inst + w.n_inst; ++i)
            for (int g = 0; g < h[i].groups; ++g)
                for (int s = 0; s < h[i].nsrc; ++s)
                    for (int r = 0; r < h[i].ray_count; r += 32) items.push_back(make_int4(i, s, g, r));
        std::stable_sort(items.begin() + begin, items.end(), [&](const int4& a, const int4& b) {
            const int wa = rt_batch::widx(h[a.x].W), wb = rt_batch::widx(h[b.x].W);
            if (wa != wb) return wa < wb;
            return h[a.x].ns > h[b.x].ns;
        });
        for (size_t k = begin; k < items.size(); ++k) w.w_count[rt_batch::widx(h[items[k].x].W)]++;
        w.w_first[0] = (int)begin;
        w.w_first[1] = w.w_first[0] + w.w_count[0];
        w.w_first[2] = w.w_first[1] + w.w_count[1];
        if (items.size() > 0x7fffffff) return fail_free(err(RT_ERR_INVALID_ARG, "rt_batch_create: too many work items"));
    }
    B->n_items = (int)items.size();
    e = cudaMalloc(&B->d_insts, sizeof(rt::BatchInst) * h.size());
    if (e == cudaSuccess) e = cudaMemcpy(B->d_insts, h.data(), sizeof(rt::BatchInst) * h.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&B->d_items, sizeof(int4) * std::max<size_t>(items.size(), 1));
    if (e == cudaSuccess && !items.empty())
        e = cudaMemcpy(B->d_items, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&B->d_counter, 3 * std::max<size_t>(B->waves.size(), 1) * sizeof(int));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaStreamCreateWithFlags(&B->side[i], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&B->join[i], cudaEventDisableTiming);
    if (e != cudaSuccess) return fail_free(cuda_err(e, "work queue"));
    B->host = std::move(h);
    B->block = 64;
    *out = B;
    return RT_OK;
}

rt_status rt_batch_run(rt_batch* B, void* cuda_stream) {
    if (!B) return err(RT_ERR_INVALID_ARG, "rt_batch_run: batch is NULL");
    int dev = -1;
    B_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev != B->device) return err(RT_ERR_INVALID_ARG, "rt_batch_run: current device differs from the batch's");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    if (!B->exec) {
        if (B->opt.autotune) {
            // plans of the dedicated instances, then the persistent march for a few block sizes,
            // timed on the real inputs (untimed clears)
            cudaEvent_t e0, e1;
            B_CUDA(cudaEventCreate(&e0), "cudaEventCreate");
            B_CUDA(cudaEventCreate(&e1), "cudaEventCreate");
            float best = 3.0e38f;
            int best_block = B->block;
            rt_status rs = RT_OK;
            for (auto& d : B->ded)
                if (rs == RT_OK) rs = B->tune_dedicated(d, B->cap, e0, e1);
            for (int blk : {32, 64, 128, 256}) {
                if (rs != RT_OK || B->waves.empty()) break;
                B->block = blk;
                if ((rs = B->enqueue(B->cap)) != RT_OK) break;   // warm-up
                cudaError_t e = cudaEventRecord(e0, B->cap);
                if (e == cudaSuccess && (rs = B->enqueue(B->cap)) != RT_OK) break;
                if (e == cudaSuccess) e = cudaEventRecord(e1, B->cap);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                float ms = 0.0f;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                if (e != cudaSuccess) { rs = cuda_err(e, "autotune run"); break; }
                if (ms < best) { best = ms; best_block = blk; }
            }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            if (rs != RT_OK) return rs;
            B->block = best_block;
        }
        cudaGraph_t graph = nullptr;
        B_CUDA(cudaStreamBeginCapture(B->cap, cudaStreamCaptureModeThreadLocal), "begin capture");
        rt_status rs = B->enqueue(B->cap);
        cudaError_t e = cudaStreamEndCapture(B->cap, &graph);
        if (rs != RT_OK) { if (graph) cudaGraphDestroy(graph); return rs; }
        if (e != cudaSuccess) return cuda_err(e, "end capture");
        e = cudaGraphInstantiate(&B->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) { B->exec = nullptr; return cuda_err(e, "graph instantiate"); }
    }
    B_CUDA(cudaGraphLaunch(B->exec, st), "graph launch");
    return RT_OK;
}

long long rt_batch_updates(const rt_batch* B) { return B ? B->updates : 0; }

rt_status rt_batch_info(const rt_batch* B, int instance, int* dedicated, int* width, int* block, int* prefetch,
                        int* tile) {
    if (!B) return err(RT_ERR_INVALID_ARG, "rt_batch_info: batch is NULL");
    if (instance < 0 || instance >= (int)B->pos.size())
        return err(RT_ERR_INVALID_ARG, "rt_batch_info: instance %d outside [0, %d)", instance, (int)B->pos.size());
    const int k = B->pos[instance];
    int dd = 0, w = B->host[k].W, bl = B->block, pf = 0, tl = 0;
    for (const auto& d : B->ded)
        if (d.inst == k) { dd = 1; w = d.W; bl = d.block; pf = d.prefetch; tl = d.tile; }
    if (dedicated) *dedicated = dd;
    if (width) *width = w;
    if (block) *block = bl;
    if (prefetch) *prefetch = pf;
    if (tile) *tile = tl;
    return RT_OK;
}

rt_status rt_batch_destroy(rt_batch* B) {
    if (!B) return RT_OK;
    B->release();
    delete B;
    return RT_OK;
}

}  // extern "C"
