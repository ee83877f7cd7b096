#!/usr/bin/env python3
"""Benchmark of the emission-absorption march: ray-substep updates per second.

One step = one rt_advance on the turbulent workload (128^3 lognormal kappa, 16 sources,
N_Omega 3072, ds 0.5, c dt 128 so N_s 256, 4 frequency bins): packing, zeroing, the march
kernel and the unpack, inputs resident in HBM. L2 is flushed (256 MiB write) before every
timed step, outside the step's CUDA-event pair. One update = one substep of one
(ray, source, bin), U = 16 * 3072 * 256 * 4 = 50,331,648 per step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

Under torchrun (N > 1) every rank runs the same workload on its own GPU (replicas, weak
scaling); the time is the max over ranks and the value counts the updates of all ranks.
`--impl reference` times the FP64 CPU oracle instead (rank 0 only) on a bounded sample.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ray-substep updates/s (forward march)"
UNIT = "updates/s"
WORKLOAD = ("turbulent lognormal kappa 128^3 (sigma_g 1, mean 0.05), 16 sources with Gaussian j blobs, "
            "N_Omega 3072, ds 0.5, c*dt 128 (N_s 256), 4 frequency bins, FP32")
FLUSH_BYTES = 256 << 20


def rank_info():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured", p
    except Exception:
        return 6800.0, "fallback", {}


def kernel_source_hash():
    h = hashlib.sha256()
    for name in ("march_fwd.cu", "march_lane.cuh", "march_common.cuh"):
        with open(os.path.join(ROOT, "paper_2511_09389_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_counter(src_hash, key="dram_bytes_per_launch", summary="march_fwd_turbulent128.md"):
    """A counter of the march kernel (DRAM bytes, L2 red sectors) from a committed ncu summary in
    profiles/, or None when the kernel source changed since it was captured."""
    path = os.path.join(ROOT, "profiles", summary)
    try:
        text = open(path).read()
    except OSError:
        return None
    m_hash = re.search(r"source_sha256_16:\s*([0-9a-f]+)", text)
    m_tr = re.search(key + r":\s*([0-9.eE+]+)", text)
    if not m_hash or not m_tr or m_hash.group(1) != src_hash:
        return None
    return float(m_tr.group(1))


def march_roofline(plan, U, kms, src_hash, hbm_peak, hbm_kind):
    """The march kernel against the bound that limits it: L2 reductions (`red`), with L2 gathers
    and HBM beside it. Peaks of the reductions and gathers are measured here by the library's
    microbenchmark with the march's access pattern (the 8 corners of a random cell of a 128^3
    cell-major grid of W-float vectors); the HBM peak is the driver's copy bandwidth. Issued
    reductions and gathers per launch are the L2 sectors ncu counted for this kernel source (the
    committed summary in profiles/, hash-checked), divided by this run's CUDA-event kernel time.
    Algorithmic counts (8 deposits and 9 gathers of a W-vector per (ray, source, bin group)
    substep) are reported beside them: merging deposits in registers issues fewer reductions than
    the algorithm names, so the algorithmic fraction can exceed 1."""
    from paper_2511_09389_gb300 import peaks
    pk = peaks.measure(edge=128, vecs=(4, 1))
    W = int(plan["width"])
    vec = 4 if W == 4 else 1
    t = kms * 1e-3
    lane_steps = U / W
    red_peak = pk[f"red_stencil_v{vec}"]["ops_per_s"]
    gather_peak = pk[f"gather_stencil_v{vec}"]["ops_per_s"]
    reds = profiled_counter(src_hash, "l2_red_sectors_per_launch")
    reads = profiled_counter(src_hash, "l2_read_sectors_per_launch")
    dram = profiled_counter(src_hash)
    fresh = reds is not None
    red_rate = (reds if fresh else 8 * lane_steps) / t
    line = {
        "bound": "l2_red", "achieved": red_rate / 1e9, "peak": red_peak / 1e9, "unit": "Gop/s",
        "frac": red_rate / red_peak, "traffic": dram,
        "peak_kind": f"measured here (rt_microbench: red.global.add.v{vec}.f32 into the 8 corners of random cells "
                     "of a 128^3 cell-major grid)",
        "basis": (f"issued L2 red sectors per launch ({int(reds)}, ncu, profiles/march_fwd_turbulent128.md) / "
                  "march-kernel CUDA-event time" if fresh else
                  "ALGORITHMIC deposits (the committed ncu count is stale for this kernel source) / kernel time"),
        "gather": {"issued_per_s": None if reads is None else reads / t,
                   "frac": None if reads is None else reads / t / gather_peak, "peak_per_s": gather_peak},
        "hbm": {"achieved_gbs": None if dram is None else dram / t / 1e9, "peak_gbs": hbm_peak, "peak_kind": hbm_kind,
                "frac": None if dram is None else dram / t / 1e9 / hbm_peak},
        "algorithmic": {"deposits_per_s": 8 * lane_steps / t, "deposit_frac": 8 * lane_steps / t / red_peak,
                        "gathers_per_s": 9 * lane_steps / t, "gather_frac": 9 * lane_steps / t / gather_peak,
                        "basis": f"8 deposits and 9 gathers of {W}-float vectors per (ray, source, bin group) substep "
                                 f"x {int(lane_steps)} substeps per launch"},
        "peaks": {k: v["ops_per_s"] for k, v in pk.items() if isinstance(v, dict)},
    }
    return line


class ClockSampler:
    """nvidia-smi clocks and throttle reasons every 200 ms while the benchmark runs."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(gpu_index)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_model():
    """CPU model from /proc/cpuinfo ("model name", or the Arm implementer / part codes)."""
    try:
        text = open("/proc/cpuinfo").read()
    except OSError:
        return "unknown"
    m = re.search(r"model name\s*:\s*(.+)", text)
    if m:
        return m.group(1).strip()
    imp = re.search(r"CPU implementer\s*:\s*(\S+)", text)
    part = re.search(r"CPU part\s*:\s*(\S+)", text)
    return f"arm implementer {imp.group(1) if imp else '?'} part {part.group(1) if part else '?'}"


def run_oracle_sample(p, src_slice, ns, threads=1):
    import oracle
    t0 = time.perf_counter()
    F = oracle.advance(p.j, p.kappa, p.sources[src_slice], p.num_rays, p.step_size, ns, geom_mode=0,
                       threads=threads, ray_block=64)
    return F, time.perf_counter() - t0


def reference_arm(args):
    """The FP64 oracle, as it stands, on all host cores (its threaded driver: (source, 64-ray
    block) items, one partial field per thread): each step is the whole benchmark step."""
    rank, world, _ = rank_info()
    if rank != 0:
        return 0
    import oracle
    from paper_2511_09389_gb300 import inputs
    p = inputs.turbulent()
    ns = oracle.num_substeps(p.step_size, p.radiation_velocity, p.time_step)
    per_step = len(p.sources) * p.num_rays * ns * p.n_freq
    cores = host_cores()
    times = []
    for i in range(args.warmup + args.steps):
        _, dt = run_oracle_sample(p, slice(0, len(p.sources)), ns, threads=cores)
        if i >= args.warmup:
            times.append(dt)
    t = statistics.mean(times)
    value = per_step / t
    sample = (f"the whole step per step ({per_step} updates: 16 sources x 3072 rays x 256 substeps x 4 bins), "
              f"FP64, {cores} threads on {cpu_model()}")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def fwd_adjoint(args, dev, flush, stream):
    """Forward + adjoint updates/s on the inverse-problem workload (64^3 lognormal kappa, 8
    sources at Gaussian blob centres, N_Omega 3072, ds 0.5, N_s 128, one bin): each step is one
    rt_advance and one rt_backward (dL/dj and dL/dkappa), L2 flushed before each step."""
    import statistics as st
    import torch
    from paper_2511_09389_gb300 import inputs
    from paper_2511_09389_gb300.api import Grid, num_substeps
    p = inputs.inverse_problem()
    U = len(p.sources) * p.num_rays * num_substeps(p.step_size, p.radiation_velocity, p.time_step) * p.n_freq
    g = Grid(p.shape, 1, profile=True, record_checkpoints=True, autotune=True, ckpt_stride=args.ckpt_stride)
    j, k, s = (torch.from_numpy(a).to(dev) for a in (p.j, p.kappa, p.sources))
    G = torch.randn(p.j.shape, device=dev)
    out = torch.empty_like(j)
    fwd, bwd, kf, kb = [], [], [], []
    for i in range(args.warmup + args.steps):
        flush.fill_(i & 0xff)
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record(stream)
        g.advance(j, k, s, p.num_rays, p.step_size, p.radiation_velocity, p.time_step, out=out)
        e[1].record(stream)
        kfwd = g.kernel_ms()
        g.backward(G, j, k, s, p.num_rays, p.step_size, p.radiation_velocity, p.time_step)
        e[2].record(stream)
        e[2].synchronize()
        if i >= args.warmup:
            fwd.append(e[0].elapsed_time(e[1]))
            bwd.append(e[1].elapsed_time(e[2]))
            kf.append(kfwd)
            kb.append(g.kernel_ms())
    stride = g.last_ckpt_stride()
    plan = g.last_plan()
    # the config-4 inversion: j recovered from zero by Adam (lr 1e-2, 200 iterations, projected
    # onto j >= 0) on the MSE of the log field, through the differentiable march
    from paper_2511_09389_gb300 import inversion
    target = g.advance(j, k, s, p.num_rays, p.step_size, p.radiation_velocity, p.time_step)
    inv = inversion.recover_emissivity(target, k, s, p.num_rays, p.step_size, p.radiation_velocity, p.time_step,
                                       iterations=200, lr=1e-2, grid=g)
    g.close()
    tf, tb = st.mean(fwd), st.mean(bwd)
    return {"value": U / ((tf + tb) * 1e-3), "unit": "updates/s", "updates_per_step": U,
            "workload": "inverse problem: lognormal kappa 64^3, 8 sources, N_Omega 3072, ds 0.5, N_s 128, 1 bin",
            "checkpoints": "recorded by the forward march, reused by the reverse march (record_checkpoints)",
            "ckpt_stride": stride, "forward_plan": plan,
            "ms_fwd": tf, "ms_bwd": tb, "fwd_kernel_ms": st.mean(kf), "adjoint_kernel_ms": st.mean(kb),
            "adjoint_updates_per_s": U / (tb * 1e-3),
            "inversion": {"iterations": inv["iterations"], "lr": 1e-2, "wall_s": inv["wall_s"],
                          "ms_per_iteration": 1e3 * inv["wall_s"] / inv["iterations"],
                          "loss_first": inv["losses"][0], "loss_last": inv["losses"][-1],
                          "correlation_with_target_j": inversion.correlation(inv["j"], j),
                          "loss": "mean (log(F + 1e-2 max F_t) - log(F_t + 1e-2 max F_t))^2",
                          "optimiser": "Adam (rt_adam_step), projected onto j >= 0, j = 0 at the start"}}


def paper_roofline(plan, acc, U, kms, peaks):
    """The paper workload's march kernel against the L2 reductions of its accumulation: issued
    L2 red sectors per update counted by ncu on the first 256 of its sources with the same plan
    (the committed summary, hash-checked), times this run's updates, over its CUDA-event time."""
    summary = "march_fwd_paper_timing.md"
    src_hash = kernel_source_hash()
    per_update = profiled_counter(src_hash, "l2_red_sectors_per_update", summary)
    text = open(os.path.join(ROOT, "profiles", summary)).read() if per_update is not None else ""
    m = re.search(r"profiled_plan:\s*([0-9,]+)\s+(\w+)", text)
    same = (m is not None and plan is not None and acc == m.group(2) and
            m.group(1) == f"{plan['width']},{plan['prefetch']},{plan['lanes_per_ray']},{plan['tile']}")
    peak_key = {"fixed": "red_stencil_u64", "fp64": "red_stencil_f64"}.get(acc, "red_stencil_v1")
    peak = (peaks or {}).get(peak_key)
    if per_update is None or not same or not peak:
        return {"bound": "l2_red", "frac": None,
                "note": "no ncu count for this kernel source, plan and accumulation" if peak else "no peak"}
    rate = per_update * U / (kms * 1e-3)
    return {"bound": "l2_red", "achieved": rate / 1e9, "peak": peak / 1e9, "unit": "Gop/s", "frac": rate / peak,
            "peak_kind": f"measured here ({peak_key}: reductions into the 8 corners of random cells of a 128^3 grid)",
            "basis": f"issued L2 red sectors per update ({per_update:.4f}, ncu on the first 256 sources, "
                     f"profiles/{summary}) x {U} updates / march-kernel CUDA-event time"}


def paper_workload(args, dev, flush, stream, peaks=None):
    """The paper's timing run on a synthetic medium (128^3 lognormal kappa, 2097 sources at the
    0.1 % highest-kappa cells, N_Omega 4096, ds 0.5, one bin; c dt 128 assumed, N_s 256): one
    rt_advance per step, autotuned during the warm-up, L2 flushed before each timed step. The
    paper's 4.49 s on one H200 is quoted beside it as context (another machine, N_s unstated)."""
    import statistics as st
    import torch
    from paper_2511_09389_gb300 import inputs
    from paper_2511_09389_gb300.api import Grid, num_substeps
    p = inputs.paper_timing()
    ns = num_substeps(p.step_size, p.radiation_velocity, p.time_step)
    U = len(p.sources) * p.num_rays * ns * p.n_freq
    g = Grid(p.shape, 1, profile=True, autotune=True)
    j, k, s = (torch.from_numpy(a).to(dev) for a in (p.j, p.kappa, p.sources))
    out = torch.empty_like(j)
    steps, kern = [], []
    for i in range(3 + max(3, min(args.steps, 10))):
        flush.fill_(i & 0xff)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g.advance(j, k, s, p.num_rays, p.step_size, p.radiation_velocity, p.time_step, out=out)
        e1.record(stream)
        e1.synchronize()
        if i >= 3:
            steps.append(e0.elapsed_time(e1))
            kern.append(g.kernel_ms())
    plan = g.last_plan()
    acc = g.last_accumulation()
    g.close()
    t = st.mean(steps)
    res = {"value": U / (t * 1e-3), "unit": "updates/s", "updates_per_step": U, "ms_per_step": t,
           "kernel_ms": st.mean(kern), "launch_plan": plan, "accumulation": acc,
           "roofline": paper_roofline(plan, acc, U, st.mean(kern), peaks),
           "workload": f"128^3 lognormal kappa, {len(p.sources)} sources at the 0.1 % highest-kappa cells, "
                       f"N_Omega {p.num_rays}, ds {p.step_size}, N_s {ns} (c dt 128 assumed), 1 bin",
           "paper": {"seconds": 4.49, "hardware": "1x H200 (JAX)", "speedup_context": 4.49 / (t * 1e-3),
                     "note": "context only: another machine; the paper does not state N_s or bins"}}
    if not args.no_cpu_baseline:
        # parity of the timed field against the FP64 oracle over all sources (all host cores)
        import numpy as np
        import oracle
        F = out.double().cpu().numpy()
        R = oracle.advance(p.j, p.kappa, p.sources, p.num_rays, p.step_size, ns, threads=host_cores(), ray_block=256)
        res["parity_vs_oracle"] = {"rel_l2": float(np.linalg.norm(F - R) / np.linalg.norm(R)),
                                   "max_abs_rel": float(np.abs(F - R).max() / np.abs(R).max()),
                                   "bar": {"rel_l2": 1e-5, "max_abs_rel": 1e-4}}
    return res


def _batch_vs_one_by_one(probs, args, dev, stream):
    """One autotuned batch (dedicated launches for instances that fill the GPU, persistent
    kernels for the rest) replayed from a CUDA graph, against the same instances advanced one
    autotuned rt_advance call at a time with the batch's FP32 sums (mean ms of each)."""
    import statistics as st
    import torch
    from paper_2511_09389_gb300.api import Batch, Grid
    dev_in = []
    for p in probs:
        d = {k: torch.from_numpy(v).to(dev) for k, v in (("j", p.j), ("kappa", p.kappa), ("sources", p.sources))}
        d.update(num_rays=p.num_rays, step_size=p.step_size, radiation_velocity=1.0, time_step=p.time_step)
        dev_in.append(d)
    b = Batch(dev_in, autotune=True)
    U = b.updates
    for _ in range(args.warmup):
        b.run()
    torch.cuda.synchronize()
    tb = []
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.run()
        e1.record(stream)
        e1.synchronize()
        tb.append(e0.elapsed_time(e1))
    # the same arithmetic as the batch, which sums in FP32: single calls would pick fixed-point
    # sums for the dense instances (automatic accumulation) and not be the same computation
    grids = [Grid(p.shape, 8, autotune=True, accumulation="fp32") for p in probs]
    outs = [torch.empty_like(d["j"]) for d in dev_in]

    def one_by_one():
        for g, d, o in zip(grids, dev_in, outs):
            g.advance(d["j"], d["kappa"], d["sources"], d["num_rays"], d["step_size"], 1.0, d["time_step"], out=o)
    for _ in range(args.warmup):
        one_by_one()
    torch.cuda.synchronize()
    t1 = []
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        one_by_one()
        e1.record(stream)
        e1.synchronize()
        t1.append(e0.elapsed_time(e1))
    rel = max(float((o - bo).norm() / bo.norm()) for o, bo in zip(outs, b.outputs))
    mb, m1 = st.mean(tb), st.mean(t1)
    b.close()
    for g in grids:
        g.close()
    return {"value": U / (mb * 1e-3), "unit": "updates/s", "updates_per_step": U, "ms_per_step": mb,
            "one_by_one": {"value": U / (m1 * 1e-3), "ms_per_step": m1}, "speedup_vs_one_by_one": m1 / mb,
            "max_rel_l2_batched_vs_one_by_one": rel}


def batched(args, dev, stream):
    """64 independent instances (edges from {32,48,64,96,128,160}, lognormal kappa with sigma_g in
    [0.5, 1.5], 1-64 sources, N_Omega from {768, 3072, 12288}, ds 0.5, c dt = edge, 1-8 bins):
    one autotuned batch replayed from a CUDA graph, against the same instances
    advanced one rt_advance call at a time. The inputs (2.6 GB) exceed L2, so no flush. Beside
    it, 256 small instances (edges {16, 24, 32}, 1-4 sources, N_Omega {192, 768}, 1-2 bins), where
    one call per instance is bound by launch and host overheads."""
    from paper_2511_09389_gb300 import inputs
    res = _batch_vs_one_by_one(inputs.batch_instances(64), args, dev, stream)
    res.update({"workload": "64 instances: edges {32..160}, 1-64 sources, N_Omega {768,3072,12288}, 1-8 bins, "
                            "c*dt = edge",
                "l2": "inputs (2.6 GB) larger than L2"})
    small = _batch_vs_one_by_one(inputs.batch_instances(256, seed=3100, edges=(16, 24, 32), ray_choices=(192, 768),
                                                        max_src=4, max_freq=2), args, dev, stream)
    small["workload"] = "256 instances: edges {16, 24, 32}, 1-4 sources, N_Omega {192, 768}, 1-2 bins, c*dt = edge"
    res["small_instances"] = small
    return res


def surrogate_leg(args, dev):
    """Learned surrogate vs the plain march on 64^3 one-bin problems (lognormal kappa with
    sigma_g in [0.5, 1.5], 1-8 Gaussian sources, N_Omega 3072, ds 0.5, c dt 64): train on march
    fields with the library's kernels, fit the per-field error estimate on a calibration split
    held out from training, then time fields/s of
    (surrogate + estimate + fallback march, bound rel-L2 <= 1e-2) against the plain march on
    held-out seeds, batch 32."""
    import time as _t
    import numpy as np
    import torch
    from paper_2511_09389_gb300 import surrogate as S
    from paper_2511_09389_gb300.api import Grid
    grid = Grid((64, 64, 64), 1)
    t0 = _t.perf_counter()
    train = S.Dataset(range(args.surrogate_train), grid)
    calib = S.Dataset(range(20_000_000, 20_000_000 + args.surrogate_calib), grid)
    held = S.Dataset(range(10_000_000, 10_000_000 + args.surrogate_heldout), grid)
    t_data = _t.perf_counter() - t0
    model = S.Surrogate(seed=0)
    t0 = _t.perf_counter()
    losses = S.train(model, train, epochs=args.surrogate_epochs, batch=32, lr=2e-3)
    torch.cuda.synchronize()
    t_train = _t.perf_counter() - t0
    errs, est = S.fit_estimator(model, calib, batch=32)   # calibrated on fields held out from training
    res = S.evaluate(model, grid, held, batch=32)
    grid.close()
    # one hidden layer of the network on its own, against the measured bf16 tensor peak
    conv = S.time_conv_layer(batch=32, edge=64, dilation=2)
    _, _, peaks = load_peaks()
    peak_tf = float(peaks.get("bf16_tflops", 1900.0))
    conv["roofline"] = {"bound": "tensor", "achieved": conv["forward_tflops"], "peak": peak_tf, "unit": "TFLOP/s",
                        "frac": conv["forward_tflops"] / peak_tf,
                        "data_grad_frac": conv["data_grad_tflops"] / peak_tf,
                        "weight_grad_frac": conv["weight_grad_tflops"] / peak_tf,
                        "peak_kind": "measured" if "bf16_tflops" in peaks else "fallback"}
    res["conv_layer"] = conv
    res.update({"train_fields": len(train), "calibration_fields": len(calib), "epochs": args.surrogate_epochs,
                "loss_per_epoch": losses, "calibration_rel_l2_median": float(np.median(errs)),
                "estimate_threshold_log10": model.est_threshold,
                "data_generation_s": t_data, "training_s": t_train,
                "workload": "64^3, 1-8 sources, N_Omega 3072, ds 0.5, c*dt 64, 1 bin; batch 32"})
    return res


def sharded_tail(args, p, g, j, k, s, out, hj, hk, hs, hout, stream, step_ms, kern_ms, wall, clocks, U, world,
                 rank, dev, sources):
    """The rest of the N > 1 run: e2e through host buffers (copy j, kappa and the sources in,
    march this rank's shard, all-reduce, copy the field out, per step), the max over ranks, and
    rank 0's JSON line. The single-GPU legs are not run."""
    import torch
    import torch.distributed as dist
    from paper_2511_09389_gb300 import sharding

    def e2e_step():
        j.copy_(hj, non_blocking=True)
        k.copy_(hk, non_blocking=True)
        s.copy_(hs, non_blocking=True)
        sharding.advance_distributed(g, j, k, s, p.num_rays, p.step_size, p.radiation_velocity, p.time_step, out)
        hout.copy_(out, non_blocking=True)

    for _ in range(max(1, args.warmup)):
        e2e_step()
    torch.cuda.synchronize()
    e2e_ms = []
    for i in range(args.steps):
        dist.barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        e2e_step()
        e1.record(stream)
        e1.synchronize()
        e2e_ms.append(e0.elapsed_time(e1))
    clk = clocks.stop()
    t = torch.tensor([statistics.mean(step_ms), statistics.mean(kern_ms), statistics.mean(e2e_ms)],
                     dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms, kms, ems = t.tolist()
    h2d = p.j.nbytes + p.kappa.nbytes + sources.nbytes
    line = {
        "metric": METRIC, "value": world * U / (ms * 1e-3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD + f"; {16 * world} sources in all, 16 per rank",
                   "updates_per_step": world * U, "l2": "flushed before every timed step (256 MiB write)",
                   "parallelism": f"(source, ray) shards x{world} (rt_shard_plan), one NCCL all-reduce of the "
                                  f"{p.j.nbytes >> 20} MiB field per step",
                   "kernel_ms": kms, "wall_s": wall, "launch_plan": g.last_plan(),
                   "accumulation": g.last_accumulation(),
                   "timing": "max over ranks of the mean over the K timed steps"},
        "e2e": {"value": world * U / (ems * 1e-3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": p.j.nbytes, "ms_per_step": ems,
                "api": "per step: pinned inputs copied in, sharding.advance_distributed, field copied out"},
        # per step, each of this rank's planned pieces is one pack, one march and one unpack
        "gpu_launches": 3 * len(sharding.plan(len(sources), p.num_rays, world, rank)) * args.steps,
        "clocks": {"sm_mhz": clk["sm_mhz"], "sm_max_mhz": clk["sm_max_mhz"], "reasons": clk["reasons"],
                   "samples": clk["samples"]},
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    g.close()
    dist.destroy_process_group()
    return 0


def native_arm(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    rank, world, local = rank_info()
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2511_09389_gb300 import build, inputs
    if rank == 0 or world == 1:
        build.build()
    if world > 1:
        dist.barrier()
    from paper_2511_09389_gb300.api import Grid

    from paper_2511_09389_gb300 import sharding
    from paper_2511_09389_gb300.api import num_substeps
    p = inputs.turbulent()
    sources = p.sources
    if world > 1:
        # weak scaling over the sharded data path: the job is one advance with 16 sources per
        # rank (rank 0's are the single-GPU workload's, the others drawn uniformly in the box
        # from seeded generators); each rank marches its planned shard of the (source, ray)
        # pairs and one all-reduce sums the partial fields
        extra = [np.random.Generator(np.random.PCG64(2100 + r)).uniform(0.0, p.shape[0] - 1.0, size=(16, 3))
                 for r in range(1, world)]
        sources = np.concatenate([p.sources] + [e.astype(np.float32) for e in extra])
    ns_ = num_substeps(p.step_size, p.radiation_velocity, p.time_step)
    U = len(p.sources) * p.num_rays * ns_ * p.n_freq          # updates per rank and step
    if args.plan:
        g = Grid(p.shape, 8, profile=True, plan=tuple(int(x) for x in args.plan.split(",")))
    else:
        g = Grid(p.shape, 8, profile=True, autotune=True)   # tuned during the warm-up calls
    j = torch.from_numpy(p.j).to(dev)
    k = torch.from_numpy(p.kappa).to(dev)
    s = torch.from_numpy(sources).to(dev)
    out = torch.empty_like(j)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        if world > 1:
            sharding.advance_distributed(g, j, k, s, p.num_rays, p.step_size, p.radiation_velocity, p.time_step, out)
        else:
            g.advance(j, k, s, p.num_rays, p.step_size, p.radiation_velocity, p.time_step, out=out)

    visible = [v for v in os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",") if v.strip()]
    clocks = ClockSampler(visible[local].strip() if local < len(visible) else local)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    step_ms, kern_ms = [], []
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.fill_(i & 0xff)                 # evict L2 before the step (not timed)
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
        ev[i][1].synchronize()
        step_ms.append(ev[i][0].elapsed_time(ev[i][1]))
        kern_ms.append(g.kernel_ms())
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    wall = time.perf_counter() - wall0

    # end to end through the host entry point: pinned inputs in, field back to the host
    pin = lambda a: torch.from_numpy(a).pin_memory()
    hj, hk, hs = pin(p.j), pin(p.kappa), pin(sources)
    hout = torch.empty(p.j.shape, dtype=torch.float32).pin_memory()
    if world > 1:
        return sharded_tail(args, p, g, j, k, s, out, hj, hk, hs, hout, stream, step_ms, kern_ms, wall, clocks,
                            U, world, rank, dev, sources)
    for _ in range(max(1, args.warmup)):
        g.advance_host(hj, hk, hs, p.num_rays, p.step_size, p.radiation_velocity, p.time_step, out=hout)
    e2e_ms = []
    for i in range(args.steps):
        flush.fill_(i & 0xff)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g.advance_host(hj, hk, hs, p.num_rays, p.step_size, p.radiation_velocity, p.time_step, out=hout)
        e1.record(stream)
        e1.synchronize()
        e2e_ms.append(e0.elapsed_time(e1))
    # the same calls pipelined (rt_advance_host_async): step i+1's inputs move in and step i-1's
    # field moves out while step i marches; two alternating host output buffers, K steps
    # between one pair of events (pipeline fill and drain included)
    houts = [hout, torch.empty(p.j.shape, dtype=torch.float32).pin_memory()]
    for i in range(max(1, args.warmup)):
        g.advance_host_async(hj, hk, hs, p.num_rays, p.step_size, p.radiation_velocity, p.time_step,
                             out=houts[i & 1], stream=stream)
    g.host_wait()
    flush.fill_(0)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(args.steps):
        g.advance_host_async(hj, hk, hs, p.num_rays, p.step_size, p.radiation_velocity, p.time_step,
                             out=houts[i & 1], stream=stream)
    g.host_join(stream)
    e1.record(stream)
    e1.synchronize()
    g.host_wait()
    pipe_ms = e0.elapsed_time(e1) / args.steps
    clk = clocks.stop()

    ms = statistics.mean(step_ms)
    kms = statistics.mean(kern_ms)
    ems = statistics.mean(e2e_ms)
    if world > 1:
        t = torch.tensor([ms, kms, ems, pipe_ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms, kms, ems, pipe_ms = t.tolist()

    peak, peak_kind, _ = load_peaks()
    src_hash = kernel_source_hash()
    h2d = p.j.nbytes + p.kappa.nbytes + p.sources.nbytes
    d2h = p.j.nbytes

    line = {
        "metric": METRIC, "value": world * U / (ms * 1e-3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "updates_per_step": U, "l2": "flushed before every timed step (256 MiB write)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "kernel_ms": kms, "wall_s": wall, "launch_plan": g.last_plan(),
                   "accumulation": g.last_accumulation(),
                   "median_ms_per_step": statistics.median(step_ms), "median_kernel_ms": statistics.median(kern_ms),
                   "timing": "value and ms_per_step use the mean over the K timed steps; medians beside them"},
        "roofline": march_roofline(g.last_plan(), U, kms, src_hash, peak, peak_kind),
        "e2e": {"value": world * U / (pipe_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": pipe_ms,
                "api": "rt_advance_host_async x K steps, one event pair around all K (fill and drain included)",
                "l2": "not flushed inside the pipeline; each step copies its 67 MB of inputs in and 34 MB out, "
                      "alternating two device buffer sets (per-step footprint with packing ~200 MB > L2)"},
        "e2e_serial": {"value": world * U / (ems * 1e-3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                       "d2h_bytes_per_step": d2h, "ms_per_step": ems,
                       "api": "rt_advance_host (copy in, march, copy out, synchronise) per step, L2 flushed before each"},
        "gpu_launches": 3 * args.steps,
        "clocks": {"sm_mhz": clk["sm_mhz"], "sm_max_mhz": clk["sm_max_mhz"], "reasons": clk["reasons"],
                   "samples": clk["samples"]},
    }

    # the same step with the deterministic (64-bit fixed-point) accumulation
    gd = Grid(p.shape, 8, deterministic=True)
    tdet = []
    for i in range(args.warmup + args.steps):
        flush.fill_(i & 0xff)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        gd.advance(j, k, s, p.num_rays, p.step_size, p.radiation_velocity, p.time_step, out=out)
        e1.record(stream)
        e1.synchronize()
        if i >= args.warmup:
            tdet.append(e0.elapsed_time(e1))
    gd.close()
    line["deterministic"] = {"value": U / (statistics.mean(tdet) * 1e-3), "unit": UNIT,
                             "ms_per_step": statistics.mean(tdet), "note": "64-bit fixed-point deposits, bitwise reproducible"}
    line["fwd_adjoint"] = fwd_adjoint(args, dev, flush, stream)
    if not args.no_paper:
        line["paper_workload"] = paper_workload(args, dev, flush, stream, line["roofline"].get("peaks"))
    if not args.no_batch:
        line["batched"] = batched(args, dev, stream)
    if args.surrogate_train > 0:
        line["surrogate"] = surrogate_leg(args, dev)

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        ns = oracle.num_substeps(p.step_size, p.radiation_velocity, p.time_step)
        cores = host_cores()
        R, dt = run_oracle_sample(p, slice(0, len(p.sources)), ns, threads=cores)
        line["cpu_baseline"] = {"value": U / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"the whole step ({U} updates), FP64, {cores} threads, {dt:.2f} s",
                                "cpu": cpu_model()}
        _, dt1 = run_oracle_sample(p, slice(0, 1), ns)
        line["cpu_baseline_1core"] = {"value": U / len(p.sources) / dt1, "unit": UNIT, "cores": 1, "kind": "oracle",
                                      "sample": f"1 of 16 sources ({U // len(p.sources)} updates), FP64, 1 thread, "
                                                f"{dt1:.2f} s"}
        F = out.double().cpu().numpy()
        rel = [float(np.linalg.norm(F[b] - R[b]) / np.linalg.norm(R[b])) for b in range(p.n_freq)]
        line["parity_vs_oracle"] = {"rel_l2_per_bin": rel}

    if rank == 0:
        print(json.dumps(line), flush=True)
    g.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--no-cpu-baseline", action="store_true", help="skip the oracle timing (faster)")
    ap.add_argument("--no-batch", action="store_true", help="skip the 64-instance batched measurement")
    ap.add_argument("--no-paper", action="store_true", help="skip the paper's 2097-source timing workload")
    ap.add_argument("--surrogate-train", type=int, default=4096, help="surrogate training fields (0: skip)")
    ap.add_argument("--surrogate-heldout", type=int, default=512)
    ap.add_argument("--surrogate-calib", type=int, default=256, help="fields held out to calibrate the estimate")
    ap.add_argument("--surrogate-epochs", type=int, default=8)
    ap.add_argument("--plan", default="", help="pin the launch plan 'bins_per_group,block,prefetch[,lanes_per_ray]' "
                                               "instead of autotuning (for reproducible profiles)")
    ap.add_argument("--ckpt-stride", type=int, default=0,
                    help="pin the adjoint checkpoint stride K (4, 8, 16 or 32) instead of tuning it (0)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return reference_arm(args)
    return native_arm(args)


if __name__ == "__main__":
    sys.exit(main())
