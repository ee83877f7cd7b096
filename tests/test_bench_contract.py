"""The benchmark's command-line contract on the CPU: the reference arm (the FP64 oracle on the
host cores) prints one JSON line with the keys the native arm's line also carries, and the
warm-up floor is enforced. The native arm needs the GPU and is exercised there."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_bench(*args, timeout=600):
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT, capture_output=True,
                          text=True, timeout=timeout)


def test_reference_arm_prints_one_json_line():
    r = run_bench("--impl", "reference", "--steps", "1", "--warmup", "3")
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference"
    assert d["unit"] == "updates/s" and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["warmup"] == 3 and d["n_gpus"] == 1
    # one step is the whole 128^3 step: 16 sources x 3072 rays x 256 substeps x 4 bins
    assert d["value"] == pytest.approx(50_331_648 / (d["ms_per_step"] * 1e-3), rel=1e-9)
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert "workload" in d["config"]


def test_warmup_floor_is_enforced():
    r = run_bench("--impl", "reference", "--steps", "1", "--warmup", "2", timeout=120)
    assert r.returncode != 0
    assert "--warmup must be >= 3" in r.stderr


def _bench_module():
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_profile_counters_are_current_and_read_back():
    """The ncu counts the benchmark divides by its own kernel time come from summaries captured
    on the current march sources: the hash check passes, and the paper leg's L2 fraction is the
    summary's reductions per update x updates / time over the peak, null for another plan."""
    b = _bench_module()
    h = b.kernel_source_hash()
    assert b.profiled_counter(h, "l2_red_sectors_per_launch") > 0
    assert b.profiled_counter(h, "l2_read_sectors_per_launch") > 0
    per_update = b.profiled_counter(h, "l2_red_sectors_per_update", "march_fwd_paper_timing.md")
    assert per_update is not None and 1.0 < per_update < 8.0
    assert b.profiled_counter("0" * 16, "l2_red_sectors_per_launch") is None
    plan = {"width": 1, "block": 32, "prefetch": 4, "lanes_per_ray": 2, "tile": 0}
    U, kms, peak = 2_198_863_872, 31.3, 195e9
    r = b.paper_roofline(plan, "fixed", U, kms, {"red_stencil_u64": peak})
    assert r["frac"] == pytest.approx(per_update * U / (kms * 1e-3) / peak, rel=1e-12)
    assert b.paper_roofline(dict(plan, lanes_per_ray=1), "fixed", U, kms, {"red_stencil_u64": peak})["frac"] is None
    assert b.paper_roofline(plan, "fp32", U, kms, {"red_stencil_v1": peak})["frac"] is None
