"""The L2 microbenchmarks that give the march's roofline its peaks (`rt_microbench`).

Every reduction adds a known constant (1 per vector element, 1/8 per stencil corner) into a
zeroed buffer, so the buffer's sum after one launch equals operations x vector width x constant
exactly (all partial sums are small multiples of 1/8, exact in FP32): every operation happened
and landed inside the buffer. The gather kinds leave the buffer unchanged.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_2511_09389_gb300 import build, _native
    build.build()
    assert torch.cuda.is_available()
    return torch, _native.load()


def run(lib, kind, vec, buf, edge, iters):
    ms, ops = ctypes.c_float(), ctypes.c_double()
    st = lib.rt_microbench(kind, vec, buf.data_ptr(), buf.numel() * 4, edge, iters, ctypes.byref(ms), ctypes.byref(ops))
    return st, ms.value, ops.value


@pytest.mark.parametrize("kind,const", [(0, 1.0), (1, 1.0), (2, 0.125)])
@pytest.mark.parametrize("vec", [1, 4])
def test_reductions_all_land_in_bounds(env, kind, const, vec):
    torch, lib = env
    edge = 40
    buf = torch.zeros(edge ** 3 * vec + 7, dtype=torch.float32, device="cuda")
    iters = 3
    st, ms, ops = run(lib, kind, vec, buf, edge, iters)
    assert st == 0, lib.rt_last_error()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert ops == 8 * sms * 256 * iters * (8 if kind == 2 else 1)
    assert ms > 0
    total = buf.double().sum().item()
    assert total == ops * vec * const
    if kind == 2:
        # stencil corners stay inside the edge^3 grid
        assert torch.count_nonzero(buf[edge ** 3 * vec:]).item() == 0


@pytest.mark.parametrize("kind", [3, 4])
def test_gathers_leave_the_buffer_unchanged(env, kind):
    torch, lib = env
    edge = 32
    buf = torch.arange(edge ** 3 * 4, dtype=torch.float32, device="cuda").remainder_(97.0)
    ref = buf.clone()
    st, ms, ops = run(lib, kind, 4, buf, edge, 4)
    assert st == 0, lib.rt_last_error()
    assert ops > 0 and ms > 0
    assert torch.equal(buf, ref)


def test_invalid_arguments(env):
    torch, lib = env
    buf = torch.zeros(1024, dtype=torch.float32, device="cuda")
    from paper_2511_09389_gb300._native import STATUS_NAMES
    for kind, vec, edge, iters in [(5, 4, 4, 1), (0, 2, 4, 1), (0, 4, 4, 0), (2, 4, 64, 1), (4, 1, 1, 1)]:
        st, _, _ = run(lib, kind, vec, buf, edge, iters)
        assert STATUS_NAMES[st] == "RT_ERR_INVALID_ARG", (kind, vec, edge, iters)
    small = torch.zeros(16, dtype=torch.float32, device="cuda")    # fewer than 32 vectors
    st, _, _ = run(lib, 0, 1, small, 2, 1)
    assert STATUS_NAMES[st] == "RT_ERR_INVALID_ARG"


def test_measure_reports_positive_rates(env):
    from paper_2511_09389_gb300 import peaks
    res = peaks.measure(edge=64, vecs=(4,), reps=1)
    for name in peaks.KINDS:
        r = res[f"{name}_v4"]
        assert np.isfinite(r["ops_per_s"]) and r["ops_per_s"] > 0
        assert r["bytes_per_s"] == pytest.approx(16 * r["ops_per_s"])
