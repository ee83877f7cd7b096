"""The C-ABI library loads and exports every symbol include/raytrax.h declares; host-only
logic (substep rule, direction lattice) agrees with the oracle. No GPU compute is called."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2511_09389_gb300 import build, _native
    build.build()
    return _native.load()


def _declared(header):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rt_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            names += _declared(h)
    assert names, "no declarations found"
    for name in names:
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"
    from paper_2511_09389_gb300 import _native
    assert set(_native.EXPORTS) <= set(names)


def test_num_substeps_matches_oracle(lib):
    cases = [(0.5, 1.0, 16.0, 0), (0.5, 1.0, 128.0, 0), (0.25, 2.0, 3.3, 0), (0.5, 1.0, 64.0, 100),
             (0.5, 1.0, 0.0, 0), (1.0, 1.0, 160.0, 0), (0.3, 1.0, 0.9, 0), (0.7, 1.3, 11.1, 7)]
    for ds, c, dt, cap in cases:
        # the library takes float arguments: give the oracle the same FP32 values
        f = [float(np.float32(v)) for v in (ds, c, dt)]
        assert lib.rt_num_substeps(*f, cap) == oracle.num_substeps(*f, cap), (ds, c, dt, cap)
    assert lib.rt_num_substeps(0.0, 1.0, 1.0, 0) == -1
    assert lib.rt_num_substeps(0.5, -1.0, 1.0, 0) == -1
    assert lib.rt_num_substeps(0.5, 1.0, -1.0, 0) == -1
    assert lib.rt_num_substeps(1e-30, 1e30, 1e30, 0) == -1


@pytest.mark.parametrize("n", [1, 2, 3, 37, 192, 768, 3072, 12288])
def test_direction_table_bit_equal_to_oracle(lib, n):
    from paper_2511_09389_gb300.api import direction_table
    assert np.array_equal(direction_table(n), oracle.fibonacci_dirs_f32(n))


def test_invalid_arguments_rejected_on_host(lib):
    h = ctypes.c_void_p()
    assert lib.rt_create_grid(ctypes.byref(h), 0, 4, 4, 1, None) == 1
    assert b"extents" in lib.rt_last_error()
    assert lib.rt_create_grid(ctypes.byref(h), 4, 4, 4, 0, None) == 1
    assert lib.rt_create_grid(ctypes.byref(h), 2048, 2048, 1024, 1, None) == 1
    assert lib.rt_destroy(None) == 0
    assert lib.rt_direction_table(0, None) == 1


@pytest.mark.parametrize("field,value,word", [("plan_lanes", 4, b"plan_lanes"), ("plan_lanes", 3, b"plan_lanes"),
                                              ("plan_prefetch", 6, b"plan_prefetch"), ("plan_width", 3, b"plan_width"),
                                              ("plan_block", 48, b"plan_block"), ("plan_tile", 3, b"plan_tile"),
                                              ("kappa_mode", 2, b"kappa_mode"), ("ckpt_stride", -1, b"ckpt_stride")])
def test_bad_options_rejected_at_creation(lib, field, value, word):
    """Launch-plan and other options are checked by rt_create_grid on the host, before any device
    call: an out-of-range value returns RT_ERR_INVALID_ARG naming the field."""
    from paper_2511_09389_gb300 import _native
    opt = _native.rt_options()
    lib.rt_default_options(ctypes.byref(opt))
    setattr(opt, field, value)
    h = ctypes.c_void_p()
    assert lib.rt_create_grid(ctypes.byref(h), 8, 8, 8, 1, ctypes.byref(opt)) == 1
    assert word in lib.rt_last_error()
    assert not h.value


@pytest.mark.parametrize("dims,max_freq", [((1291, 1291, 1291), 1), ((1024, 1024, 512), 1), ((1024, 1024, 512), 4),
                                           ((1024, 512, 512), 5), ((2, 1 << 30, 1), 1), ((0, 8, 8), 1),
                                           ((8, -1, 8), 1), ((8, 8, 8), 0)])
def test_grid_limits_rejected_at_creation(lib, dims, max_freq):
    """The kernels index cells and packed bin groups with 32-bit integers: a grid whose
    n0 n1 n2 times the bins rounded up to a group of four reaches 2^31 is refused on the host,
    before any device call, as are empty extents and max_freq < 1."""
    h = ctypes.c_void_p()
    assert lib.rt_create_grid(ctypes.byref(h), *dims, max_freq, None) == 1
    msg = lib.rt_last_error()
    assert (b"too large" in msg) or (b">= 1" in msg)
    assert not h.value


@pytest.mark.parametrize("field,value", [("plan_lanes", 2), ("plan_tile", 2), ("plan_prefetch", 2),
                                         ("plan_prefetch", 4), ("plan_prefetch", 3)])
def test_deterministic_rejects_plans_it_cannot_run(lib, field, value):
    """The fixed-point march runs one lane per ray with corner slots and no tiles: a pinned plan
    asking for two lanes, tiles or another gathers mode is refused at creation, naming the mode,
    instead of being accepted and then ignored."""
    from paper_2511_09389_gb300 import _native
    opt = _native.rt_options()
    lib.rt_default_options(ctypes.byref(opt))
    opt.deterministic = 1
    setattr(opt, field, value)
    h = ctypes.c_void_p()
    assert lib.rt_create_grid(ctypes.byref(h), 8, 8, 8, 1, ctypes.byref(opt)) == 1
    assert b"deterministic" in lib.rt_last_error()
    assert not h.value



def test_invert_emissivity_rejects_a_null_grid(lib):
    """rt_invert_emissivity checks the handle on the host before any device call (the other
    argument checks need a device grid: tests/test_gpu_adjoint.py)."""
    assert lib.rt_invert_emissivity(None, None, None, None, 1, 8, 0.5, 1.0, 1.0, 1, 1, 1e-2, 1e-2, None, None,
                                    None) == 1
    assert b"grid" in lib.rt_last_error()
