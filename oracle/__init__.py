"""FP64 CPU oracle for the Ray-trax march (paper Sec. 2, Eq. 2) -- TEST INFRASTRUCTURE.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline / reference legs of
``bench.py`` may import this package. The product path (the CUDA library and its Python
binding) never imports, links or executes anything here, and this package never imports
the product package.

The arithmetic lives in ``rt_oracle.c`` (plain loops, FP64, ``-ffp-contract=off``); this
module compiles it with the host C compiler and marshals numpy arrays through ctypes.
Every function states the passage of the paper it follows; the readings taken where the
paper is silent are listed at the top of ``rt_oracle.c`` (R1-R6).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rt_oracle.c")
_CONV_SRC = os.path.join(_HERE, "conv_oracle.c")
_THREADS_SRC = os.path.join(_HERE, "rt_oracle_threads.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_fp = ctypes.POINTER(ctypes.c_float)
_lp = ctypes.POINTER(ctypes.c_long)


def build(force: bool = False) -> str:
    """Compile the oracle C sources into ``oracle/liboracle.so`` (no fast-math, no FMA)."""
    srcs = [_SRC, _THREADS_SRC] + ([_CONV_SRC] if os.path.exists(_CONV_SRC) else [])
    newest = max(os.path.getmtime(s) for s in srcs)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["cc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-pthread",
           "-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        i, d = ctypes.c_int, ctypes.c_double
        lib.oracle_num_substeps.argtypes = [d, d, d, i]
        lib.oracle_num_substeps.restype = i
        lib.oracle_fibonacci_dirs.argtypes = [i, _dp]
        lib.oracle_fibonacci_dirs.restype = None
        lib.oracle_fibonacci_dirs_f32.argtypes = [i, _fp]
        lib.oracle_fibonacci_dirs_f32.restype = None
        common = [_dp, _dp, i, i, i, i, _dp, i, i, d, i, i, i, i, i]
        lib.oracle_advance.argtypes = common + [_dp]
        lib.oracle_advance.restype = i
        lib.oracle_advance_threads.argtypes = common + [i, i, _dp]
        lib.oracle_advance_threads.restype = i
        lib.oracle_source_gradient.argtypes = [_dp, _dp, i, i, i, i, _dp, i, i, d, i, i, i, _dp, _dp]
        lib.oracle_source_gradient.restype = i
        lib.oracle_advance_state.argtypes = [_dp, _dp, i, i, i, i, _dp, i, i, d, i, i, i, i, _dp, _dp, _dp, _dp]
        lib.oracle_advance_state.restype = i
        lib.oracle_backward.argtypes = common + [_dp, _dp, _dp]
        lib.oracle_backward.restype = i
        lib.oracle_trace_ray.argtypes = [_dp, _dp, i, i, i, _dp, i, i, d, i, i, i, _lp, _lp, _dp]
        lib.oracle_trace_ray.restype = i
        if hasattr(lib, "oracle_conv3d_fwd"):
            conv = [_dp, _dp, _dp, i, i, i, i, i, i, i]
            lib.oracle_conv3d_fwd.argtypes = conv + [_dp]
            lib.oracle_conv3d_fwd.restype = i
            lib.oracle_conv3d_bwd.argtypes = conv + [_dp, _dp, _dp, _dp]
            lib.oracle_conv3d_bwd.restype = i
        _lib = lib
        return lib


def _ptr(a: np.ndarray, ty=_dp):
    return a.ctypes.data_as(ty)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def num_substeps(step_size: float, radiation_velocity: float, time_step: float, cap: int = 0) -> int:
    """N_s = ceil(c dt / ds), or the cap (Sec. 2 after Eq. 2; App. A). Reading R4."""
    n = _load().oracle_num_substeps(float(step_size), float(radiation_velocity), float(time_step), int(cap))
    if n < 0:
        raise ValueError("invalid step_size / radiation_velocity / time_step")
    return n


def fibonacci_dirs(num_rays: int) -> np.ndarray:
    """Golden-angle lattice on S^2 (Sec. 2), FP64, shape [num_rays, 3]. Reading R1."""
    out = np.empty((num_rays, 3), np.float64)
    _load().oracle_fibonacci_dirs(int(num_rays), _ptr(out))
    return out


def fibonacci_dirs_f32(num_rays: int) -> np.ndarray:
    """The FP64 lattice rounded once to FP32, shape [num_rays, 3]."""
    out = np.empty((num_rays, 3), np.float32)
    _load().oracle_fibonacci_dirs_f32(int(num_rays), _ptr(out, _fp))
    return out


def _grid_args(j, kappa):
    j = _f64(j)
    kappa = _f64(kappa)
    if j.ndim == 3:
        j = j[None]
    if kappa.ndim == 3:
        kappa = kappa[None]
    if j.shape != kappa.shape or j.ndim != 4:
        raise ValueError("j and kappa must both be [n_freq, n0, n1, n2] (or [n0, n1, n2])")
    return np.ascontiguousarray(j), np.ascontiguousarray(kappa)


def advance(j, kappa, source_pos, num_rays: int, step_size: float, num_steps: int,
            geom_mode: int = 0, kappa_mode: int = 0, ray_range=None, threads: int = 1,
            ray_block: int = 256) -> np.ndarray:
    """Field after one dt: (4 pi / N_Omega) sum_src sum_rays sum_k W(x_k) I_{k+1} (Sec. 2, Eq. 2).

    j, kappa: [n_freq, n0, n1, n2] (or 3-D for one bin); source_pos: [n_src, 3] in grid
    coordinates; num_steps = N_s. geom_mode 0 reproduces FP32 geometry (reading R6), 1 is
    pure FP64. ray_range=(begin, end) traces a shard of the lattice. threads > 1 splits the
    (source, block of ray_block rays) items over host threads, each summing into its own
    partial field (added in thread order). Returns FP64 [n_freq, n0, n1, n2].
    """
    j, kappa = _grid_args(j, kappa)
    nf, n0, n1, n2 = j.shape
    src = _f64(source_pos).reshape(-1, 3)
    rb, re = (0, num_rays) if ray_range is None else ray_range
    out = np.zeros_like(j)
    args = (_ptr(j), _ptr(kappa), nf, n0, n1, n2, _ptr(src), src.shape[0], int(num_rays), float(step_size),
            int(num_steps), int(geom_mode), int(kappa_mode), int(rb), int(re))
    if threads > 1:
        rc = _load().oracle_advance_threads(*args, int(threads), int(ray_block), _ptr(out))
    else:
        rc = _load().oracle_advance(*args, _ptr(out))
    if rc != 0:
        raise ValueError("oracle_advance: invalid arguments")
    return out


class MarchState:
    """Per-ray state carried between stateful advances: positions [n_src, num_rays, 3] and
    I, tau [n_freq, n_src, num_rays] (FP64)."""

    def __init__(self, n_freq: int, n_src: int, num_rays: int):
        self.pos = np.zeros((n_src, num_rays, 3))
        self.I = np.zeros((n_freq, n_src, num_rays))
        self.tau = np.zeros((n_freq, n_src, num_rays))


def advance_state(j, kappa, source_pos, num_rays: int, step_size: float, num_steps: int, state: MarchState,
                  restart: bool, geom_mode: int = 0, kappa_mode: int = 0) -> np.ndarray:
    """One advance of the march continued across calls (Sec. 3: time integration with a fixed dt): rays start
    from `state` (or, with restart, at their sources with I = tau = 0), march num_steps
    substeps of Eq. 2 through this call's j and kappa, deposit them, and leave their new state
    in `state`. Returns the call's field, FP64 [n_freq, n0, n1, n2]."""
    j, kappa = _grid_args(j, kappa)
    nf, n0, n1, n2 = j.shape
    src = _f64(source_pos).reshape(-1, 3)
    if state.pos.shape != (src.shape[0], num_rays, 3) or state.I.shape != (nf, src.shape[0], num_rays):
        raise ValueError("advance_state: state shape does not match the call")
    out = np.zeros_like(j)
    rc = _load().oracle_advance_state(_ptr(j), _ptr(kappa), nf, n0, n1, n2, _ptr(src), src.shape[0],
                                      int(num_rays), float(step_size), int(num_steps), int(geom_mode),
                                      int(kappa_mode), int(bool(restart)), _ptr(state.pos), _ptr(state.I),
                                      _ptr(state.tau), _ptr(out))
    if rc != 0:
        raise ValueError("oracle_advance_state: invalid arguments")
    return out


def backward(j, kappa, source_pos, num_rays: int, step_size: float, num_steps: int, grad_out,
             geom_mode: int = 0, kappa_mode: int = 0, ray_range=None):
    """Reverse-mode adjoint of :func:`advance`: returns (dL/dj, dL/dkappa) for G = dL/d(out)."""
    j, kappa = _grid_args(j, kappa)
    nf, n0, n1, n2 = j.shape
    G = _f64(grad_out).reshape(j.shape)
    src = _f64(source_pos).reshape(-1, 3)
    rb, re = (0, num_rays) if ray_range is None else ray_range
    dj = np.zeros_like(j)
    dk = np.zeros_like(j)
    rc = _load().oracle_backward(_ptr(j), _ptr(kappa), nf, n0, n1, n2, _ptr(src), src.shape[0],
                                 int(num_rays), float(step_size), int(num_steps), int(geom_mode),
                                 int(kappa_mode), int(rb), int(re), _ptr(G), _ptr(dj), _ptr(dk))
    if rc != 0:
        raise ValueError("oracle_backward: invalid arguments")
    return dj, dk


def source_gradient(j, kappa, source_pos, num_rays: int, step_size: float, num_steps: int, grad_out,
                    geom_mode: int = 0, kappa_mode: int = 0) -> np.ndarray:
    """dL/d(source positions) [n_src, 3] for G = dL/d(out): each ray's positions are the source
    plus multiples of n ds, so the gradient sums dL/dx_k over the source's rays and substeps
    (trilinear deposit and gather weights; the kappa cell is piecewise constant)."""
    j, kappa = _grid_args(j, kappa)
    nf, n0, n1, n2 = j.shape
    G = _f64(grad_out).reshape(j.shape)
    src = _f64(source_pos).reshape(-1, 3)
    out = np.zeros_like(src)
    rc = _load().oracle_source_gradient(_ptr(j), _ptr(kappa), nf, n0, n1, n2, _ptr(src), src.shape[0],
                                        int(num_rays), float(step_size), int(num_steps), int(geom_mode),
                                        int(kappa_mode), _ptr(G), _ptr(out))
    if rc != 0:
        raise ValueError("oracle_source_gradient: invalid arguments")
    return out


def trace_ray(j, kappa, source, num_rays: int, ray: int, step_size: float, num_steps: int,
              geom_mode: int = 0, kappa_mode: int = 0):
    """Per-substep record of one ray (bin 0): base corner flat index, kappa cell, I_{k+1}."""
    j, kappa = _grid_args(j, kappa)
    _, n0, n1, n2 = j.shape
    src = _f64(source).reshape(3)
    base = np.zeros(num_steps, np.int64)
    nn = np.zeros(num_steps, np.int64)
    I = np.zeros(num_steps, np.float64)
    rc = _load().oracle_trace_ray(_ptr(j[0]), _ptr(kappa[0]), n0, n1, n2, _ptr(src), int(num_rays),
                                  int(ray), float(step_size), int(num_steps), int(geom_mode),
                                  int(kappa_mode), _ptr(base, _lp), _ptr(nn, _lp), _ptr(I))
    if rc != 0:
        raise ValueError("oracle_trace_ray: invalid arguments")
    return base, nn, I


def conv3d_fwd(x, w, bias=None, dilation: int = 1) -> np.ndarray:
    """3x3x3 'same' cross-correlation with zero padding and dilation (conv_oracle.c), FP64.
    x: [B, Ci, D, H, W]; w: [Co, Ci, 3, 3, 3]; bias: [Co] or None. Returns [B, Co, D, H, W]."""
    x = _f64(x)
    w = _f64(w)
    B, Ci, D, H, W = x.shape
    Co = w.shape[0]
    assert w.shape == (Co, Ci, 3, 3, 3)
    b = None if bias is None else _f64(bias)
    y = np.empty((B, Co, D, H, W), np.float64)
    rc = _load().oracle_conv3d_fwd(_ptr(x), _ptr(w), _ptr(b) if b is not None else None, B, Ci, Co, D, H, W,
                                   int(dilation), _ptr(y))
    if rc != 0:
        raise ValueError("oracle_conv3d_fwd: invalid arguments")
    return y


def conv3d_bwd(x, w, gy, dilation: int = 1):
    """(dL/dx, dL/dw, dL/dbias) of conv3d_fwd for dL/dy = gy, FP64."""
    x = _f64(x)
    w = _f64(w)
    gy = _f64(gy)
    B, Ci, D, H, W = x.shape
    Co = w.shape[0]
    gx = np.empty_like(x)
    gw = np.empty_like(w)
    gb = np.empty(Co, np.float64)
    rc = _load().oracle_conv3d_bwd(_ptr(x), _ptr(w), None, B, Ci, Co, D, H, W, int(dilation), _ptr(gy),
                                   _ptr(gx), _ptr(gw), _ptr(gb))
    if rc != 0:
        raise ValueError("oracle_conv3d_bwd: invalid arguments")
    return gx, gw, gb
