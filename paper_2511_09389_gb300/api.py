"""Python binding of the C ABI (include/raytrax.h): argument marshalling only.

PyTorch supplies device memory and streams; every step of the march runs in the CUDA
library. Tensors are float32, C-contiguous, shape [n_freq, n0, n1, n2] (a 3-D grid is one
bin); source positions are [n_src, 3] grid coordinates. Calls are asynchronous on the
current torch stream unless a stream is given.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _native
from ._native import RTError, check


def _stream_ptr(stream, device) -> int:
    s = stream if stream is not None else torch.cuda.current_stream(device)
    return int(s.cuda_stream)


def _grid_tensor(t: torch.Tensor, name: str) -> torch.Tensor:
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor (the library has no CPU path)")
    if t.dtype != torch.float32:
        raise TypeError(f"{name} must be float32")
    if t.dim() == 3:
        t = t.unsqueeze(0)
    if t.dim() != 4:
        raise ValueError(f"{name} must be [n_freq, n0, n1, n2] or [n0, n1, n2]")
    return t.contiguous()


def num_substeps(step_size: float, radiation_velocity: float, time_step: float, cap: int = 0) -> int:
    """N_s = ceil(c dt / ds) (or the cap), as the library computes it."""
    n = _native.load().rt_num_substeps(float(step_size), float(radiation_velocity), float(time_step), int(cap))
    if n < 0:
        raise ValueError("invalid step_size / radiation_velocity / time_step")
    return n


def direction_table(num_rays: int) -> np.ndarray:
    """The library's FP32 Fibonacci lattice in lattice order, [num_rays, 3]."""
    out = np.empty((num_rays, 3), np.float32)
    check(_native.load().rt_direction_table(int(num_rays), out.ctypes.data))
    return out


class Grid:
    """A library handle for one grid shape (owns its scratch on one device).

    accumulation: "auto" (FP32 while a call deposits fewer than 32 updates per cell and bin on
    average, else 64-bit fixed point, or FP64 where the fixed-point unit would be coarse and in
    continued marches), "fp32", "fp64" or "fixed"; deterministic=True also sums in fixed point,
    with one launch plan.

    plan=(bins_per_group, block, gathers[, lanes_per_ray[, tile]]) pins the forward launch plan,
    gathers 0 = corner slots (a shared face keeps its gathers and sums), 1 = one step ahead,
    2 = both, 3 = the whole corner set reused while unchanged, 4 = corner slots with the entering
    corners gathered a substep ahead; lanes_per_ray 1 or 2 (2: gathers 0 or 4); tile 0 / 1 =
    source deposit tiles off / on (the library's default when not given; ignored when
    autotune=True, which times the candidates on the first call of each shape class)."""

    ACCUMULATION = {"auto": 0, "fp32": 1, "fp64": 2, "fixed": 3}

    def __init__(self, shape, max_freq: int = 8, *, deterministic: bool = False, kappa_mode: int = 0,
                 ns_cap: int = 0, autotune: bool = False, ckpt_stride: int = 0, profile: bool = False,
                 plan=None, check_inputs: bool = False, record_checkpoints: bool = False,
                 accumulation: str = "auto", device=None):
        self._lib = _native.load()
        self.shape = tuple(int(s) for s in shape)
        if len(self.shape) != 3:
            raise ValueError("shape must be (n0, n1, n2)")
        self.max_freq = int(max_freq)
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None
                                   else torch.device(device).index or 0)
        pw, pb, pp, pl, pt = (0, 0, 0, 0, 0) if plan is None else (
            int(plan[0]), int(plan[1]), int(plan[2]) + 1, int(plan[3]) if len(plan) > 3 else 1,
            int(plan[4]) + 1 if len(plan) > 4 else 0)
        if accumulation not in self.ACCUMULATION:
            raise ValueError(f"accumulation must be one of {sorted(self.ACCUMULATION)}")
        opt = _native.rt_options(int(bool(deterministic)), int(kappa_mode), int(ns_cap), int(bool(autotune)),
                                 int(ckpt_stride), int(bool(profile)), pw, pb, pp, pl, pt, int(bool(check_inputs)),
                                 int(bool(record_checkpoints)), self.ACCUMULATION[accumulation])
        self.options = opt
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            check(self._lib.rt_create_grid(ctypes.byref(h), *self.shape, self.max_freq, ctypes.byref(opt)))
        self._h = h
        self._inflight = []   # host buffers of enqueued advance_host_async calls

    # -- lifetime -------------------------------------------------------------------------
    def close(self):
        h, self._h = getattr(self, "_h", None), None
        if h is not None and h.value:
            with torch.cuda.device(self.device):
                self._lib.rt_destroy(h)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- helpers --------------------------------------------------------------------------
    def _inputs(self, j, kappa, sources):
        j = _grid_tensor(j, "j")
        kappa = _grid_tensor(kappa, "kappa")
        if j.shape != kappa.shape:
            raise ValueError("j and kappa must have the same shape")
        if tuple(j.shape[1:]) != self.shape:
            raise ValueError(f"grid shape {tuple(j.shape[1:])} differs from the handle's {self.shape}")
        if j.device != self.device or kappa.device != self.device:
            raise ValueError(f"tensors must live on {self.device}")
        src = torch.as_tensor(sources, dtype=torch.float32, device=self.device).reshape(-1, 3).contiguous()
        return j, kappa, src

    # -- forward --------------------------------------------------------------------------
    def advance(self, j, kappa, sources, num_rays: int, step_size: float, radiation_velocity: float = 1.0,
                time_step: float = 1.0, *, out=None, accumulate: bool = False, ray_range=None,
                stream=None) -> torch.Tensor:
        """One dt of the field: out[b] (+)= (4 pi / N_Omega) sum_src sum_rays sum_k W(x_k) I_{k+1}."""
        j, kappa, src = self._inputs(j, kappa, sources)
        nf = j.shape[0]
        if out is None:
            out = torch.empty_like(j)
            accumulate = False
        elif out.shape != j.shape or out.dtype != torch.float32 or not out.is_contiguous() \
                or out.device != self.device:
            raise ValueError("out must be a contiguous float32 tensor shaped like j on the handle's device")
        sp = _stream_ptr(stream, self.device)
        with torch.cuda.device(self.device):
            if ray_range is None:
                st = self._lib.rt_advance(self._h, j.data_ptr(), kappa.data_ptr(), src.data_ptr(), src.shape[0],
                                          int(num_rays), float(step_size), float(radiation_velocity),
                                          float(time_step), nf, out.data_ptr(), int(bool(accumulate)), sp)
            else:
                rb, re = ray_range
                st = self._lib.rt_advance_rays(self._h, j.data_ptr(), kappa.data_ptr(), src.data_ptr(),
                                               src.shape[0], int(num_rays), int(rb), int(re), float(step_size),
                                               float(radiation_velocity), float(time_step), nf, out.data_ptr(),
                                               int(bool(accumulate)), sp)
        check(st)
        return out

    def advance_continue(self, j, kappa, sources, num_rays: int, step_size: float,
                         radiation_velocity: float = 1.0, time_step: float = 1.0, *, out=None,
                         accumulate: bool = False, restart: bool = False, stream=None) -> torch.Tensor:
        """rt_advance_continue: one more dt of a march that continues across calls (each ray resumes
        where the previous call on this handle left it; restart=True, or a change of sources /
        rays / bins / step size, starts the rays at their sources again)."""
        j, kappa, src = self._inputs(j, kappa, sources)
        nf = j.shape[0]
        if out is None:
            out = torch.empty_like(j)
            accumulate = False
        elif out.shape != j.shape or out.dtype != torch.float32 or not out.is_contiguous() \
                or out.device != self.device:
            raise ValueError("out must be a contiguous float32 tensor shaped like j on the handle's device")
        sp = _stream_ptr(stream, self.device)
        with torch.cuda.device(self.device):
            st = self._lib.rt_advance_continue(self._h, j.data_ptr(), kappa.data_ptr(), src.data_ptr(), src.shape[0],
                                               int(num_rays), float(step_size), float(radiation_velocity),
                                               float(time_step), nf, out.data_ptr(), int(bool(accumulate)),
                                               int(bool(restart)), sp)
        check(st)
        return out

    def _host_call(self, fn, j, kappa, sources, num_rays, step_size, radiation_velocity, time_step, out,
                   stream):
        def host(a, name):
            if isinstance(a, torch.Tensor):
                if a.is_cuda or a.dtype != torch.float32 or not a.is_contiguous():
                    raise ValueError(f"{name} must be a contiguous float32 CPU tensor")
                return a, a.data_ptr(), tuple(a.shape)
            a = np.ascontiguousarray(a, dtype=np.float32)
            return a, a.ctypes.data, a.shape
        jh, jp, jshape = host(j, "j")
        kh, kp, kshape = host(kappa, "kappa")
        sh, spp, sshape = host(sources, "sources")
        if len(jshape) == 3:
            jshape = (1,) + tuple(jshape)
        if tuple(jshape) != tuple(kshape if len(kshape) == 4 else (1,) + tuple(kshape)) or tuple(jshape[1:]) != self.shape:
            raise ValueError("j / kappa shapes do not match the handle")
        nsrc = int(np.prod(sshape)) // 3
        if out is None:
            out = np.empty(jshape, np.float32)
        oh, op, oshape = host(out, "out")
        if tuple(oshape) != tuple(jshape):
            raise ValueError("out has the wrong shape")
        with torch.cuda.device(self.device):
            st = fn(self._h, jp, kp, spp, nsrc, int(num_rays), float(step_size), float(radiation_velocity),
                    float(time_step), jshape[0], op, _stream_ptr(stream, self.device))
        check(st)
        return oh, (jh, kh, sh, oh)

    def advance_host(self, j: np.ndarray, kappa: np.ndarray, sources: np.ndarray, num_rays: int,
                     step_size: float, radiation_velocity: float = 1.0, time_step: float = 1.0, *,
                     out: np.ndarray | None = None, stream=None) -> np.ndarray:
        """rt_advance_host: host (numpy / pinned torch CPU) buffers in, host field out, synchronous."""
        oh, _ = self._host_call(self._lib.rt_advance_host, j, kappa, sources, num_rays, step_size,
                                radiation_velocity, time_step, out, stream)
        return oh

    def advance_host_async(self, j, kappa, sources, num_rays: int, step_size: float,
                           radiation_velocity: float = 1.0, time_step: float = 1.0, *, out=None, stream=None):
        """rt_advance_host_async: enqueue one host-buffer advance and return at once; the field is
        in the returned buffer (``out`` if given) after :meth:`host_wait`. Consecutive calls overlap
        their copies with the march of their neighbours when the host buffers are pinned. The
        handle keeps references to the buffers until :meth:`host_wait`."""
        oh, keep = self._host_call(self._lib.rt_advance_host_async, j, kappa, sources, num_rays, step_size,
                                   radiation_velocity, time_step, out, stream)
        self._inflight.append(keep)
        return oh

    def host_wait(self) -> None:
        """rt_host_wait: block until every :meth:`advance_host_async` call has landed on the host."""
        with torch.cuda.device(self.device):
            st = self._lib.rt_host_wait(self._h)
        self._inflight.clear()
        check(st)

    def host_join(self, stream=None) -> None:
        """rt_host_join: make ``stream`` wait on the device for the enqueued host calls."""
        with torch.cuda.device(self.device):
            check(self._lib.rt_host_join(self._h, _stream_ptr(stream, self.device)))

    # -- adjoint --------------------------------------------------------------------------
    def backward(self, grad_out, j, kappa, sources, num_rays: int, step_size: float,
                 radiation_velocity: float = 1.0, time_step: float = 1.0, *, need_j: bool = True,
                 need_kappa: bool = True, need_sources: bool = False, stream=None):
        """(dL/dj, dL/dkappa) for G = dL/d(out) of :meth:`advance` (either may be None if not
        needed); with need_sources=True also dL/d(source positions) [n_src, 3] as a third entry."""
        j, kappa, src = self._inputs(j, kappa, sources)
        g = _grid_tensor(grad_out, "grad_out")
        if g.shape != j.shape or g.device != self.device:
            raise ValueError("grad_out must be shaped like j on the handle's device")
        gj = torch.empty_like(j) if need_j else None
        gk = torch.empty_like(j) if need_kappa else None
        gs = torch.empty_like(src) if need_sources else None
        ptr = lambda t: t.data_ptr() if t is not None else None
        with torch.cuda.device(self.device):
            if need_sources:
                st = self._lib.rt_backward_sources(self._h, g.data_ptr(), j.data_ptr(), kappa.data_ptr(),
                                                   src.data_ptr(), src.shape[0], int(num_rays), float(step_size),
                                                   float(radiation_velocity), float(time_step), j.shape[0], ptr(gj),
                                                   ptr(gk), ptr(gs), _stream_ptr(stream, self.device))
            else:
                st = self._lib.rt_backward(self._h, g.data_ptr(), j.data_ptr(), kappa.data_ptr(), src.data_ptr(),
                                           src.shape[0], int(num_rays), float(step_size), float(radiation_velocity),
                                           float(time_step), j.shape[0], ptr(gj), ptr(gk),
                                           _stream_ptr(stream, self.device))
        check(st)
        return (gj, gk, gs) if need_sources else (gj, gk)

    def invert_emissivity(self, target, kappa, sources, num_rays: int, step_size: float,
                          radiation_velocity: float = 1.0, time_step: float = 1.0, *, iterations: int = 200,
                          lr: float = 1e-2, eps_rel: float = 1e-2, j=None, stream=None):
        """rt_invert_emissivity: `iterations` projected Adam steps on the log-field misfit to
        `target`, from j (default zero). Returns (the recovered j, the device tensor of the
        iterations + 1 losses); nothing is synchronised."""
        t = _grid_tensor(target, "target")
        j = torch.zeros_like(t) if j is None else _grid_tensor(j, "j").clone()
        j, kappa, src = self._inputs(j, kappa, sources)
        if t.shape != j.shape:
            raise ValueError("target must be shaped like kappa")
        losses = torch.empty(int(iterations) + 1, dtype=torch.float32, device=self.device)
        with torch.cuda.device(self.device):
            check(self._lib.rt_invert_emissivity(self._h, t.data_ptr(), kappa.data_ptr(), src.data_ptr(), src.shape[0],
                                                 int(num_rays), float(step_size), float(radiation_velocity),
                                                 float(time_step), j.shape[0], int(iterations), float(lr),
                                                 float(eps_rel), j.data_ptr(), losses.data_ptr(),
                                                 _stream_ptr(stream, self.device)))
        return j, losses

    def kernel_ms(self) -> float:
        """Duration of the last call's march kernel (needs profile=True)."""
        ms = ctypes.c_float()
        check(self._lib.rt_kernel_ms(self._h, ctypes.byref(ms)))
        return float(ms.value)

    def last_plan(self) -> dict:
        """Launch plan of the last forward call (width, block, prefetch, lanes, tile, tuned_ms)."""
        w, b, p, n, tl, t = (ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int(),
                             ctypes.c_float())
        check(self._lib.rt_last_plan(self._h, ctypes.byref(w), ctypes.byref(b), ctypes.byref(p), ctypes.byref(n),
                                     ctypes.byref(tl), ctypes.byref(t)))
        return {"width": w.value, "block": b.value, "prefetch": p.value, "lanes_per_ray": n.value, "tile": tl.value,
                "tuned_ms": t.value}

    def last_ckpt_stride(self) -> dict:
        """Checkpoint stride K of the last backward call and its tuned reverse-march ms (-1: not tuned)."""
        k, t = ctypes.c_int(), ctypes.c_float()
        check(self._lib.rt_last_ckpt_stride(self._h, ctypes.byref(k), ctypes.byref(t)))
        return {"stride": k.value, "tuned_ms": t.value}

    def last_accumulation(self) -> str:
        """How the last forward call summed its deposits: "fp32", "fp64" or "fixed" (deterministic)."""
        m = ctypes.c_int()
        check(self._lib.rt_last_accumulation(self._h, ctypes.byref(m)))
        return {1: "fp32", 2: "fp64", 3: "fixed"}[m.value]

    def tuning_report(self) -> str:
        """Candidates and times of the last autotuning pass ("" if none)."""
        buf = ctypes.create_string_buffer(8192)
        check(self._lib.rt_tuning_report(self._h, buf, len(buf)))
        return buf.value.decode()

    # -- test hook ------------------------------------------------------------------------
    def trace_cells(self, source, num_rays: int, ray: int, step_size: float, num_steps: int):
        """Per-substep (base corner, kappa cell) flat indices of one lattice ray, from the device."""
        src = np.ascontiguousarray(np.asarray(source, np.float32).reshape(3))
        base = np.zeros(num_steps, np.int64)
        nn = np.zeros(num_steps, np.int64)
        llp = ctypes.POINTER(ctypes.c_longlong)
        with torch.cuda.device(self.device):
            st = self._lib.rt_trace_cells(self._h, src.ctypes.data, int(num_rays), int(ray), float(step_size),
                                          int(num_steps), base.ctypes.data_as(llp), nn.ctypes.data_as(llp))
        check(st)
        return base, nn


class Batch:
    """Many independent problems advanced by one persistent launch replayed from a CUDA graph.

    instances: sequence of dicts with keys j, kappa, sources (CUDA float32 tensors), num_rays,
    step_size, radiation_velocity, time_step and optionally out. The tensors are bound to the
    batch: each run() reads them and overwrites the outputs in place (`outputs`).
    """

    def __init__(self, instances, *, kappa_mode: int = 0, autotune: bool = False, ns_cap: int = 0):
        self._lib = _native.load()
        self.device = torch.device("cuda", torch.cuda.current_device())
        self._keep, self.outputs = [], []
        arr = (_native.rt_instance * len(instances))()
        for i, d in enumerate(instances):
            j = _grid_tensor(d["j"], "j")
            k = _grid_tensor(d["kappa"], "kappa")
            if j.shape != k.shape:
                raise ValueError(f"instance {i}: j and kappa shapes differ")
            src = torch.as_tensor(d["sources"], dtype=torch.float32, device=j.device).reshape(-1, 3).contiguous()
            out = d.get("out")
            out = torch.empty_like(j) if out is None else out
            if out.shape != j.shape or not out.is_contiguous() or out.dtype != torch.float32:
                raise ValueError(f"instance {i}: bad out tensor")
            self._keep += [j, k, src, out]
            self.outputs.append(out)
            nf, n0, n1, n2 = j.shape
            arr[i] = _native.rt_instance(j.data_ptr(), k.data_ptr(), src.data_ptr(), src.shape[0], n0, n1, n2, nf,
                                         int(d["num_rays"]), float(d["step_size"]),
                                         float(d.get("radiation_velocity", 1.0)), float(d.get("time_step", 1.0)),
                                         out.data_ptr())
        opt = _native.rt_options(0, int(kappa_mode), int(ns_cap), int(bool(autotune)), 0, 0, 0, 0, 0, 0)
        h = ctypes.c_void_p()
        check(self._lib.rt_batch_create(ctypes.byref(h), arr, len(instances), ctypes.byref(opt)))
        self._h = h

    @property
    def updates(self) -> int:
        return int(self._lib.rt_batch_updates(self._h))

    def info(self, instance: int) -> dict:
        """rt_batch_info: how an instance is marched (its own launches or the persistent kernels)
        and with which plan."""
        vals = [ctypes.c_int() for _ in range(5)]
        check(self._lib.rt_batch_info(self._h, int(instance), *[ctypes.byref(v) for v in vals]))
        keys = ("dedicated", "bins_per_thread", "block", "gathers", "tile")
        return {k: v.value for k, v in zip(keys, vals)}

    def run(self, stream=None):
        check(self._lib.rt_batch_run(self._h, _stream_ptr(stream, self.device)))
        return self.outputs

    def close(self):
        h, self._h = getattr(self, "_h", None), None
        if h is not None and h.value:
            self._lib.rt_batch_destroy(h)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_grid_cache: dict = {}


def _cached_grid(shape, n_freq, device, **opts) -> Grid:
    key = (tuple(shape), int(device.index), tuple(sorted(opts.items())))
    g = _grid_cache.get(key)
    if g is None or g.max_freq < n_freq:
        g = Grid(shape, max(8, n_freq), device=device, **opts)
        _grid_cache[key] = g
    return g


def adam_step(params: torch.Tensor, grads: torch.Tensor, m: torch.Tensor, v: torch.Tensor, lr: float, step: int,
              beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8, stream=None) -> None:
    """One bias-corrected Adam step (rt_adam_step) on float32 CUDA tensors of one size, in place."""
    for t in (params, grads, m, v):
        if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous() and t.numel() == params.numel()):
            raise ValueError("adam_step needs contiguous float32 CUDA tensors of one size")
    with torch.cuda.device(params.device):
        check(_native.load().rt_adam_step(params.data_ptr(), grads.data_ptr(), m.data_ptr(), v.data_ptr(),
                                          params.numel(), float(lr), float(beta1), float(beta2), float(eps),
                                          int(step), _stream_ptr(stream, params.device)))


def advance(j, kappa, sources, num_rays: int, step_size: float, radiation_velocity: float = 1.0,
            time_step: float = 1.0, **opts) -> torch.Tensor:
    """Functional form of :meth:`Grid.advance` with a cached handle per (shape, device, options)."""
    jj = _grid_tensor(j, "j")
    g = _cached_grid(jj.shape[1:], jj.shape[0], jj.device, **opts)
    out = g.advance(jj, kappa, sources, num_rays, step_size, radiation_velocity, time_step)
    return out if j.dim() == 4 else out[0]


__all__ = ["Grid", "Batch", "advance", "adam_step", "num_substeps", "direction_table", "RTError"]
