"""Peaks of the march's memory operations on the current GPU, from the library's microbenchmark
kernels (`rt_microbench`): L2 reductions (`red.global.add`) and read-only gathers on an
L2-resident array, with random, warp-coherent and 8-corner-stencil addresses.

The march's deposit is a `red.global.add.v4.f32` into the 8 corners of a cell of a cell-major
accumulator and its gather is 8 + 1 16-byte loads, so the stencil kinds with 16-byte vectors
are the denominators of its roofline fractions; the 8-byte stencil reductions (u64, f64) are
those of the fixed-point deposits. The paper has no counterpart.

    python -m paper_2511_09389_gb300.peaks [--edge 128] [--out peaks.json]
"""
from __future__ import annotations

import ctypes
import json

import torch

from . import _native
from ._native import check

KINDS = {"red_random": 0, "red_coherent": 1, "red_stencil": 2, "gather_random": 3, "gather_stencil": 4}


def measure(edge: int = 128, vecs=(4, 1), reps: int = 3, device=None) -> dict:
    """Best-of-`reps` rate of every kind for each vector width in `vecs` on an edge^3 grid of
    4-float cells (edge 128: 32 MiB, the march's packed accumulator at 128^3 with 4 bins).
    Returns {"<kind>_v<vec>": {"ops_per_s", "bytes_per_s", "ms", "ops"}, ...}."""
    lib = _native.load()
    dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
    buf = torch.zeros(edge ** 3 * 4, dtype=torch.float32, device=dev)
    out = {"edge": edge, "buffer_bytes": buf.numel() * 4,
           "launch": "8 blocks of 256 threads per SM; each thread 256 operations, or 64 stencil iterations of 8"}
    ms = ctypes.c_float()
    ops = ctypes.c_double()
    with torch.cuda.device(dev):
        torch.cuda.synchronize(dev)
        for vec in vecs:
            for name, kind in KINDS.items():
                iters = 64 if kind in (2, 4) else 256
                best = None
                for r in range(reps + 1):          # the first launch is a warm-up
                    check(lib.rt_microbench(kind, vec, buf.data_ptr(), buf.numel() * 4, edge, iters, ctypes.byref(ms),
                                            ctypes.byref(ops)))
                    if r > 0 and (best is None or ms.value < best):
                        best = ms.value
                rate = ops.value / (best * 1e-3)
                out[f"{name}_v{vec}"] = {"ops_per_s": rate, "bytes_per_s": rate * 4 * vec, "ms": best,
                                         "ops": ops.value}
        # the stencil with 8-byte reductions: the fixed-point deposit (u64) and FP64
        for name, kind in (("red_stencil_u64", 5), ("red_stencil_f64", 6)):
            best = None
            for r in range(reps + 1):
                check(lib.rt_microbench(kind, 1, buf.data_ptr(), buf.numel() * 4, edge, 64, ctypes.byref(ms),
                                        ctypes.byref(ops)))
                if r > 0 and (best is None or ms.value < best):
                    best = ms.value
            rate = ops.value / (best * 1e-3)
            out[name] = {"ops_per_s": rate, "bytes_per_s": rate * 8, "ms": best, "ops": ops.value}
    return out


if __name__ == "__main__":
    import argparse

    ap = argparse.ArgumentParser(description="measure L2 reduction / gather peaks with the library's kernels")
    ap.add_argument("--edge", type=int, default=128)
    ap.add_argument("--out", default="")
    a = ap.parse_args()
    from . import build as _build
    _build.build()
    res = measure(a.edge)
    text = json.dumps(res, indent=1)
    print(text)
    if a.out:
        with open(a.out, "w") as f:
            f.write(text + "\n")
