"""GB300-native (sm_103a) emission-absorption ray march of Ray-trax (arXiv 2511.09389).

The march (paper Sec. 2, Eq. 2) runs in hand-written CUDA kernels behind a C ABI
(include/raytrax.h, built into ``librt_gb300.so``); this package is its thin Python binding.
Importing the package does not load the library; the first call that needs it does, and
raises if it has not been built (there is no CPU fallback).
"""
__all__ = ["Grid", "advance", "num_substeps", "direction_table", "RTError", "RTFunction"]


def __getattr__(name):
    if name in ("Grid", "advance", "num_substeps", "direction_table", "RTError"):
        from . import api
        return getattr(api, name)
    if name == "RTFunction":
        from . import autograd
        return autograd.RTFunction
    raise AttributeError(name)
