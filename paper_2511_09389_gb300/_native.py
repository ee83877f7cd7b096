"""ctypes loader for the in-tree CUDA library ``librt_gb300.so`` (C ABI of include/raytrax.h).

There is no fallback: if the library is missing or fails to load, every entry point raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "librt_gb300.so")

RT_OK = 0
STATUS_NAMES = {0: "RT_OK", 1: "RT_ERR_INVALID_ARG", 2: "RT_ERR_CUDA", 3: "RT_ERR_OOM",
                4: "RT_ERR_TIMEOUT", 5: "RT_ERR_INTERNAL", 6: "RT_ERR_UNSUPPORTED"}

# every symbol include/raytrax.h declares
EXPORTS = ("rt_default_options", "rt_create_grid", "rt_destroy", "rt_last_error", "rt_num_substeps",
           "rt_direction_table", "rt_advance", "rt_advance_rays", "rt_advance_continue", "rt_advance_host",
           "rt_advance_host_async", "rt_host_wait", "rt_host_join", "rt_backward", "rt_backward_sources", "rt_invert_emissivity",
           "rt_trace_cells", "rt_kernel_ms", "rt_last_plan",
           "rt_tuning_report", "rt_last_accumulation", "rt_last_ckpt_stride", "rt_shard_plan", "rt_advance_noalloc", "rt_batch_create", "rt_batch_run", "rt_batch_updates",
           "rt_batch_info",
           "rt_batch_destroy", "rt_c32_from_f32", "rt_c32_to_f32", "rt_conv3d_pack_weights",
           "rt_conv3d_forward", "rt_device_status", "rt_conv3d_weight_grad",
           "rt_surrogate_features", "rt_field_max", "rt_log_field_loss", "rt_field_error", "rt_c32_channel_mean",
           "rt_adam_step", "rt_microbench", "rt_neg_exp", "rt_advance_batch", "rt_sync_status")


class RTError(RuntimeError):
    """A non-zero rt_status, with the library's thread-local message."""

    def __init__(self, status: int, message: str):
        self.status = status
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")


class rt_options(ctypes.Structure):
    _fields_ = [("deterministic", ctypes.c_int), ("kappa_mode", ctypes.c_int), ("ns_cap", ctypes.c_int),
                ("autotune", ctypes.c_int), ("ckpt_stride", ctypes.c_int),
                ("profile", ctypes.c_int), ("plan_width", ctypes.c_int), ("plan_block", ctypes.c_int),
                ("plan_prefetch", ctypes.c_int), ("plan_lanes", ctypes.c_int), ("plan_tile", ctypes.c_int),
                ("check_inputs", ctypes.c_int), ("record_checkpoints", ctypes.c_int),
                ("accumulation", ctypes.c_int)]


class rt_instance(ctypes.Structure):
    _fields_ = [("j_map", ctypes.c_void_p), ("kappa_map", ctypes.c_void_p), ("source_pos", ctypes.c_void_p),
                ("num_sources", ctypes.c_int), ("n0", ctypes.c_int), ("n1", ctypes.c_int), ("n2", ctypes.c_int),
                ("n_freq", ctypes.c_int), ("num_rays", ctypes.c_int), ("step_size", ctypes.c_float),
                ("radiation_velocity", ctypes.c_float), ("time_step", ctypes.c_float),
                ("out_field", ctypes.c_void_p)]


_lock = threading.Lock()
_lib = None


def load(path: str = LIB_PATH):
    """Load the library (once) and declare the argument types of every export."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise ImportError(f"CUDA library {path} is not built; run __graft_entry__.build() "
                              "(there is no CPU fallback)")
        lib = ctypes.CDLL(path)
        vp, fp, i, f = ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_float
        llp = ctypes.POINTER(ctypes.c_longlong)
        lib.rt_default_options.argtypes = [ctypes.POINTER(rt_options)]
        lib.rt_default_options.restype = None
        lib.rt_create_grid.argtypes = [ctypes.POINTER(vp), i, i, i, i, ctypes.POINTER(rt_options)]
        lib.rt_create_grid.restype = i
        lib.rt_destroy.argtypes = [vp]
        lib.rt_destroy.restype = i
        lib.rt_last_error.argtypes = []
        lib.rt_last_error.restype = ctypes.c_char_p
        lib.rt_num_substeps.argtypes = [f, f, f, i]
        lib.rt_num_substeps.restype = i
        lib.rt_direction_table.argtypes = [i, fp]
        lib.rt_direction_table.restype = i
        lib.rt_advance.argtypes = [vp, fp, fp, fp, i, i, f, f, f, i, fp, i, vp]
        lib.rt_advance.restype = i
        lib.rt_advance_rays.argtypes = [vp, fp, fp, fp, i, i, i, i, f, f, f, i, fp, i, vp]
        lib.rt_advance_rays.restype = i
        lib.rt_advance_continue.argtypes = [vp, fp, fp, fp, i, i, f, f, f, i, fp, i, i, vp]
        lib.rt_advance_continue.restype = i
        lib.rt_advance_host.argtypes = [vp, fp, fp, fp, i, i, f, f, f, i, fp, vp]
        lib.rt_advance_host.restype = i
        lib.rt_advance_host_async.argtypes = [vp, fp, fp, fp, i, i, f, f, f, i, fp, vp]
        lib.rt_advance_host_async.restype = i
        lib.rt_host_wait.argtypes = [vp]
        lib.rt_host_wait.restype = i
        lib.rt_host_join.argtypes = [vp, vp]
        lib.rt_host_join.restype = i
        lib.rt_backward.argtypes = [vp, fp, fp, fp, fp, i, i, f, f, f, i, fp, fp, vp]
        lib.rt_backward.restype = i
        lib.rt_backward_sources.argtypes = [vp, fp, fp, fp, fp, i, i, f, f, f, i, fp, fp, fp, vp]
        lib.rt_backward_sources.restype = i
        lib.rt_invert_emissivity.argtypes = [vp, fp, fp, fp, i, i, f, f, f, i, i, f, f, fp, fp, vp]
        lib.rt_invert_emissivity.restype = i
        lib.rt_trace_cells.argtypes = [vp, fp, i, i, f, i, llp, llp]
        lib.rt_trace_cells.restype = i
        lib.rt_shard_plan.argtypes = [i, i, i, i, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
        lib.rt_shard_plan.restype = i
        lib.rt_last_ckpt_stride.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_float)]
        lib.rt_last_ckpt_stride.restype = i
        lib.rt_last_accumulation.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
        lib.rt_last_accumulation.restype = i
        lib.rt_kernel_ms.argtypes = [vp, ctypes.POINTER(ctypes.c_float)]
        lib.rt_kernel_ms.restype = i
        ip = ctypes.POINTER(ctypes.c_int)
        lib.rt_last_plan.argtypes = [vp, ip, ip, ip, ip, ip, ctypes.POINTER(ctypes.c_float)]
        lib.rt_last_plan.restype = i
        lib.rt_tuning_report.argtypes = [vp, ctypes.c_char_p, i]
        lib.rt_tuning_report.restype = i
        lib.rt_advance_noalloc.argtypes = [fp, fp, fp, i, i, i, i, i, f, f, f, i, fp, vp]
        lib.rt_advance_noalloc.restype = i
        lib.rt_batch_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(rt_instance), i, ctypes.POINTER(rt_options)]
        lib.rt_batch_create.restype = i
        lib.rt_batch_run.argtypes = [vp, vp]
        lib.rt_batch_run.restype = i
        lib.rt_batch_updates.argtypes = [vp]
        lib.rt_batch_updates.restype = ctypes.c_longlong
        ip = ctypes.POINTER(ctypes.c_int)
        lib.rt_batch_info.argtypes = [vp, i, ip, ip, ip, ip, ip]
        lib.rt_batch_info.restype = i
        lib.rt_batch_destroy.argtypes = [vp]
        lib.rt_batch_destroy.restype = i
        lib.rt_c32_from_f32.argtypes = [vp, i, i, i, i, i, vp, vp]
        lib.rt_c32_from_f32.restype = i
        lib.rt_c32_to_f32.argtypes = [vp, i, i, i, i, i, vp, vp]
        lib.rt_c32_to_f32.restype = i
        lib.rt_conv3d_pack_weights.argtypes = [vp, i, i, i, vp, vp]
        lib.rt_conv3d_pack_weights.restype = i
        lib.rt_conv3d_forward.argtypes = [vp, i, i, i, i, i, vp, vp, i, i, i, f, vp, vp, vp, vp]
        lib.rt_conv3d_forward.restype = i
        lib.rt_conv3d_weight_grad.argtypes = [vp, vp, i, i, i, i, i, i, i, vp, vp, vp]
        lib.rt_conv3d_weight_grad.restype = i
        ll = ctypes.c_longlong
        lib.rt_surrogate_features.argtypes = [vp, vp, i, i, i, i, vp, vp]
        lib.rt_surrogate_features.restype = i
        lib.rt_field_max.argtypes = [vp, i, ll, vp, vp]
        lib.rt_field_max.restype = i
        lib.rt_log_field_loss.argtypes = [vp, vp, i, ll, vp, f, f, f, vp, vp, vp]
        lib.rt_log_field_loss.restype = i
        lib.rt_field_error.argtypes = [vp, vp, i, ll, vp, f, f, f, vp, vp]
        lib.rt_field_error.restype = i
        lib.rt_microbench.argtypes = [i, i, vp, ll, i, i, ctypes.POINTER(ctypes.c_float),
                                      ctypes.POINTER(ctypes.c_double)]
        lib.rt_microbench.restype = i
        lib.rt_neg_exp.argtypes = [fp, fp, ll, vp]
        lib.rt_neg_exp.restype = i
        lib.rt_advance_batch.argtypes = [vp, vp, i, vp]
        lib.rt_advance_batch.restype = i
        lib.rt_sync_status.argtypes = [vp]
        lib.rt_sync_status.restype = i
        lib.rt_c32_channel_mean.argtypes = [vp, i, i, ll, vp, vp]
        lib.rt_c32_channel_mean.restype = i
        lib.rt_adam_step.argtypes = [vp, vp, vp, vp, ll, f, f, f, f, i, vp]
        lib.rt_adam_step.restype = i
        lib.rt_device_status.argtypes = [ctypes.POINTER(ctypes.c_int)]
        lib.rt_device_status.restype = i
        _lib = lib
        return lib


def check(status: int) -> None:
    if status != RT_OK:
        msg = _lib.rt_last_error().decode() if _lib is not None else ""
        raise RTError(status, msg)
