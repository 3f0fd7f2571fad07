"""ctypes binding of ``liblb.so``: argument marshalling only.

Every function here forwards to the C ABI in ``include/lb.h``; all work runs in
the library's CUDA kernels.  If the library is missing, importing the binding
raises: there is no CPU or PyTorch fallback.
"""
from __future__ import annotations

import ctypes
import os

from . import buildlib as _build

_lib = None


class LBError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}" + (f" ({detail})" if detail else ""))


STATUS_NAMES = {0: "LB_OK", 1: "LB_ERR_INVALID_ARG", 2: "LB_ERR_CUDA", 3: "LB_ERR_OOM", 4: "LB_ERR_UNSUPPORTED",
                5: "LB_ERR_TIMEOUT", 6: "LB_ERR_BAD_INPUT"}


class PlanOpts(ctypes.Structure):
    _fields_ = [("num_cols", ctypes.c_int32), ("items_per_thread", ctypes.c_int32), ("group_size", ctypes.c_int32),
                ("ctas_per_sm", ctypes.c_int32), ("validate", ctypes.c_int32), ("mp_variant", ctypes.c_int32),
                ("wave_items", ctypes.c_int32), ("units_per_cta", ctypes.c_int32),
                ("tiles_per_share", ctypes.c_int32), ("items_per_thread_t", ctypes.c_int32),
                ("row_weight", ctypes.c_int32), ("staged", ctypes.c_int32)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("schedule", ctypes.c_int32), ("num_tiles", ctypes.c_int32), ("num_cols", ctypes.c_int32),
                ("num_atoms", ctypes.c_int64), ("block_threads", ctypes.c_int32), ("grid", ctypes.c_int32),
                ("items_per_tile", ctypes.c_int32), ("tiles_per_cta", ctypes.c_int32), ("num_workers", ctypes.c_int32),
                ("mp_variant", ctypes.c_int32), ("num_waves", ctypes.c_int32), ("num_waves_t", ctypes.c_int32),
                ("num_splits", ctypes.c_int64),
                ("group_size", ctypes.c_int32), ("num_sms", ctypes.c_int32), ("kernels_per_spmv", ctypes.c_int32),
                ("has_transpose", ctypes.c_int32)]


TUNE_MAX_CANDIDATES = 20
TUNE_MP_WARP, TUNE_MP_CTA, TUNE_THREAD, TUNE_GROUP = 1, 2, 4, 8


class TuneOpts(ctypes.Structure):
    _fields_ = [("num_cols", ctypes.c_int32), ("reps", ctypes.c_int32), ("prune_factor", ctypes.c_float),
                ("cold_l2", ctypes.c_int32), ("no_cache", ctypes.c_int32), ("families", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 2)]


class TuneCandidate(ctypes.Structure):
    _fields_ = [("schedule", ctypes.c_int32), ("items_per_thread", ctypes.c_int32), ("group_size", ctypes.c_int32),
                ("mp_variant", ctypes.c_int32), ("units_per_cta", ctypes.c_int32), ("row_weight", ctypes.c_int32),
                ("staged", ctypes.c_int32), ("ms", ctypes.c_float),
                ("gbps", ctypes.c_float),
                ("reps", ctypes.c_int32), ("status", ctypes.c_int32)]


class TuneResult(ctypes.Structure):
    _fields_ = [("num_candidates", ctypes.c_int32), ("best", ctypes.c_int32), ("heuristic", ctypes.c_int32),
                ("from_cache", ctypes.c_int32), ("best_schedule", ctypes.c_int32), ("best_opts", PlanOpts),
                ("candidates", TuneCandidate * TUNE_MAX_CANDIDATES)]


class BatchTuneCandidate(ctypes.Structure):
    _fields_ = [("opts", PlanOpts), ("ms", ctypes.c_float), ("gbps", ctypes.c_float), ("reps", ctypes.c_int32),
                ("status", ctypes.c_int32)]


class BatchTuneResult(ctypes.Structure):
    _fields_ = [("num_candidates", ctypes.c_int32), ("best", ctypes.c_int32), ("from_cache", ctypes.c_int32),
                ("passes", ctypes.c_int32), ("best_opts", PlanOpts),
                ("candidates", BatchTuneCandidate * TUNE_MAX_CANDIDATES)]


TUNE_PASS_FWD, TUNE_PASS_DX, TUNE_PASS_DVALS = 1, 2, 4

# name -> (restype, argtypes); the declarations of include/lb.h
VP, I32, I64, SZ = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
PLANP = ctypes.POINTER(ctypes.c_void_p)
SIGNATURES = {
    "lb_plan": (I32, [PLANP, VP, I32, I32, I32]),
    "lb_plan_ex": (I32, [PLANP, VP, I32, I32, I32, ctypes.POINTER(PlanOpts), VP]),
    "lb_plan_destroy": (None, [VP]),
    "lb_plan_get_info": (I32, [VP, ctypes.POINTER(PlanInfo)]),
    "lb_plan_splits": (I32, [VP, I32, VP, VP, SZ, ctypes.POINTER(SZ)]),
    "lb_spmv": (I32, [VP, VP, VP, VP, VP, VP]),
    "lb_prepare_backward": (I32, [VP, I32, VP, VP]),
    "lb_plan_transpose": (I32, [VP, VP, VP, VP, VP]),
    "lb_spmv_backward": (I32, [VP, I32, VP, VP, VP, VP, VP, VP, VP]),
    "lb_atom_tiles": (I32, [VP, VP, VP]),
    "lb_spmv_noalloc": (I32, [VP, I32, I32, VP, VP, VP, VP, VP]),
    "lb_status": (I32, [VP, VP]),
    "lb_autotune": (I32, [VP, I32, I32, VP, VP, VP, VP, ctypes.POINTER(TuneOpts), ctypes.POINTER(TuneResult), PLANP,
                          VP]),
    "lb_batch_autotune": (I32, [I32, VP, VP, VP, VP, VP, VP, VP, VP, VP, VP, VP, I32, ctypes.POINTER(TuneOpts),
                                ctypes.POINTER(BatchTuneResult), PLANP, VP]),
    "lb_autotune_cache_clear": (None, []),
    "lb_autotune_cache_size": (I32, []),
    "lb_autotune_cache_save": (I32, [ctypes.c_char_p]),
    "lb_autotune_cache_load": (I32, [ctypes.c_char_p, ctypes.POINTER(I32)]),
    "lb_coo_to_csr": (I32, [I32, I32, VP, VP, VP, VP, VP, VP, VP]),
    "lb_csc_to_csr": (I32, [I32, I32, I32, VP, VP, VP, VP, VP, VP, VP]),
    "lb_sssp": (I32, [VP, I32, I32, VP, VP, I32, I32, VP, ctypes.POINTER(I32), VP]),
    "lb_spmm": (I32, [VP, I32, VP, VP, VP, I64, VP, I64, VP]),
    "lb_prepare_spmm": (I32, [VP, VP]),
    "lb_batch_plan": (I32, [PLANP, I32, VP, VP, VP, VP, ctypes.POINTER(PlanOpts), VP]),
    "lb_batch_spmv": (I32, [VP, VP, VP, VP, VP, VP]),
    "lb_batch_prepare_backward": (I32, [VP, VP, VP]),
    "lb_batch_spmv_backward": (I32, [VP, VP, VP, VP, VP, VP, VP, VP]),
    "lb_heuristic_schedule": (I32, [I32, I32, I64]),
    "lb_merge_diagonals": (I32, [I64, I32, I32, VP, SZ, ctypes.POINTER(SZ), ctypes.POINTER(I32)]),
    "lb_probe_gather": (I32, [VP, VP, VP, I64, VP, I32, VP]),
    "lb_probe_gather_grid": (I32, []),
    "lb_probe_gather_tma": (I32, [VP, VP, VP, I64, I32, VP, I32, VP, VP]),
    "lb_probe_gather_tma_grid": (I32, []),
    "lb_selftest": (I32, [I32, VP]),
    "lb_status_string": (ctypes.c_char_p, [I32]),
    "lb_last_error": (ctypes.c_char_p, []),
    "lb_version": (I32, []),
}


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load liblb.so (building it in-tree first if sources changed)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        _build.build()
    path = _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"liblb.so not found at {path}: build it with paper_2301_04792_gb300.build.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(status: int, where: str):
    if status != 0:
        lib = load()
        raise LBError(status, where, lib.lb_last_error().decode(errors="replace"))
