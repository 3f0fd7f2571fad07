"""Load-balanced sparse matrix-vector multiply for GB300 (sm_103a).

GB300-native implementation of the data-parallel hot path of "A Programming
Model for GPU Load Balancing" (Osama, Porumbescu, Owens, PPoPP'23): CSR SpMV
with work stated as tiles (rows) of atoms (nonzeros), scheduled thread-mapped,
group-mapped (warp / block / any group size) or merge-path, plus a
differentiable backward and a batched persistent form.  The compute lives in
``liblb.so`` (C ABI ``include/lb.h``); this package marshals arguments.
"""
from .buildlib import build  # noqa: F401
from .lb import (BatchPlan, LBBatchSpMV, LBSpMV, Plan, Schedule, autotune, autotune_cache_clear,  # noqa: F401
                 autotune_cache_load, autotune_cache_save, autotune_cache_size, batch_autotune, batch_spmv, coo_to_csr, csc_to_csr,
                 heuristic_schedule, merge_diagonals, spmv, sssp)

__all__ = ["build", "Plan", "BatchPlan", "Schedule", "LBSpMV", "LBBatchSpMV", "spmv", "batch_spmv",
           "heuristic_schedule", "merge_diagonals", "autotune", "autotune_cache_clear", "autotune_cache_save",
           "autotune_cache_load", "autotune_cache_size", "batch_autotune", "sssp", "coo_to_csr", "csc_to_csr"]
