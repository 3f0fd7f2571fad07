"""PyTorch-facing wrapper of the load-balanced SpMV library.

PyTorch supplies device memory and streams; every step of SpMV, its backward,
the transpose and the plan runs in ``liblb.so``'s kernels through the C ABI
(``include/lb.h``).  Tensors must be CUDA, contiguous, int32 for indices and
float32 for values.
"""
from __future__ import annotations

import ctypes
from enum import IntEnum

import numpy as np
import torch

from . import _lib
from ._lib import BatchTuneResult, PlanInfo, PlanOpts, TuneOpts, TuneResult, check


class Schedule(IntEnum):
    """Load-balancing schedules (Sec. 4.2 and 5.2)."""
    THREAD_MAPPED = 0
    WARP_MAPPED = 1
    BLOCK_MAPPED = 2
    MERGE_PATH = 3
    GROUP_MAPPED = 4
    AUTO = 5

    @classmethod
    def parse(cls, s) -> "Schedule":
        if isinstance(s, Schedule):
            return s
        if isinstance(s, int):
            return cls(s)
        return cls[str(s).upper().replace("-", "_")]


def _stream(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _need(t: torch.Tensor, dtype, name: str, numel=None):
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} must have {numel} elements, got {t.numel()}")
    return t


def heuristic_schedule(rows: int, cols: int, nnz: int) -> Schedule:
    """Sec. 6.2 rule: merge-path unless (rows or cols < 500) and nnz < 10000."""
    return Schedule(_lib.load().lb_heuristic_schedule(int(rows), int(cols), int(nnz)))


def merge_diagonals(items: int, grid: int, items_per_tile: int):
    """(diagonals, tiles_per_cta) of a merge-path plan, computed on the host."""
    lib = _lib.load()
    cnt = ctypes.c_size_t(0)
    tpc = ctypes.c_int32(0)
    check(lib.lb_merge_diagonals(int(items), int(grid), int(items_per_tile), None, 0, ctypes.byref(cnt),
                                 ctypes.byref(tpc)), "lb_merge_diagonals")
    out = np.empty(cnt.value, dtype=np.int64)
    check(lib.lb_merge_diagonals(int(items), int(grid), int(items_per_tile),
                                 out.ctypes.data_as(ctypes.c_void_p), out.shape[0], ctypes.byref(cnt),
                                 ctypes.byref(tpc)), "lb_merge_diagonals")
    return out, int(tpc.value)


class Plan:
    """A plan for y = A x over one CSR tile set (tile_offsets = row offsets)."""

    def __init__(self, tile_offsets: torch.Tensor, num_atoms: int | None = None, schedule="merge_path",
                 num_cols: int = 0, items_per_thread: int = 0, group_size: int = 0, ctas_per_sm: int = 0,
                 validate: bool = False, mp_variant: int = 0, units_per_cta: int = 0, tiles_per_share: int = 0,
                 items_per_thread_t: int = 0, row_weight: int = 0, staged: bool = False, stream=None):
        self._lib = _lib.load()
        _need(tile_offsets, torch.int32, "tile_offsets")
        self.tile_offsets = tile_offsets
        self.num_tiles = tile_offsets.numel() - 1
        if self.num_tiles < 0:
            raise ValueError("tile_offsets needs at least one entry")
        if num_atoms is None:
            num_atoms = int(tile_offsets[-1].item()) if self.num_tiles > 0 else 0
        self.num_atoms = int(num_atoms)
        self.num_cols = int(num_cols)
        opts = PlanOpts(num_cols=int(num_cols), items_per_thread=int(items_per_thread), group_size=int(group_size),
                        ctas_per_sm=int(ctas_per_sm), validate=int(bool(validate)), mp_variant=int(mp_variant),
                        units_per_cta=int(units_per_cta), tiles_per_share=int(tiles_per_share),
                        items_per_thread_t=int(items_per_thread_t), row_weight=int(row_weight),
                        staged=int(bool(staged)))
        h = ctypes.c_void_p()
        check(self._lib.lb_plan_ex(ctypes.byref(h), _ptr(tile_offsets), self.num_tiles, self.num_atoms,
                                   int(Schedule.parse(schedule)), ctypes.byref(opts), ctypes.c_void_p(_stream(stream))),
              "lb_plan")
        self._h = h

    @classmethod
    def _adopt(cls, handle: ctypes.c_void_p, tile_offsets: torch.Tensor, num_atoms: int, num_cols: int) -> "Plan":
        """Wraps a plan handle made by the library (the autotuner's winner)."""
        self = cls.__new__(cls)
        self._lib = _lib.load()
        self.tile_offsets = tile_offsets
        self.num_tiles = tile_offsets.numel() - 1
        self.num_atoms = int(num_atoms)
        self.num_cols = int(num_cols)
        self._h = handle
        return self

    # ------------------------------------------------------------------ util
    @property
    def handle(self):
        if self._h is None:
            raise RuntimeError("plan destroyed")
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None:
            self._lib.lb_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> dict:
        inf = PlanInfo()
        check(self._lib.lb_plan_get_info(self.handle, ctypes.byref(inf)), "lb_plan_get_info")
        d = {f: getattr(inf, f) for f, _ in PlanInfo._fields_}
        d["schedule"] = Schedule(d["schedule"]).name.lower()
        return d

    def splits(self, which: int = 0):
        """(diagonals int64 [n], splits int32 [n, 2]) of the merge-path table."""
        cnt = ctypes.c_size_t(0)
        check(self._lib.lb_plan_splits(self.handle, int(which), None, None, 0, ctypes.byref(cnt)), "lb_plan_splits")
        d = np.empty(cnt.value, dtype=np.int64)
        ij = np.empty((cnt.value, 2), dtype=np.int32)
        check(self._lib.lb_plan_splits(self.handle, int(which), d.ctypes.data_as(ctypes.c_void_p),
                                       ij.ctypes.data_as(ctypes.c_void_p), cnt.value, ctypes.byref(cnt)),
              "lb_plan_splits")
        return d, ij

    def status(self, stream=None):
        check(self._lib.lb_status(self.handle, ctypes.c_void_p(_stream(stream))), "lb_status")

    # --------------------------------------------------------------- compute
    def spmv(self, col_idx: torch.Tensor, vals: torch.Tensor, x: torch.Tensor, y: torch.Tensor | None = None,
             stream=None) -> torch.Tensor:
        _need(col_idx, torch.int32, "col_idx", self.num_atoms)
        _need(vals, torch.float32, "vals", self.num_atoms)
        _need(x, torch.float32, "x")
        if y is None:
            y = torch.empty(self.num_tiles, dtype=torch.float32, device=x.device)
        _need(y, torch.float32, "y", self.num_tiles)
        check(self._lib.lb_spmv(self.handle, _ptr(col_idx), _ptr(vals), _ptr(x), _ptr(y),
                                ctypes.c_void_p(_stream(stream))), "lb_spmv")
        return y

    def spmm(self, col_idx: torch.Tensor, vals: torch.Tensor, B: torch.Tensor, C: torch.Tensor | None = None,
             stream=None) -> torch.Tensor:
        """C = A B (``lb_spmm``) for a dense B [num_cols, K] whose rows are contiguous
        (row stride >= K, unit column stride); C [num_tiles, K] likewise."""
        _need(col_idx, torch.int32, "col_idx", self.num_atoms)
        _need(vals, torch.float32, "vals", self.num_atoms)
        if not isinstance(B, torch.Tensor) or B.dim() != 2 or not B.is_cuda or B.dtype != torch.float32:
            raise TypeError("B must be a 2-D float32 CUDA tensor")
        if B.stride(1) != 1 or B.stride(0) < B.shape[1]:
            raise ValueError("B must have unit column stride and row stride >= its width")
        K = B.shape[1]
        if C is None:
            C = torch.empty(self.num_tiles, K, dtype=torch.float32, device=B.device)
        if C.dim() != 2 or C.shape != (self.num_tiles, K) or C.stride(1) != 1 or C.dtype != torch.float32:
            raise ValueError("C must be float32 [num_tiles, K] with unit column stride")
        check(self._lib.lb_spmm(self.handle, int(K), _ptr(col_idx), _ptr(vals), _ptr(B), int(B.stride(0)), _ptr(C),
                                int(C.stride(0)), ctypes.c_void_p(_stream(stream))), "lb_spmm")
        return C

    def prepare_backward(self, num_cols: int, col_idx: torch.Tensor, stream=None):
        _need(col_idx, torch.int32, "col_idx", self.num_atoms)
        check(self._lib.lb_prepare_backward(self.handle, int(num_cols), _ptr(col_idx),
                                            ctypes.c_void_p(_stream(stream))), "lb_prepare_backward")
        self.num_cols = int(num_cols)

    def transpose(self, stream=None):
        """(cp, riT, perm) of the cached transpose (after prepare_backward)."""
        dev = self.tile_offsets.device
        cp = torch.empty(self.num_cols + 1, dtype=torch.int32, device=dev)
        riT = torch.empty(self.num_atoms, dtype=torch.int32, device=dev)
        perm = torch.empty(self.num_atoms, dtype=torch.int32, device=dev)
        check(self._lib.lb_plan_transpose(self.handle, _ptr(cp), _ptr(riT), _ptr(perm),
                                          ctypes.c_void_p(_stream(stream))), "lb_plan_transpose")
        return cp, riT, perm

    def backward(self, num_cols: int, col_idx, vals, x, dy, want_dx=True, want_dvals=True, dx=None, dvals=None,
                 stream=None):
        dev = dy.device
        _need(dy, torch.float32, "dy", self.num_tiles)
        if want_dx and dx is None:
            dx = torch.empty(int(num_cols), dtype=torch.float32, device=dev)
        if want_dvals and dvals is None:
            dvals = torch.empty(self.num_atoms, dtype=torch.float32, device=dev)
        check(self._lib.lb_spmv_backward(self.handle, int(num_cols), _ptr(col_idx), _ptr(vals), _ptr(x), _ptr(dy),
                                         _ptr(dx) if want_dx else None, _ptr(dvals) if want_dvals else None,
                                         ctypes.c_void_p(_stream(stream))), "lb_spmv_backward")
        self.num_cols = int(num_cols)
        return (dx if want_dx else None), (dvals if want_dvals else None)

    def atom_tiles(self, out=None, stream=None) -> torch.Tensor:
        if out is None:
            out = torch.empty(self.num_atoms, dtype=torch.int32, device=self.tile_offsets.device)
        check(self._lib.lb_atom_tiles(self.handle, _ptr(out), ctypes.c_void_p(_stream(stream))), "lb_atom_tiles")
        return out


def _candidate_name(c) -> str:
    s = Schedule(c.schedule)
    if s == Schedule.THREAD_MAPPED and c.staged:
        return "thread_mapped_staged"
    if s == Schedule.MERGE_PATH:
        u = f"_u{c.units_per_cta}" if c.units_per_cta > 1 else ""
        w = f"_w{c.row_weight}" if c.row_weight > 1 else ""
        return f"merge_path_ipt{c.items_per_thread}_v{c.mp_variant}{u}{w}"
    if s == Schedule.GROUP_MAPPED:
        return f"group_mapped_g{c.group_size}"
    return s.name.lower()


def autotune(tile_offsets: torch.Tensor, col_idx: torch.Tensor, vals: torch.Tensor, x: torch.Tensor,
             num_cols: int | None = None, y: torch.Tensor | None = None, reps: int = 0, prune_factor: float = 0.0,
             cold_l2: bool = False, use_cache: bool = True, families: int = 0, stream=None):
    """Times every candidate schedule on this matrix (``lb_autotune``) and returns
    ``(plan, report)``: the winner's Plan and a dict with the timed table.  ``y``
    (allocated if None) holds A x by the winner afterwards (``report["y"]``)."""
    lib = _lib.load()
    _need(tile_offsets, torch.int32, "tile_offsets")
    R = tile_offsets.numel() - 1
    N = int(col_idx.numel())
    _need(col_idx, torch.int32, "col_idx")
    _need(vals, torch.float32, "vals", N)
    _need(x, torch.float32, "x")
    C = int(x.numel()) if num_cols is None else int(num_cols)
    if y is None:
        y = torch.empty(R, dtype=torch.float32, device=x.device)
    _need(y, torch.float32, "y", R)
    o = TuneOpts(num_cols=C, reps=int(reps), prune_factor=float(prune_factor), cold_l2=int(bool(cold_l2)),
                 no_cache=int(not use_cache), families=int(families))
    res = TuneResult()
    h = ctypes.c_void_p()
    check(lib.lb_autotune(_ptr(tile_offsets), R, N, _ptr(col_idx), _ptr(vals), _ptr(x), _ptr(y), ctypes.byref(o),
                          ctypes.byref(res), ctypes.byref(h), ctypes.c_void_p(_stream(stream))), "lb_autotune")
    cands = []
    for i in range(res.num_candidates):
        c = res.candidates[i]
        cands.append({"name": _candidate_name(c), "schedule": Schedule(c.schedule).name.lower(),
                      "items_per_thread": c.items_per_thread, "group_size": c.group_size,
                      "mp_variant": c.mp_variant, "units_per_cta": c.units_per_cta, "row_weight": c.row_weight,
                      "staged": c.staged,
                      "ms": c.ms, "gbps": c.gbps, "reps": c.reps, "status": c.status})
    report = {"candidates": cands, "best": cands[res.best]["name"],
              "heuristic": cands[res.heuristic]["name"] if res.heuristic >= 0 else None,
              "from_cache": bool(res.from_cache), "best_schedule": Schedule(res.best_schedule).name.lower(),
              "best_opts": {f: getattr(res.best_opts, f) for f, _ in PlanOpts._fields_},
              "y": y}
    return Plan._adopt(h, tile_offsets, N, C), report


def coo_to_csr(num_rows: int, row_idx: torch.Tensor, col_idx: torch.Tensor, vals: torch.Tensor, stream=None):
    """(tile_offsets, col_idx, vals) of a COO matrix as a CSR tile set (``lb_coo_to_csr``)."""
    lib = _lib.load()
    N = int(row_idx.numel())
    _need(row_idx, torch.int32, "row_idx")
    _need(col_idx, torch.int32, "col_idx", N)
    _need(vals, torch.float32, "vals", N)
    dev = row_idx.device
    rp = torch.empty(int(num_rows) + 1, dtype=torch.int32, device=dev)
    ci = torch.empty(N, dtype=torch.int32, device=dev)
    v = torch.empty(N, dtype=torch.float32, device=dev)
    check(lib.lb_coo_to_csr(int(num_rows), N, _ptr(row_idx), _ptr(col_idx), _ptr(vals), _ptr(rp), _ptr(ci), _ptr(v),
                            ctypes.c_void_p(_stream(stream))), "lb_coo_to_csr")
    return rp, ci, v


def csc_to_csr(num_rows: int, col_offsets: torch.Tensor, row_idx: torch.Tensor, vals: torch.Tensor, stream=None):
    """(tile_offsets, col_idx, vals) of a CSC matrix as a CSR tile set (``lb_csc_to_csr``)."""
    lib = _lib.load()
    _need(col_offsets, torch.int32, "col_offsets")
    C = col_offsets.numel() - 1
    N = int(row_idx.numel())
    _need(row_idx, torch.int32, "row_idx")
    _need(vals, torch.float32, "vals", N)
    dev = col_offsets.device
    rp = torch.empty(int(num_rows) + 1, dtype=torch.int32, device=dev)
    ci = torch.empty(N, dtype=torch.int32, device=dev)
    v = torch.empty(N, dtype=torch.float32, device=dev)
    check(lib.lb_csc_to_csr(int(num_rows), C, N, _ptr(col_offsets), _ptr(row_idx), _ptr(vals), _ptr(rp), _ptr(ci),
                            _ptr(v), ctypes.c_void_p(_stream(stream))), "lb_csc_to_csr")
    return rp, ci, v


def sssp(tile_offsets: torch.Tensor, col_idx: torch.Tensor, weights: torch.Tensor, source: int, group_size: int = 0,
         dist: torch.Tensor | None = None, stream=None):
    """Single-source shortest paths (``lb_sssp``, Listing 5): returns (dist, iterations)."""
    lib = _lib.load()
    _need(tile_offsets, torch.int32, "tile_offsets")
    V = tile_offsets.numel() - 1
    E = int(col_idx.numel())
    _need(col_idx, torch.int32, "col_idx")
    _need(weights, torch.float32, "weights", E)
    if dist is None:
        dist = torch.empty(V, dtype=torch.float32, device=tile_offsets.device)
    _need(dist, torch.float32, "dist", V)
    it = ctypes.c_int32(0)
    check(lib.lb_sssp(_ptr(tile_offsets), V, E, _ptr(col_idx), _ptr(weights), int(source), int(group_size),
                      _ptr(dist), ctypes.byref(it), ctypes.c_void_p(_stream(stream))), "lb_sssp")
    return dist, int(it.value)


def autotune_cache_clear():
    """Empties the autotuner's in-memory cache (files are not touched)."""
    _lib.load().lb_autotune_cache_clear()


def autotune_cache_size() -> int:
    return int(_lib.load().lb_autotune_cache_size())


def autotune_cache_save(path: str):
    """Writes the autotuner's cache to ``path`` (one JSON object per line)."""
    check(_lib.load().lb_autotune_cache_save(str(path).encode()), "lb_autotune_cache_save")


def autotune_cache_load(path: str) -> int:
    """Merges the entries of a file written by autotune_cache_save; returns how many were taken."""
    n = ctypes.c_int32(0)
    check(_lib.load().lb_autotune_cache_load(str(path).encode(), ctypes.byref(n)), "lb_autotune_cache_load")
    return int(n.value)


class BatchPlan:
    """One persistent merge-path plan over a batch of CSR matrices."""

    def __init__(self, rows, cols, nnz, rp_cat: torch.Tensor, items_per_thread: int = 0, ctas_per_sm: int = 0,
                 mp_variant: int = 0, wave_items: int = 0, units_per_cta: int = 0, tiles_per_share: int = 0,
                 items_per_thread_t: int = 0, stream=None):
        """mp_variant 0 walks a long batch in waves of whole matrices; mp_variant 3
        (look-back shares, capped at 8 tiles) with items_per_thread 4 measured
        fastest for fwd + bwd of many large matrices on GB300."""
        self._lib = _lib.load()
        _need(rp_cat, torch.int32, "rp_cat")
        self.rows = np.ascontiguousarray(rows, dtype=np.int32)
        self.cols = np.ascontiguousarray(cols, dtype=np.int32)
        self.nnz = np.ascontiguousarray(nnz, dtype=np.int64)
        if not (self.rows.shape == self.cols.shape == self.nnz.shape):
            raise ValueError("rows, cols, nnz must have the same length")
        if rp_cat.numel() != int(self.rows.sum()) + self.rows.shape[0]:
            raise ValueError("rp_cat must hold rows[m] + 1 offsets per matrix")
        self.rp_cat = rp_cat
        self.total_rows = int(self.rows.sum())
        self.total_cols = int(self.cols.sum())
        self.total_nnz = int(self.nnz.sum())
        opts = PlanOpts(items_per_thread=int(items_per_thread), ctas_per_sm=int(ctas_per_sm),
                        mp_variant=int(mp_variant), wave_items=int(wave_items), units_per_cta=int(units_per_cta),
                        tiles_per_share=int(tiles_per_share), items_per_thread_t=int(items_per_thread_t))
        h = ctypes.c_void_p()
        check(self._lib.lb_batch_plan(ctypes.byref(h), self.rows.shape[0], self.rows.ctypes.data_as(ctypes.c_void_p),
                                      self.cols.ctypes.data_as(ctypes.c_void_p),
                                      self.nnz.ctypes.data_as(ctypes.c_void_p), _ptr(rp_cat), ctypes.byref(opts),
                                      ctypes.c_void_p(_stream(stream))), "lb_batch_plan")
        self._h = h

    @classmethod
    def _adopt(cls, handle: ctypes.c_void_p, rows, cols, nnz, rp_cat: torch.Tensor) -> "BatchPlan":
        """Wraps a batch plan handle made by the library (the batch autotuner's winner)."""
        self = cls.__new__(cls)
        self._lib = _lib.load()
        self.rows = np.ascontiguousarray(rows, dtype=np.int32)
        self.cols = np.ascontiguousarray(cols, dtype=np.int32)
        self.nnz = np.ascontiguousarray(nnz, dtype=np.int64)
        self.rp_cat = rp_cat
        self.total_rows = int(self.rows.sum())
        self.total_cols = int(self.cols.sum())
        self.total_nnz = int(self.nnz.sum())
        self._h = handle
        return self

    @property
    def handle(self):
        if self._h is None:
            raise RuntimeError("plan destroyed")
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None:
            self._lib.lb_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> dict:
        inf = PlanInfo()
        check(self._lib.lb_plan_get_info(self.handle, ctypes.byref(inf)), "lb_plan_get_info")
        return {f: getattr(inf, f) for f, _ in PlanInfo._fields_}

    def spmv(self, col_cat, vals_cat, x_cat, y_cat=None, stream=None):
        _need(col_cat, torch.int32, "col_cat", self.total_nnz)
        _need(vals_cat, torch.float32, "vals_cat", self.total_nnz)
        _need(x_cat, torch.float32, "x_cat", self.total_cols)
        if y_cat is None:
            y_cat = torch.empty(self.total_rows, dtype=torch.float32, device=x_cat.device)
        _need(y_cat, torch.float32, "y_cat", self.total_rows)
        check(self._lib.lb_batch_spmv(self.handle, _ptr(col_cat), _ptr(vals_cat), _ptr(x_cat), _ptr(y_cat),
                                      ctypes.c_void_p(_stream(stream))), "lb_batch_spmv")
        return y_cat

    def prepare_backward(self, col_cat, stream=None):
        _need(col_cat, torch.int32, "col_cat", self.total_nnz)
        check(self._lib.lb_batch_prepare_backward(self.handle, _ptr(col_cat), ctypes.c_void_p(_stream(stream))),
              "lb_batch_prepare_backward")

    def backward(self, col_cat, vals_cat, x_cat, dy_cat, want_dx=True, want_dvals=True, dx_cat=None, dvals_cat=None,
                 stream=None):
        dev = dy_cat.device
        _need(dy_cat, torch.float32, "dy_cat", self.total_rows)
        if want_dx and dx_cat is None:
            dx_cat = torch.empty(self.total_cols, dtype=torch.float32, device=dev)
        if want_dvals and dvals_cat is None:
            dvals_cat = torch.empty(self.total_nnz, dtype=torch.float32, device=dev)
        check(self._lib.lb_batch_spmv_backward(self.handle, _ptr(col_cat), _ptr(vals_cat), _ptr(x_cat), _ptr(dy_cat),
                                               _ptr(dx_cat) if want_dx else None,
                                               _ptr(dvals_cat) if want_dvals else None,
                                               ctypes.c_void_p(_stream(stream))), "lb_batch_spmv_backward")
        return (dx_cat if want_dx else None), (dvals_cat if want_dvals else None)

    def atom_tiles(self, out=None, stream=None):
        if out is None:
            out = torch.empty(self.total_nnz, dtype=torch.int32, device=self.rp_cat.device)
        check(self._lib.lb_atom_tiles(self.handle, _ptr(out), ctypes.c_void_p(_stream(stream))), "lb_atom_tiles")
        return out


def _batch_candidate_name(o) -> str:
    s = f"batch_ipt{o.items_per_thread}_v{o.mp_variant}"
    if o.tiles_per_share > 1:
        s += f"_tps{o.tiles_per_share}"
    if o.units_per_cta > 1:
        s += f"_u{o.units_per_cta}"
    if o.wave_items:
        s += f"_wave{o.wave_items}"
    return s


def batch_autotune(rows, cols, nnz, rp_cat: torch.Tensor, col_cat: torch.Tensor, vals_cat: torch.Tensor,
                   x_cat: torch.Tensor, dy_cat: torch.Tensor | None = None, passes: str = "fwd", y_cat=None,
                   dx_cat=None, dvals_cat=None, reps: int = 0, cold_l2: bool = False, use_cache: bool = True,
                   stream=None):
    """Times the batch plan candidates (``lb_batch_autotune``) over the passes named in
    ``passes`` ("fwd", "dx", "dvals" joined by "+", e.g. "fwd+dx+dvals") and returns
    ``(plan, report)``: the winner's BatchPlan and a dict with the timed table and the
    outputs of the timed passes by the winner."""
    lib = _lib.load()
    rows = np.ascontiguousarray(rows, dtype=np.int32)
    cols = np.ascontiguousarray(cols, dtype=np.int32)
    nnz = np.ascontiguousarray(nnz, dtype=np.int64)
    R, C, N = int(rows.sum()), int(cols.sum()), int(nnz.sum())
    bits = {"fwd": _lib.TUNE_PASS_FWD, "dx": _lib.TUNE_PASS_DX, "dvals": _lib.TUNE_PASS_DVALS}
    mask = 0
    for part in str(passes).split("+"):
        mask |= bits[part.strip()]
    _need(rp_cat, torch.int32, "rp_cat", R + rows.shape[0])
    _need(col_cat, torch.int32, "col_cat", N)
    _need(vals_cat, torch.float32, "vals_cat", N)
    _need(x_cat, torch.float32, "x_cat", C)
    dev = x_cat.device
    if mask & _lib.TUNE_PASS_FWD and y_cat is None:
        y_cat = torch.empty(R, dtype=torch.float32, device=dev)
    if mask & (_lib.TUNE_PASS_DX | _lib.TUNE_PASS_DVALS):
        _need(dy_cat, torch.float32, "dy_cat", R)
    if mask & _lib.TUNE_PASS_DX and dx_cat is None:
        dx_cat = torch.empty(C, dtype=torch.float32, device=dev)
    if mask & _lib.TUNE_PASS_DVALS and dvals_cat is None:
        dvals_cat = torch.empty(N, dtype=torch.float32, device=dev)
    o = TuneOpts(reps=int(reps), cold_l2=int(bool(cold_l2)), no_cache=int(not use_cache))
    res = BatchTuneResult()
    h = ctypes.c_void_p()
    check(lib.lb_batch_autotune(rows.shape[0], rows.ctypes.data_as(ctypes.c_void_p),
                                cols.ctypes.data_as(ctypes.c_void_p), nnz.ctypes.data_as(ctypes.c_void_p),
                                _ptr(rp_cat), _ptr(col_cat), _ptr(vals_cat), _ptr(x_cat), _ptr(y_cat), _ptr(dy_cat),
                                _ptr(dx_cat), _ptr(dvals_cat), mask, ctypes.byref(o), ctypes.byref(res),
                                ctypes.byref(h), ctypes.c_void_p(_stream(stream))), "lb_batch_autotune")
    cands = []
    for i in range(res.num_candidates):
        c = res.candidates[i]
        cands.append({"name": _batch_candidate_name(c.opts), "ms": c.ms, "gbps": c.gbps, "reps": c.reps,
                      "status": c.status,
                      "opts": {f: getattr(c.opts, f) for f, _ in PlanOpts._fields_}})
    report = {"candidates": cands, "best": cands[res.best]["name"], "from_cache": bool(res.from_cache),
              "passes": passes, "best_opts": {f: getattr(res.best_opts, f) for f, _ in PlanOpts._fields_},
              "y": y_cat, "dx": dx_cat, "dvals": dvals_cat}
    return BatchPlan._adopt(h, rows, cols, nnz, rp_cat), report


class LBSpMV(torch.autograd.Function):
    """y = A x with A in CSR (values differentiable) and x differentiable.

    forward runs lb_spmv; backward runs lb_spmv_backward, which gives
    dx = A^T dy (the plan's schedule over the cached transpose) and
    dvals[k] = dy[row(k)] x[col(k)].
    """

    @staticmethod
    def forward(ctx, plan: Plan, col_idx, vals, x):
        y = plan.spmv(col_idx, vals.detach(), x.detach())
        ctx.plan = plan
        ctx.save_for_backward(col_idx, vals, x)
        return y

    @staticmethod
    def backward(ctx, dy):
        col_idx, vals, x = ctx.saved_tensors
        plan: Plan = ctx.plan
        want_dvals = ctx.needs_input_grad[2]
        want_dx = ctx.needs_input_grad[3]
        dx, dvals = plan.backward(x.numel(), col_idx, vals.detach(), x.detach(), dy.contiguous(), want_dx=want_dx,
                                  want_dvals=want_dvals)
        return None, None, dvals, dx


class LBBatchSpMV(torch.autograd.Function):
    """Batched y_cat = blockdiag(A_m) x_cat with the same gradients as LBSpMV."""

    @staticmethod
    def forward(ctx, plan: BatchPlan, col_cat, vals_cat, x_cat):
        y = plan.spmv(col_cat, vals_cat.detach(), x_cat.detach())
        ctx.plan = plan
        ctx.save_for_backward(col_cat, vals_cat, x_cat)
        return y

    @staticmethod
    def backward(ctx, dy):
        col_cat, vals_cat, x_cat = ctx.saved_tensors
        dx, dvals = ctx.plan.backward(col_cat, vals_cat.detach(), x_cat.detach(), dy.contiguous(),
                                      want_dx=ctx.needs_input_grad[3], want_dvals=ctx.needs_input_grad[2])
        return None, None, dvals, dx


def spmv(plan: Plan, col_idx, vals, x):
    """Differentiable y = A x through the plan."""
    return LBSpMV.apply(plan, col_idx, vals, x)


def batch_spmv(plan: BatchPlan, col_cat, vals_cat, x_cat):
    return LBBatchSpMV.apply(plan, col_cat, vals_cat, x_cat)
