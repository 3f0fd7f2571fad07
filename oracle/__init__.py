"""ORACLE -- test infrastructure only.

Python wrapper around ``oracle.c``: plain FP64 CPU implementations of what the
load-balanced SpMV path computes (SpMV, merge-path splits, the merged work
list, atom->tile mapping, get_tile, the stable CSR->CSC transpose, and the
gradients of y = A x).  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library and never calls it.

Parity is pinned for every function here by the ``-m "not gpu"`` tests in
``tests/test_oracle_pins.py`` (dense brute force, closed forms, invariants,
brute-force merges); no function is unpinned.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

# Acceptance bound for FP32 results against the FP64 oracle: |y - y64| <= TOL * b,
# b = sum |a_ij x_j| over the row (or column for dx).
TOL = 1e-5


def _build_lib(force: bool = False) -> str:
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O1", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` in-tree (plain gcc)."""
    global _lib
    with _lock:
        path = _build_lib(force)
        _lib = None
    return path


def _bind(lib):
    i8p = ctypes.POINTER(ctypes.c_int8)
    i32p = ctypes.POINTER(ctypes.c_int32)
    i64p = ctypes.POINTER(ctypes.c_int64)
    f32p = ctypes.POINTER(ctypes.c_float)
    f64p = ctypes.POINTER(ctypes.c_double)
    lib.or_spmv.argtypes = [ctypes.c_int32, i32p, i32p, f32p, f32p, f64p, f64p]
    lib.or_spmv_rows.argtypes = [ctypes.c_int64, i64p, i32p, i32p, f32p, f32p, f64p, f64p]
    lib.or_coo_to_csr.argtypes = [ctypes.c_int32, ctypes.c_int64, i32p, i32p, i32p, i32p, i32p]
    lib.or_sssp.argtypes = [ctypes.c_int32, i32p, i32p, f32p, ctypes.c_int32, f32p]
    lib.or_sssp.restype = ctypes.c_int32
    lib.or_spmm.argtypes = [ctypes.c_int32, i32p, i32p, f32p, f32p, ctypes.c_int64, ctypes.c_int32, f64p, f64p]
    lib.or_merge_split.argtypes = [ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, i32p]
    lib.or_merge_split.restype = ctypes.c_int32
    lib.or_merge_splits.argtypes = [ctypes.c_int64, i64p, ctypes.c_int32, ctypes.c_int32, i32p, i32p]
    lib.or_merge_sequence.argtypes = [ctypes.c_int32, ctypes.c_int32, i32p, i8p, i32p]
    lib.or_weighted_diagonals.argtypes = [ctypes.c_int32, ctypes.c_int32, i32p, ctypes.c_int32, ctypes.c_int32,
                                          ctypes.c_int32, ctypes.c_int32, i64p]
    lib.or_row_of_atom.argtypes = [ctypes.c_int32, i32p, i32p]
    lib.or_get_tile.argtypes = [i32p, ctypes.c_int32, ctypes.c_int32]
    lib.or_get_tile.restype = ctypes.c_int32
    lib.or_transpose.argtypes = [ctypes.c_int32, ctypes.c_int32, i32p, i32p, i32p, i32p, i32p]
    lib.or_grad.argtypes = [ctypes.c_int32, ctypes.c_int32, i32p, i32p, f32p, f32p, f32p, f64p, f64p, f32p]
    return lib


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _p(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


class Oracle:
    """The oracle's functions bound to one compiled copy of ``oracle.c``.

    The module-level functions use the in-tree build; tests may bind a second
    copy (for instance one compiled from a deliberately broken source) to show
    that the pins catch the mistake.
    """

    def __init__(self, lib_path: str):
        self.lib = _bind(ctypes.CDLL(lib_path))

    def spmv(self, rp, ci, v, x):
        """(y64, b): y = A x in FP64 and b[i] = sum_k |v[k] x[ci[k]]|."""
        rp, ci, v, x = _c(rp, np.int32), _c(ci, np.int32), _c(v, np.float32), _c(x, np.float32)
        R = rp.shape[0] - 1
        y = np.empty(R, dtype=np.float64)
        b = np.empty(R, dtype=np.float64)
        self.lib.or_spmv(R, _p(rp, ctypes.c_int32), _p(ci, ctypes.c_int32), _p(v, ctypes.c_float),
                         _p(x, ctypes.c_float), _p(y, ctypes.c_double), _p(b, ctypes.c_double))
        return y, b

    def spmm(self, rp, ci, v, B):
        """(C64, b), both [R, K]: C = A B in FP64 for a dense row-major B [num_cols, K] and
        b[i, j] = sum_k |v[k] B[ci[k], j]|."""
        rp, ci, v = _c(rp, np.int32), _c(ci, np.int32), _c(v, np.float32)
        B = _c(B, np.float32)
        R, K = rp.shape[0] - 1, B.shape[1]
        C = np.empty((R, K), dtype=np.float64)
        b = np.empty((R, K), dtype=np.float64)
        self.lib.or_spmm(R, _p(rp, ctypes.c_int32), _p(ci, ctypes.c_int32), _p(v, ctypes.c_float),
                         _p(B, ctypes.c_float), K, K, _p(C, ctypes.c_double), _p(b, ctypes.c_double))
        return C, b

    def sssp(self, rp, ci, w, source: int):
        """float32 [V] shortest distances from `source` (+inf if unreachable), Listing 5's float
        arithmetic, by Dijkstra's algorithm."""
        rp, ci, w = _c(rp, np.int32), _c(ci, np.int32), _c(w, np.float32)
        V = rp.shape[0] - 1
        dist = np.empty(V, dtype=np.float32)
        self.lib.or_sssp(V, _p(rp, ctypes.c_int32), _p(ci, ctypes.c_int32), _p(w, ctypes.c_float), int(source),
                         _p(dist, ctypes.c_float))
        return dist

    def spmv_threads(self, rp, ci, v, x, threads: int):
        """(y64, b) as spmv, the rows cut into `threads` blocks of about equal rows + atoms,
        each block run by or_spmv on its own host thread (ctypes releases the GIL); every
        row is summed exactly as in spmv, so the results are identical."""
        import threading
        rp, ci, v, x = _c(rp, np.int32), _c(ci, np.int32), _c(v, np.float32), _c(x, np.float32)
        R = rp.shape[0] - 1
        y = np.empty(R, dtype=np.float64)
        b = np.empty(R, dtype=np.float64)
        T = max(1, min(int(threads), max(R, 1)))
        work = rp.astype(np.int64) + np.arange(R + 1, dtype=np.int64)  # rows + atoms before each row
        cuts = np.searchsorted(work, np.linspace(0, work[-1], T + 1), side="left").clip(0, R)
        cuts[0], cuts[-1] = 0, R

        def block(r0, r1):
            if r1 > r0:
                self.lib.or_spmv(int(r1 - r0), _p(rp[r0:], ctypes.c_int32), _p(ci, ctypes.c_int32),
                                 _p(v, ctypes.c_float), _p(x, ctypes.c_float), _p(y[r0:], ctypes.c_double),
                                 _p(b[r0:], ctypes.c_double))

        ts = [threading.Thread(target=block, args=(int(cuts[t]), int(cuts[t + 1]))) for t in range(T)]
        for t in ts:
            t.start()
        for t in ts:
            t.join()
        return y, b

    def spmv_rows(self, rows, rp, ci, v, x):
        """(y64, b) for the selected rows only."""
        rows = _c(rows, np.int64)
        rp, ci, v, x = _c(rp, np.int32), _c(ci, np.int32), _c(v, np.float32), _c(x, np.float32)
        n = rows.shape[0]
        y = np.empty(n, dtype=np.float64)
        b = np.empty(n, dtype=np.float64)
        self.lib.or_spmv_rows(n, _p(rows, ctypes.c_int64), _p(rp, ctypes.c_int32), _p(ci, ctypes.c_int32),
                              _p(v, ctypes.c_float), _p(x, ctypes.c_float), _p(y, ctypes.c_double),
                              _p(b, ctypes.c_double))
        return y, b

    def merge_split(self, d, rp):
        rp = _c(rp, np.int32)
        R = rp.shape[0] - 1
        i = self.lib.or_merge_split(int(d), R, int(rp[-1]), _p(rp, ctypes.c_int32))
        return int(i), int(d) - int(i)

    def merge_splits(self, diags, rp):
        """int32 [n, 2] array of (i, j) for each diagonal."""
        diags = _c(diags, np.int64)
        rp = _c(rp, np.int32)
        R = rp.shape[0] - 1
        out = np.empty((diags.shape[0], 2), dtype=np.int32)
        self.lib.or_merge_splits(diags.shape[0], _p(diags, ctypes.c_int64), R, int(rp[-1]),
                                 _p(rp, ctypes.c_int32), _p(out, ctypes.c_int32))
        return out

    def merge_sequence(self, rp):
        """(kind, idx): the merged work list, kind 0 = row end, 1 = atom."""
        rp = _c(rp, np.int32)
        R = rp.shape[0] - 1
        N = int(rp[-1])
        kind = np.empty(R + N, dtype=np.int8)
        idx = np.empty(R + N, dtype=np.int32)
        self.lib.or_merge_sequence(R, N, _p(rp, ctypes.c_int32), _p(kind, ctypes.c_int8), _p(idx, ctypes.c_int32))
        return kind, idx

    def weighted_diagonals(self, rp, w: int, shares: int, items_per_tile: int, tiles_per_share: int):
        """int64 [shares * (tiles_per_share + 1)]: table diagonals with row ends weighted w."""
        rp = _c(rp, np.int32)
        R = rp.shape[0] - 1
        out = np.empty(shares * (tiles_per_share + 1), dtype=np.int64)
        self.lib.or_weighted_diagonals(R, int(rp[-1]), _p(rp, ctypes.c_int32), int(w), int(shares),
                                       int(items_per_tile), int(tiles_per_share), _p(out, ctypes.c_int64))
        return out

    def row_of_atom(self, rp):
        rp = _c(rp, np.int32)
        R = rp.shape[0] - 1
        out = np.empty(int(rp[-1]), dtype=np.int32)
        self.lib.or_row_of_atom(R, _p(rp, ctypes.c_int32), _p(out, ctypes.c_int32))
        return out

    def get_tile(self, prefix, a):
        prefix = _c(prefix, np.int32)
        n = prefix.shape[0] - 1
        return int(self.lib.or_get_tile(_p(prefix, ctypes.c_int32), n, int(a)))

    def transpose(self, rp, ci, num_cols):
        """(cp, riT, perm) of the stable counting-sort CSR->CSC transpose."""
        rp, ci = _c(rp, np.int32), _c(ci, np.int32)
        R = rp.shape[0] - 1
        N = int(rp[-1])
        cp = np.empty(num_cols + 1, dtype=np.int32)
        riT = np.empty(N, dtype=np.int32)
        perm = np.empty(N, dtype=np.int32)
        self.lib.or_transpose(R, int(num_cols), _p(rp, ctypes.c_int32), _p(ci, ctypes.c_int32),
                              _p(cp, ctypes.c_int32), _p(riT, ctypes.c_int32), _p(perm, ctypes.c_int32))
        return cp, riT, perm

    def coo_to_csr(self, num_rows, row, col, val):
        """(rp, ci, v) of the COO atoms (row[k], col[k], val[k]) as a CSR tile set; atoms of a
        row keep their input order."""
        row, col, val = _c(row, np.int32), _c(col, np.int32), _c(val, np.float32)
        N = row.shape[0]
        rp = np.empty(num_rows + 1, dtype=np.int32)
        ci = np.empty(N, dtype=np.int32)
        perm = np.empty(N, dtype=np.int32)
        self.lib.or_coo_to_csr(int(num_rows), N, _p(row, ctypes.c_int32), _p(col, ctypes.c_int32),
                               _p(rp, ctypes.c_int32), _p(ci, ctypes.c_int32), _p(perm, ctypes.c_int32))
        return rp, ci, val[perm]

    def csc_to_csr(self, num_rows, cp, ri, val):
        """(rp, ci, v) of a CSC matrix (column offsets cp, row ids ri) as a CSR tile set: the
        CSC arrays read as the CSR of A^T, transposed by the stable counting sort (columns
        ascend within each row)."""
        cp, ri, val = _c(cp, np.int32), _c(ri, np.int32), _c(val, np.float32)
        rp, ci, perm = self.transpose(cp, ri, num_rows)
        return rp, ci, val[perm]

    def grad(self, rp, ci, v, x, dy, num_cols, want_dx=True, want_dvals=True):
        """(dx64, bx, dvals32) for L = dy . (A x)."""
        rp, ci, v, x, dy = (_c(rp, np.int32), _c(ci, np.int32), _c(v, np.float32), _c(x, np.float32),
                            _c(dy, np.float32))
        R = rp.shape[0] - 1
        N = int(rp[-1])
        dx = np.empty(num_cols, dtype=np.float64) if want_dx else None
        bx = np.empty(num_cols, dtype=np.float64) if want_dx else None
        dv = np.empty(N, dtype=np.float32) if want_dvals else None
        self.lib.or_grad(R, int(num_cols), _p(rp, ctypes.c_int32), _p(ci, ctypes.c_int32), _p(v, ctypes.c_float),
                         _p(x, ctypes.c_float), _p(dy, ctypes.c_float),
                         _p(dx, ctypes.c_double) if want_dx else None, _p(bx, ctypes.c_double) if want_dx else None,
                         _p(dv, ctypes.c_float) if want_dvals else None)
        return dx, bx, dv


def default() -> Oracle:
    global _lib
    with _lock:
        if _lib is None:
            _lib = Oracle(_build_lib())
        return _lib


def spmv(rp, ci, v, x):
    return default().spmv(rp, ci, v, x)


def spmv_rows(rows, rp, ci, v, x):
    return default().spmv_rows(rows, rp, ci, v, x)


def spmv_threads(rp, ci, v, x, threads: int):
    return default().spmv_threads(rp, ci, v, x, threads)


def spmm(rp, ci, v, B):
    return default().spmm(rp, ci, v, B)


def sssp(rp, ci, w, source: int):
    return default().sssp(rp, ci, w, source)


def merge_split(d, rp):
    return default().merge_split(d, rp)


def merge_splits(diags, rp):
    return default().merge_splits(diags, rp)


def merge_sequence(rp):
    return default().merge_sequence(rp)


def row_of_atom(rp):
    return default().row_of_atom(rp)


def weighted_diagonals(rp, w, shares, items_per_tile, tiles_per_share):
    return default().weighted_diagonals(rp, w, shares, items_per_tile, tiles_per_share)


def get_tile(prefix, a):
    return default().get_tile(prefix, a)


def transpose(rp, ci, num_cols):
    return default().transpose(rp, ci, num_cols)


def grad(rp, ci, v, x, dy, num_cols, want_dx=True, want_dvals=True):
    return default().grad(rp, ci, v, x, dy, num_cols, want_dx, want_dvals)


def coo_to_csr(num_rows, row, col, val):
    return default().coo_to_csr(num_rows, row, col, val)


def csc_to_csr(num_rows, cp, ri, val):
    return default().csc_to_csr(num_rows, cp, ri, val)


def source_path() -> str:
    return _SRC


def within_bound(y32, y64, b, tol=TOL):
    """Boolean mask of entries with |y32 - y64| <= tol * b (exact when b == 0)."""
    y32 = np.asarray(y32, dtype=np.float64)
    return np.abs(y32 - y64) <= tol * b
