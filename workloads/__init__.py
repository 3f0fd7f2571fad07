"""Seeded synthetic CSR workloads (no method arithmetic lives here).

Every generator returns plain numpy arrays: ``rp`` (int32 row offsets, R+1),
``ci`` (int32 column indices, sorted and distinct within each row), ``v``
(float32 values) and dense float32 vectors.  The CUDA path and the CPU oracle
both consume exactly these arrays.  The drawing itself is done by ``gen.c``
(splitmix64 -> xoshiro256**, one stream per row / vector block / edge block),
so results do not depend on the number of threads.

The workload shapes stand in for the paper's SuiteSparse corpus (Sec. 6),
which is not available here; each recipe is listed in ``RECIPES``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_LIB = os.path.join(_HERE, "libworkloads.so")
_lock = threading.Lock()
_lib = None

U_PM1, U_01, NORMAL = 0, 1, 2

RECIPES = {
    "plain": "R=C=2000, exactly 10 nnz/row, columns uniform without replacement and sorted, v,x ~ U(-1,1)",
    "powerlaw": "R=C=1e6, L_r=min(floor(c*K_r),200000), K_r~Zipf(2) on 1..200000, rows empty w.p. 0.05, "
                "c by bisection to ~20M nnz, >=3 rows of >100k (planted if needed), v,x ~ U(-1,1)",
    "rmat": "R-MAT scale 22, 16*2^22 edges, (a,b,c,d)=(0.57,0.19,0.19,0.05), duplicates merged, "
            "self loops kept, weights U(0,1), x ~ U(-1,1)",
    "stencil27": "27-point stencil on 160^3, x fastest, non-periodic, off-diagonals N(0,1), diagonal 27",
    "batch": "512 square matrices, R_m log-uniform [1e3,2e5], mean row length log-uniform [1,64], "
             "per-row lengths Zipf(2)-weighted (largest remainder), clipped to C_m",
    "diff": "64 matrices 2^20 x 2^20 power-law (as 'powerlaw', ~16M nnz each, seeds 0..63), dy ~ N(0,1)",
}


def _build_lib(force: bool = False) -> str:
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-pthread", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def build(force: bool = False) -> str:
    """Compile ``libworkloads.so`` in-tree (gcc, a second or two)."""
    global _lib
    with _lock:
        path = _build_lib(force)
        _lib = None
    return path


def _L():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(_build_lib())
            i32p = ctypes.POINTER(ctypes.c_int32)
            i64p = ctypes.POINTER(ctypes.c_int64)
            f32p = ctypes.POINTER(ctypes.c_float)
            lib.wl_fill_vector.argtypes = [ctypes.c_int64, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, f32p,
                                           ctypes.c_int]
            lib.wl_fill_csr.argtypes = [ctypes.c_int32, ctypes.c_int32, i32p, ctypes.c_uint64, ctypes.c_uint64,
                                        ctypes.c_int, i32p, f32p, ctypes.c_int]
            lib.wl_powerlaw_lengths.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, ctypes.c_int32,
                                                ctypes.c_double, ctypes.c_int, ctypes.c_uint64, i32p,
                                                ctypes.POINTER(ctypes.c_double)]
            lib.wl_powerlaw_lengths.restype = ctypes.c_int64
            lib.wl_apportioned_lengths.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64,
                                                   ctypes.c_uint64, i32p]
            lib.wl_apportioned_lengths.restype = ctypes.c_int64
            lib.wl_batch_dims.argtypes = [ctypes.c_int32, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_uint64, i32p, i64p]
            lib.wl_rmat.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_uint64, i32p, i32p, ctypes.c_int]
            lib.wl_rmat.restype = ctypes.c_int64
            lib.wl_stencil27.argtypes = [ctypes.c_int32, ctypes.c_float, ctypes.c_uint64, i32p, i32p, f32p,
                                         ctypes.c_int]
            lib.wl_stencil27.restype = ctypes.c_int64
            _lib = lib
        return _lib


def _p(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _threads() -> int:
    return max(1, min(64, os.cpu_count() or 1))


@dataclass
class CSR:
    """A CSR matrix: tiles are rows, atoms are nonzeros (Sec. 3.1, Listing 1)."""
    rp: np.ndarray
    ci: np.ndarray
    v: np.ndarray
    num_cols: int
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def num_rows(self) -> int:
        return int(self.rp.shape[0] - 1)

    @property
    def nnz(self) -> int:
        return int(self.rp[-1])


def vector(n: int, kind: int = U_PM1, seed: int = 0, tag: int = 0) -> np.ndarray:
    out = np.empty(int(n), dtype=np.float32)
    if n:
        _L().wl_fill_vector(int(n), int(kind), int(seed), int(tag), _p(out, ctypes.c_float), _threads())
    return out


def from_lengths(L: np.ndarray, num_cols: int, seed: int, tag: int = 0, val_kind: int = U_PM1,
                 name: str = "") -> CSR:
    """CSR with the given row lengths, sorted distinct uniform columns, seeded values."""
    L = np.ascontiguousarray(L, dtype=np.int64)
    R = int(L.shape[0])
    rp = np.zeros(R + 1, dtype=np.int64)
    np.cumsum(L, out=rp[1:])
    if rp[-1] >= 2 ** 31:
        raise ValueError("nnz exceeds int32 range")
    if R and int(L.max(initial=0)) > num_cols:
        raise ValueError("row length exceeds number of columns")
    rp = rp.astype(np.int32)
    N = int(rp[-1])
    ci = np.empty(N, dtype=np.int32)
    v = np.empty(N, dtype=np.float32)
    if R:
        _L().wl_fill_csr(R, int(num_cols), _p(rp, ctypes.c_int32), int(seed), int(tag), int(val_kind),
                         _p(ci, ctypes.c_int32), _p(v, ctypes.c_float), _threads())
    return CSR(rp, ci, v, int(num_cols), name)


def powerlaw_lengths(R: int, C: int, target_nnz: int, lmax: int = 200_000, empty_frac: float = 0.05,
                     plant_long: bool = True, seed: int = 0):
    L = np.empty(max(R, 1), dtype=np.int32)
    c = ctypes.c_double(0.0)
    total = _L().wl_powerlaw_lengths(int(R), int(C), int(target_nnz), int(lmax), float(empty_frac),
                                     int(bool(plant_long)), int(seed), _p(L, ctypes.c_int32), ctypes.byref(c))
    return L[:R].copy(), int(total), float(c.value)


def plain(R: int = 2000, C: int = 2000, per_row: int = 10, seed: int = 0) -> CSR:
    m = from_lengths(np.full(R, per_row, dtype=np.int64), C, seed, tag=1, name=f"plain_{R}x{C}_{per_row}")
    return m


def powerlaw(R: int = 1_000_000, C: int = 1_000_000, target_nnz: int = 20_000_000, lmax: int = 200_000,
             empty_frac: float = 0.05, plant_long: bool = True, seed: int = 0) -> CSR:
    L, total, c = powerlaw_lengths(R, C, target_nnz, lmax, empty_frac, plant_long, seed)
    m = from_lengths(L, C, seed, tag=2, name=f"powerlaw_{R}x{C}_{total}")
    m.meta.update(c=c, target_nnz=target_nnz)
    return m


def rmat(scale: int = 22, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = 0) -> CSR:
    R = 1 << scale
    E = edge_factor * R
    rp = np.empty(R + 1, dtype=np.int32)
    ci = np.empty(E, dtype=np.int32)
    n = _L().wl_rmat(int(scale), int(E), float(a), float(b), float(c), int(seed), _p(rp, ctypes.c_int32),
                     _p(ci, ctypes.c_int32), _threads())
    ci = ci[:n].copy()
    v = np.empty(n, dtype=np.float32)
    _L().wl_fill_csr(R, R, _p(rp, ctypes.c_int32), int(seed), 3, U_01, None, _p(v, ctypes.c_float), _threads())
    return CSR(rp, ci, v, R, f"rmat_s{scale}_e{edge_factor}", {"edges_generated": E})


def stencil27(n: int = 160, seed: int = 0) -> CSR:
    R = n ** 3
    nnz = (3 * n - 2) ** 3
    rp = np.empty(R + 1, dtype=np.int32)
    ci = np.empty(nnz, dtype=np.int32)
    v = np.empty(nnz, dtype=np.float32)
    got = _L().wl_stencil27(int(n), ctypes.c_float(27.0), int(seed), _p(rp, ctypes.c_int32),
                            _p(ci, ctypes.c_int32), _p(v, ctypes.c_float), _threads())
    assert got == nnz
    return CSR(rp, ci, v, R, f"stencil27_{n}")


@dataclass
class Batch:
    """Concatenation of square CSR matrices: per-matrix offsets start at 0."""
    mats: list

    @property
    def num(self) -> int:
        return len(self.mats)

    def rows(self) -> np.ndarray:
        return np.array([m.num_rows for m in self.mats], dtype=np.int32)

    def cols(self) -> np.ndarray:
        return np.array([m.num_cols for m in self.mats], dtype=np.int32)

    def nnz(self) -> np.ndarray:
        return np.array([m.nnz for m in self.mats], dtype=np.int64)

    def rp_cat(self) -> np.ndarray:
        return np.concatenate([m.rp for m in self.mats]).astype(np.int32, copy=False)

    def ci_cat(self) -> np.ndarray:
        return np.concatenate([m.ci for m in self.mats]).astype(np.int32, copy=False)

    def v_cat(self) -> np.ndarray:
        return np.concatenate([m.v for m in self.mats]).astype(np.float32, copy=False)


def batch(num: int = 512, rmin: float = 1e3, rmax: float = 2e5, mmin: float = 1.0, mmax: float = 64.0,
          seed: int = 0) -> Batch:
    R = np.empty(num, dtype=np.int32)
    Nt = np.empty(num, dtype=np.int64)
    _L().wl_batch_dims(int(num), float(rmin), float(rmax), float(mmin), float(mmax), int(seed),
                       _p(R, ctypes.c_int32), _p(Nt, ctypes.c_int64))
    mats = []
    for m in range(num):
        Rm = int(R[m])
        L = np.empty(Rm, dtype=np.int32)
        _L().wl_apportioned_lengths(Rm, Rm, int(Nt[m]), int(seed), int(m), _p(L, ctypes.c_int32))
        mats.append(from_lengths(L, Rm, seed, tag=1000 + m, name=f"batch{m}"))
    return Batch(mats)


def diff_batch(num: int = 64, R: int = 1 << 20, target_nnz: int = 16_000_000, first_seed: int = 0) -> Batch:
    return Batch([powerlaw(R, R, target_nnz, seed=first_seed + s) for s in range(num)])


def x_for(m: CSR, seed: int = 0, tag: int = 11) -> np.ndarray:
    return vector(m.num_cols, U_PM1, seed, tag)


def dy_for(m: CSR, seed: int = 0, tag: int = 12) -> np.ndarray:
    return vector(m.num_rows, NORMAL, seed, tag)


def config(name: str, seed: int = 0):
    """The five evaluation workloads by name (full size)."""
    if name == "plain":
        return plain(seed=seed)
    if name == "powerlaw":
        return powerlaw(seed=seed)
    if name == "rmat":
        return rmat(seed=seed)
    if name == "stencil27":
        return stencil27(seed=seed)
    if name == "batch":
        return batch(seed=seed)
    if name == "diff":
        return diff_batch(first_seed=seed)
    raise KeyError(name)
