"""Shared helpers for the GPU parity tests (inputs, oracle comparisons)."""
import numpy as np

import oracle
import workloads as W

TOL = oracle.TOL  # |y - y64| <= 1e-5 * sum |a_ij x_j|

# every schedule and option set the library offers for one matrix (forward parity runs all of them)
SCHEDULES = [("thread_mapped", {}), ("thread_mapped", {"staged": True}), ("warp_mapped", {}), ("block_mapped", {}),
             ("group_mapped", {"group_size": 4}), ("group_mapped", {"group_size": 8}),
             ("group_mapped", {"group_size": 16}), ("group_mapped", {"group_size": 64}),
             ("group_mapped", {"group_size": 128}),
             ("merge_path", {"items_per_thread": 4}), ("merge_path", {"items_per_thread": 8}),
             ("merge_path", {"items_per_thread": 16}),
             ("merge_path", {"items_per_thread": 4, "mp_variant": 1}),
             ("merge_path", {"items_per_thread": 8, "mp_variant": 1}),
             ("merge_path", {"items_per_thread": 16, "mp_variant": 1}),
             ("merge_path", {"items_per_thread": 4, "mp_variant": 2}),
             ("merge_path", {"items_per_thread": 8, "mp_variant": 2}),
             ("merge_path", {"items_per_thread": 16, "mp_variant": 2}),
             ("merge_path", {"items_per_thread": 8, "units_per_cta": 4}),
             ("merge_path", {"items_per_thread": 4, "units_per_cta": 16}),
             ("merge_path", {"items_per_thread": 4, "row_weight": 2}),
             ("merge_path", {"items_per_thread": 8, "row_weight": 5}),
             ("merge_path", {"items_per_thread": 8, "mp_variant": 3}),
             ("merge_path", {"items_per_thread": 4, "mp_variant": 3, "tiles_per_share": 3}),
             ("merge_path", {"items_per_thread": 16, "mp_variant": 3, "tiles_per_share": 2})]
SCHED_IDS = [s + "".join(f"_{k}{v}" for k, v in o.items()) for s, o in SCHEDULES]


def to_dev(*arrs):
    import torch
    return [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrs]


def assert_within_bound(y32, y64, b, what="y", tol=TOL):
    y32 = np.asarray(y32, dtype=np.float64)
    err = np.abs(y32 - y64)
    bad = err > tol * b
    if bad.any():
        i = int(np.argmax(bad))
        raise AssertionError(f"{what}: {int(bad.sum())} of {len(y64)} entries outside the bound; first at {i}: "
                             f"got {y32[i]!r}, oracle {y64[i]!r}, bound {tol * b[i]!r}")


def small_cases():
    """(name, CSR, x) at sizes the oracle finishes instantly, spanning many tiles and ragged tails."""
    out = []
    m = W.plain(2000, 2000, 10, seed=0)
    out.append(("plain_2000", m))
    m = W.powerlaw(20000, 20000, 400_000, lmax=20000, plant_long=False, seed=1)
    out.append(("powerlaw_20k", m))
    # a few very long rows crossing many tiles and CTAs, many empty rows
    L = np.zeros(3001, dtype=np.int64)
    L[::7] = 3
    L[5] = 60000
    L[1500] = 45000
    L[3000] = 70000
    out.append(("long_rows", W.from_lengths(L, 80000, seed=2)))
    # ragged: lengths 0..40 cycling, odd total
    L = (np.arange(4999) * 7919) % 41
    out.append(("ragged", W.from_lengths(L, 5000, seed=3)))
    out.append(("rmat_s12", W.rmat(scale=12, edge_factor=8, seed=4)))
    out.append(("stencil_12", W.stencil27(12)))
    return out


def edge_cases():
    """Degenerate tile sets: empty, all-empty rows, one row, one column, 1x1."""
    cases = []
    cases.append(("one_row", W.from_lengths(np.array([100_000]), 200_000, seed=5)))
    cases.append(("all_empty", W.from_lengths(np.zeros(1000, np.int64), 10, seed=6)))
    cases.append(("one_col", W.from_lengths(np.ones(3333, np.int64), 1, seed=7)))
    cases.append(("one_by_one", W.from_lengths(np.ones(1, np.int64), 1, seed=8)))
    L = np.zeros(2048, np.int64)
    L[-1] = 5000
    cases.append(("last_row_only", W.from_lengths(L, 6000, seed=9)))
    L = np.zeros(257, np.int64)
    L[0] = 1
    cases.append(("first_row_only", W.from_lengths(L, 3, seed=10)))
    return cases
