"""The C ABI library builds, loads without a GPU and exports every symbol the header declares.

Only host-side functions are called here (no GPU needed): the Sec. 6.2
schedule heuristic and the merge-path diagonal layout.
"""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2301_04792_gb300 import _lib, buildlib as lb_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\**\s+(lb_[a-z_0-9]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    lb_build.build()
    return _lib.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("lb_plan", "lb_spmv", "lb_spmv_backward", "lb_plan_destroy", "lb_batch_plan",
                     "lb_batch_spmv", "lb_batch_spmv_backward", "lb_status", "lb_plan_splits", "lb_plan_transpose"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    raw = ctypes.CDLL(_lib.library_path())
    missing = [n for n in declared_functions() if not hasattr(raw, n)]
    assert not missing, missing
    # and the binding's signature table covers the header exactly
    assert sorted(_lib.SIGNATURES) == declared_functions()


def test_version_and_status_strings(lib):
    assert lib.lb_version() >= 10100
    for s in range(7):
        assert lib.lb_status_string(s).decode().startswith(_lib.STATUS_NAMES[s])


def test_heuristic_matches_sec_6_2(lib):
    # merge-path unless (rows < 500 or cols < 500) and nnz < 10000
    TM, MP = 0, 3
    assert lib.lb_heuristic_schedule(499, 10 ** 6, 9999) == TM
    assert lib.lb_heuristic_schedule(10 ** 6, 499, 9999) == TM
    assert lib.lb_heuristic_schedule(499, 499, 10000) == MP
    assert lib.lb_heuristic_schedule(500, 500, 5) == MP
    assert lib.lb_heuristic_schedule(2000, 2000, 20000) == MP


@pytest.mark.parametrize("items,grid,ipt", [(0, 1, 2048), (1, 1, 2048), (21_000_000, 456, 2048),
                                            (22_000, 86, 2048), (1000, 7, 3), (123457, 152, 1024)])
def test_merge_diagonals_layout(lib, items, grid, ipt):
    from paper_2301_04792_gb300 import merge_diagonals
    d, tpc = merge_diagonals(items, grid, ipt)
    assert d.shape[0] == grid * (tpc + 1)
    d = d.reshape(grid, tpc + 1)
    begins = np.array([c * items // grid for c in range(grid)])
    ends = np.array([(c + 1) * items // grid for c in range(grid)])
    assert np.array_equal(d[:, 0], begins) and np.array_equal(d[:, -1], ends)  # equal shares, contiguous
    assert (np.diff(d, axis=1) >= 0).all() and (np.diff(d, axis=1) <= ipt).all()  # tiles of at most ipt items
    assert d.min() >= 0 and d.max() <= items
    # ceil(share / ipt) tiles suffice for the largest share
    assert tpc == max(1, -(-(-(-items // grid)) // ipt))


def test_merge_diagonals_rejects_bad_args(lib):
    n = ctypes.c_size_t(0)
    t = ctypes.c_int32(0)
    assert lib.lb_merge_diagonals(-1, 1, 1, None, 0, ctypes.byref(n), ctypes.byref(t)) == 1
    assert lib.lb_merge_diagonals(10, 0, 1, None, 0, ctypes.byref(n), ctypes.byref(t)) == 1
    assert b"items" in lib.lb_last_error()


def test_autotune_rejects_bad_args_before_any_launch(lib):
    res = _lib.TuneResult()
    opts = _lib.TuneOpts(num_cols=10)
    plan = ctypes.c_void_p()
    # no result / no opts
    assert lib.lb_autotune(None, 0, 0, None, None, None, None, ctypes.byref(opts), None, None, None) == 1
    assert lib.lb_autotune(None, 0, 0, None, None, None, None, None, ctypes.byref(res), None, None) == 1
    # atoms without buffers, negative sizes, atoms without columns
    assert lib.lb_autotune(None, 5, 10, None, None, None, None, ctypes.byref(opts), ctypes.byref(res),
                           ctypes.byref(plan), None) == 1
    assert lib.lb_autotune(None, -1, 0, None, None, None, None, ctypes.byref(opts), ctypes.byref(res), None,
                           None) == 1
    fake = ctypes.c_void_p(256)  # never dereferenced: the call is refused first
    opts0 = _lib.TuneOpts(num_cols=0)
    assert lib.lb_autotune(fake, 5, 10, fake, fake, fake, fake, ctypes.byref(opts0), ctypes.byref(res),
                           None, None) == 1
    assert b"num_cols" in lib.lb_last_error()
    assert plan.value is None
    assert ctypes.sizeof(_lib.PlanOpts) == 12 * 4
    assert ctypes.sizeof(_lib.TuneResult) == 5 * 4 + ctypes.sizeof(_lib.PlanOpts) + 20 * 44


def test_plan_rejects_row_weight_out_of_range_before_any_launch(lib):
    plan = ctypes.c_void_p()
    for w in (-1, 65):
        opts = _lib.PlanOpts(row_weight=w)
        assert lib.lb_plan_ex(ctypes.byref(plan), None, 0, 0, 3, ctypes.byref(opts), None) == 1
        assert b"row_weight" in lib.lb_last_error()
    assert plan.value is None


def test_candidate_names_carry_units_and_row_weight():
    from paper_2301_04792_gb300 import lb as lbm
    c = _lib.TuneCandidate(schedule=3, items_per_thread=4, mp_variant=0, units_per_cta=1, row_weight=2)
    assert lbm._candidate_name(c) == "merge_path_ipt4_v0_w2"
    c = _lib.TuneCandidate(schedule=3, items_per_thread=8, mp_variant=0, units_per_cta=4, row_weight=1)
    assert lbm._candidate_name(c) == "merge_path_ipt8_v0_u4"
    c = _lib.TuneCandidate(schedule=3, items_per_thread=8, mp_variant=3, units_per_cta=1, row_weight=0)
    assert lbm._candidate_name(c) == "merge_path_ipt8_v3"
    c = _lib.TuneCandidate(schedule=0, staged=1)
    assert lbm._candidate_name(c) == "thread_mapped_staged"
    assert ctypes.sizeof(_lib.TuneCandidate) == 11 * 4


def test_selftest_rejects_unknown_case_without_launching(lib):
    assert lib.lb_selftest(0, None) == 1
    assert lib.lb_selftest(3, None) == 1
    assert b"which" in lib.lb_last_error()


def test_autotune_cache_file_round_trip(lib, tmp_path):
    """The persisted autotuner cache (no GPU needed): a file of entries loads,
    saves back to the same text, reloads after a clear; lines of another
    library version or that do not parse are skipped."""
    ver = lib.lb_version()
    cands = "[[3,8,0,0,1,1,0,0,5,0.5,1900.25],[3,4,0,0,1,2,0,0,5,0.25,3800.5],[0,0,0,0,1,1,1,0,1,12.5,7.75]]"
    opts = ",".join(str(v) for v in (1000000, 4, 0, 0, 0, 0, 0, 1, 0, 0, 2, 0))

    def line(v, rows, fp):
        return ('{"format":"lb_autotune_cache","version":%d,"device":"NVIDIA GB300/152/10.3","rows":%d,'
                '"atoms":20000016,"cols":1000000,"fingerprint":"0x%016x","families":15,"cold_l2":1,"best":1,'
                '"heuristic":0,"best_schedule":3,"best_opts":[%s],"candidates":%s}\n' % (v, rows, fp, opts, cands))
    good = [line(ver, 1000000, 0x0123456789abcdef), line(ver, 5, 0xfedcba9876543210)]
    src = tmp_path / "cache.jsonl"
    src.write_text(good[0] + line(ver + 1, 7, 1) + "not json\n" + good[1])
    lib.lb_autotune_cache_clear()
    n = ctypes.c_int32(-1)
    assert lib.lb_autotune_cache_load(str(src).encode(), ctypes.byref(n)) == 0
    assert n.value == 2 and lib.lb_autotune_cache_size() == 2
    out = tmp_path / "saved.jsonl"
    assert lib.lb_autotune_cache_save(str(out).encode()) == 0
    assert sorted(out.read_text().splitlines(keepends=True)) == sorted(good)
    lib.lb_autotune_cache_clear()
    assert lib.lb_autotune_cache_size() == 0
    assert lib.lb_autotune_cache_load(str(out).encode(), ctypes.byref(n)) == 0 and n.value == 2
    lib.lb_autotune_cache_clear()
    assert lib.lb_autotune_cache_load(str(tmp_path / "missing.jsonl").encode(), None) == 1
    assert lib.lb_autotune_cache_save(b"") == 1


def test_batch_autotune_rejects_bad_arguments(lib):
    """Argument checks of lb_batch_autotune run on the host, before any launch."""
    res = _lib.BatchTuneResult()
    opts = _lib.TuneOpts()
    rows = (ctypes.c_int32 * 1)(10)
    nnz = (ctypes.c_int64 * 1)(20)
    fake = ctypes.c_void_p(16)
    args = [1, rows, rows, nnz, fake, fake, fake, fake, fake, None, None, None]
    # passes out of range, no result, num_mats 0, dy missing for a backward pass
    assert lib.lb_batch_autotune(*args, 0, ctypes.byref(opts), ctypes.byref(res), None, None) == 1
    assert lib.lb_batch_autotune(*args, 1, ctypes.byref(opts), None, None, None) == 1
    assert lib.lb_batch_autotune(0, *args[1:], 1, ctypes.byref(opts), ctypes.byref(res), None, None) == 1
    assert lib.lb_batch_autotune(*args, 3, ctypes.byref(opts), ctypes.byref(res), None, None) == 1


def test_batch_autotune_cache_lines_round_trip(lib, tmp_path):
    """Batch autotuner entries share the cache file: a handwritten batch line loads beside a
    single-matrix line and both save back to the same text."""
    ver = lib.lb_version()
    opts = ",".join(str(v) for v in (0, 4, 0, 0, 0, 3, 0, 0, 2, 0, 0, 0))
    cand = "[%s,0,3,16.125,1928.5],[%s,0,3,17.75,1750.25]" % (opts, opts)
    bline = ('{"format":"lb_batch_autotune_cache","version":%d,"device":"NVIDIA GB300/152/10.3","mats":64,'
             '"rows":67108864,"cols":67108864,"atoms":1024724164,"fingerprint":"0x00000000000000ff","passes":7,'
             '"cold_l2":0,"best":0,"best_opts":[%s],"candidates":[%s]}\n' % (ver, opts, cand))
    sline = ('{"format":"lb_autotune_cache","version":%d,"device":"NVIDIA GB300/152/10.3","rows":10,"atoms":20,'
             '"cols":10,"fingerprint":"0x0000000000000001","families":15,"cold_l2":0,"best":0,"heuristic":0,'
             '"best_schedule":3,"best_opts":[%s],"candidates":[[3,8,0,0,1,1,0,0,5,0.5,1.5]]}\n' % (ver, opts))
    src = tmp_path / "both.jsonl"
    src.write_text(sline + bline + bline.replace('"best":0', '"best":5'))  # last: best out of range
    lib.lb_autotune_cache_clear()
    n = ctypes.c_int32(-1)
    assert lib.lb_autotune_cache_load(str(src).encode(), ctypes.byref(n)) == 0 and n.value == 2
    out = tmp_path / "saved.jsonl"
    assert lib.lb_autotune_cache_save(str(out).encode()) == 0
    assert sorted(out.read_text().splitlines(keepends=True)) == sorted([sline, bline])
    lib.lb_autotune_cache_clear()
