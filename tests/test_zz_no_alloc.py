"""lb_spmv_noalloc: merge-path SpMV for callers that cannot allocate device memory.

Such callers (allocator-free real-time loops that reserve all device memory up
front, hosts whose memory pool belongs to another framework) get their scratch
from a fixed device array built into the library instead of from cudaMalloc.
This checks, through the C ABI, that two calls in a row give the same result as
the planned entry point lb_spmv within the tolerance the parity tests use
(|y - y64| <= 1e-5 * sum_j |a_ij x_j| against the FP64 oracle), that the two
calls are bit-identical, that atom arrays which are not 16-byte aligned (the
scalar-load kernel) give the same, and that a problem too large for the fixed
scratch is refused before any launch.  This file runs last so that a failure
here leaves every other test already run.
"""
import ctypes

import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_noalloc_matches_planned_spmv_twice():
    import torch
    import paper_2301_04792_gb300 as lb
    from paper_2301_04792_gb300 import _lib
    lb.build()
    lib = _lib.load()
    vp = ctypes.c_void_p
    cases = [W.plain(2000, 2000, 10, seed=0),
             W.powerlaw(50_000, 50_000, 1_000_000, lmax=40_000, plant_long=False, seed=2)]
    L = np.zeros(3001, dtype=np.int64)
    L[::5] = 3
    L[17] = 60_000
    cases.append(W.from_lengths(L, 70_000, seed=4))
    for m in cases:
        x = W.x_for(m)
        y64, b = oracle.spmv(m.rp, m.ci, m.v, x)
        rp, xd = _dev(m.rp), _dev(x)
        # 16-byte aligned atom arrays (vector loads), then the same arrays one element into larger
        # buffers (not 16-byte aligned: the scalar-load kernel)
        ci_buf = torch.zeros(m.nnz + 1, dtype=torch.int32, device="cuda")
        v_buf = torch.zeros(m.nnz + 1, dtype=torch.float32, device="cuda")
        ci_buf[1:] = _dev(m.ci)
        v_buf[1:] = _dev(m.v)
        for ci, v in ((_dev(m.ci), _dev(m.v)), (ci_buf[1:], v_buf[1:])):
            plan = lb.Plan(rp, m.nnz, "merge_path", num_cols=m.num_cols)
            y_plan = plan.spmv(ci, v, xd)
            ref = y_plan.cpu().numpy().astype(np.float64)
            stream = torch.cuda.current_stream().cuda_stream
            got = []
            for call in range(2):
                y = torch.full((m.num_rows,), float("nan"), device="cuda")
                st = lib.lb_spmv_noalloc(vp(rp.data_ptr()), m.num_rows, m.nnz, vp(ci.data_ptr()), vp(v.data_ptr()),
                                         vp(xd.data_ptr()), vp(y.data_ptr()), vp(stream))
                assert st == 0, lib.lb_last_error()
                torch.cuda.synchronize()
                got.append(y.cpu().numpy())
                g64 = got[-1].astype(np.float64)
                assert np.all(np.abs(g64 - y64) <= oracle.TOL * b), (m.name, call, ci.data_ptr() % 16)
                assert np.all(np.abs(g64 - ref) <= oracle.TOL * b), (m.name, call, ci.data_ptr() % 16)
            assert np.array_equal(got[0].view(np.uint32), got[1].view(np.uint32)), (m.name, "calls differ")


def test_noalloc_refuses_oversized_problem():
    import torch
    from paper_2301_04792_gb300 import _lib
    lib = _lib.load()
    vp = ctypes.c_void_p
    tiny = torch.zeros(4, dtype=torch.int32, device="cuda")
    y = torch.zeros(4, device="cuda")
    st = lib.lb_spmv_noalloc(vp(tiny.data_ptr()), 2_000_000_000, 2_000_000_000, vp(tiny.data_ptr()),
                             vp(y.data_ptr()), vp(y.data_ptr()), vp(y.data_ptr()), None)
    assert st == 4  # LB_ERR_UNSUPPORTED, nothing launched
    assert b"scratch" in lib.lb_last_error()
    torch.cuda.synchronize()
