"""The roofline probes gather the right values: the load-unit probe
(lb_probe_gather) and the TMA gather4 probe (lb_probe_gather_tma) both reduce
sum_k vals[k] * x[idx[k]] to per-thread partials whose total matches an FP64
sum on the host within 1e-5 of sum_k |vals[k] * x[idx[k]]| (the TMA probe
reads 0 for indices in a trailing partial row of 8 floats, as documented)."""
import ctypes

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import paper_2301_04792_gb300 as lb
    from paper_2301_04792_gb300 import _lib
    lb.build()
    return _lib.load()


@pytest.mark.parametrize("num_x", [1_000_000, 999_997])
def test_probes_reduce_the_gathered_products(lib, num_x):
    import torch
    vp = ctypes.c_void_p
    n = 128 * 40_000
    idx = np.minimum((W.vector(n, W.U_01, 3, 51).astype(np.float64) * num_x).astype(np.int64), num_x - 1)
    idx = idx.astype(np.int32)
    v = W.vector(n, W.U_PM1, 3, 52)
    x = W.vector(num_x, W.U_PM1, 3, 53)
    prod = v.astype(np.float64) * x[idx].astype(np.float64)
    ci_d, v_d, x_d = (torch.from_numpy(a).cuda() for a in (idx, v, x))
    s = vp(torch.cuda.current_stream().cuda_stream)
    grid = lib.lb_probe_gather_grid()
    out = torch.zeros(grid * 256, dtype=torch.float32, device="cuda")
    assert lib.lb_probe_gather(vp(ci_d.data_ptr()), vp(v_d.data_ptr()), vp(x_d.data_ptr()), n, vp(out.data_ptr()),
                               grid, s) == 0
    total = float(out.double().sum().item())
    assert abs(total - prod.sum()) <= 1e-5 * np.abs(prod).sum()
    tgrid = lib.lb_probe_gather_tma_grid()
    assert tgrid > 0
    tout = torch.zeros(tgrid * 256, dtype=torch.float32, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert lib.lb_probe_gather_tma(vp(ci_d.data_ptr()), vp(v_d.data_ptr()), vp(x_d.data_ptr()), n, num_x,
                                   vp(tout.data_ptr()), tgrid, vp(err.data_ptr()), s) == 0, lib.lb_last_error()
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    inside = idx < 8 * (num_x // 8)
    expect = prod[inside].sum()
    assert abs(float(tout.double().sum().item()) - expect) <= 1e-5 * np.abs(prod).sum()
    # argument checks: n not a multiple of 128, unaligned x
    assert lib.lb_probe_gather_tma(vp(ci_d.data_ptr()), vp(v_d.data_ptr()), vp(x_d.data_ptr()), n - 4, num_x,
                                   vp(tout.data_ptr()), tgrid, vp(err.data_ptr()), s) == 1
    assert lib.lb_probe_gather_tma(vp(ci_d.data_ptr()), vp(v_d.data_ptr()), vp(x_d.data_ptr() + 4), n, num_x - 1,
                                   vp(tout.data_ptr()), tgrid, vp(err.data_ptr()), s) == 1
