"""GPU parity of SpMM C = A B (Listing 4) on the merge-path and thread-mapped
schedules against the FP64 oracle: every element within 1e-5 of sum |v B| per
element, bit-identical repeats, row-pitched B and C, panels of columns, and the
degenerate cases."""
import numpy as np
import pytest

import oracle
import workloads as W
from helpers import edge_cases, small_cases, to_dev

pytestmark = pytest.mark.gpu

TOL = oracle.TOL


@pytest.fixture(scope="module")
def lbmod():
    import paper_2301_04792_gb300 as lb
    lb.build()
    return lb


def dense_b(C, K, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(-1, 1, (C, K)).astype(np.float32)


def check(lb, m, K, schedule, seed=0, pad_b=0, pad_c=0, reps=2, **kw):
    import torch
    B = dense_b(m.num_cols, K, seed)
    c64, bnd = oracle.spmm(m.rp, m.ci, m.v, B)
    rp, ci, v = to_dev(m.rp, m.ci, m.v)
    Bw = torch.zeros(m.num_cols, K + pad_b, device="cuda")
    Bw[:, :K] = torch.from_numpy(B).cuda()
    Bd = Bw[:, :K]
    plan = lb.Plan(rp, m.nnz, schedule, num_cols=m.num_cols, **kw)
    outs = []
    for _ in range(reps):
        Cw = torch.full((m.num_rows, K + pad_c), 7.0, device="cuda")
        outs.append((plan.spmm(ci, v, Bd, Cw[:, :K]), Cw))
    got = outs[0][0].cpu().numpy().astype(np.float64)
    err = np.abs(got - c64)
    assert (err <= TOL * bnd).all(), f"{m.name} K={K} {schedule}: max excess {np.max(err - TOL * bnd)}"
    if pad_c:
        assert (outs[0][1][:, K:] == 7.0).all(), "C written outside its K columns"
    for c2, _ in outs[1:]:
        assert torch.equal(c2.view(torch.int32), outs[0][0].view(torch.int32)), "SpMM not bit-identical"


@pytest.mark.parametrize("K", [1, 4, 7, 8, 16, 20, 32, 33, 64, 100, 128, 130, 256])
def test_spmm_small_cases(lbmod, K):
    for name, m in small_cases() + edge_cases():
        check(lbmod, m, K, "merge_path")
        if K in (1, 33):
            check(lbmod, m, K, "thread_mapped")


def test_spmm_pitched_and_long_rows(lbmod):
    m = W.from_lengths(np.array([30_000, 3, 0, 0, 45_000, 1, 900, 0]), 50_000, seed=12)
    for K in (16, 96, 257):
        check(lbmod, m, K, "merge_path", pad_b=5, pad_c=3, reps=3)   # scalar path (pitch not a multiple of 4)
    for K in (8, 32, 124):
        check(lbmod, m, K, "merge_path", pad_b=4, pad_c=8, reps=3)   # 16-byte rows of B and C
    check(lbmod, W.plain(300, 300, 3, seed=2), 40, "thread_mapped", pad_b=2, pad_c=1)


def test_spmm_powerlaw(lbmod):
    m = W.powerlaw(200_000, 150_000, 3_000_000, lmax=100_000, plant_long=False, seed=13)
    check(lbmod, m, 32, "merge_path", reps=3)


def test_spmm_shares_of_several_tiles(lbmod):
    """Enough rows + atoms that every warp share spans several tiles, so the partial sum of a row open
    at a tile's end crosses into the next tile of the same share, including tiles that start at a row's
    end marker (the row closes where the tile starts)."""
    m = W.powerlaw(600_000, 400_000, 12_000_000, lmax=60_000, seed=21)
    for K in (8, 32, 12, 7):  # 16-byte rows of B (K = 12: a partly idle lane group) and scalar ones
        check(lbmod, m, K, "merge_path", seed=K)


def test_spmm_unsupported_and_bad_arguments(lbmod):
    import torch
    from paper_2301_04792_gb300 import _lib
    m = W.plain(100, 100, 3, seed=3)
    rp, ci, v = to_dev(m.rp, m.ci, m.v)
    B = torch.ones(100, 8, device="cuda")
    with pytest.raises(_lib.LBError):
        lbmod.Plan(rp, m.nnz, "warp_mapped").spmm(ci, v, B)
    lib = _lib.load()
    plan = lbmod.Plan(rp, m.nnz, "merge_path")
    C = torch.empty(100, 8, device="cuda")
    import ctypes
    vp = ctypes.c_void_p
    # ldb < K, ldc < K, K < 0
    assert lib.lb_spmm(plan.handle, 8, vp(ci.data_ptr()), vp(v.data_ptr()), vp(B.data_ptr()), 4, vp(C.data_ptr()),
                       8, None) == 1
    assert lib.lb_spmm(plan.handle, 8, vp(ci.data_ptr()), vp(v.data_ptr()), vp(B.data_ptr()), 8, vp(C.data_ptr()),
                       7, None) == 1
    assert lib.lb_spmm(plan.handle, -1, None, None, None, 0, None, 0, None) == 1
    # K = 0 is a no-op
    assert lib.lb_spmm(plan.handle, 0, None, None, None, 0, None, 0, None) == 0
