"""GPU parity of the forward SpMV schedules against the FP64 oracle, through the C ABI.

Floating point: |y - y64| <= 1e-5 * sum_j |a_ij x_j| per row, and bit-identical
results on repeated runs of the same plan.  Integer parts (merge-path splits,
atom->tile map) must match the oracle bit for bit.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from helpers import SCHED_IDS, SCHEDULES, assert_within_bound, edge_cases, small_cases, to_dev

pytestmark = pytest.mark.gpu



@pytest.fixture(scope="module")
def lbmod():
    import paper_2301_04792_gb300 as lb
    lb.build()
    return lb


def run_case(lb, m, x, schedule, opts, repeats=3):
    import torch
    rp, ci, v, xd = to_dev(m.rp, m.ci, m.v, x)
    plan = lb.Plan(rp, m.nnz, schedule, num_cols=m.num_cols, **opts)
    outs = []
    for _ in range(repeats):
        y = torch.full((m.num_rows,), float("nan"), device="cuda")
        plan.spmv(ci, v, xd, y)
        outs.append(y.cpu().numpy())
    torch.cuda.synchronize()
    return plan, outs


@pytest.mark.parametrize("schedule,opts", SCHEDULES, ids=SCHED_IDS)
def test_small_cases_all_schedules(lbmod, schedule, opts):
    for name, m in small_cases() + edge_cases():
        x = W.x_for(m, seed=1)
        y64, b = oracle.spmv(m.rp, m.ci, m.v, x)
        _, outs = run_case(lbmod, m, x, schedule, opts)
        assert_within_bound(outs[0], y64, b, f"{name}/{schedule}")
        for o in outs[1:]:
            assert np.array_equal(o.view(np.uint32), outs[0].view(np.uint32)), f"{name}: not bit-identical"


def test_empty_tile_set(lbmod):
    import torch
    rp = torch.zeros(1, dtype=torch.int32, device="cuda")
    for s in ("thread_mapped", "warp_mapped", "merge_path"):
        p = lbmod.Plan(rp, 0, s)
        y = p.spmv(torch.zeros(0, dtype=torch.int32, device="cuda"), torch.zeros(0, device="cuda"),
                   torch.zeros(4, device="cuda"))
        assert y.numel() == 0


def test_row_sums_and_identity_exact(lbmod):
    import torch
    # x = 1 with small-integer values: row sums are exact in any order
    m = W.powerlaw(5000, 5000, 100_000, lmax=4000, plant_long=False, seed=11)
    vi = np.random.default_rng(0).integers(-4, 5, m.nnz).astype(np.float32)
    ones = np.ones(m.num_cols, np.float32)
    y64, _ = oracle.spmv(m.rp, m.ci, vi, ones)
    for s, o in SCHEDULES:
        mm = W.CSR(m.rp, m.ci, vi, m.num_cols)
        _, outs = run_case(lbmod, mm, ones, s, o, repeats=1)
        assert np.array_equal(outs[0].astype(np.float64), y64), s
    # identity: y = x bit for bit
    n = 10007
    I = W.CSR(np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), np.ones(n, np.float32), n)
    x = W.vector(n, W.U_PM1, 3, 3)
    for s, o in SCHEDULES:
        _, outs = run_case(lbmod, I, x, s, o, repeats=1)
        assert np.array_equal(outs[0], x), s


def test_unaligned_buffers_take_scalar_path(lbmod):
    import torch
    m = W.powerlaw(3000, 3000, 60_000, lmax=3000, plant_long=False, seed=12)
    x = W.x_for(m)
    y64, b = oracle.spmv(m.rp, m.ci, m.v, x)
    rp = to_dev(m.rp)[0]
    # offset the atom arrays by one element inside larger buffers
    ci_buf = torch.zeros(m.nnz + 1, dtype=torch.int32, device="cuda")
    v_buf = torch.zeros(m.nnz + 1, dtype=torch.float32, device="cuda")
    ci_buf[1:] = torch.from_numpy(m.ci).cuda()
    v_buf[1:] = torch.from_numpy(m.v).cuda()
    ci, v = ci_buf[1:], v_buf[1:]
    assert ci.data_ptr() % 16 != 0
    for s, o in SCHEDULES:
        plan = lbmod.Plan(rp, m.nnz, s, **o)
        y = plan.spmv(ci, v, to_dev(x)[0])
        assert_within_bound(y.cpu().numpy(), y64, b, f"unaligned/{s}")


def test_merge_path_splits_bit_exact(lbmod):
    for name, m in small_cases() + edge_cases():
        for ipt, var, w in ((4, 0, 1), (8, 0, 1), (16, 0, 1), (8, 1, 1), (4, 2, 1), (16, 2, 1), (8, 3, 1),
                            (4, 0, 2), (8, 0, 3), (16, 0, 64)):
            rp = to_dev(m.rp)[0]
            plan = lbmod.Plan(rp, m.nnz, "merge_path", items_per_thread=ipt, mp_variant=var, row_weight=w)
            diag, ij = plan.splits()
            info = plan.info()
            R, N = m.num_rows, m.nnz
            if w > 1:
                # shares cut with row ends weighted w: the oracle's walk along the merged list
                expect = oracle.weighted_diagonals(m.rp, w, info["num_workers"], info["items_per_tile"],
                                                   info["tiles_per_cta"])
                assert np.array_equal(diag, expect), (name, ipt, w)
            elif var == 3:
                # guided shares: tiles of items_per_tile items in order, each share ending where
                # the next begins, the last at R + N
                assert diag[0] == 0 and diag[-1] == R + N and (np.diff(diag) >= 0).all()
                assert (np.diff(diag) <= info["items_per_tile"]).all()
            else:
                # the plan's diagonals follow the documented layout
                d_host, tpc = lbmod.merge_diagonals(R + N, info["num_workers"], info["items_per_tile"])
                assert tpc == info["tiles_per_cta"]
                assert np.array_equal(diag, d_host), name
            assert np.array_equal(ij, oracle.merge_splits(diag, m.rp)), f"{name} ipt={ipt}"


def test_atom_tiles_bit_exact(lbmod):
    for name, m in small_cases() + edge_cases():
        rp = to_dev(m.rp)[0]
        for var in (0, 1, 2):
            plan = lbmod.Plan(rp, m.nnz, "thread_mapped", mp_variant=var)
            got = plan.atom_tiles().cpu().numpy()
            assert np.array_equal(got, oracle.row_of_atom(m.rp)), (name, var)


def test_validation_reports_bad_inputs(lbmod):
    import torch
    from paper_2301_04792_gb300._lib import LBError
    m = W.plain(500, 500, 5, seed=3)
    rp, ci, v, x = to_dev(m.rp, m.ci, m.v, W.x_for(m))
    bad_rp = rp.clone()
    bad_rp[10] = bad_rp[11] + 1  # decreasing offsets
    with pytest.raises(LBError) as ei:
        lbmod.Plan(bad_rp, m.nnz, "merge_path", validate=True)
    assert ei.value.status == 1
    bad_end = rp.clone()
    bad_end[-1] = m.nnz - 1
    with pytest.raises(LBError):
        lbmod.Plan(bad_end, m.nnz, "thread_mapped", validate=True)
    # out-of-range columns read as 0 and are reported by lb_status
    bad_ci = ci.clone()
    bad_ci[17] = 500
    for s, kw in (("thread_mapped", {}), ("thread_mapped", {"staged": True}), ("warp_mapped", {}),
                  ("merge_path", {}), ("merge_path", {"mp_variant": 3})):
        p = lbmod.Plan(rp, m.nnz, s, num_cols=500, validate=True, **kw)
        p.spmv(ci, v, x)
        p.status()  # clean
        p.spmv(bad_ci, v, x)
        with pytest.raises(LBError) as ei:
            p.status()
        assert ei.value.status == 6
        p.status()  # cleared
    # backward rejects out-of-range columns before using them as addresses
    p = lbmod.Plan(rp, m.nnz, "merge_path")
    with pytest.raises(LBError) as ei:
        p.prepare_backward(500, bad_ci)
    assert ei.value.status == 6


def test_bad_arguments_do_not_launch(lbmod):
    import torch
    from paper_2301_04792_gb300._lib import LBError
    m = W.plain(100, 100, 3, seed=3)
    rp = to_dev(m.rp)[0]
    with pytest.raises(LBError):
        lbmod.Plan(rp, m.nnz, "group_mapped", group_size=12)
    with pytest.raises(LBError):
        lbmod.Plan(rp, m.nnz, "merge_path", items_per_thread=5)
    with pytest.raises(LBError):
        lbmod.Plan(rp, -1, "merge_path")


def test_auto_schedule_follows_heuristic(lbmod):
    small = W.plain(400, 400, 10, seed=1)  # 4000 nnz, rows < 500
    big = W.plain(2000, 2000, 10, seed=1)
    assert lbmod.Plan(to_dev(small.rp)[0], small.nnz, "auto", num_cols=400).info()["schedule"] == "thread_mapped"
    assert lbmod.Plan(to_dev(big.rp)[0], big.nnz, "auto", num_cols=2000).info()["schedule"] == "merge_path"


# ------------------------------------------------------------ full sizes --

def full_size_check(lb, m, x, schedules, sample_rows=None):
    """Every row (or the sampled ones) within the bound, 3 runs bit-identical."""
    import torch
    rp, ci, v, xd = to_dev(m.rp, m.ci, m.v, x)
    if sample_rows is None:
        y64, b = oracle.spmv(m.rp, m.ci, m.v, x)
    else:
        y64, b = oracle.spmv_rows(sample_rows, m.rp, m.ci, m.v, x)
    for s, o in schedules:
        plan = lb.Plan(rp, m.nnz, s, num_cols=m.num_cols, **o)
        ys = []
        for _ in range(3):
            y = torch.empty(m.num_rows, device="cuda")
            plan.spmv(ci, v, xd, y)
            ys.append(y)
        y0 = ys[0].cpu().numpy()
        got = y0 if sample_rows is None else y0[sample_rows]
        assert_within_bound(got, y64, b, f"{m.name}/{s}")
        for y in ys[1:]:
            assert torch.equal(y.view(torch.int32), ys[0].view(torch.int32)), f"{m.name}/{s}: not bit-identical"
        del plan
    torch.cuda.synchronize()


def test_full_plain_2000(lbmod):
    m = W.plain()
    full_size_check(lbmod, m, W.x_for(m), [("thread_mapped", {}), ("merge_path", {})])


def test_full_powerlaw_1M(lbmod):
    m = W.powerlaw()
    assert (np.diff(m.rp) > 100_000).sum() >= 3
    full_size_check(lbmod, m, W.x_for(m), SCHEDULES)


def test_full_rmat_and_stencil(lbmod):
    sched = [("thread_mapped", {}), ("thread_mapped", {"staged": True}), ("warp_mapped", {}), ("block_mapped", {}),
             ("merge_path", {}), ("merge_path", {"items_per_thread": 8, "mp_variant": 3})]
    m = W.rmat()
    full_size_check(lbmod, m, W.x_for(m), sched)
    del m
    m = W.stencil27()
    assert m.nnz == 109_215_352
    full_size_check(lbmod, m, W.x_for(m), sched)


def test_lookback_rows_spanning_many_shares(lbmod):
    """Variant 3 with one-tile shares: rows of 50,000 and 70,000 atoms span hundreds
    of shares, so the look-back walks many 32-share windows; repeated runs are
    bit-identical."""
    import torch
    m = W.from_lengths(np.array([50_000, 3, 0, 70_000, 1, 0, 0, 40, 5000]), 120_000, seed=8)
    x = W.x_for(m)
    y64, b = oracle.spmv(m.rp, m.ci, m.v, x)
    rp, ci, v, xd = to_dev(m.rp, m.ci, m.v, x)
    for ipt in (4, 8):
        plan = lbmod.Plan(rp, m.nnz, "merge_path", items_per_thread=ipt, mp_variant=3, tiles_per_share=1)
        assert plan.info()["num_workers"] >= m.nnz // (32 * ipt)
        ys = [plan.spmv(ci, v, xd) for _ in range(3)]
        assert_within_bound(ys[0].cpu().numpy(), y64, b, f"lookback ipt={ipt}")
        for y in ys[1:]:
            assert torch.equal(y.view(torch.int32), ys[0].view(torch.int32))
        plan.status()
