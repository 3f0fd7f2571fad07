"""Accuracy on long all-positive rows and columns.

With values and x drawn from U(0,1) nothing cancels: every partial sum of a
row grows towards its total, so a summation order that adds thousands of
terms one after another into a single FP32 accumulator is where the bound
|y - y64| <= 1e-5 * sum_j |a_ij x_j| would fail first (the worst case of a
sequential sum of n terms is (n-1) * 2^-24 of the total).  These tests drive
rows of 100,000 to 200,000 atoms through every forward schedule, the
look-back shares with one tile per share (the most shares per row), the
batched plans, and dx over a column of 200,000 atoms; every result must stay
inside the bound and be bit-identical when repeated.
"""
import numpy as np
import pytest

import oracle
import workloads as W
from helpers import SCHEDULES, assert_within_bound, to_dev

pytestmark = pytest.mark.gpu

LONG = (100_000, 150_000, 200_000)


@pytest.fixture(scope="module")
def lbmod():
    import paper_2301_04792_gb300 as lb
    lb.build()
    return lb


def long_positive_rows(seed=21):
    """Rows of 100k, 150k and 200k atoms among 30,000 short rows (0-24 atoms,
    some empty), v and x ~ U(0,1)."""
    L = (np.arange(30_000, dtype=np.int64) * 7919) % 25
    for pos, n in zip((3, 12_345, 29_998), LONG):
        L[pos] = n
    m = W.from_lengths(L, 250_000, seed=seed, val_kind=W.U_01, name="long_positive")
    x = W.vector(m.num_cols, W.U_01, seed, 31)
    return m, x


def long_positive_column(seed=22):
    """A tile set whose column 0 holds 200,000 atoms: rows 0..199,999 are
    {0, c_r} with c_r uniform in [1, 4000); 5,000 more rows of 0-9 atoms.  v, x,
    dy ~ U(0,1), so dx[0] sums 200,000 positive terms."""
    n_long, C = 200_000, 4000
    tail = W.from_lengths((np.arange(5000, dtype=np.int64) * 31) % 10, C, seed=seed, val_kind=W.U_01)
    # second column of the long rows, drawn from the seeded vector stream and mapped into [1, C)
    u = W.vector(n_long, W.U_01, seed, 41).astype(np.float64)
    c2 = 1 + np.minimum((u * (C - 1)).astype(np.int64), C - 2)
    rp = np.concatenate([np.arange(0, 2 * n_long + 1, 2, dtype=np.int64), 2 * n_long + tail.rp[1:].astype(np.int64)])
    ci = np.empty(2 * n_long, dtype=np.int32)
    ci[0::2] = 0
    ci[1::2] = c2
    ci = np.concatenate([ci, tail.ci])
    v = np.concatenate([W.vector(2 * n_long, W.U_01, seed, 42), tail.v])
    m = W.CSR(rp.astype(np.int32), ci, v, C, name="long_positive_column")
    x = W.vector(C, W.U_01, seed, 43)
    dy = W.vector(m.num_rows, W.U_01, seed, 44)
    return m, x, dy


def test_long_positive_rows_all_schedules(lbmod):
    import torch
    m, x = long_positive_rows()
    assert sorted(np.diff(m.rp))[-3:] == list(LONG)
    y64, b = oracle.spmv(m.rp, m.ci, m.v, x)
    rp, ci, v, xd = to_dev(m.rp, m.ci, m.v, x)
    extra = [("merge_path", {"items_per_thread": 4, "mp_variant": 3, "tiles_per_share": 1}),
             ("merge_path", {"items_per_thread": 8, "mp_variant": 3, "tiles_per_share": 1})]
    for s, o in SCHEDULES + extra:
        plan = lbmod.Plan(rp, m.nnz, s, num_cols=m.num_cols, **o)
        ys = [plan.spmv(ci, v, xd) for _ in range(3)]
        assert_within_bound(ys[0].cpu().numpy(), y64, b, f"long positive rows/{s}{o}")
        for y in ys[1:]:
            assert torch.equal(y.view(torch.int32), ys[0].view(torch.int32)), f"{s}{o}: not bit-identical"


def test_long_positive_rows_batched(lbmod):
    import torch
    m, x = long_positive_rows()
    others = [W.powerlaw(20_000, 20_000, 300_000, lmax=20_000, plant_long=False, seed=5),
              W.from_lengths(np.array([180_000, 0, 7]), 200_000, seed=6, val_kind=W.U_01)]
    b = W.Batch([others[0], m, others[1]])
    xs = [W.vector(others[0].num_cols, W.U_01, 1, 31), x, W.vector(others[1].num_cols, W.U_01, 2, 31)]
    y64 = np.concatenate([oracle.spmv(mm.rp, mm.ci, mm.v, xx)[0] for mm, xx in zip(b.mats, xs)])
    yb = np.concatenate([oracle.spmv(mm.rp, mm.ci, mm.v, xx)[1] for mm, xx in zip(b.mats, xs)])
    rp_cat, ci, v, xd = to_dev(b.rp_cat(), b.ci_cat(), b.v_cat(), np.concatenate(xs))
    for kw in (dict(items_per_thread=4, mp_variant=3), dict(items_per_thread=8, mp_variant=3, tiles_per_share=1),
               dict(items_per_thread=4), dict(items_per_thread=8, wave_items=100_000)):
        plan = lbmod.BatchPlan(b.rows(), b.cols(), b.nnz(), rp_cat, **kw)
        ys = [plan.spmv(ci, v, xd) for _ in range(3)]
        assert_within_bound(ys[0].cpu().numpy(), y64, yb, f"batched long positive rows {kw}")
        for y in ys[1:]:
            assert torch.equal(y.view(torch.int32), ys[0].view(torch.int32))


def test_long_positive_column_dx(lbmod):
    import torch
    from helpers import SCHEDULES as S
    m, x, dy = long_positive_column()
    dx64, bx, dv32 = oracle.grad(m.rp, m.ci, m.v, x, dy, m.num_cols)
    cp, _, _ = oracle.transpose(m.rp, m.ci, m.num_cols)
    assert cp[1] - cp[0] >= 200_000
    rp, ci, v, xd, dyd = to_dev(m.rp, m.ci, m.v, x, dy)
    extra = [("merge_path", {"items_per_thread": 4, "mp_variant": 3, "tiles_per_share": 1})]
    for s, o in S + extra:
        plan = lbmod.Plan(rp, m.nnz, s, num_cols=m.num_cols, **o)
        outs = [plan.backward(m.num_cols, ci, v, xd, dyd) for _ in range(2)]
        dx, dvals = outs[0]
        assert_within_bound(dx.cpu().numpy(), dx64, bx, f"long positive column dx/{s}{o}")
        assert np.array_equal(dvals.cpu().numpy().view(np.uint32), dv32.view(np.uint32))
        assert torch.equal(outs[1][0].view(torch.int32), dx.view(torch.int32))
    # the same column through a batched plan (look-back shares, the configuration the bench times)
    b = W.Batch([m])
    rp_cat = to_dev(b.rp_cat())[0]
    plan = lbmod.BatchPlan(b.rows(), b.cols(), b.nnz(), rp_cat, mp_variant=3, items_per_thread=4)
    dx, dvals = plan.backward(ci, v, xd, dyd)
    assert_within_bound(dx.cpu().numpy(), dx64, bx, "batched long positive column dx")
    assert np.array_equal(dvals.cpu().numpy().view(np.uint32), dv32.view(np.uint32))
