"""GPU parity of the batched persistent merge-path form (forward and backward),
its CUDA-graph replay, and the batched workloads at full size."""
import numpy as np
import pytest

import oracle
import workloads as W
from helpers import assert_within_bound, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbmod():
    import paper_2301_04792_gb300 as lb
    lb.build()
    return lb


def batch_inputs(b, seed=0):
    xs = [W.x_for(m, seed=seed + i) for i, m in enumerate(b.mats)]
    dys = [W.dy_for(m, seed=seed + i) for i, m in enumerate(b.mats)]
    return xs, dys


def oracle_batch(b, xs, dys):
    y64, yb, dx64, dxb, dv = [], [], [], [], []
    for m, x, dy in zip(b.mats, xs, dys):
        y, bb = oracle.spmv(m.rp, m.ci, m.v, x)
        d, db, g = oracle.grad(m.rp, m.ci, m.v, x, dy, m.num_cols)
        y64.append(y), yb.append(bb), dx64.append(d), dxb.append(db), dv.append(g)
    cat = lambda a, dt: np.concatenate(a).astype(dt) if a else np.zeros(0, dt)
    return (cat(y64, np.float64), cat(yb, np.float64), cat(dx64, np.float64), cat(dxb, np.float64),
            cat(dv, np.float32))


def make_plan(lb, b, **kw):
    rp_cat, ci, v = to_dev(b.rp_cat(), b.ci_cat(), b.v_cat())
    plan = lb.BatchPlan(b.rows(), b.cols(), b.nnz(), rp_cat, **kw)
    return plan, rp_cat, ci, v


def check_batch(lb, b, ipts=(8,), variants=(0, 1, 2, 3), wave_items=0, units=0):
    import torch
    xs, dys = batch_inputs(b)
    y64, yb, dx64, dxb, dv32 = oracle_batch(b, xs, dys)
    xd, dyd = to_dev(np.concatenate(xs), np.concatenate(dys))
    row_of = np.concatenate([oracle.row_of_atom(m.rp) for m in b.mats])
    for ipt, var in [(i, v) for i in ipts for v in variants]:
        plan, rp_cat, ci, v = make_plan(lb, b, items_per_thread=ipt, mp_variant=var, wave_items=wave_items,
                                        units_per_cta=units)
        ys = [plan.spmv(ci, v, xd) for _ in range(3)]
        assert_within_bound(ys[0].cpu().numpy(), y64, yb, "batch y")
        for y in ys[1:]:
            assert torch.equal(y.view(torch.int32), ys[0].view(torch.int32))
        tiles = plan.atom_tiles().cpu().numpy()
        row_base = np.concatenate([[0], np.cumsum(b.rows())])[:-1]
        mat_of_atom = np.repeat(np.arange(b.num), b.nnz())
        assert np.array_equal(tiles - row_base[mat_of_atom], row_of)
        outs = [plan.backward(ci, v, xd, dyd) for _ in range(2)]
        dx, dvals = outs[0]
        assert_within_bound(dx.cpu().numpy(), dx64, dxb, "batch dx")
        assert np.array_equal(dvals.cpu().numpy().view(np.uint32), dv32.view(np.uint32))
        assert torch.equal(outs[1][0].view(torch.int32), dx.view(torch.int32))


def test_small_batch(lbmod):
    b = W.batch(num=40, rmin=50, rmax=5000, mmin=1, mmax=64, seed=3)
    check_batch(lbmod, b, ipts=(4, 8, 16))
    check_batch(lbmod, b, ipts=(8,), variants=(0,), units=8)  # dynamic units, one wave


def test_small_batch_in_waves(lbmod):
    """Waves of whole matrices (forced small) give the same results."""
    b = W.batch(num=40, rmin=50, rmax=5000, mmin=1, mmax=64, seed=3)
    for wave_items in (1, 20_000, 100_000):
        plan, rp_cat, ci, v = make_plan(lbmod, b, wave_items=wave_items)
        assert plan.info()["num_waves"] > 1
    check_batch(lbmod, b, ipts=(4, 8), variants=(0,), wave_items=20_000)
    check_batch(lbmod, b, ipts=(8,), variants=(0,), wave_items=1)
    check_batch(lbmod, b, ipts=(4,), variants=(0,), wave_items=20_000, units=4)


def test_batch_with_degenerate_members(lbmod):
    mats = [W.from_lengths(np.zeros(5, np.int64), 3, seed=1),           # all-empty rows
            W.from_lengths(np.array([1]), 1, seed=2),                   # 1x1
            W.powerlaw(3000, 3000, 50_000, lmax=3000, plant_long=False, seed=3),
            W.from_lengths(np.array([20000]), 30000, seed=4),           # one long row
            W.from_lengths(np.ones(7, np.int64), 1, seed=5),            # one column
            W.plain(300, 300, 3, seed=6)]
    check_batch(lbmod, W.Batch(mats), ipts=(4, 16))


def test_single_matrix_batch_equals_oracle(lbmod):
    b = W.Batch([W.powerlaw(20000, 20000, 400_000, lmax=20000, plant_long=False, seed=9)])
    check_batch(lbmod, b)


def test_batched_graph_replay(lbmod):
    """Forward + backward captured once in a CUDA graph and replayed give the same bits."""
    import torch
    b = W.batch(num=24, rmin=100, rmax=20000, seed=4)
    xs, dys = batch_inputs(b)
    y64, yb, dx64, dxb, dv32 = oracle_batch(b, xs, dys)
    plan, rp_cat, ci, v = make_plan(lbmod, b, wave_items=50_000)
    assert plan.info()["num_waves"] > 1
    xd, dyd = to_dev(np.concatenate(xs), np.concatenate(dys))
    plan.prepare_backward(ci)
    y = torch.empty(plan.total_rows, device="cuda")
    dx = torch.empty(plan.total_cols, device="cuda")
    dv = torch.empty(plan.total_nnz, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        plan.spmv(ci, v, xd, y)
        plan.backward(ci, v, xd, dyd, dx_cat=dx, dvals_cat=dv)
    torch.cuda.current_stream().wait_stream(s)
    ref = (y.clone(), dx.clone(), dv.clone())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        plan.spmv(ci, v, xd, y)
        plan.backward(ci, v, xd, dyd, dx_cat=dx, dvals_cat=dv)
    for _ in range(3):
        y.zero_(), dx.zero_(), dv.zero_()
        g.replay()
        torch.cuda.synchronize()
        for a, r in zip((y, dx, dv), ref):
            assert torch.equal(a.view(torch.int32), r.view(torch.int32))
    assert_within_bound(y.cpu().numpy(), y64, yb, "graph y")
    assert_within_bound(dx.cpu().numpy(), dx64, dxb, "graph dx")


# the configuration bench.py times for both batched workloads (look-back shares, items_per_thread 4)
BENCHED = dict(mp_variant=3, items_per_thread=4)


def test_full_batch_512(lbmod):
    """The 512-matrix batch at full size: forward on every row, for the library's
    default batch plan and for the plan the bench times; repeated runs bit-identical."""
    import torch
    b = W.batch()
    xs = [W.x_for(m, seed=i) for i, m in enumerate(b.mats)]
    ref = [oracle.spmv(m.rp, m.ci, m.v, x) for m, x in zip(b.mats, xs)]
    y64 = np.concatenate([r[0] for r in ref])
    yb = np.concatenate([r[1] for r in ref])
    xd = to_dev(np.concatenate(xs))[0]
    for kw in ({}, BENCHED):
        plan, rp_cat, ci, v = make_plan(lbmod, b, **kw)
        ys = [plan.spmv(ci, v, xd) for _ in range(4)]
        assert_within_bound(ys[0].cpu().numpy(), y64, yb, f"batch512 y {kw}")
        for y in ys[1:]:
            assert torch.equal(y.view(torch.int32), ys[0].view(torch.int32)), f"batch512 {kw}: not bit-identical"
        plan.close()
        del rp_cat, ci, v


def test_full_differentiable_batch_64(lbmod):
    """64 power-law matrices of 2^20 rows (~16M nnz each): y, dx and dvals of
    every matrix against the oracle (y and dx within the bound, dvals bit-exact),
    for the default batch plan and for the plan the bench times; a second pass
    bit-identical."""
    import torch
    b = W.diff_batch()
    xs, dys = batch_inputs(b)
    xd, dyd = to_dev(np.concatenate(xs), np.concatenate(dys))
    rows, cols, nnz = b.rows(), b.cols(), b.nnz()
    rb = np.concatenate([[0], np.cumsum(rows)])
    cb = np.concatenate([[0], np.cumsum(cols)])
    nb = np.concatenate([[0], np.cumsum(nnz)])
    results = {}
    for name, kw in (("default", {}), ("benched", BENCHED)):
        plan, rp_cat, ci, v = make_plan(lbmod, b, **kw)
        y = plan.spmv(ci, v, xd)
        dx, dvals = plan.backward(ci, v, xd, dyd)
        y2 = plan.spmv(ci, v, xd)
        dx2, dvals2 = plan.backward(ci, v, xd, dyd)
        assert torch.equal(y.view(torch.int32), y2.view(torch.int32)), name
        assert torch.equal(dx.view(torch.int32), dx2.view(torch.int32)), name
        assert torch.equal(dvals.view(torch.int32), dvals2.view(torch.int32)), name
        results[name] = (y.cpu().numpy(), dx.cpu().numpy(), dvals.cpu().numpy())
        plan.close()
        del rp_cat, ci, v, y, dx, dvals, y2, dx2, dvals2
        torch.cuda.empty_cache()
    for mi, m in enumerate(b.mats):
        y64, yb = oracle.spmv(m.rp, m.ci, m.v, xs[mi])
        dx64, dxb, dv32 = oracle.grad(m.rp, m.ci, m.v, xs[mi], dys[mi], m.num_cols)
        for name, (y, dx, dvals) in results.items():
            assert_within_bound(y[rb[mi]:rb[mi + 1]], y64, yb, f"diff y m{mi} {name}")
            assert_within_bound(dx[cb[mi]:cb[mi + 1]], dx64, dxb, f"diff dx m{mi} {name}")
            assert np.array_equal(dvals[nb[mi]:nb[mi + 1]].view(np.uint32), dv32.view(np.uint32)), (mi, name)


def test_batch_autotune_fwd_bwd_matches_oracle(lbmod):
    """lb_batch_autotune times every batch candidate over fwd + dx + dvals, picks the
    fastest, and the winner's outputs and plan agree with the oracle; a second call
    is a cache hit with the same choice."""
    import torch
    b = W.batch(num=40, rmin=50, rmax=5000, mmin=1, mmax=64, seed=3)
    xs, dys = batch_inputs(b)
    y64, yb, dx64, dxb, dv32 = oracle_batch(b, xs, dys)
    rp_cat, ci, v, xd, dyd = to_dev(b.rp_cat(), b.ci_cat(), b.v_cat(), np.concatenate(xs), np.concatenate(dys))
    lbmod.autotune_cache_clear()
    plan, rep = lbmod.batch_autotune(b.rows(), b.cols(), b.nnz(), rp_cat, ci, v, xd, dyd, passes="fwd+dx+dvals",
                                     reps=3)
    cands = rep["candidates"]
    assert len(cands) == 7 and all(c["status"] == 0 and c["ms"] > 0 for c in cands), cands
    best_ms = min(c["ms"] for c in cands)
    assert rep["best"] == next(c["name"] for c in cands if c["ms"] == best_ms)
    assert not rep["from_cache"]
    assert_within_bound(rep["y"].cpu().numpy(), y64, yb, "tuned batch y")
    assert_within_bound(rep["dx"].cpu().numpy(), dx64, dxb, "tuned batch dx")
    assert np.array_equal(rep["dvals"].cpu().numpy().view(np.uint32), dv32.view(np.uint32))
    # the returned plan is the winner and runs on its own
    assert plan.info()["mp_variant"] == rep["best_opts"]["mp_variant"]
    y = plan.spmv(ci, v, xd)
    assert torch.equal(y.view(torch.int32), rep["y"].view(torch.int32))
    _, rep2 = lbmod.batch_autotune(b.rows(), b.cols(), b.nnz(), rp_cat, ci, v, xd, dyd, passes="fwd+dx+dvals",
                                   reps=3)
    assert rep2["from_cache"] and rep2["best"] == rep["best"]
    assert_within_bound(rep2["y"].cpu().numpy(), y64, yb, "cached tuned batch y")
    # forward only is another key
    _, rep3 = lbmod.batch_autotune(b.rows(), b.cols(), b.nnz(), rp_cat, ci, v, xd, passes="fwd", reps=2)
    assert not rep3["from_cache"] and rep3["dx"] is None
    assert_within_bound(rep3["y"].cpu().numpy(), y64, yb, "fwd-only tuned batch y")
    lbmod.autotune_cache_clear()
