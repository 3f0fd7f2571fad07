"""GPU parity of the differentiable path: transpose (bit-exact), dx = A^T dy (bound),
dvals = fl32(dy[row] x[col]) (bit-exact), the autograd Function and FP64 finite differences."""
import numpy as np
import pytest

import oracle
import workloads as W
from helpers import assert_within_bound, edge_cases, small_cases, to_dev

pytestmark = pytest.mark.gpu

BWD_SCHEDULES = [("thread_mapped", {}), ("thread_mapped", {"staged": True}), ("warp_mapped", {}), ("block_mapped", {}),
                 ("group_mapped", {"group_size": 8}), ("merge_path", {"items_per_thread": 4}),
                 ("merge_path", {"items_per_thread": 8}), ("merge_path", {"items_per_thread": 16}),
                 ("merge_path", {"items_per_thread": 8, "mp_variant": 1}),
                 ("merge_path", {"items_per_thread": 8, "mp_variant": 2}),
                 ("merge_path", {"items_per_thread": 8, "units_per_cta": 8}),
                 ("merge_path", {"items_per_thread": 4, "row_weight": 3}),
                 ("merge_path", {"items_per_thread": 8, "mp_variant": 3, "tiles_per_share": 2})]


@pytest.fixture(scope="module")
def lbmod():
    import paper_2301_04792_gb300 as lb
    lb.build()
    return lb


def check_backward(lb, m, schedules, seed=0):
    import torch
    x = W.x_for(m, seed=seed)
    dy = W.dy_for(m, seed=seed)
    dx64, bx, dv32 = oracle.grad(m.rp, m.ci, m.v, x, dy, m.num_cols)
    cp_o, riT_o, perm_o = oracle.transpose(m.rp, m.ci, m.num_cols)
    rp, ci, v, xd, dyd = to_dev(m.rp, m.ci, m.v, x, dy)
    for s, o in schedules:
        plan = lb.Plan(rp, m.nnz, s, num_cols=m.num_cols, **o)
        plan.prepare_backward(m.num_cols, ci)
        cp, riT, perm = plan.transpose()
        assert np.array_equal(cp.cpu().numpy(), cp_o), f"{m.name}: cp"
        assert np.array_equal(riT.cpu().numpy(), riT_o), f"{m.name}: riT"
        assert np.array_equal(perm.cpu().numpy(), perm_o), f"{m.name}: perm"
        outs = [plan.backward(m.num_cols, ci, v, xd, dyd) for _ in range(3)]
        dx, dvals = outs[0]
        assert_within_bound(dx.cpu().numpy(), dx64, bx, f"{m.name}/{s}: dx")
        assert np.array_equal(dvals.cpu().numpy().view(np.uint32), dv32.view(np.uint32)), f"{m.name}/{s}: dvals"
        for dx2, dv2 in outs[1:]:
            assert torch.equal(dx2.view(torch.int32), dx.view(torch.int32)), "dx not bit-identical"
            assert torch.equal(dv2.view(torch.int32), dvals.view(torch.int32))
        # transposed merge-path table is bit-exact too
        if s == "merge_path":
            diag, ij = plan.splits(1)
            assert np.array_equal(ij, oracle.merge_splits(diag, cp_o))


def test_backward_small_cases(lbmod):
    for name, m in small_cases() + edge_cases():
        check_backward(lbmod, m, BWD_SCHEDULES)


def test_backward_only_one_output(lbmod):
    m = W.plain(1000, 800, 7, seed=5)
    x, dy = W.x_for(m), W.dy_for(m)
    dx64, bx, dv32 = oracle.grad(m.rp, m.ci, m.v, x, dy, m.num_cols)
    rp, ci, v, xd, dyd = to_dev(m.rp, m.ci, m.v, x, dy)
    p = lbmod.Plan(rp, m.nnz, "merge_path")
    dx, dv = p.backward(m.num_cols, ci, v, xd, dyd, want_dx=False)
    assert dx is None and np.array_equal(dv.cpu().numpy(), dv32)
    dx, dv = p.backward(m.num_cols, ci, v, xd, dyd, want_dvals=False)
    assert dv is None
    assert_within_bound(dx.cpu().numpy(), dx64, bx, "dx only")


def test_dvals_and_atom_tiles_on_unaligned_buffers(lbmod):
    """The expand kernel loads column indices as 16-byte vectors and stores a vector lying wholly inside
    a tile with one 16-byte store only when the buffers are 16-byte aligned: every mix of aligned and
    offset buffers gives the same bits, and nothing is written outside the output."""
    import torch
    m = W.powerlaw(20_000, 20_000, 400_000, lmax=20_000, seed=4)
    x, dy = W.x_for(m), W.dy_for(m)
    _, _, dv32 = oracle.grad(m.rp, m.ci, m.v, x, dy, m.num_cols, want_dx=False)
    rows = oracle.row_of_atom(m.rp)
    rp, v, xd, dyd = to_dev(m.rp, m.v, x, dy)
    ci_buf = torch.zeros(m.nnz + 1, dtype=torch.int32, device="cuda")
    for opts in ({"items_per_thread": 4}, {"items_per_thread": 8}, {"items_per_thread": 4, "mp_variant": 3}):
        plan = lbmod.Plan(rp, m.nnz, "merge_path", num_cols=m.num_cols, **opts)
        for ci_off in (0, 1):
            ci = ci_buf[ci_off:ci_off + m.nnz]
            ci.copy_(torch.from_numpy(m.ci))
            for out_off in (0, 1, 3):
                dv_buf = torch.full((m.nnz + 4,), float("nan"), device="cuda")
                dv = dv_buf[out_off:out_off + m.nnz]
                plan.backward(m.num_cols, ci, v, xd, dyd, want_dx=False, dvals=dv)
                assert np.array_equal(dv.cpu().numpy().view(np.uint32), dv32.view(np.uint32)), (opts, ci_off, out_off)
                assert torch.isnan(dv_buf[:out_off]).all() and torch.isnan(dv_buf[out_off + m.nnz:]).all()
        for out_off in (0, 1, 2):
            t_buf = torch.full((m.nnz + 4,), -7, dtype=torch.int32, device="cuda")
            t = t_buf[out_off:out_off + m.nnz]
            plan.atom_tiles(out=t)
            assert np.array_equal(t.cpu().numpy(), rows), (opts, out_off)
            assert bool((t_buf[:out_off] == -7).all()) and bool((t_buf[out_off + m.nnz:] == -7).all())


def test_autograd_function(lbmod):
    import torch
    m = W.powerlaw(4000, 3000, 60_000, lmax=3000, plant_long=False, seed=6)
    x, dy = W.x_for(m), W.dy_for(m)
    y64, b = oracle.spmv(m.rp, m.ci, m.v, x)
    dx64, bx, dv32 = oracle.grad(m.rp, m.ci, m.v, x, dy, m.num_cols)
    rp, ci, v, xd, dyd = to_dev(m.rp, m.ci, m.v, x, dy)
    for s in ("thread_mapped", "block_mapped", "merge_path"):
        plan = lbmod.Plan(rp, m.nnz, s, num_cols=m.num_cols)
        vv = v.clone().requires_grad_(True)
        xx = xd.clone().requires_grad_(True)
        y = lbmod.spmv(plan, ci, vv, xx)
        assert_within_bound(y.detach().cpu().numpy(), y64, b, f"autograd fwd {s}")
        (y * dyd).sum().backward()
        assert_within_bound(xx.grad.cpu().numpy(), dx64, bx, f"autograd dx {s}")
        assert np.array_equal(vv.grad.cpu().numpy(), dv32)


def test_finite_differences_500x500(lbmod):
    """FP64 central differences of L = dy . (A x) on the 500x500, 5000-nnz instance."""
    m = W.from_lengths(np.full(500, 10), 500, seed=5)
    x = W.vector(500, W.U_PM1, 5, 1)
    dy = W.vector(500, W.NORMAL, 5, 2)
    rp, ci, v, xd, dyd = to_dev(m.rp, m.ci, m.v, x, dy)
    plan = lbmod.Plan(rp, m.nnz, "merge_path", num_cols=500)
    dx, dvals = plan.backward(500, ci, v, xd, dyd)
    dx, dvals = dx.cpu().numpy().astype(np.float64), dvals.cpu().numpy().astype(np.float64)
    row_of = np.repeat(np.arange(500), np.diff(m.rp))
    A = np.zeros((500, 500))
    A[row_of, m.ci] = m.v
    d64 = dy.astype(np.float64)
    h = 1e-3
    for c in range(0, 500, 7):
        e = np.zeros(500)
        e[c] = h
        fd = (d64 @ (A @ (x + e)) - d64 @ (A @ (x - e))) / (2 * h)
        bound = np.abs(A[:, c]) @ np.abs(d64)
        assert abs(dx[c] - fd) <= 1e-5 * bound + 1e-12, c
    xs = x.astype(np.float64)[m.ci]
    for k in range(0, m.nnz, 37):
        fd = d64[row_of[k]] * xs[k]  # exact derivative of the bilinear loss in v_k
        Ap = A.copy()
        Ap[row_of[k], m.ci[k]] += h
        Am = A.copy()
        Am[row_of[k], m.ci[k]] -= h
        fdn = (d64 @ (Ap @ x) - d64 @ (Am @ x)) / (2 * h)
        assert abs(fdn - fd) <= 1e-9
        assert abs(dvals[k] - fdn) <= 1e-6 * abs(fdn) + 1e-12


def test_full_powerlaw_backward(lbmod):
    m = W.powerlaw()
    check_backward(lbmod, m, [("thread_mapped", {}), ("merge_path", {})])
