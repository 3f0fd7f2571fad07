"""The synthetic workload generators produce the shapes and structure they claim."""
import numpy as np
import pytest

import workloads as W


def check_csr(m):
    rp, ci = m.rp, m.ci
    assert rp.dtype == np.int32 and ci.dtype == np.int32 and m.v.dtype == np.float32
    assert rp[0] == 0 and (np.diff(rp) >= 0).all() and rp[-1] == len(ci) == len(m.v)
    assert ci.min(initial=0) >= 0 and ci.max(initial=-1) < m.num_cols
    # strictly increasing within each row: distinct and sorted
    d = np.diff(ci.astype(np.int64))
    row_start = np.zeros(len(ci), dtype=bool)
    row_start[rp[:-1][np.diff(rp) > 0]] = True
    assert (d[~row_start[1:]] > 0).all()


def test_plain_is_exact_and_deterministic():
    m = W.plain()
    check_csr(m)
    assert m.num_rows == 2000 and m.num_cols == 2000 and m.nnz == 20000
    assert (np.diff(m.rp) == 10).all()
    assert (np.abs(m.v) <= 1).all() and m.v.min() < -0.9 and m.v.max() > 0.9
    m2 = W.plain()
    assert np.array_equal(m.ci, m2.ci) and np.array_equal(m.v, m2.v)
    m3 = W.plain(seed=1)
    assert not np.array_equal(m.ci, m3.ci)
    # U(-1,1) values lie on the 2^-23 grid (exact in FP32)
    assert np.array_equal(np.round(m.v.astype(np.float64) * 2 ** 23), m.v.astype(np.float64) * 2 ** 23)


def test_powerlaw_small_shape():
    m = W.powerlaw(R=20000, C=20000, target_nnz=400000, lmax=15000, plant_long=False, seed=3)
    check_csr(m)
    L = np.diff(m.rp)
    assert abs(m.nnz - 400000) <= 0.03 * 400000
    assert 0.04 < (L == 0).mean() < 0.06
    assert L.max() <= 15000


@pytest.mark.slow
def test_powerlaw_full_size():
    m = W.powerlaw()
    check_csr(m)
    L = np.diff(m.rp)
    assert m.num_rows == 1_000_000
    assert abs(m.nnz - 20_000_000) <= 0.01 * 20_000_000
    assert (L > 100_000).sum() >= 3 and L.max() <= 200_000
    assert 0.045 < (L == 0).mean() < 0.055


def test_rmat_small_shape():
    m = W.rmat(scale=10, edge_factor=8, seed=2)
    check_csr(m)
    assert m.num_rows == 1024 and m.num_cols == 1024
    assert 0 < m.nnz <= 8 * 1024
    assert (m.v >= 0).all() and (m.v < 1).all()
    # skew: top-left quadrant (a = 0.57) holds the most edges
    row_of = np.repeat(np.arange(1024), np.diff(m.rp))
    tl = ((row_of < 512) & (m.ci < 512)).sum()
    br = ((row_of >= 512) & (m.ci >= 512)).sum()
    assert tl > 4 * br


def test_stencil_counts():
    n = 7
    m = W.stencil27(n)
    check_csr(m)
    assert m.nnz == (3 * n - 2) ** 3
    L = np.diff(m.rp)
    assert set(np.unique(L).tolist()) <= {8, 12, 18, 27}
    # diagonal entries are 27
    row_of = np.repeat(np.arange(n ** 3), L)
    diag = m.ci == row_of
    assert diag.sum() == n ** 3 and (m.v[diag] == 27).all()
    # pattern symmetric
    A = set(zip(row_of.tolist(), m.ci.tolist()))
    assert all((c, r) in A for (r, c) in A)


def test_batch_shapes():
    b = W.batch(num=16, rmin=100, rmax=2000, seed=1)
    assert b.num == 16
    R = b.rows()
    assert (R >= 100).all() and (R <= 2000).all()
    for m in b.mats:
        check_csr(m)
        assert m.num_rows == m.num_cols
    assert b.rp_cat().shape[0] == R.sum() + 16


def test_vectors():
    x = W.vector(10000, W.U_PM1, 0, 1)
    assert (np.abs(x) <= 1).all() and abs(x.mean()) < 0.05
    z = W.vector(100000, W.NORMAL, 0, 2)
    assert abs(z.mean()) < 0.02 and abs(z.std() - 1) < 0.02
    u = W.vector(10000, W.U_01, 0, 3)
    assert (u >= 0).all() and (u < 1).all()
    assert np.array_equal(W.vector(5000, W.U_PM1, 9, 1), W.vector(5000, W.U_PM1, 9, 1))
