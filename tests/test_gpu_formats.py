"""COO and CSC inputs turned into CSR tile sets on the GPU: bit-identical to the
oracle's stable counting sort, and SpMV over the result equals SpMV over the
original CSR."""
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


def coo_of(m, rng, shuffle=True):
    row = np.repeat(np.arange(m.num_rows, dtype=np.int32), np.diff(m.rp))
    order = rng.permutation(m.nnz) if shuffle else np.arange(m.nnz)
    return row[order], m.ci[order], m.v[order]


def test_coo_to_csr_matches_oracle(lbmod):
    rng = np.random.default_rng(41)
    cases = [W.plain(300, 200, 5, seed=1), W.powerlaw(20_000, 15_000, 300_000, lmax=8000, plant_long=False, seed=2),
             W.from_lengths(np.array([0, 0, 7, 0, 1, 0]), 9, seed=3), W.from_lengths(np.zeros(4, np.int64), 3, seed=4)]
    for m in cases:
        for shuffle in (True, False):
            row, col, val = coo_of(m, rng, shuffle)
            rp_o, ci_o, v_o = oracle.coo_to_csr(m.num_rows, row, col, val)
            rp, ci, v = lbmod.coo_to_csr(m.num_rows, *to_dev(row, col, val))
            assert np.array_equal(rp.cpu().numpy(), rp_o)
            assert np.array_equal(ci.cpu().numpy(), ci_o)
            assert np.array_equal(v.cpu().numpy().view(np.int32), v_o.view(np.int32))
            if not shuffle:  # a row-sorted COO comes back as the CSR it came from
                assert np.array_equal(rp_o, m.rp) and np.array_equal(ci_o, m.ci)
    # duplicates keep their input order
    row = np.array([2, 0, 2, 2, 0], np.int32)
    col = np.array([1, 1, 1, 0, 1], np.int32)
    val = np.array([1, 2, 3, 4, 5], np.float32)
    rp, ci, v = lbmod.coo_to_csr(3, *to_dev(row, col, val))
    assert rp.cpu().tolist() == [0, 2, 2, 5] and v.cpu().tolist() == [2, 5, 1, 3, 4]


def test_csc_to_csr_then_spmv(lbmod):
    for m in (W.powerlaw(30_000, 25_000, 500_000, lmax=10_000, plant_long=False, seed=5), W.plain(500, 700, 9, seed=6)):
        cp, riT, perm = oracle.transpose(m.rp, m.ci, m.num_cols)
        rp_o, ci_o, v_o = oracle.csc_to_csr(m.num_rows, cp, riT, m.v[perm])
        rp, ci, v = lbmod.csc_to_csr(m.num_rows, *to_dev(cp, riT, m.v[perm]))
        assert np.array_equal(rp.cpu().numpy(), rp_o) and np.array_equal(ci.cpu().numpy(), ci_o)
        assert np.array_equal(v.cpu().numpy(), v_o)
        assert np.array_equal(rp_o, m.rp) and np.array_equal(ci_o, m.ci)  # sorted columns: back to the original
        x = W.x_for(m)
        y64, b = oracle.spmv(m.rp, m.ci, m.v, x)
        plan = lbmod.Plan(rp, m.nnz, "merge_path")
        assert_within_bound(plan.spmv(ci, v, to_dev(x)[0]).cpu().numpy(), y64, b, "SpMV after CSC input")


def test_formats_reject_bad_input(lbmod):
    from paper_2301_04792_gb300 import _lib
    row = np.array([0, 5], np.int32)
    col = np.array([0, 0], np.int32)
    val = np.ones(2, np.float32)
    with pytest.raises(_lib.LBError):
        lbmod.coo_to_csr(5, *to_dev(row, col, val))             # row 5 of 5
    cp = np.array([0, 2, 1], np.int32)                          # decreasing offsets
    with pytest.raises(_lib.LBError):
        lbmod.csc_to_csr(3, *to_dev(cp, np.array([0, 1], np.int32), val))
