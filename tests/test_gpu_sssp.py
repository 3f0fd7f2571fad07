"""GPU SSSP (Listing 5, group-mapped) against the oracle's float Dijkstra: the
distances are the least fixed point of dist[v] = min fl32(dist[u] + w), so they
must agree bit for bit, for every group size, on degenerate graphs and on the
full R-MAT graph."""
import numpy as np
import pytest

import oracle
import workloads as W
from helpers import to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbmod():
    import paper_2301_04792_gb300 as lb
    lb.build()
    return lb


def graph(V, lengths_seed, zero_frac=0.0, lmax=12):
    rng = np.random.default_rng(lengths_seed)
    m = W.from_lengths(np.minimum(rng.integers(0, lmax + 1, V), V).astype(np.int64), V, seed=lengths_seed)
    w = np.abs(m.v).astype(np.float32)
    w[rng.random(w.shape[0]) < zero_frac] = 0.0
    return m.rp, m.ci, w


def check(lb, rp, ci, w, source, groups=(32,)):
    d_ref = oracle.sssp(rp, ci, w, source)
    rpd, cid, wd = to_dev(rp, ci, w)
    for G in groups:
        outs = [lb.sssp(rpd, cid, wd, source, group_size=G) for _ in range(2)]
        for d, it in outs:
            got = d.cpu().numpy()
            assert np.array_equal(got.view(np.int32), d_ref.view(np.int32)), \
                f"G={G}: {int((got != d_ref).sum())} distances differ"
            assert it >= 1


def test_sssp_small_graphs_all_group_sizes(lbmod):
    for V, seed, zf in ((1, 0, 0.0), (2, 1, 0.0), (50, 2, 0.0), (300, 3, 0.2), (2000, 4, 0.0), (5000, 5, 0.5)):
        rp, ci, w = graph(V, seed, zf)
        check(lbmod, rp, ci, w, 0, groups=(4, 8, 16, 32, 64, 128, 256))
        if V > 1:
            check(lbmod, rp, ci, w, V - 1)


def test_sssp_degenerate_graphs(lbmod):
    # self loops and duplicate edges, an isolated source, a chain, all-zero weights
    rp = np.array([0, 3, 4, 6, 6], np.int32)
    ci = np.array([0, 1, 1, 2, 2, 3], np.int32)
    w = np.array([0.5, 0.25, 0.125, 1.0, 0.75, 2.0], np.float32)
    check(lbmod, rp, ci, w, 0, groups=(4, 32, 256))
    check(lbmod, rp, ci, w, 3)                      # no out-edges: only the source is reachable
    n = 4000
    rp = np.arange(n + 1, dtype=np.int32)
    rp[-1] = n - 1
    rp = np.minimum(rp, n - 1)
    ci = np.arange(1, n, dtype=np.int32)
    w = np.full(n - 1, 0.1, np.float32)
    check(lbmod, rp, ci, w, 0)                      # a chain: n - 1 frontier iterations
    rpz, ciz, wz = graph(1000, 7)
    check(lbmod, rpz, ciz, np.zeros_like(wz), 5)    # zero weights: every reachable vertex at 0


def test_sssp_full_rmat(lbmod):
    m = W.rmat()
    check(lbmod, m.rp, m.ci, m.v.astype(np.float32), 0)


def test_sssp_rejects_bad_input(lbmod):
    import torch
    from paper_2301_04792_gb300 import _lib
    rp, ci, w = graph(100, 9)
    rpd, cid, wd = to_dev(rp, ci, w)
    with pytest.raises(_lib.LBError):
        lbmod.sssp(rpd, cid, wd, 100)                         # source out of range
    with pytest.raises(_lib.LBError):
        lbmod.sssp(rpd, cid, wd, 0, group_size=48)            # not a power of two
    wn = wd.clone()
    wn[3] = -1.0
    with pytest.raises(_lib.LBError):
        lbmod.sssp(rpd, cid, wn, 0)                           # negative weight
    cb = cid.clone()
    cb[0] = 100
    with pytest.raises(_lib.LBError):
        lbmod.sssp(rpd, cb, wd, 0)                            # head out of range
    d, it = lbmod.sssp(rpd, cid, wd, 0)                       # the context still works
    assert np.array_equal(d.cpu().numpy(), oracle.sssp(rp, ci, w, 0))
