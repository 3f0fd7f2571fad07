"""Pins for the CPU oracle against facts that do not come from the oracle itself.

Each check below uses an independent route: a dense brute-force product, a
closed form (row sums of small integers, identity, diagonal), a brute-force
merge built by sorting tagged items, a library special case (numpy's stable
argsort is a stable counting sort by column; searchsorted is get_tile), or a
finite difference of an exactly bilinear loss.  The mutation tests at the end
compile deliberately broken copies of ``oracle.c`` and show that these pins
reject each plausible mistake.
"""
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
from oracle import Oracle


def rand_csr(rng, R, C, density=None, empty_rows=(), full_rows=(), lengths=None):
    rows = []
    for i in range(R):
        if lengths is not None:
            L = int(lengths[i])
        elif i in empty_rows:
            L = 0
        elif i in full_rows:
            L = C
        else:
            dens = density if density is not None else rng.uniform(0, 1)
            L = int(rng.binomial(C, dens)) if C else 0
        cols = np.sort(rng.choice(C, size=L, replace=False)) if L else np.zeros(0, np.int64)
        rows.append(cols)
    rp = np.zeros(R + 1, dtype=np.int32)
    rp[1:] = np.cumsum([len(r) for r in rows]) if R else []
    ci = np.concatenate(rows).astype(np.int32) if R and rp[-1] else np.zeros(0, np.int32)
    v = rng.uniform(-1, 1, size=int(rp[-1])).astype(np.float32)
    return rp, ci, v


def dense_of(rp, ci, v, C):
    R = len(rp) - 1
    A = np.zeros((R, C), dtype=np.float64)
    for i in range(R):
        for k in range(rp[i], rp[i + 1]):
            A[i, ci[k]] += float(v[k])
    return A


def tiny_cases(seed=0, n=40):
    rng = np.random.default_rng(seed)
    out = []
    for t in range(n):
        R = int(rng.integers(0, 40))
        C = int(rng.integers(1, 40))
        empty = set(rng.choice(R, size=min(R, int(rng.integers(0, 5))), replace=False).tolist()) if R else set()
        full = {int(rng.integers(0, R))} if R and t % 3 == 0 else set()
        full -= empty
        out.append((C,) + rand_csr(rng, R, C, empty_rows=empty, full_rows=full))
    # hand-made degenerate shapes
    out.append((5, np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0, np.float32)))           # R = 0
    out.append((5, np.zeros(4, np.int32), np.zeros(0, np.int32), np.zeros(0, np.float32)))           # N = 0
    out.append((1, np.array([0, 1], np.int32), np.array([0], np.int32), np.array([0.5], np.float32)))  # 1x1
    return out


# ----------------------------------------------------------------- SpMV pins --

def check_spmv_dense(orc):
    rng = np.random.default_rng(7)
    for C, rp, ci, v in tiny_cases(1):
        x = rng.uniform(-1, 1, size=C).astype(np.float32)
        A = dense_of(rp, ci, v, C)
        y, b = orc.spmv(rp, ci, v, x)
        np.testing.assert_allclose(y, A @ x.astype(np.float64), rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(b, np.abs(A) @ np.abs(x.astype(np.float64)), rtol=1e-12, atol=1e-12)


def test_spmv_matches_dense_bruteforce():
    check_spmv_dense(oracle.default())


def test_spmv_rowsums_of_small_integers_are_exact():
    rng = np.random.default_rng(3)
    rp, ci, _ = rand_csr(rng, 50, 60, density=0.3, empty_rows={4, 9}, full_rows={7})
    v = rng.integers(-8, 9, size=len(ci)).astype(np.float32)
    y, b = oracle.spmv(rp, ci, v, np.ones(60, np.float32))
    expect = np.array([v[rp[i]:rp[i + 1]].astype(np.int64).sum() for i in range(50)])
    assert np.array_equal(y, expect.astype(np.float64))
    assert np.array_equal(b, np.array([np.abs(v[rp[i]:rp[i + 1]]).astype(np.int64).sum() for i in range(50)],
                                      dtype=np.float64))


def test_spmv_identity_and_diagonal():
    rng = np.random.default_rng(4)
    n = 33
    rp = np.arange(n + 1, dtype=np.int32)
    ci = np.arange(n, dtype=np.int32)
    x = rng.uniform(-1, 1, n).astype(np.float32)
    y, _ = oracle.spmv(rp, ci, np.ones(n, np.float32), x)
    assert np.array_equal(y, x.astype(np.float64))
    d = rng.uniform(-1, 1, n).astype(np.float32)
    y, _ = oracle.spmv(rp, ci, d, x)
    assert np.array_equal(y, d.astype(np.float64) * x.astype(np.float64))
    assert np.array_equal(y.astype(np.float32), d * x)  # fl32(d*x) from the exact product


def test_spmv_rows_subset_matches_full():
    rng = np.random.default_rng(5)
    rp, ci, v = rand_csr(rng, 80, 70, density=0.2, empty_rows={0, 79})
    x = rng.uniform(-1, 1, 70).astype(np.float32)
    rows = np.array([79, 0, 5, 5, 40])
    A = dense_of(rp, ci, v, 70)
    y, b = oracle.spmv_rows(rows, rp, ci, v, x)
    np.testing.assert_allclose(y, (A @ x.astype(np.float64))[rows], rtol=1e-12, atol=1e-12)


# ----------------------------------------------------------- merge-path pins --

def brute_merge(rp):
    """The merged work list by sorting tagged items: marker A[r] = rp[r+1] sorts
    as (rp[r+1], 0, r), atom k as (k, 1, k); so A[r] precedes atom k iff rp[r+1] <= k."""
    R = len(rp) - 1
    items = [(int(rp[r + 1]), 0, r) for r in range(R)] + [(k, 1, k) for k in range(int(rp[-1]))]
    items.sort()
    return [(t, i) for (_, t, i) in items]


def check_merge(orc):
    for C, rp, ci, v in tiny_cases(2):
        seq = brute_merge(rp)
        kind, idx = orc.merge_sequence(rp)
        assert [(int(a), int(b)) for a, b in zip(kind, idx)] == seq
        R, N = len(rp) - 1, int(rp[-1])
        diags = np.arange(R + N + 1)
        sp = orc.merge_splits(diags, rp)
        for d in range(R + N + 1):
            i_bf = sum(1 for (t, _) in seq[:d] if t == 0)
            assert (int(sp[d, 0]), int(sp[d, 1])) == (i_bf, d - i_bf), (rp, d)
            assert orc.merge_split(d, rp) == (i_bf, d - i_bf)


def test_merge_path_matches_bruteforce_merge():
    check_merge(oracle.default())


def check_weighted_diagonals(orc):
    """Shares cut with row ends weighted w: against the brute-force merged list
    (cost of every prefix by a cumulative sum, last prefix within each share's
    bound by a search), against the unweighted layout written out for w = 1,
    and the size bound a table relies on."""
    for t, (C, rp, ci, v) in enumerate(tiny_cases(5)):
        seq = brute_merge(rp)
        R, N = len(rp) - 1, int(rp[-1])
        for w in (1, 2, 3, 7):
            cost = np.concatenate([[0], np.cumsum([w if kind == 0 else 1 for kind, _ in seq])]).astype(np.int64)
            T = w * R + N
            for S, ipt in ((1, 4), (3, 2), (5, 3), (16, 1)):
                tpc = (-(-T // S) + w + ipt - 1) // ipt
                d = orc.weighted_diagonals(rp, w, S, ipt, tpc).reshape(S, tpc + 1)
                bounds = np.arange(S + 1, dtype=np.int64) * T // S
                pts = np.searchsorted(cost, bounds, side="right") - 1   # last prefix of cost <= bound
                assert np.array_equal(d[:, 0], pts[:-1]) and np.array_equal(d[:, -1], pts[1:]), (t, w, S)
                for c in range(S):
                    expect = np.minimum(pts[c] + np.arange(tpc + 1) * ipt, pts[c + 1])
                    assert np.array_equal(d[c], expect), (t, w, S, c)
                assert (pts[1:] - pts[:-1] <= tpc * ipt).all()            # every share fits its tiles
                if w == 1:
                    assert np.array_equal(pts, bounds)                    # the equal rows + atoms shares
                assert pts[0] == 0 and pts[-1] == R + N


def test_weighted_shares_match_bruteforce():
    check_weighted_diagonals(oracle.default())


def test_merge_path_split_invariants_and_coverage():
    rng = np.random.default_rng(11)
    import workloads as W
    L, _, _ = W.powerlaw_lengths(3000, 3000, 40000, lmax=2500, empty_frac=0.05, plant_long=False, seed=1)
    m = W.from_lengths(L, 3000, seed=1)
    rp = m.rp
    R, N = m.num_rows, m.nnz
    for W_items in (1, 7, 64, 2048, R + N + 5):
        P = -(-(R + N) // W_items)
        diags = np.minimum(np.arange(P + 1, dtype=np.int64) * W_items, R + N)
        sp = oracle.merge_splits(diags, rp).astype(np.int64)
        assert np.array_equal(sp.sum(1), diags)                       # on its diagonal
        assert tuple(sp[0]) == (0, 0) and tuple(sp[-1]) == (R, N)      # endpoints
        assert (np.diff(sp[:, 0]) >= 0).all() and (np.diff(sp[:, 1]) >= 0).all()  # monotone
        i, j = sp[:, 0], sp[:, 1]
        rp_ext = np.concatenate([rp, [N]]).astype(np.int64)
        assert (rp_ext[i] <= j).all() and (j <= rp_ext[i + 1]).all()   # split sits inside row i
        # every marker and atom covered exactly once: window p holds markers
        # [i_p, i_{p+1}) and atoms [j_p, j_{p+1}); their counts must tile the list
        assert np.array_equal(np.diff(i) + np.diff(j), np.diff(diags))
    kind, idx = oracle.merge_sequence(rp)
    assert (kind == 0).sum() == R and (kind == 1).sum() == N
    assert np.array_equal(np.sort(idx[kind == 0]), np.arange(R))
    assert np.array_equal(idx[kind == 1], np.arange(N))


# ---------------------------------------------------------- get_tile pins --

def test_get_tile_and_row_of_atom():
    rng = np.random.default_rng(12)
    for C, rp, ci, v in tiny_cases(3):
        N = int(rp[-1])
        row_of = oracle.row_of_atom(rp)
        assert np.array_equal(row_of, np.repeat(np.arange(len(rp) - 1), np.diff(rp)).astype(np.int32))
        if len(rp) > 1:
            for a in range(N):
                # largest t with prefix[t] <= a == searchsorted(side='right') - 1
                assert oracle.get_tile(rp, a) == int(np.searchsorted(rp, a, side="right")) - 1
                assert oracle.get_tile(rp, a) == row_of[a]


# --------------------------------------------------------- transpose pins --

def check_transpose(orc):
    for C, rp, ci, v in tiny_cases(4):
        cp, riT, perm = orc.transpose(rp, ci, C)
        row_of = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
        expect_perm = np.argsort(ci, kind="stable")
        assert np.array_equal(perm, expect_perm)
        assert np.array_equal(riT, row_of[expect_perm])
        assert np.array_equal(cp, np.concatenate([[0], np.cumsum(np.bincount(ci, minlength=C))]))
        # dense transpose
        At = dense_of(cp, riT, v[perm], len(rp) - 1)
        assert np.array_equal(At, dense_of(rp, ci, v, C).T)
        # (A^T)^T = A, bit for bit
        rp2, ci2, perm2 = orc.transpose(cp, riT, len(rp) - 1)
        assert np.array_equal(rp2, rp) and np.array_equal(ci2, ci)
        assert np.array_equal(perm[perm2], np.arange(len(ci)))


def test_transpose_is_stable_counting_sort():
    check_transpose(oracle.default())


# ---------------------------------------------------------- gradient pins --

def check_grad(orc):
    rng = np.random.default_rng(21)
    for C, rp, ci, v in tiny_cases(5, n=15):
        R = len(rp) - 1
        x = rng.uniform(-1, 1, C).astype(np.float32)
        dy = rng.normal(size=R).astype(np.float32)
        A = dense_of(rp, ci, v, C)
        dx, bx, dv = orc.grad(rp, ci, v, x, dy, C)
        np.testing.assert_allclose(dx, A.T @ dy.astype(np.float64), rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(bx, np.abs(A.T) @ np.abs(dy.astype(np.float64)), rtol=1e-12, atol=1e-12)
        # central finite differences of the bilinear loss L(v) = dy . (A(v) x), in FP64
        row_of = np.repeat(np.arange(R), np.diff(rp))
        h = 1e-3
        vv = v.astype(np.float64)

        def loss(vals):
            y = np.zeros(R)
            np.add.at(y, row_of, vals * x.astype(np.float64)[ci])
            return float(dy.astype(np.float64) @ y)

        for k in range(len(ci)):
            e = np.zeros_like(vv)
            e[k] = h
            fd = (loss(vv + e) - loss(vv - e)) / (2 * h)
            assert abs(float(dv[k]) - fd) <= 1e-6 * abs(fd) + 1e-12


def test_gradients_against_dense_and_finite_differences():
    check_grad(oracle.default())


def test_fd_instance_500x500():
    """The FP64 finite-difference instance of the differentiable workload (500x500, 5000 nnz)."""
    import workloads as W
    m = W.from_lengths(np.full(500, 10), 500, seed=5)
    x = W.vector(500, W.U_PM1, 5, 1)
    dy = W.vector(500, W.NORMAL, 5, 2)
    dx, _, dv = oracle.grad(m.rp, m.ci, m.v, x, dy, 500)
    h = 1e-3
    rng = np.random.default_rng(0)
    A = dense_of(m.rp, m.ci, m.v, 500)
    for c in rng.choice(500, 20, replace=False):
        e = np.zeros(500)
        e[c] = h
        xp = x.astype(np.float64) + e
        xm = x.astype(np.float64) - e
        fd = (dy.astype(np.float64) @ (A @ xp) - dy.astype(np.float64) @ (A @ xm)) / (2 * h)
        assert abs(dx[c] - fd) <= 1e-9 * max(1.0, abs(fd))


def check_spmm(orc):
    """SpMM (Listing 4) against dense brute force, the identity and SpMV column by column."""
    rng = np.random.default_rng(11)
    for R, C, K in ((0, 3, 4), (1, 1, 1), (7, 5, 3), (40, 33, 32), (33, 40, 33), (20, 20, 64)):
        dens = rng.uniform(0.0, 0.6)
        mask = rng.random((R, C)) < dens
        if R > 2:
            mask[1, :] = False          # an empty row
            mask[2, :] = True           # a full row
        rp = np.concatenate([[0], np.cumsum(mask.sum(1))]).astype(np.int32)
        ci = np.nonzero(mask)[1].astype(np.int32)
        v = rng.uniform(-1, 1, ci.shape[0]).astype(np.float32)
        B = rng.uniform(-1, 1, (C, K)).astype(np.float32)
        out, b = orc.spmm(rp, ci, v, B)
        A = dense_of(rp, ci, v, C)
        ref = A @ B.astype(np.float64)
        assert out.shape == (R, K)
        assert (np.abs(out - ref) <= 1e-12 * (np.abs(A) @ np.abs(B.astype(np.float64))) + 1e-300).all()
        assert np.allclose(b, np.abs(A) @ np.abs(B.astype(np.float64)), rtol=1e-12, atol=0)
        # one column of B at a time is SpMV
        for j in (0, K - 1):
            y, _ = orc.spmv(rp, ci, v, B[:, j].copy())
            assert np.array_equal(out[:, j], y)
    # identity: C = B exactly; a row permutation permutes B's rows
    n, K = 50, 17
    B = rng.uniform(-1, 1, (n, K)).astype(np.float32)
    rp = np.arange(n + 1, dtype=np.int32)
    out, _ = orc.spmm(rp, np.arange(n, dtype=np.int32), np.ones(n, np.float32), B)
    assert np.array_equal(out, B.astype(np.float64))
    perm = rng.permutation(n).astype(np.int32)
    out, _ = orc.spmm(rp, perm, np.ones(n, np.float32), B)
    assert np.array_equal(out, B[perm].astype(np.float64))


def test_spmm_against_dense_identity_and_spmv():
    check_spmm(oracle.default())


def bellman_ford32(rp, ci, w, src):
    """Plain Bellman-Ford in float32: relax every edge, in edge order, until nothing changes."""
    V = len(rp) - 1
    d = np.full(V, np.inf, dtype=np.float32)
    if V == 0:
        return d
    d[src] = np.float32(0)
    row = np.repeat(np.arange(V), np.diff(rp))
    for _ in range(V + 1):
        changed = False
        for k in range(len(ci)):
            nd = np.float32(d[row[k]] + w[k])
            if nd < d[ci[k]]:
                d[ci[k]] = nd
                changed = True
        if not changed:
            break
    return d


def random_graph(rng, V, E, wmax=1.0, zero_frac=0.0):
    src = rng.integers(0, V, E)
    dst = rng.integers(0, V, E)
    order = np.lexsort((dst, src))
    src, dst = src[order], dst[order]
    rp = np.concatenate([[0], np.cumsum(np.bincount(src, minlength=V))]).astype(np.int32)
    w = rng.uniform(0, wmax, E).astype(np.float32)
    w[rng.random(E) < zero_frac] = 0.0
    return rp, dst.astype(np.int32), w


def check_sssp(orc):
    """SSSP (Listing 5, float distances) against Bellman-Ford in float32 (bit-exact), BFS levels for
    unit weights, and scipy's FP64 Dijkstra within the float rounding of the path sums."""
    rng = np.random.default_rng(21)
    cases = [(1, 0, 0.0), (2, 1, 0.0), (6, 10, 0.0), (30, 90, 0.0), (50, 60, 0.0), (40, 200, 0.3), (64, 400, 0.0)]
    for V, E, zf in cases:
        rp, ci, w = random_graph(rng, V, E, zero_frac=zf)
        for s in sorted({0, V - 1}):
            d = orc.sssp(rp, ci, w, s)
            ref = bellman_ford32(rp, ci, w, s)
            assert np.array_equal(d.view(np.int32), ref.view(np.int32)), (V, E, s)
    # unit weights: breadth-first levels
    rp, ci, _ = random_graph(rng, 80, 240)
    d = orc.sssp(rp, ci, np.ones(len(ci), np.float32), 3)
    lev = np.full(80, np.inf)
    lev[3] = 0
    front = [3]
    while front:
        nxt = []
        for u in front:
            for k in range(rp[u], rp[u + 1]):
                if lev[ci[k]] == np.inf:
                    lev[ci[k]] = lev[u] + 1
                    nxt.append(ci[k])
        front = nxt
    assert np.array_equal(d.astype(np.float64), lev)
    # FP64 Dijkstra of a library: the same reachable set, distances within path-sum rounding
    sp = pytest.importorskip("scipy.sparse")
    csg = pytest.importorskip("scipy.sparse.csgraph")
    rp, ci, w = random_graph(rng, 500, 3000)
    w = w + np.float32(0.01)
    d = orc.sssp(rp, ci, w, 0)
    A = sp.csr_matrix((w.astype(np.float64), ci, rp), shape=(500, 500))
    d64 = csg.dijkstra(A, directed=True, indices=0)
    assert np.array_equal(np.isinf(d), np.isinf(d64))
    fin = np.isfinite(d64)
    assert (np.abs(d[fin] - d64[fin]) <= 1e-5 * d64[fin] + 1e-30).all()


def test_sssp_against_bellman_ford_bfs_and_fp64_dijkstra():
    check_sssp(oracle.default())


def check_formats(orc):
    """COO and CSC inputs as CSR tile sets: the same dense matrix, rows in order, a row's atoms in
    input order (COO) or ascending column (CSC), and round trips CSR -> COO -> CSR, CSR -> CSC -> CSR."""
    rng = np.random.default_rng(31)
    for R, C, N in ((0, 4, 0), (1, 1, 1), (5, 7, 0), (9, 6, 30), (40, 33, 500), (64, 64, 2000)):
        row = rng.integers(0, max(R, 1), N).astype(np.int32) if R else np.zeros(0, np.int32)
        col = rng.integers(0, C, N).astype(np.int32)
        val = rng.uniform(-1, 1, N).astype(np.float32)
        rp, ci, v = orc.coo_to_csr(R, row, col, val)
        assert rp[0] == 0 and rp[-1] == N and (np.diff(rp) >= 0).all()
        D = np.zeros((R, C))
        np.add.at(D, (row, col), val.astype(np.float64))
        assert np.array_equal(dense_of(rp, ci, v, C), D)
        order = np.argsort(row, kind="stable")           # stable by row: the input order within a row
        assert np.array_equal(ci, col[order]) and np.array_equal(v, val[order])
        # CSR -> COO (expand the row ids) -> CSR is the identity
        r2 = np.repeat(np.arange(R, dtype=np.int32), np.diff(rp))
        rp2, ci2, v2 = orc.coo_to_csr(R, r2, ci, v)
        assert np.array_equal(rp2, rp) and np.array_equal(ci2, ci) and np.array_equal(v2, v)
        # CSC of the same matrix (sorted by column, rows ascending) -> CSR
        oc = np.lexsort((row, col))
        cp = np.concatenate([[0], np.cumsum(np.bincount(col, minlength=C))]).astype(np.int32)
        rp3, ci3, v3 = orc.csc_to_csr(R, cp, row[oc], val[oc])
        assert np.array_equal(dense_of(rp3, ci3, v3, C), D)
        for r in range(R):
            seg = ci3[rp3[r]:rp3[r + 1]]
            assert (np.diff(seg) >= 0).all()              # columns ascend within a row


def test_coo_and_csc_inputs():
    check_formats(oracle.default())


# ------------------------------------------------------------ mutation tests --

MUTANTS = {
    # a dropped term: the first atom of every row is skipped
    "dropped_term": ("i < R; ++i) {\n    double s = 0.0, a = 0.0;\n    for (int32_t k = rp[i]; k",
                     "i < R; ++i) {\n    double s = 0.0, a = 0.0;\n    for (int32_t k = rp[i] + 1; k",
                     check_spmv_dense),
    # wrong tie-break: atoms before row ends with the same index
    "merge_ties_to_atoms": ("if ((int64_t)rp[mid + 1] > d - mid - 1) hi = mid;",
                            "if ((int64_t)rp[mid + 1] >= d - mid - 1) hi = mid;", check_merge),
    "sequence_ties_to_atoms": ("(j >= N || rp[i + 1] <= j)", "(j >= N || rp[i + 1] < j)", check_merge),
    # weighted shares that stop one item short (a point whose cost equals the bound left out)
    "weighted_share_short": ("if (cost + step > W) break;", "if (cost + step >= W) break;", check_weighted_diagonals),
    # unstable transpose: rows visited bottom-up
    "unstable_transpose": ("for (int32_t r = 0; r < R; ++r) {\n    for (int32_t k = rp[r]; k < rp[r + 1]; ++k) {\n"
                           "      int32_t p = cur",
                           "for (int32_t r = R - 1; r >= 0; --r) {\n    for (int32_t k = rp[r]; k < rp[r + 1]; ++k) {\n"
                           "      int32_t p = cur", check_transpose),
    # transposed operand in the gradient: dvals uses x[row] instead of x[col]
    "dvals_wrong_operand": ("dvals[k] = (float)((double)dy[r] * (double)x[ci[k]]);",
                            "dvals[k] = (float)((double)dy[r] * (double)x[r % C]);", check_grad),
    # sign error in dx
    "dx_sign": ("dx[ci[k]] += p;", "dx[ci[k]] -= p;", check_grad),
    # SSSP relaxing with a dropped weight (distance of the source carried unchanged)
    "sssp_dropped_weight": ("float nd = dist[it.v] + w[k];", "float nd = dist[it.v] + 0.0f * w[k];", check_sssp),
    # COO rows placed unstably (atoms of a row reversed)
    "coo_unstable": ("int32_t p = cur[row[k]]++;", "int32_t p = rp[row[k] + 1] - 1 - (cur[row[k]]++ - rp[row[k]]);",
                     check_formats),
    # wrong column of B in SpMM: the columns of B read in reverse order
    "spmm_wrong_b_column": ("(double)B[(int64_t)ci[k] * ldb + j];", "(double)B[(int64_t)ci[k] * ldb + (K - 1 - j)];",
                            check_spmm),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_reject_planted_mistakes(name):
    old, new, check = MUTANTS[name]
    src = open(oracle.source_path()).read()
    assert src.count(old) == 1, name
    d = tempfile.mkdtemp(prefix="oracle_mutant_")
    try:
        c = os.path.join(d, "mutant.c")
        so = os.path.join(d, "libmutant.so")
        open(c, "w").write(src.replace(old, new))
        subprocess.check_call(["gcc", "-O1", "-fPIC", "-shared", "-o", so, c, "-lm"])
        with pytest.raises(AssertionError):
            check(Oracle(so))
    finally:
        shutil.rmtree(d, ignore_errors=True)


def test_threaded_oracle_runner_is_identical():
    import workloads as W
    """spmv_threads only splits the rows over host threads: bit-identical to spmv."""
    for R, C, L, seed in ((0, 5, 1, 0), (1, 7, 3, 1), (37, 50, 9, 2), (5000, 3000, 40, 3)):
        m = W.powerlaw(R, C, max(R * L // 3, 0), lmax=min(C, 200), plant_long=False, seed=seed) if R > 1 \
            else W.from_lengths(np.full(R, min(L, C), dtype=np.int64), C, seed=seed)
        x = W.x_for(m)
        y, b = oracle.spmv(m.rp, m.ci, m.v, x)
        for T in (1, 2, 7, 64):
            yt, bt = oracle.spmv_threads(m.rp, m.ci, m.v, x, T)
            assert np.array_equal(y.view(np.int64), yt.view(np.int64)) and np.array_equal(b, bt), (R, T)
