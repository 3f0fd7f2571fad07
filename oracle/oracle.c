/*
 * ORACLE -- test infrastructure only.
 *
 * Plain, slow, obviously correct CPU implementations of what the load-balanced
 * SpMV path computes, in FP64 where floating point is involved.  Only the test
 * suite, the smoke check and the benchmark's CPU-baseline leg use this file;
 * the product path never links or calls it, and it shares no code, header,
 * table or helper with the CUDA library.
 *
 * Notation (Sec. 3.1, Listing 1): a tile is a CSR row, an atom is a nonzero;
 * rp[R+1] are the row offsets, ci[N] the column indices, v[N] the values.
 * The atoms of tile t are [rp[t], rp[t+1]) (Listing 2, atoms()).
 *
 * Every function states the passage it follows.  Where the paper is silent the
 * reading used is stated at the function (tie-break in the merge, summation
 * order, empty rows).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/*
 * y = A x by the definition of SpMV (Sec. 1; Listing 3 body): for every row i,
 * y[i] = sum over k in [rp[i], rp[i+1]) of v[k] * x[ci[k]], accumulated in
 * FP64 in atom order.  Also returns the error scale b[i] = sum |v[k] x[ci[k]]|
 * used by the acceptance bound |y32 - y64| <= tol * b.  Empty rows give 0.
 */
void or_spmv(int32_t R, const int32_t* rp, const int32_t* ci, const float* v, const float* x, double* y,
             double* b) {
  for (int32_t i = 0; i < R; ++i) {
    double s = 0.0, a = 0.0;
    for (int32_t k = rp[i]; k < rp[i + 1]; ++k) {
      double p = (double)v[k] * (double)x[ci[k]];
      s += p;
      a += fabs(p);
    }
    y[i] = s;
    if (b) b[i] = a;
  }
}

/*
 * C = A B for a dense row-major B (num_cols rows of K values, row pitch ldb):
 * for every row i and column j of B, C[i][j] = sum over k in [rp[i], rp[i+1])
 * of v[k] * B[ci[k]][j] -- the SpMV loop of Listing 3 inside a loop over the
 * columns of B, as Sec. 7 (Listing 4) extends it; B is read at the atom's
 * column index.  FP64 in atom order; bnd[i][j] = sum |v[k] B[ci[k]][j]| for the
 * acceptance bound.  C and bnd are row-major R x K.  Empty rows give 0.
 */
void or_spmm(int32_t R, const int32_t* rp, const int32_t* ci, const float* v, const float* B, int64_t ldb,
             int32_t K, double* C, double* bnd) {
  for (int32_t i = 0; i < R; ++i) {
    for (int32_t j = 0; j < K; ++j) {
      double s = 0.0, a = 0.0;
      for (int32_t k = rp[i]; k < rp[i + 1]; ++k) {
        double p = (double)v[k] * (double)B[(int64_t)ci[k] * ldb + j];
        s += p;
        a += fabs(p);
      }
      C[(int64_t)i * K + j] = s;
      if (bnd) bnd[(int64_t)i * K + j] = a;
    }
  }
}

/*
 * Same as or_spmv for a subset of rows (sampled parity at full size).
 */
void or_spmv_rows(int64_t nsel, const int64_t* rows, const int32_t* rp, const int32_t* ci, const float* v,
                  const float* x, double* y, double* b) {
  for (int64_t q = 0; q < nsel; ++q) {
    int64_t i = rows[q];
    double s = 0.0, a = 0.0;
    for (int32_t k = rp[i]; k < rp[i + 1]; ++k) {
      double p = (double)v[k] * (double)x[ci[k]];
      s += p;
      a += fabs(p);
    }
    y[q] = s;
    if (b) b[q] = a;
  }
}

/*
 * Merge-path split (Sec. 5.2.1; Merrill & Garland's merge-based SpMV, cited
 * there).  The work list is the merge of list A (row-end markers
 * A[r] = rp[r+1], r < R) with list B (atom indices B[k] = k, k < N).
 * Reading of the tie, which the paper leaves open: A[r] precedes B[k] exactly
 * when A[r] <= k, i.e. a row ends before the atom with the same index starts.
 *
 * The split of diagonal d (0 <= d <= R+N) is the pair (i, j), i + j = d, that
 * puts the first i markers and the first j atoms before the rest.  It is the
 * smallest i in [max(0, d-N), min(d, R)] for which either i is that upper
 * limit or atom j-1 = d-i-1 precedes marker A[i] (rp[i+1] > d-i-1); the test
 * is monotone in i, so a bisection along the diagonal finds it.
 * Returns i; j = d - i.
 */
int32_t or_merge_split(int64_t d, int32_t R, int32_t N, const int32_t* rp) {
  int64_t lo = d - (int64_t)N;
  if (lo < 0) lo = 0;
  int64_t hi = d < (int64_t)R ? d : (int64_t)R;
  while (lo < hi) {
    int64_t mid = (lo + hi) / 2;
    if ((int64_t)rp[mid + 1] > d - mid - 1) hi = mid;
    else lo = mid + 1;
  }
  return (int32_t)lo;
}

/* Splits for a list of diagonals: out[2q] = i, out[2q+1] = j. */
void or_merge_splits(int64_t nd, const int64_t* diag, int32_t R, int32_t N, const int32_t* rp, int32_t* out) {
  for (int64_t q = 0; q < nd; ++q) {
    int32_t i = or_merge_split(diag[q], R, N, rp);
    out[2 * q] = i;
    out[2 * q + 1] = (int32_t)(diag[q] - i);
  }
}

/*
 * The full merged work list, written out item by item (Sec. 5.2.1): kind[q] is
 * 0 for a row-end marker and 1 for an atom, idx[q] the row or atom index.
 * Same tie reading as or_merge_split.  Length R + N.
 */
void or_merge_sequence(int32_t R, int32_t N, const int32_t* rp, int8_t* kind, int32_t* idx) {
  int32_t i = 0, j = 0;
  int64_t q = 0;
  while (i < R || j < N) {
    if (i < R && (j >= N || rp[i + 1] <= j)) {
      kind[q] = 0;
      idx[q] = i++;
    } else {
      kind[q] = 1;
      idx[q] = j++;
    }
    ++q;
  }
}

/*
 * Table diagonals of a merge path whose worker shares are cut with row ends
 * weighted w (the library's row_weight option, a cost model for its warp
 * tiles; the paper's shares are the w = 1 case, Sec. 5.2.1).  The point after
 * i row ends and j atoms costs w*i + j.  Share c of S runs from the last point
 * of cost <= floor(c*T/S) to the last point of cost <= floor((c+1)*T/S),
 * T = w*R + N; its table entry k (k = 0..tpc) is its first diagonal plus
 * k*ipt, clamped to its last.  The points are found by walking the merged list
 * from the start, one item at a time.  diag: S*(tpc+1) entries.
 */
void or_weighted_diagonals(int32_t R, int32_t N, const int32_t* rp, int32_t w, int32_t S, int32_t ipt, int32_t tpc,
                           int64_t* diag) {
  const int64_t T = (int64_t)w * R + N;
  int64_t* point = (int64_t*)malloc(sizeof(int64_t) * ((size_t)S + 1));
  /* one walk along the merged list; the bounds c*T/S only grow with c */
  int32_t i = 0, j = 0;
  int64_t cost = 0;
  for (int32_t c = 0; c <= S; ++c) {
    const int64_t W = (int64_t)c * T / S;
    while (i < R || j < N) {
      const int row_end = i < R && (j == N || j >= rp[i + 1]); /* ties: the row end first */
      const int64_t step = row_end ? w : 1;
      if (cost + step > W) break;
      cost += step;
      if (row_end) ++i;
      else ++j;
    }
    point[c] = (int64_t)i + j;
  }
  for (int32_t c = 0; c < S; ++c)
    for (int32_t k = 0; k <= tpc; ++k) {
      const int64_t d = point[c] + (int64_t)k * ipt;
      diag[(int64_t)c * (tpc + 1) + k] = d < point[c + 1] ? d : point[c + 1];
    }
  free(point);
}

/*
 * Tile of every atom (the mapping a schedule's get_tile returns, Sec. 5.2.3):
 * row_of[k] = the row r with rp[r] <= k < rp[r+1], by walking the rows.
 */
void or_row_of_atom(int32_t R, const int32_t* rp, int32_t* row_of) {
  for (int32_t r = 0; r < R; ++r)
    for (int32_t k = rp[r]; k < rp[r + 1]; ++k) row_of[k] = r;
}

/*
 * get_tile(a) of the group-mapped schedule (Sec. 5.2.3): given the exclusive
 * prefix sum prefix[0..n] of the atoms-per-tile of a group's tiles, the tile
 * of flattened atom a is the largest t < n with prefix[t] <= a (empty tiles,
 * whose prefix equals the next one's, are skipped).  Linear scan.
 */
int32_t or_get_tile(const int32_t* prefix, int32_t n, int32_t a) {
  int32_t t = -1;
  for (int32_t q = 0; q < n; ++q)
    if (prefix[q] <= a) t = q;
  return t;
}

/*
 * CSR -> CSC by a stable counting sort over the atoms in CSR order
 * (the transpose the differentiable form needs for dx = A^T dy):
 * cnt[c] = number of atoms in column c; cp = exclusive prefix of cnt;
 * atoms are then placed in increasing k, so rows ascend within each column.
 * perm[p] = source atom k of CSC slot p, riT[p] = row of that atom.
 */
void or_transpose(int32_t R, int32_t C, const int32_t* rp, const int32_t* ci, int32_t* cp, int32_t* riT,
                  int32_t* perm) {
  int32_t N = rp[R];
  for (int32_t c = 0; c <= C; ++c) cp[c] = 0;
  for (int32_t k = 0; k < N; ++k) cp[ci[k] + 1] += 1;
  for (int32_t c = 0; c < C; ++c) cp[c + 1] += cp[c];
  int32_t* cur = (int32_t*)malloc(sizeof(int32_t) * (size_t)(C > 0 ? C : 1));
  for (int32_t c = 0; c < C; ++c) cur[c] = cp[c];
  for (int32_t r = 0; r < R; ++r) {
    for (int32_t k = rp[r]; k < rp[r + 1]; ++k) {
      int32_t p = cur[ci[k]]++;
      perm[p] = k;
      riT[p] = r;
    }
  }
  free(cur);
}

/*
 * Gradients of y = A x for the loss L = sum_i dy[i] y[i]:
 *   dx[c]    = sum over atoms k with ci[k] = c of v[k] dy[row(k)]   (A^T dy)
 *   dvals[k] = dy[row(k)] x[ci[k]]
 * dx is accumulated in FP64 by scattering over the CSR atoms in k order, with
 * bound bx[c] = sum |v[k] dy[row(k)]|.  dvals is one product of two FP32
 * numbers; the FP64 product is exact, so rounding it to FP32 gives the
 * correctly rounded FP32 product.
 */
void or_grad(int32_t R, int32_t C, const int32_t* rp, const int32_t* ci, const float* v, const float* x,
             const float* dy, double* dx, double* bx, float* dvals) {
  if (dx) {
    for (int32_t c = 0; c < C; ++c) dx[c] = 0.0;
    if (bx)
      for (int32_t c = 0; c < C; ++c) bx[c] = 0.0;
  }
  for (int32_t r = 0; r < R; ++r) {
    for (int32_t k = rp[r]; k < rp[r + 1]; ++k) {
      if (dx) {
        double p = (double)v[k] * (double)dy[r];
        dx[ci[k]] += p;
        if (bx) bx[ci[k]] += fabs(p);
      }
      if (dvals) dvals[k] = (float)((double)dy[r] * (double)x[ci[k]]);
    }
  }
}

/*
 * Single-source shortest paths (Sec. 7, Listing 5) with the listing's float
 * distances: dist[source] = 0 and, for every other vertex v reachable from the
 * source, dist[v] = min over edges (u, v) of fl32(dist[u] + w(u, v)); +inf if
 * unreachable.  Vertices are tiles, their out-edges atoms (CSR rp / ci, edge
 * weights w >= 0).  Dijkstra's algorithm: settle vertices in order of
 * distance from a binary min-heap (entries pushed on every improvement, stale
 * ones skipped when popped).  Returns the number of vertices settled.
 */
typedef struct {
  float d;
  int32_t v;
} or_heap_item;

static void or_heap_push(or_heap_item* h, int64_t* n, float d, int32_t v) {
  int64_t i = (*n)++;
  while (i > 0) {
    int64_t p = (i - 1) / 2;
    if (h[p].d <= d) break;
    h[i] = h[p];
    i = p;
  }
  h[i].d = d;
  h[i].v = v;
}

static or_heap_item or_heap_pop(or_heap_item* h, int64_t* n) {
  or_heap_item top = h[0];
  or_heap_item last = h[--(*n)];
  int64_t i = 0;
  for (;;) {
    int64_t c = 2 * i + 1;
    if (c >= *n) break;
    if (c + 1 < *n && h[c + 1].d < h[c].d) ++c;
    if (last.d <= h[c].d) break;
    h[i] = h[c];
    i = c;
  }
  if (*n > 0) h[i] = last;
  return top;
}

int32_t or_sssp(int32_t V, const int32_t* rp, const int32_t* ci, const float* w, int32_t src, float* dist) {
  for (int32_t v = 0; v < V; ++v) dist[v] = INFINITY;
  if (V == 0) return 0;
  int64_t cap = (int64_t)rp[V] + 1;
  or_heap_item* h = (or_heap_item*)malloc(sizeof(or_heap_item) * (size_t)cap);
  unsigned char* done = (unsigned char*)calloc((size_t)V, 1);
  int64_t n = 0;
  int32_t settled = 0;
  dist[src] = 0.0f;
  or_heap_push(h, &n, 0.0f, src);
  while (n > 0) {
    or_heap_item it = or_heap_pop(h, &n);
    if (done[it.v] || it.d > dist[it.v]) continue;
    done[it.v] = 1;
    ++settled;
    for (int32_t k = rp[it.v]; k < rp[it.v + 1]; ++k) {
      int32_t u = ci[k];
      float nd = dist[it.v] + w[k];
      if (nd < dist[u]) {
        dist[u] = nd;
        or_heap_push(h, &n, nd, u);
      }
    }
  }
  free(h);
  free(done);
  return settled;
}

/*
 * COO -> CSR tile set ("other formats only need their own atom and tile
 * iterators", Sec. 4): the tiles are the rows, so the tile offsets are the
 * run lengths of the atoms' row ids, prefix-summed, and the atoms are placed
 * by a stable counting sort on the row id (atoms of a row keep their input
 * order).  rp[R+1]; perm[p] = input atom of CSR slot p; col_out[p] = its column.
 * Row ids must lie in [0, R).
 */
void or_coo_to_csr(int32_t R, int64_t N, const int32_t* row, const int32_t* col, int32_t* rp, int32_t* col_out,
                   int32_t* perm) {
  for (int32_t r = 0; r <= R; ++r) rp[r] = 0;
  for (int64_t k = 0; k < N; ++k) rp[row[k] + 1]++;
  for (int32_t r = 0; r < R; ++r) rp[r + 1] += rp[r];
  int32_t* cur = (int32_t*)malloc(sizeof(int32_t) * (size_t)(R > 0 ? R : 1));
  for (int32_t r = 0; r < R; ++r) cur[r] = rp[r];
  for (int64_t k = 0; k < N; ++k) {
    int32_t p = cur[row[k]]++;
    perm[p] = (int32_t)k;
    col_out[p] = col[k];
  }
  free(cur);
}
