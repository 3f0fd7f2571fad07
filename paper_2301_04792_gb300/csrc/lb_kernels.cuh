// Device kernels of the load-balanced SpMV path (sm_103a).
//
// Work vocabulary (Sec. 3.1, Listing 1): tiles are rows of a CSR tile set,
// atoms its nonzeros.  Four schedules (Sec. 4.2, 5.2) consume the same tile
// set: thread-mapped, group-mapped (warp / block / any power-of-two group) and
// merge-path.  Everything here is deterministic: the order in which partial
// sums are combined depends only on the plan, never on timing, and no
// floating-point atomics are used.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <climits>

namespace lbk {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kDevErrColumn = 1;  // device error bit: column index out of range

// ------------------------------------------------------------- load helpers --

__device__ __forceinline__ int ld_stream(const int* p) { return __ldcs(p); }
__device__ __forceinline__ float ld_stream(const float* p) { return __ldcs(p); }
__device__ __forceinline__ int4 ld_stream(const int4* p) { return __ldcs(p); }
__device__ __forceinline__ float4 ld_stream(const float4* p) { return __ldcs(p); }

// ------------------------------------------------------------- atom views --

// How atom j of a tile set becomes a product.  idx[j] selects the entry of the
// dense vector (a column for y = A x, a row for dx = A^T dy); the value is
// val[j], or val[perm[j]] when the tile set is a transpose that gathers the
// original values.  `vbase` offsets perm for batched transposes (perm is
// matrix-local there).  With check > 0 every index is checked against it;
// an out-of-range index reads as 0 and sets a bit in *status.
struct AtomView {
  const int32_t* idx;
  const float* val;
  const int32_t* perm;
  const float* vec;
  int32_t check;
  int* status;

  __device__ __forceinline__ float value(int64_t j, int64_t vbase) const {
    return perm ? __ldg(val + vbase + ld_stream(perm + j)) : ld_stream(val + j);
  }
  __device__ __forceinline__ float gather(int c, int64_t xbase) const {
    if (check > 0 && (unsigned)c >= (unsigned)check) {
      atomicOr(status, kDevErrColumn);
      return 0.f;
    }
    return __ldg(vec + xbase + c);
  }
  __device__ __forceinline__ float product(int64_t j, int64_t vbase, int64_t xbase) const {
    const int c = ld_stream(idx + j);
    return value(j, vbase) * gather(c, xbase);
  }
};

// ----------------------------------------------------------- block scans --

// Inclusive segmented scan over the threads of a block, in thread order.
// Thread t holds (f, v); a flagged element starts a new segment.  `prefix` is
// an unflagged element placed before thread 0.  Returns the inclusive value,
// and through excl / total the exclusive value of this thread and the
// inclusive value of the last thread.  Contains two __syncthreads; the
// scratch arrays may be reused only after the caller's next barrier.
template <int BLOCK>
__device__ __forceinline__ float block_seg_scan(float v, int f, float prefix, float* s_wv, int* s_wf,
                                                float* s_incl, float& excl, float& total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const float vo = __shfl_up_sync(kFull, v, o);
    const int fo = __shfl_up_sync(kFull, f, o);
    if (lane >= o) {
      if (!f) v = vo + v;
      f |= fo;
    }
  }
  if (lane == 31) {
    s_wv[warp] = v;
    s_wf[warp] = f;
  }
  __syncthreads();
  float pv = prefix;
  for (int w = 0; w < warp; ++w) pv = s_wf[w] ? s_wv[w] : pv + s_wv[w];
  if (!f) v = pv + v;
  s_incl[threadIdx.x] = v;
  __syncthreads();
  excl = threadIdx.x ? s_incl[threadIdx.x - 1] : prefix;
  total = s_incl[BLOCK - 1];
  return v;
}

// Exclusive prefix sum of one int per thread over a group of G threads that
// lies inside one warp (G <= 32, width-G shuffles).
template <int G>
__device__ __forceinline__ int group_excl_scan_small(int x, int lane_in_group, int& total) {
  int incl = x;
#pragma unroll
  for (int o = 1; o < G; o <<= 1) {
    const int n = __shfl_up_sync(kFull, incl, o, G);
    if (lane_in_group >= o) incl += n;
  }
  total = __shfl_sync(kFull, incl, G - 1, G);
  return incl - x;
}

// ------------------------------------------------------------ merge path --

// One split of the merged list of row ends and atoms: i row ends and j atoms
// precede it; m is the matrix it falls in (batched tile sets only).
struct Split64 {
  int64_t i, j;
  int32_t m, pad;
};

// Arguments of the merge-path kernels.  `splits` holds, for every persistent
// CTA c, tiles_per_cta + 1 consecutive splits (its tile boundaries).
struct MpArgs {
  const int32_t* rp;        // single: tile offsets; batch: per-matrix offsets back to back
  const int64_t* row_base;  // batch: first global tile of each matrix [M+1]
  const int64_t* nnz_base;  // batch: first global atom of each matrix [M+1]
  const int64_t* vec_base;  // batch: first entry of each matrix's dense input vector [M+1]
  AtomView atoms;
  float* out;               // per-tile result (y or dx)
  const void* splits;       // int2 (single) or Split64 (batch)
  int tiles_per_cta;
  int num_ctas;
  int64_t num_tiles;
  float* carry_val;         // [num_ctas]
  int64_t* carry_row;       // [num_ctas]
  unsigned* ticket;         // zero between launches
  // expand kernels
  const float* dy;          // dvals: upstream gradient per tile
  float* dvals;             // dvals output per atom
  int32_t* tile_of_atom;    // atom -> tile output
};

template <bool BATCH>
__device__ __forceinline__ Split64 load_split(const MpArgs& a, size_t e) {
  if constexpr (BATCH) {
    return reinterpret_cast<const Split64*>(a.splits)[e];
  } else {
    const int2 s = __ldg(reinterpret_cast<const int2*>(a.splits) + e);
    Split64 r;
    r.i = s.x;
    r.j = s.y;
    r.m = 0;
    r.pad = 0;
    return r;
  }
}

// Largest m in [lo, hi] with base[m] <= g (the matrix holding global index g).
__device__ __forceinline__ int find_matrix(const int64_t* base, int lo, int hi, int64_t g) {
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(base + mid) <= g) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Row ends of the tile's rows, relative to its first atom, into s_end[0..nrows).
template <int BLOCK, bool BATCH>
__device__ __forceinline__ void stage_row_ends(const MpArgs& a, const Split64& cur, const Split64& nxt, int nrows,
                                               int* s_end) {
  if constexpr (!BATCH) {
    const int32_t* rp = a.rp + cur.i + 1;
    const int j0 = (int)cur.j;
    for (int r = threadIdx.x; r < nrows; r += BLOCK) s_end[r] = __ldg(rp + r) - j0;
  } else {
    for (int r = threadIdx.x; r < nrows; r += BLOCK) {
      const int64_t g = cur.i + r;
      const int m = (cur.m == nxt.m) ? cur.m : find_matrix(a.row_base, cur.m, nxt.m, g);
      const int64_t end = __ldg(a.nnz_base + m) + __ldg(a.rp + g + m + 1);
      s_end[r] = (int)(end - cur.j);
    }
  }
}

// Products of the tile's atoms into s_prod[off + l], l in [0, nnz), with
// off = (first atom) & 3 so that 16-byte vectors of col_idx / vals land on
// 16-byte shared-memory boundaries.  VEC: col_idx, vals (or perm) 16-byte aligned.
template <int BLOCK, int IPT, bool BATCH, bool VEC>
__device__ __forceinline__ void stage_products(const MpArgs& a, const Split64& cur, const Split64& nxt, int nnz,
                                               float* s_prod) {
  const int64_t j0 = cur.j;
  const int off = (int)(j0 & 3);
  const AtomView& at = a.atoms;
  int m_uni = 0;
  int64_t vb = 0, xb = 0;
  const bool uniform = !BATCH || cur.m == nxt.m;
  if constexpr (BATCH) {
    m_uni = cur.m;
    vb = __ldg(a.nnz_base + m_uni);
    xb = __ldg(a.vec_base + m_uni);
  }
  if constexpr (VEC) {
    const int64_t g0 = j0 - off;  // multiple of 4
    const int nv = (off + nnz) >> 2;
    constexpr int NV = (BLOCK * IPT + 4) / 4 / BLOCK + 1;
    const int4* idx4 = reinterpret_cast<const int4*>(at.idx + g0);
    if (uniform && at.perm == nullptr) {
      const float4* val4 = reinterpret_cast<const float4*>(at.val + g0);
      int4 c[NV];
      float4 w[NV];
#pragma unroll
      for (int u = 0; u < NV; ++u) {
        const int q = threadIdx.x + u * BLOCK;
        if (q < nv) {
          c[u] = ld_stream(idx4 + q);
          w[u] = ld_stream(val4 + q);
        }
      }
#pragma unroll
      for (int u = 0; u < NV; ++u) {
        const int q = threadIdx.x + u * BLOCK;
        if (q < nv) {
          // slots below `off` belong to atoms before the tile; in a batch they may
          // belong to another matrix, so they are not gathered
          const int s0 = 4 * q;
          float4 p;
          p.x = (BATCH && s0 + 0 < off) ? 0.f : w[u].x * at.gather(c[u].x, xb);
          p.y = (BATCH && s0 + 1 < off) ? 0.f : w[u].y * at.gather(c[u].y, xb);
          p.z = (BATCH && s0 + 2 < off) ? 0.f : w[u].z * at.gather(c[u].z, xb);
          p.w = w[u].w * at.gather(c[u].w, xb);
          *reinterpret_cast<float4*>(s_prod + s0) = p;
        }
      }
    } else if (uniform) {
      const int4* perm4 = reinterpret_cast<const int4*>(at.perm + g0);
      int4 c[NV], pm[NV];
#pragma unroll
      for (int u = 0; u < NV; ++u) {
        const int q = threadIdx.x + u * BLOCK;
        if (q < nv) {
          c[u] = ld_stream(idx4 + q);
          pm[u] = ld_stream(perm4 + q);
        }
      }
#pragma unroll
      for (int u = 0; u < NV; ++u) {
        const int q = threadIdx.x + u * BLOCK;
        if (q < nv) {
          const int s0 = 4 * q;
          float4 p;
          p.x = (BATCH && s0 + 0 < off) ? 0.f : __ldg(at.val + vb + pm[u].x) * at.gather(c[u].x, xb);
          p.y = (BATCH && s0 + 1 < off) ? 0.f : __ldg(at.val + vb + pm[u].y) * at.gather(c[u].y, xb);
          p.z = (BATCH && s0 + 2 < off) ? 0.f : __ldg(at.val + vb + pm[u].z) * at.gather(c[u].z, xb);
          p.w = __ldg(at.val + vb + pm[u].w) * at.gather(c[u].w, xb);
          *reinterpret_cast<float4*>(s_prod + s0) = p;
        }
      }
    } else {
      // tile spans several matrices (batch): per-atom matrix lookup, scalar loads
      for (int l = threadIdx.x; l < nnz; l += BLOCK) {
        const int64_t j = j0 + l;
        const int m = find_matrix(a.nnz_base, cur.m, nxt.m, j);
        s_prod[off + l] = at.product(j, __ldg(a.nnz_base + m), __ldg(a.vec_base + m));
      }
      return;
    }
    // ragged tail past the last full vector
    const int tail0 = 4 * nv > off ? 4 * nv : off;
    for (int l = tail0 + threadIdx.x; l < off + nnz; l += BLOCK) {
      s_prod[l] = at.product(g0 + l, vb, xb);
    }
  } else {
    for (int l = threadIdx.x; l < nnz; l += BLOCK) {
      const int64_t j = j0 + l;
      int64_t vbj = vb, xbj = xb;
      if (!uniform) {
        const int m = find_matrix(a.nnz_base, cur.m, nxt.m, j);
        vbj = __ldg(a.nnz_base + m);
        xbj = __ldg(a.vec_base + m);
      }
      s_prod[off + l] = at.product(j, vbj, xbj);
    }
  }
}

// Split of local diagonal d inside a tile: smallest ti with
// ti == min(d, nrows) or s_end[ti] > d - ti - 1 (row end ti comes after atom
// d - ti - 1; a row end precedes the atom with the same index).
__device__ __forceinline__ int tile_search(const int* s_end, int d, int nrows, int nnz) {
  int lo = d - nnz > 0 ? d - nnz : 0;
  int hi = d < nrows ? d : nrows;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (s_end[mid] > d - mid - 1) hi = mid;
    else lo = mid + 1;
  }
  return lo;
}

template <int BLOCK, int IPT>
constexpr size_t mp_smem_bytes() {
  return sizeof(int) * (BLOCK * IPT) + sizeof(float) * (BLOCK * IPT + 4) + sizeof(float) * (BLOCK * IPT) + 64;
}

// Merge-path SpMV (Sec. 5.2.1) as a persistent kernel: CTA c owns an equal
// share of rows + atoms and walks it tile by tile.  Per tile: stage row ends
// and atom products in shared memory, split the tile evenly over the threads
// by a search along each thread's diagonal, walk IPT items per thread
// (complete rows are written directly; the partial row at each thread's end is
// its carry-out), resolve carries across threads with a segmented scan and
// across tiles with a running CTA carry.  Rows split between CTAs are fixed up
// by the last CTA to finish (ticket), in CTA order.
template <int BLOCK, int IPT, bool BATCH, bool VEC>
__global__ void __launch_bounds__(BLOCK) mp_spmv_kernel(MpArgs a) {
  constexpr int T = BLOCK * IPT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* s_prod = reinterpret_cast<float*>(smem_raw);     // T + 4
  int* s_end = reinterpret_cast<int*>(s_prod + T + 4);    // T
  float* s_y = reinterpret_cast<float*>(s_end + T);       // T
  __shared__ float s_wv[BLOCK / 32];
  __shared__ int s_wf[BLOCK / 32];
  __shared__ float s_incl[BLOCK];
  __shared__ int s_last;

  const int tid = threadIdx.x;
  const size_t base = (size_t)blockIdx.x * (a.tiles_per_cta + 1);
  float carry = 0.f;
  Split64 cur = load_split<BATCH>(a, base);
  for (int k = 0; k < a.tiles_per_cta; ++k) {
    const Split64 nxt = load_split<BATCH>(a, base + k + 1);
    const int nrows = (int)(nxt.i - cur.i);
    const int nnz = (int)(nxt.j - cur.j);
    const int items = nrows + nnz;
    if (items == 0) break;
    stage_row_ends<BLOCK, BATCH>(a, cur, nxt, nrows, s_end);
    stage_products<BLOCK, IPT, BATCH, VEC>(a, cur, nxt, nnz, s_prod);
    const int off = (int)(cur.j & 3);
    __syncthreads();

    const int d = min(tid * IPT, items);
    int ti = tile_search(s_end, d, nrows, nnz);
    int tj = d - ti;
    const int ti0 = ti;
    const int dend = min(d + IPT, items);
    float acc = 0.f, first = 0.f;
    int any = 0;
    int nend = ti < nrows ? s_end[ti] : INT_MAX;
#pragma unroll
    for (int it = 0; it < IPT; ++it) {
      if (d + it < dend) {
        if (tj >= nend) {
          if (any) s_y[ti] = acc;
          else {
            first = acc;
            any = 1;
          }
          acc = 0.f;
          ++ti;
          nend = ti < nrows ? s_end[ti] : INT_MAX;
        } else {
          acc += s_prod[off + tj];
          ++tj;
        }
      }
    }
    float excl, total;
    block_seg_scan<BLOCK>(acc, any, carry, s_wv, s_wf, s_incl, excl, total);
    if (any) s_y[ti0] = excl + first;
    carry = total;
    __syncthreads();
    for (int r = tid; r < nrows; r += BLOCK) a.out[cur.i + r] = s_y[r];
    cur = nxt;
  }

  // carry-out of this CTA: the row left open at the end of its share
  if (tid == 0) {
    a.carry_row[blockIdx.x] = cur.i < a.num_tiles ? cur.i : -1;
    a.carry_val[blockIdx.x] = carry;
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) s_last = (atomicAdd(a.ticket, 1u) == (unsigned)(a.num_ctas - 1));
  __syncthreads();
  if (!s_last) return;
  __threadfence();

  // Fix-up by the last CTA: y[row] += sum of the carries of all CTAs that left
  // `row` open, combined in CTA order by a segmented scan keyed by row.
  float run = 0.f;
  for (int b = 0; b < a.num_ctas; b += BLOCK) {
    const int e = b + tid;
    const bool valid = e < a.num_ctas;
    const int64_t row = valid ? __ldcg(a.carry_row + e) : -2;
    const float val = valid ? __ldcg(a.carry_val + e) : 0.f;
    const int64_t prev = (e == 0) ? -3 : (valid ? __ldcg(a.carry_row + e - 1) : -2);
    const int64_t next = (e + 1 < a.num_ctas) ? __ldcg(a.carry_row + e + 1) : -4;
    float excl, total;
    const float incl = block_seg_scan<BLOCK>(val, row != prev, run, s_wv, s_wf, s_incl, excl, total);
    if (valid && row >= 0 && row != next) {
      float* py = a.out + row;
      __stcg(py, __ldcg(py) + incl);
    }
    run = total;
    __syncthreads();
  }
  if (tid == 0) *a.ticket = 0u;
}

// Merge-path expand: the tile of every atom from the same walk (the
// schedule's get_tile for all atoms at once), then per atom either
// tile_of_atom[j] = tile or dvals[j] = dy[tile] * x[col[j]].
template <int BLOCK, int IPT, bool BATCH, bool DVALS>
__global__ void __launch_bounds__(BLOCK) mp_expand_kernel(MpArgs a) {
  constexpr int T = BLOCK * IPT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int* s_end = reinterpret_cast<int*>(smem_raw);  // T
  int* s_row = s_end + T;                          // T
  const int tid = threadIdx.x;
  const size_t base = (size_t)blockIdx.x * (a.tiles_per_cta + 1);
  Split64 cur = load_split<BATCH>(a, base);
  for (int k = 0; k < a.tiles_per_cta; ++k) {
    const Split64 nxt = load_split<BATCH>(a, base + k + 1);
    const int nrows = (int)(nxt.i - cur.i);
    const int nnz = (int)(nxt.j - cur.j);
    const int items = nrows + nnz;
    if (items == 0) break;
    stage_row_ends<BLOCK, BATCH>(a, cur, nxt, nrows, s_end);
    __syncthreads();
    const int d = min(tid * IPT, items);
    int ti = tile_search(s_end, d, nrows, nnz);
    int tj = d - ti;
    const int dend = min(d + IPT, items);
    int nend = ti < nrows ? s_end[ti] : INT_MAX;
#pragma unroll
    for (int it = 0; it < IPT; ++it) {
      if (d + it < dend) {
        if (tj >= nend) {
          ++ti;
          nend = ti < nrows ? s_end[ti] : INT_MAX;
        } else {
          s_row[tj] = ti;
          ++tj;
        }
      }
    }
    __syncthreads();
    for (int l = tid; l < nnz; l += BLOCK) {
      const int64_t j = cur.j + l;
      const int64_t row = cur.i + s_row[l];
      if constexpr (DVALS) {
        int64_t xb = 0, yb = 0;
        if constexpr (BATCH) {
          const int m = (cur.m == nxt.m) ? cur.m : find_matrix(a.nnz_base, cur.m, nxt.m, j);
          xb = __ldg(a.vec_base + m);
          (void)yb;
        }
        const int c = ld_stream(a.atoms.idx + j);
        __stcs(a.dvals + j, __fmul_rn(__ldg(a.dy + row), a.atoms.gather(c, xb)));
      } else {
        a.tile_of_atom[j] = (int32_t)row;
      }
    }
    __syncthreads();
    cur = nxt;
  }
}

// ---------------------------------------------------------- thread-mapped --

// Thread-mapped schedule (Listing 2 / Listing 3): tile t to thread t with a
// grid-sized stride; the thread walks the tile's atoms in order.  Atoms are
// summed in chunks of 256 whose partials are then added in order, which bounds
// the rounding error on very long tiles.
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK) tm_spmv_kernel(const int32_t* __restrict__ rp, int32_t num_tiles,
                                                        AtomView at, float* __restrict__ out) {
  constexpr int CHUNK = 256;
  for (int64_t t = (int64_t)blockIdx.x * BLOCK + threadIdx.x; t < num_tiles; t += (int64_t)gridDim.x * BLOCK) {
    const int b = __ldg(rp + t), e = __ldg(rp + t + 1);
    float total = 0.f;
    for (int k0 = b; k0 < e; k0 += CHUNK) {
      const int k1 = min(e, k0 + CHUNK);
      float part = 0.f;
      for (int k = k0; k < k1; ++k) part += at.product(k, 0, 0);
      total += part;
    }
    out[t] = total;
  }
}

// ----------------------------------------------------------- group-mapped --

// Group-mapped schedule (Sec. 5.2.3), G threads per group, G a power of two
// (G = 32 is the warp-mapped and G = BLOCK the block-mapped schedule of
// Sec. 5.2.2).  A group takes a chunk of G consecutive tiles, writes their atom
// counts' exclusive prefix sum to shared memory, then walks the chunk's
// flattened atoms with stride G; get_tile(a) = largest t with prefix[t] <= a
// (a binary search in shared memory).  Products are reduced per tile by a
// warp-shuffle segmented scan; each warp adds its segment totals into its own
// per-tile partials, and the warps' partials are added in warp order at the
// end, so the result does not depend on timing.
template <int BLOCK, int G>
__global__ void __launch_bounds__(BLOCK) gm_spmv_kernel(const int32_t* __restrict__ rp, int32_t num_tiles,
                                                        AtomView at, float* __restrict__ out) {
  constexpr int GPB = BLOCK / G;               // groups per block
  constexpr int WPG = G >= 32 ? G / 32 : 1;    // warps per group
  constexpr int SW = G < 32 ? G : 32;          // shuffle width
  __shared__ int s_pre[GPB][G + 1];
  __shared__ float s_part[GPB][WPG][G];
  __shared__ int s_wsum[GPB][WPG];
  const int g = threadIdx.x / G;
  const int lane = threadIdx.x % G;             // rank in group
  const int sl = threadIdx.x % SW;              // rank in shuffle segment
  const int wg = lane / 32;                     // warp within group (G >= 32)

  auto group_sync = [&]() {
    if constexpr (G <= 32) {
      __syncwarp();
    } else if constexpr (G == BLOCK) {
      __syncthreads();
    } else {
      asm volatile("bar.sync %0, %1;" ::"r"(g + 1), "r"(G) : "memory");
    }
  };

  // block-uniform outer loop: every group of the block runs the same number of
  // iterations (groups past the end see empty chunks), so shuffles and
  // barriers stay convergent
  for (int64_t bc = blockIdx.x; bc * GPB * G < num_tiles; bc += gridDim.x) {
    const int64_t chunk = bc * GPB + g;
    const int64_t t0 = chunk * G;
    const int64_t t = t0 + lane;
    const int len = t < num_tiles ? __ldg(rp + t + 1) - __ldg(rp + t) : 0;
    // exclusive prefix of the chunk's atom counts
    int wtotal;
    int ex = group_excl_scan_small<SW>(len, sl, wtotal);
    if constexpr (G > 32) {
      if (sl == 0) s_wsum[g][wg] = wtotal;
      group_sync();
      int before = 0;
      for (int w = 0; w < wg; ++w) before += s_wsum[g][w];
      ex += before;
    }
    s_pre[g][lane] = ex;
    if (lane == G - 1) s_pre[g][G] = ex + len;
#pragma unroll
    for (int w = 0; w < WPG; ++w) s_part[g][w][lane] = 0.f;
    group_sync();
    const int total = s_pre[g][G];
    const int64_t abase = t0 < num_tiles ? __ldg(rp + t0) : 0;
    // sub-warp groups share a warp: iterate to the largest total among them
    int rounds_total = total;
    if constexpr (G < 32) rounds_total = __reduce_max_sync(kFull, total);
    for (int a0 = 0; a0 < rounds_total; a0 += G) {
      const int aa = a0 + lane;
      const bool valid = aa < total;
      int tile = G;  // sentinel for idle lanes
      float p = 0.f;
      if (valid) {
        int lo = 0, hi = G - 1;
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (s_pre[g][mid] <= aa) lo = mid;
          else hi = mid - 1;
        }
        tile = lo;
        p = at.product(abase + aa, 0, 0);
      }
      float v = p;
#pragma unroll
      for (int o = 1; o < SW; o <<= 1) {
        const float vo = __shfl_up_sync(kFull, v, o, SW);
        const int to = __shfl_up_sync(kFull, tile, o, SW);
        if (sl >= o && to == tile) v += vo;
      }
      const int nt = __shfl_down_sync(kFull, tile, 1, SW);
      const bool tail = valid && (sl == SW - 1 || nt != tile);
      if (tail) s_part[g][wg][tile] += v;
      __syncwarp();
    }
    group_sync();
    if (t < num_tiles) {
      float s = s_part[g][0][lane];
#pragma unroll
      for (int w = 1; w < WPG; ++w) s += s_part[g][w][lane];
      out[t] = s;
    }
    group_sync();
  }
}

}  // namespace lbk
