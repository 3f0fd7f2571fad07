// Device kernels of the load-balanced SpMV path (sm_103a).
//
// Work vocabulary (Sec. 3.1, Listing 1): tiles are rows of a CSR tile set,
// atoms its nonzeros.  Four schedules (Sec. 4.2, 5.2) consume the same tile
// set: thread-mapped, group-mapped (warp / block / any power-of-two group) and
// merge-path.  Everything here is deterministic: the order in which partial
// sums are combined depends only on the plan, never on timing, and no
// floating-point atomics are used.
//
// A batch of matrices is run as one block-diagonal tile set: its row offsets
// are made global once at plan time, and each atom's dense-vector entry is
// offset by the first column of its matrix (found from the split table's
// per-split matrix index).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <climits>

namespace lbk {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kDevErrColumn = 1;   // device error bit: column index out of range
constexpr int kDevErrTimeout = 2;  // device error bit: a bounded wait gave up
constexpr int kStages = 3;         // shared-memory ring depth of the merge-path pipeline
constexpr long long kSpinLimit = 1LL << 26;
constexpr long long kLookbackSpins = 1LL << 22;  // with 64 ns sleeps: a few tenths of a second

// resident CTAs per SM the look-back kernel is compiled for at items_per_thread 4
#ifndef LB_LOOKBACK_IPT4_CTAS
#define LB_LOOKBACK_IPT4_CTAS 4
#endif

// ------------------------------------------------------------- load helpers --

__device__ __forceinline__ int ld_stream(const int* p) { return __ldcs(p); }
__device__ __forceinline__ float ld_stream(const float* p) { return __ldcs(p); }
__device__ __forceinline__ int4 ld_stream(const int4* p) { return __ldcs(p); }
__device__ __forceinline__ float4 ld_stream(const float4* p) { return __ldcs(p); }

// ------------------------------------------------------------- atom views --

// How atom j of a tile set becomes a product.  idx[j] selects the entry of the
// dense vector (a column for y = A x, a row for dx = A^T dy); the value is
// val[j], or val[perm[j]] when the tile set is a transpose that gathers the
// original values.  With check > 0 every index is checked against it; an
// out-of-range index reads as 0 and sets a bit in *status.
struct AtomView {
  const int32_t* idx;
  const float* val;
  const int32_t* perm;
  const float* vec;
  int32_t check;
  int* status;

  __device__ __forceinline__ float value(int64_t j) const {
    return perm ? __ldg(val + ld_stream(perm + j)) : ld_stream(val + j);
  }
  __device__ __forceinline__ float gather(int c, int64_t xbase) const {
    if (check > 0 && (unsigned)c >= (unsigned)check) {
      if (status) atomicOr(status, kDevErrColumn);
      return 0.f;
    }
    return __ldg(vec + xbase + c);
  }
  __device__ __forceinline__ float product(int64_t j, int64_t xbase) const {
    const int c = ld_stream(idx + j);
    return value(j) * gather(c, xbase);
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

// ------------------------------------------------------ mbarrier and TMA --

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Bounded wait for a phase of `bar`: gives up after `limit` polls and
// returns false (the caller records kDevErrTimeout and winds down).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, long long limit = kSpinLimit) {
  for (long long n = 0; n < limit; ++n)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// 1-D bulk copy (TMA) global -> shared, completion counted on `bar`.
// dst, src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// ------------------------------------------------------------ merge path --

// One wave of a batched merge-path table: a run of whole matrices whose items
// are shared out evenly over all workers; its split entries start at
// entry_base, `tpc` tiles per worker.
struct WaveDesc {
  int64_t entry_base;
  int32_t tpc;
  int32_t row_end;  // first row after the wave: no carry may name it (its rows belong to the next wave)
};

// Arguments of the merge-path kernels.  `splits` holds, for every persistent
// CTA c, tiles_per_cta + 1 consecutive (row, atom) splits: the boundaries of
// its tiles, each on the diagonal given by the plan.
struct MpArgs {
  const int32_t* rp;        // row offsets [num_tiles + 1] (global ones for a batch)
  AtomView atoms;
  float* out;               // per-tile result (y or dx)
  const int2* splits;
  const int32_t* split_m;   // batch: matrix of every split's atom (nullptr otherwise)
  const int64_t* nnz_base;  // batch: first atom of each matrix
  const int64_t* vec_base;  // batch: first dense-vector entry of each matrix
  int tiles_per_cta;         // tiles per worker (a worker is a CTA or, for the warp kernels, a warp)
  int num_ctas;              // CTAs launched
  int num_workers;           // split-table owners = carry slots
  int items_per_tile;
  int32_t num_tiles;
  int64_t num_atoms;         // length of the atom arrays (bounds of vector loads)
  int32_t num_entries;       // split-table entries
  const WaveDesc* waves;    // batched tables: the waves in order; nullptr = one wave
  int num_waves;
  float* carry_val;         // [num_waves x num_ctas], one slot per work unit
  int32_t* carry_row;       // [num_waves x num_ctas]
  unsigned* ticket;         // [0] fix-up ticket, [1] next work unit (zero between launches), [2] launch
                            // epoch of the look-back flags (never 0)
  // look-back kernel (guided shares): first split entry of every share [S + 1],
  // its first two split entries, and the published records [S]
  const int64_t* share_ent;
  const int4* share_head;
  unsigned long long* records;
  int* status;
  // warp kernels: the carries settled run by run (nullptr: the last CTA to
  // finish combines every carry); a run is a span of consecutive work units
  // whose carries name the same row, and the unit after it closes that row
  const int2* unit_runs;    // per work unit: (run it belongs to, run it closes), -1 = none
  const int4* runs;         // per run: first unit, last unit, row, participants (units + 1)
  unsigned* run_cnt;        // per run: participants done in this launch (back to 0 by the last)
  // expand kernels
  const float* dy;          // dvals: upstream gradient per tile
  float* dvals;             // dvals output per atom
  int32_t* tile_of_atom;    // atom -> tile output
};

// Largest m in [lo, hi] with base[m] <= g (the matrix holding global index g).
__device__ __forceinline__ int find_matrix(const int64_t* base, int lo, int hi, int64_t g) {
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(base + mid) <= g) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Dense-vector offset of atom j of a tile whose atoms lie in matrices [m0, m1].
template <bool XB>
__device__ __forceinline__ int64_t atom_xbase(const MpArgs& a, int m0, int m1, int64_t xb0, int64_t j) {
  if constexpr (!XB) {
    return 0;
  } else {
    if (m0 == m1) return xb0;
    return __ldg(a.vec_base + find_matrix(a.nnz_base, m0, m1, j));
  }
}

// Split of local diagonal d inside a tile: smallest ti with
// ti == min(d, nrows) or end(ti) > d - ti - 1 (row end ti comes after atom
// d - ti - 1; a row end precedes the atom with the same index), where end(r)
// is the row end relative to the tile's first atom.
template <class End>
__device__ __forceinline__ int tile_search(End end, int d, int nrows, int nnz) {
  int lo = d - nnz > 0 ? d - nnz : 0;
  int hi = d < nrows ? d : nrows;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (end(mid) > d - mid - 1) hi = mid;
    else lo = mid + 1;
  }
  return lo;
}

// Fix-up of rows split between CTAs, run by the last CTA to finish:
// y[row] += the carries of all CTAs that left `row` open, combined in
// CTA order.  The carries are taken in passes of BLOCK * 8: each thread
// loads 8 consecutive carries at once and sums the runs of equal rows in its
// slice, a block segmented scan (thread order, the previous pass's open run in
// front) joins runs that cross threads, and the thread holding a run's last
// carry updates its row.  Resets the ticket for the next launch.
template <int BLOCK>
__device__ __forceinline__ void last_cta_fixup(const MpArgs& a, int num_slots, float* s_wv, int* s_wf,
                                               float* s_incl) {
  constexpr int KC = 8;
  const int P = num_slots;  // one carry slot per CTA and wave, waves in order: rows never decrease
  const int32_t* carry_row = a.carry_row;
  const float* carry_val = a.carry_val;
  float run_in = 0.f;  // open run at the end of the previous pass
  for (int base = 0; base < P; base += BLOCK * KC) {
    const int e0 = base + threadIdx.x * KC;
    int row[KC];
    float val[KC];
#pragma unroll
    for (int q = 0; q < KC; ++q) {
      const int e = e0 + q;
      row[q] = e < P ? __ldcg(carry_row + e) : -2;
      val[q] = e < P ? __ldcg(carry_val + e) : 0.f;
    }
    const int prev = e0 == 0 ? -3 : (e0 - 1 < P ? __ldcg(carry_row + e0 - 1) : -2);
    const int next = e0 + KC < P ? __ldcg(carry_row + e0 + KC) : -4;
    // this slice: does a run start in it, and the sum of its last (open) run
    float tail = 0.f;
    int head = 0, pr = prev;
#pragma unroll
    for (int q = 0; q < KC; ++q) {
      if (row[q] != pr) {
        head = 1;
        tail = val[q];
      } else {
        tail = tail + val[q];
      }
      pr = row[q];
    }
    float excl, total;
    block_seg_scan<BLOCK>(tail, head, run_in, s_wv, s_wf, s_incl, excl, total);
    float run = excl;
    pr = prev;
#pragma unroll
    for (int q = 0; q < KC; ++q) {
      run = (row[q] != pr) ? val[q] : run + val[q];
      pr = row[q];
      const int nx = q + 1 < KC ? row[q + 1] : next;
      if (row[q] >= 0 && row[q] != nx) {
        float* py = a.out + row[q];
        __stcg(py, __ldcg(py) + run);
      }
    }
    run_in = total;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    a.ticket[0] = 0u;
    a.ticket[1] = 0u;
  }
}

// Ticket that elects the last CTA to finish, after every thread of this CTA
// has written its carries.  Returns true in the last CTA (all threads).
__device__ __forceinline__ bool cta_ticket(const MpArgs& a, int* s_last) {
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) *s_last = (atomicAdd(a.ticket, 1u) == (unsigned)(a.num_ctas - 1));
  __syncthreads();
  const bool last = *s_last != 0;
  if (last) __threadfence();
  return last;
}

// Carry-out of a CTA worker (the CTA-tile kernels) and the ticket.
template <int BLOCK>
__device__ __forceinline__ bool publish_carry(const MpArgs& a, int32_t open_row, float carry, int* s_last) {
  if (threadIdx.x == 0) {
    a.carry_row[blockIdx.x] = open_row < a.num_tiles ? open_row : -1;
    a.carry_val[blockIdx.x] = carry;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) *s_last = (atomicAdd(a.ticket, 1u) == (unsigned)(a.num_ctas - 1));
  __syncthreads();
  const bool last = *s_last != 0;
  if (last) __threadfence();
  return last;
}

// Shared-memory layout of the pipelined merge-path kernel: kStages ring slots,
// each holding the tile's window of atom indices, of values (or perm), and of
// row offsets, each W = T + 8 words (the window starts at the 16-byte boundary
// at or below the tile's first element); then per-tile scratch: the row whose
// last atom sits in each slot, one bit per slot marking those row ends, and the
// tile's row results.
template <int BLOCK, int IPT>
struct MpLayout {
  static constexpr int T = BLOCK * IPT;
  static constexpr int W = T + 8;
  static constexpr int NBW = (W + 31) / 32;
  static constexpr size_t stage_words = 3 * (size_t)W;
  static constexpr size_t bytes = sizeof(int) * (kStages * stage_words + W + NBW + T);
};

template <int BLOCK, int IPT>
constexpr size_t mp_smem_bytes() {
  return MpLayout<BLOCK, IPT>::bytes;
}

// Merge-path SpMV (Sec. 5.2.1) as a persistent, pipelined kernel.  CTA c owns
// an equal share of rows + atoms (the setup step: the plan's split table cuts
// it into tiles of T = BLOCK * IPT merge items, each split found by the search
// along its diagonal).  Within a tile the T items are again split evenly over
// the threads, in two passes instead of one interleaved walk: every thread
// takes at most IPT of the tile's rows (marking where each non-empty row ends)
// and at most IPT of its atoms (accumulating products and closing a row at
// each mark), so no thread holds more than about IPT + 1 items.  Per tile:
//   1. one thread streams the tile's atom indices, values (or perm) and row
//      offsets into a ring slot with 1-D bulk copies (TMA), two tiles ahead;
//   2. one tile ahead, every thread issues the dense-vector gathers of its
//      atoms into registers;
//   3. row pass: empty rows get 0, a row that closes at the tile's start gets
//      the running carry, every other row marks the slot of its last atom;
//   4. atom pass: products are summed per thread in atom order, a mark closes
//      the row; a block segmented scan in thread order resolves rows that
//      cross threads (with the CTA's running carry in front);
//   5. the tile's rows are stored coalesced.
// Rows split between CTAs are fixed up by the last CTA to finish.
// Requires 16-byte aligned idx, val/perm and rp.
template <int BLOCK, int IPT, bool XB, bool PERM>
__global__ void __launch_bounds__(BLOCK) mp_spmv_tma_kernel(MpArgs a) {
  static_assert(IPT % 4 == 0 && 32 % IPT == 0, "IPT must be 4, 8 or 16");
  using L = MpLayout<BLOCK, IPT>;
  constexpr int W = L::W;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  int* s_ring = reinterpret_cast<int*>(smem_raw);
  int* s_endrow = s_ring + kStages * L::stage_words;       // W
  unsigned* s_bits = reinterpret_cast<unsigned*>(s_endrow + W);  // NBW
  float* s_y = reinterpret_cast<float*>(s_bits + L::NBW);  // T
  __shared__ __align__(8) uint64_t s_bar[kStages];
  __shared__ float s_wv[BLOCK / 32];
  __shared__ int s_wf[BLOCK / 32];
  __shared__ float s_incl[BLOCK];
  __shared__ int s_last;
  __shared__ int s_abort;

  const int tid = threadIdx.x;
  const int2* sp = a.splits + (size_t)blockIdx.x * (a.tiles_per_cta + 1);
  const int32_t* sm = XB ? a.split_m + (size_t)blockIdx.x * (a.tiles_per_cta + 1) : nullptr;
  const AtomView& at = a.atoms;

  // number of non-empty tiles of this CTA (tiles hold a.items_per_tile <= T - 4 items)
  int ntiles = 0;
  {
    const int2 e0 = __ldg(sp);
    const int2 e1 = __ldg(sp + a.tiles_per_cta);
    const int64_t share = (int64_t)(e1.x - e0.x) + (e1.y - e0.y);
    ntiles = (int)((share + a.items_per_tile - 1) / a.items_per_tile);
  }

  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) mbar_init(&s_bar[s], 1);
    fence_mbar_init();
    s_abort = 0;
  }
  for (int w = tid; w < L::NBW; w += BLOCK) s_bits[w] = 0u;
  __syncthreads();

  auto idx_slot = [&](int s) { return s_ring + (size_t)s * L::stage_words; };
  auto val_slot = [&](int s) { return s_ring + (size_t)s * L::stage_words + W; };
  auto rp_slot = [&](int s) { return s_ring + (size_t)s * L::stage_words + 2 * W; };

  // Stream tile t into its ring slot: bulk copies of the 16-byte aligned body,
  // plain loads of the (at most 3-element) ragged ends.
  auto issue = [&](int t) {
    const int s = t % kStages;
    const int2 c0 = __ldg(sp + t), c1 = __ldg(sp + t + 1);
    const int a_lo = c0.y & ~3, a_hi = c1.y & ~3;
    const int p_lo = (c0.x + 1) & ~3, p_hi = (c1.x + 1) & ~3;
    const int32_t* vsrc = PERM ? at.perm : reinterpret_cast<const int32_t*>(at.val);
    if (tid == 0) {
      const uint32_t ab = a_hi > a_lo ? (uint32_t)(a_hi - a_lo) * 4u : 0u;
      const uint32_t pb = p_hi > p_lo ? (uint32_t)(p_hi - p_lo) * 4u : 0u;
      fence_proxy_async_smem();
      mbar_arrive_expect_tx(&s_bar[s], 2 * ab + pb);
      if (ab) {
        tma_load_1d(idx_slot(s), at.idx + a_lo, ab, &s_bar[s]);
        tma_load_1d(val_slot(s), vsrc + a_lo, ab, &s_bar[s]);
      }
      if (pb) tma_load_1d(rp_slot(s), a.rp + p_lo, pb, &s_bar[s]);
    } else if (tid >= 32 && tid < 35) {
      const int j = (a_hi > c0.y ? a_hi : c0.y) + (tid - 32);
      if (j < c1.y) {
        idx_slot(s)[j - a_lo] = __ldg(at.idx + j);
        val_slot(s)[j - a_lo] = __ldg(vsrc + j);
      }
    } else if (tid >= 64 && tid < 67) {
      const int q = (p_hi > c0.x + 1 ? p_hi : c0.x + 1) + (tid - 64);
      if (q < c1.x + 1) rp_slot(s)[q - p_lo] = __ldg(a.rp + q);
    }
  };

  // gathers of this thread's atoms of one tile, issued a tile ahead
  struct Gath {
    float xg[IPT];
    float vg[PERM ? IPT : 1];
  };
  auto clear = [&](Gath& g) {
#pragma unroll
    for (int q = 0; q < IPT; ++q) {
      g.xg[q] = 0.f;
      if constexpr (PERM) g.vg[q] = 0.f;
    }
  };

  // returns false if the wait gave up: the slot's contents must then not be used
  auto wait_tile = [&](int t) -> bool {
    if (!mbar_wait_bounded(&s_bar[t % kStages], (uint32_t)((t / kStages) & 1))) {
      atomicOr(&s_abort, 1);
      if (a.status) atomicOr(a.status, kDevErrTimeout);
      return false;
    }
    return true;
  };

  auto prefetch = [&](int t, Gath& g) {
    const int s = t % kStages;
    const int2 c0 = __ldg(sp + t), c1 = __ldg(sp + t + 1);
    const int nnz = c1.y - c0.y, off = c0.y & 3, j0 = c0.y;
    int m0 = 0, m1 = 0;
    int64_t xb0 = 0;
    if constexpr (XB) {
      m0 = __ldg(sm + t);
      m1 = __ldg(sm + t + 1);
      xb0 = __ldg(a.vec_base + m0);
    }
    const int s0 = tid * IPT;
    int c[IPT];
    int pm[PERM ? IPT : 1];
#pragma unroll
    for (int q = 0; q < IPT; q += 4) {
      const int4 c4 = *reinterpret_cast<const int4*>(idx_slot(s) + s0 + q);
      c[q] = c4.x;
      c[q + 1] = c4.y;
      c[q + 2] = c4.z;
      c[q + 3] = c4.w;
      if constexpr (PERM) {
        const int4 p4 = *reinterpret_cast<const int4*>(val_slot(s) + s0 + q);
        pm[q] = p4.x;
        pm[q + 1] = p4.y;
        pm[q + 2] = p4.z;
        pm[q + 3] = p4.w;
      }
    }
#pragma unroll
    for (int q = 0; q < IPT; ++q) {
      const int l = s0 + q - off;
      g.xg[q] = 0.f;
      if constexpr (PERM) g.vg[q] = 0.f;
      if ((unsigned)l < (unsigned)nnz) {
        g.xg[q] = at.gather(c[q], atom_xbase<XB>(a, m0, m1, xb0, (int64_t)j0 + l));
        if constexpr (PERM) g.vg[q] = __ldg(at.val + pm[q]);
      }
    }
  };

  float carry = 0.f;
  int32_t open_row = __ldg(sp).x;
  int issued = 0;  // tiles [0, issued) have bulk copies issued
  int waited = 0;  // tiles [0, waited) have been waited for
  Gath cur, nxt;
  clear(cur);
  clear(nxt);
  if (ntiles > 0) {
    issue(0);
    if (ntiles > 1) issue(1);
    issued = ntiles > 1 ? 2 : 1;
    __syncthreads();  // plain-loaded ends of tiles 0 and 1 visible
    if (wait_tile(0)) prefetch(0, cur);
    waited = 1;
  }
  for (int k = 0; k < ntiles; ++k) {
    if (k + 2 < ntiles) {
      issue(k + 2);
      issued = k + 3;
    }
    if (k + 1 < ntiles) {
      if (wait_tile(k + 1)) prefetch(k + 1, nxt);
      else clear(nxt);
      waited = k + 2;
    }
    const int s = k % kStages;
    const int2 c0 = __ldg(sp + k), c1 = __ldg(sp + k + 1);
    const int nrows = c1.x - c0.x, nnz = c1.y - c0.y;
    const int off = c0.y & 3, roff = (c0.x + 1) & 3, j0 = c0.y;
    const int* rps = rp_slot(s) + roff;

    // row pass
    for (int r = tid; r < nrows; r += BLOCK) {
      const int e = rps[r] - j0;
      const int pe = r ? rps[r - 1] - j0 : -1;
      if (r > 0 && e == pe) {
        s_y[r] = 0.f;  // empty row
      } else if (e == 0) {
        s_y[r] = carry;  // first row, closed at the tile's start
      } else {
        const int slot = e - 1 + off;
        s_endrow[slot] = r;
        atomicOr(&s_bits[slot >> 5], 1u << (slot & 31));
      }
    }
    const float prefix = (nrows > 0 && rps[0] == j0) ? 0.f : carry;
    __syncthreads();

    // atom pass
    const int s0 = tid * IPT;
    const unsigned bits = s_bits[s0 >> 5] >> (s0 & 31);
    const int* vsl = val_slot(s);
    float vv[IPT];
#pragma unroll
    for (int q = 0; q < IPT; q += 4) {
      const float4 v4 = *reinterpret_cast<const float4*>(vsl + s0 + q);
      vv[q] = v4.x;
      vv[q + 1] = v4.y;
      vv[q + 2] = v4.z;
      vv[q + 3] = v4.w;
    }
    float acc = 0.f, first = 0.f;
    int any = 0, first_row = 0;
#pragma unroll
    for (int q = 0; q < IPT; ++q) {
      const int l = s0 + q - off;
      const float v = PERM ? cur.vg[q] : ((unsigned)l < (unsigned)nnz ? vv[q] : 0.f);
      acc += v * cur.xg[q];
      if ((bits >> q) & 1u) {
        const int r = s_endrow[s0 + q];
        if (any) {
          s_y[r] = acc;
        } else {
          first = acc;
          first_row = r;
          any = 1;
        }
        acc = 0.f;
      }
    }
    float excl, total;
    block_seg_scan<BLOCK>(acc, any, prefix, s_wv, s_wf, s_incl, excl, total);
    if (any) s_y[first_row] = excl + first;
    carry = total;
    __syncthreads();
    for (int r = tid; r < nrows; r += BLOCK) a.out[c0.x + r] = s_y[r];
    for (int w = tid; w < L::NBW; w += BLOCK) s_bits[w] = 0u;
    open_row = c1.x;
#pragma unroll
    for (int q = 0; q < IPT; ++q) {
      cur.xg[q] = nxt.xg[q];
      if constexpr (PERM) cur.vg[q] = nxt.vg[q];
    }
    __syncthreads();  // ring slot k % kStages and the tile scratch free again
    if (s_abort) break;
  }
  if (s_abort && tid == 0) {
    // wind down: wait for this CTA's bulk copies still in flight, each with four
    // times the normal bound, so that no copy lands in shared memory after the
    // CTA has left.  The copies read in-bounds global ranges taken from the
    // plan's split table, so they complete; one that outlasts both bounds means
    // the device has stopped making progress altogether
    for (int t = waited > 0 ? waited - 1 : 0; t < issued; ++t)
      mbar_wait_bounded(&s_bar[t % kStages], (uint32_t)((t / kStages) & 1), 4 * kSpinLimit);
  }
  if (!publish_carry<BLOCK>(a, open_row, carry, &s_last)) return;
  last_cta_fixup<BLOCK>(a, a.num_ctas, s_wv, s_wf, s_incl);
}

// Merge-path SpMV without bulk copies, for buffers that are not 16-byte
// aligned: per tile, row ends and atom products are staged in shared memory
// with plain loads, then walked as above.
template <int BLOCK, int IPT, bool XB>
__global__ void __launch_bounds__(BLOCK) mp_spmv_plain_kernel(MpArgs a) {
  constexpr int T = BLOCK * IPT;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float* s_prod = reinterpret_cast<float*>(smem_raw);  // T
  int* s_end = reinterpret_cast<int*>(s_prod + T);     // T
  float* s_y = reinterpret_cast<float*>(s_end + T);    // T
  __shared__ float s_wv[BLOCK / 32];
  __shared__ int s_wf[BLOCK / 32];
  __shared__ float s_incl[BLOCK];
  __shared__ int s_last;

  const int tid = threadIdx.x;
  const int2* sp = a.splits + (size_t)blockIdx.x * (a.tiles_per_cta + 1);
  const int32_t* sm = XB ? a.split_m + (size_t)blockIdx.x * (a.tiles_per_cta + 1) : nullptr;
  float carry = 0.f;
  int2 cur = __ldg(sp);
  for (int k = 0; k < a.tiles_per_cta; ++k) {
    const int2 nxt = __ldg(sp + k + 1);
    const int nrows = nxt.x - cur.x, nnz = nxt.y - cur.y, items = nrows + nnz;
    if (items == 0) break;
    int m0 = 0, m1 = 0;
    int64_t xb0 = 0;
    if constexpr (XB) {
      m0 = __ldg(sm + k);
      m1 = __ldg(sm + k + 1);
      xb0 = __ldg(a.vec_base + m0);
    }
    for (int r = tid; r < nrows; r += BLOCK) s_end[r] = __ldg(a.rp + cur.x + 1 + r) - cur.y;
    for (int l = tid; l < nnz; l += BLOCK) {
      const int64_t j = (int64_t)cur.y + l;
      s_prod[l] = a.atoms.product(j, atom_xbase<XB>(a, m0, m1, xb0, j));
    }
    __syncthreads();
    auto end = [&](int r) { return s_end[r]; };
    const int d = min(tid * IPT, items);
    int ti = tile_search(end, d, nrows, nnz);
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
          acc += s_prod[tj];
          ++tj;
        }
      }
    }
    float excl, total;
    block_seg_scan<BLOCK>(acc, any, carry, s_wv, s_wf, s_incl, excl, total);
    if (any) s_y[ti0] = excl + first;
    carry = total;
    __syncthreads();
    for (int r = tid; r < nrows; r += BLOCK) a.out[cur.x + r] = s_y[r];
    cur = nxt;
  }
  if (!publish_carry<BLOCK>(a, cur.x, carry, &s_last)) return;
  last_cta_fixup<BLOCK>(a, a.num_ctas, s_wv, s_wf, s_incl);
}

template <int BLOCK, int IPT>
constexpr size_t mp_plain_smem_bytes() {
  return sizeof(float) * 3 * (size_t)(BLOCK * IPT);
}

// Merge-path expand: the tile of every atom from the same walk (the
// schedule's get_tile for all atoms at once), then per atom either
// tile_of_atom[j] = tile or dvals[j] = dy[tile] * x[col[j]] (one correctly
// rounded FP32 product).
template <int BLOCK, int IPT, bool XB, bool DVALS>
__global__ void __launch_bounds__(BLOCK) mp_expand_kernel(MpArgs a) {
  constexpr int T = BLOCK * IPT;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  int* s_end = reinterpret_cast<int*>(smem_raw);  // T
  int* s_row = s_end + T;                          // T
  const int tid = threadIdx.x;
  const int2* sp = a.splits + (size_t)blockIdx.x * (a.tiles_per_cta + 1);
  const int32_t* sm = XB ? a.split_m + (size_t)blockIdx.x * (a.tiles_per_cta + 1) : nullptr;
  int2 cur = __ldg(sp);
  for (int k = 0; k < a.tiles_per_cta; ++k) {
    const int2 nxt = __ldg(sp + k + 1);
    const int nrows = nxt.x - cur.x, nnz = nxt.y - cur.y, items = nrows + nnz;
    if (items == 0) break;
    for (int r = tid; r < nrows; r += BLOCK) s_end[r] = __ldg(a.rp + cur.x + 1 + r) - cur.y;
    __syncthreads();
    auto end = [&](int r) { return s_end[r]; };
    const int d = min(tid * IPT, items);
    int ti = tile_search(end, d, nrows, nnz);
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
    int m0 = 0, m1 = 0;
    int64_t xb0 = 0;
    if constexpr (XB && DVALS) {
      m0 = __ldg(sm + k);
      m1 = __ldg(sm + k + 1);
      xb0 = __ldg(a.vec_base + m0);
    }
    for (int l = tid; l < nnz; l += BLOCK) {
      const int64_t j = (int64_t)cur.y + l;
      const int row = cur.x + s_row[l];
      if constexpr (DVALS) {
        const int c = ld_stream(a.atoms.idx + j);
        __stcs(a.dvals + j,
               __fmul_rn(__ldg(a.dy + row), a.atoms.gather(c, atom_xbase<XB>(a, m0, m1, xb0, j))));
      } else {
        a.tile_of_atom[j] = row;
      }
    }
    __syncthreads();
    cur = nxt;
  }
}

// -------------------------------------------------- warp-worker merge path --

// Per-warp shared scratch of the warp-worker kernels: one bit per slot of the
// warp tile marking the slot that holds a row's last atom, the row of each
// marked slot, and the tile's row results.
template <int IPT>
struct WarpScratch {
  static constexpr int W = 32 * IPT;
  unsigned bits[IPT];  // W / 32 words
  int endrow[W];
  float y[W];
};

// Atom indices and values (or perm) of this lane's IPT slots of a warp tile:
// slot s holds atom a_lo + s, a_lo = first atom rounded down to a multiple of
// 4, so each lane's slots are whole 16-byte vectors.  Vectors wholly inside
// the array are loaded as int4; a ragged end of the array with scalars.
// Vectors wholly past the tile's last atom are skipped.
template <int IPT>
__device__ __forceinline__ void load_lane_atoms(const int32_t* __restrict__ idx, const int32_t* __restrict__ val,
                                                int64_t a_lo, int s0, int64_t j_end, int64_t n, int* c, int* vb) {
#pragma unroll
  for (int u = 0; u < IPT / 4; ++u) {
    const int64_t g4 = a_lo + s0 + 4 * u;
    if (g4 >= j_end) {
      c[4 * u] = c[4 * u + 1] = c[4 * u + 2] = c[4 * u + 3] = 0;
      vb[4 * u] = vb[4 * u + 1] = vb[4 * u + 2] = vb[4 * u + 3] = 0;
    } else if (g4 + 3 < n) {
      const int4 ci4 = ld_stream(reinterpret_cast<const int4*>(idx + g4));
      const int4 vb4 = ld_stream(reinterpret_cast<const int4*>(val + g4));
      c[4 * u] = ci4.x;
      c[4 * u + 1] = ci4.y;
      c[4 * u + 2] = ci4.z;
      c[4 * u + 3] = ci4.w;
      vb[4 * u] = vb4.x;
      vb[4 * u + 1] = vb4.y;
      vb[4 * u + 2] = vb4.z;
      vb[4 * u + 3] = vb4.w;
    } else {
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int64_t g = g4 + e;
        c[4 * u + e] = g < n ? ld_stream(idx + g) : 0;
        vb[4 * u + e] = g < n ? ld_stream(val + g) : 0;
      }
    }
  }
}

// Row pass of a warp tile: rows [i0, i0 + nrows) whose ends fall in the tile.
// An empty row gets 0, a first row that closes at the tile's first atom gets
// the running carry; every other row marks the slot of its last atom.  Lane l
// takes rows l, l + 32, ...; the previous row's end comes from the next-lower
// lane (a shuffle) instead of a second load.
// e_pre: rp[i0 + 1 + lane] when lane < nrows (loaded ahead by the caller).
template <int IPT, bool WRITE_Y>
__device__ __forceinline__ void warp_row_pass(const int32_t* __restrict__ rp, int i0, int nrows, int j0, int off,
                                              float carry, int e_pre, WarpScratch<IPT>& sc) {
  const int lane = threadIdx.x & 31;
  int last_e = -1;  // end of row r - 32 seen by lane 31, carried to lane 0
  for (int rb = 0; rb < nrows; rb += 32) {
    const int r = rb + lane;
    const int e = r < nrows ? (rb == 0 ? e_pre : __ldg(rp + i0 + 1 + r)) - j0 : 0;
    int pe = __shfl_up_sync(kFull, e, 1);
    if (lane == 0) pe = last_e;
    last_e = __shfl_sync(kFull, e, 31);
    if (r < nrows) {
      if (r > 0 && e == pe) {
        if (WRITE_Y) sc.y[r] = 0.f;
      } else if (e == 0) {
        if (WRITE_Y) sc.y[r] = carry;
      } else {
        const int slot = e - 1 + off;
        sc.endrow[slot] = r;
        atomicOr(&sc.bits[slot >> 5], 1u << (slot & 31));
      }
    }
  }
}

// The split-table entries of one warp, held 32 at a time in lane registers
// (lane l holds entry 32 * chunk + l) and handed out by shuffles.
struct WarpSplits {
  const int2* sp;
  int count;  // entries owned by the warp
  int chunk = -1;
  int2 reg;
  __device__ __forceinline__ int2 get(int e) {
    const int lane = threadIdx.x & 31;
    const int ch = e >> 5;
    if (ch != chunk) {
      chunk = ch;
      const int idx = ch * 32 + lane;
      reg = idx < count ? __ldg(sp + idx) : make_int2(0, 0);
    }
    return make_int2(__shfl_sync(kFull, reg.x, e & 31), __shfl_sync(kFull, reg.y, e & 31));
  }
};

// One warp's walk over one merge-path share (Sec. 5.2.1): the share's
// split-table entries start at `wbase` (tpc + 1 of them, the last one its
// end).  Tile by tile (32 * IPT - 4 merge items) the lanes gather the dense
// vector for the tile's atoms (atoms loaded as 16-byte vectors one tile
// ahead), split the tile's rows evenly (row pass: empty rows 0, marks at each
// row's last atom) and its atoms evenly (IPT consecutive atoms per lane,
// closing a row at each mark); a warp-shuffle segmented scan in lane order,
// with the running carry in front, resolves rows that cross lanes, and the
// tile's finished rows are stored together.  The row open at the share's
// start gets only this share's part; walk() returns the split at the share's
// end, with the partial sum of the row left open there in `carry`.
// VEC: idx and val (or perm) are 16-byte aligned (vector loads); otherwise
// every atom is loaded on its own.  ONE_ROW: a tile inside a single row is
// summed without the row pass and the segmented scan (the look-back kernel,
// whose guided shares gain from it; the static kernel measured faster without).
// SPLIT_CHECK: whether the launch validates column indices is tested once per
// tile (the same answer for every warp), so an unvalidated launch gathers
// without a test per atom (the look-back kernel: the stencil 285 -> 261 us;
// the static kernel measured slower in that form and keeps the per-atom one).
template <int IPT, bool XB, bool PERM, bool VEC, bool ONE_ROW = false, bool SPLIT_CHECK = false>
struct WarpWalker {
  static_assert(IPT % 4 == 0 && 32 % IPT == 0, "IPT must be 4, 8 or 16");
  const MpArgs& a;
  WarpScratch<IPT>& sc;
  const int lane, s0;
  const int32_t* vsrc;

  __device__ __forceinline__ WarpWalker(const MpArgs& args, WarpScratch<IPT>& scratch)
      : a(args), sc(scratch), lane(threadIdx.x & 31), s0((threadIdx.x & 31) * IPT),
        vsrc(PERM ? args.atoms.perm : reinterpret_cast<const int32_t*>(args.atoms.val)) {
    if (lane < IPT) sc.bits[lane] = 0u;
    __syncwarp();
  }

  // tiles of a share whose split entries run from t0 to e1
  __device__ __forceinline__ int num_tiles(int2 t0, int2 e1) const {
    const int64_t share = (int64_t)(e1.x - t0.x) + (e1.y - t0.y);
    return (int)((share + a.items_per_tile - 1) / a.items_per_tile);
  }

  // this lane's atom indices and values (or perm) of tile (t0, t1)
  __device__ __forceinline__ void load_atoms(int2 t0, int2 t1, int (&c)[IPT], int (&vb)[IPT]) const {
    const int j0 = t0.y, off = j0 & 3, nnz = t1.y - t0.y;
    if constexpr (VEC) {
      load_lane_atoms<IPT>(a.atoms.idx, vsrc, (int64_t)(j0 - off), s0, t1.y, a.num_atoms, c, vb);
    } else {
#pragma unroll
      for (int q = 0; q < IPT; ++q) {
        const int l = s0 + q - off;
        const bool in = (unsigned)l < (unsigned)nnz;
        c[q] = in ? ld_stream(a.atoms.idx + j0 + l) : 0;
        vb[q] = in ? ld_stream(vsrc + j0 + l) : 0;
      }
    }
  }

  // row ends of the first 32 rows of tile (t0, t1), one per lane
  __device__ __forceinline__ int load_ends(int2 t0, int2 t1) const {
    return lane < t1.x - t0.x ? __ldg(a.rp + t0.x + 1 + lane) : 0;
  }

  // gathers of tile (t0, t1) whose atoms are in c / vb: x[col] and the value
  // (read through perm for the transposed tile set); 0 past the tile.  sm: the
  // matrix of the tile's first and last split (batches)
  __device__ __forceinline__ void gather_tile(const int32_t* sm, int2 t0, int2 t1, const int (&c)[IPT],
                                              const int (&vb)[IPT], float (&xg)[IPT], float (&vv)[IPT]) const {
    const int nnz = t1.y - t0.y, j0 = t0.y, off = j0 & 3;
    int m0 = 0, m1 = 0;
    int64_t xb0 = 0;
    if constexpr (XB) {
      m0 = __ldg(sm);
      m1 = __ldg(sm + 1);
      xb0 = __ldg(a.vec_base + m0);
    }
    if (SPLIT_CHECK && a.atoms.check <= 0) {
#pragma unroll
      for (int q = 0; q < IPT; ++q) {
        const int l = s0 + q - off;
        xg[q] = 0.f;
        vv[q] = 0.f;
        if ((unsigned)l < (unsigned)nnz) {
          xg[q] = __ldg(a.atoms.vec + atom_xbase<XB>(a, m0, m1, xb0, (int64_t)j0 + l) + c[q]);
          vv[q] = PERM ? __ldg(a.atoms.val + vb[q]) : __int_as_float(vb[q]);
        }
      }
      return;
    }
#pragma unroll
    for (int q = 0; q < IPT; ++q) {
      const int l = s0 + q - off;
      xg[q] = 0.f;
      vv[q] = 0.f;
      if ((unsigned)l < (unsigned)nnz) {
        xg[q] = a.atoms.gather(c[q], atom_xbase<XB>(a, m0, m1, xb0, (int64_t)j0 + l));
        vv[q] = PERM ? __ldg(a.atoms.val + vb[q]) : __int_as_float(vb[q]);
      }
    }
  }

  // tile (t0, t1) with its gathered products: row pass, atom pass, segmented
  // scan in lane order with the running carry in front, coalesced row stores;
  // e_t = load_ends(t0, t1)
  __device__ __forceinline__ void reduce_tile(int2 t0, int2 t1, int e_t, const float (&xg)[IPT],
                                              const float (&vv)[IPT], float& carry) {
    const int nrows = t1.x - t0.x, j0 = t0.y, off = j0 & 3;
    if (ONE_ROW && nrows == 0) {
      // the tile lies inside one row (the usual case in long rows): no row ends, so its products
      // are one sum -- each lane's in order, the lanes' by a fixed butterfly -- added to the carry
      float acc = 0.f;
#pragma unroll
      for (int q = 0; q < IPT; ++q) acc += vv[q] * xg[q];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
      carry = carry + acc;
      return;
    }
    warp_row_pass<IPT, true>(a.rp, t0.x, nrows, j0, off, carry, e_t, sc);
    const float prefix = (nrows > 0 && __shfl_sync(kFull, e_t, 0) == j0) ? 0.f : carry;
    __syncwarp();
    const unsigned bits = sc.bits[s0 >> 5] >> (s0 & 31);
    // the lane's first row end keeps its partial sum for the scan; a later one (a row that
    // lies inside the lane, rare) stores its sum at once; selects, no branch per slot
    float acc = 0.f, first = 0.f;
    int first_q = -1;
#pragma unroll
    for (int q = 0; q < IPT; ++q) {
      acc += vv[q] * xg[q];
      const bool m = (bits >> q) & 1u;
      if (m && first_q >= 0) sc.y[sc.endrow[s0 + q]] = acc;
      first = (m && first_q < 0) ? acc : first;
      first_q = (m && first_q < 0) ? q : first_q;
      acc = m ? 0.f : acc;
    }
    const int any = first_q >= 0;
    const int first_row = any ? sc.endrow[s0 + first_q] : 0;
    // segment heads at or below this lane: the scan adds lane - o only while no head lies in between
    const unsigned heads = __ballot_sync(kFull, any) & (0xffffffffu >> (31 - lane));
    const int head = heads ? 31 - __clz(heads) : -1;
    float v = acc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const float vo = __shfl_up_sync(kFull, v, o);
      if (lane >= o && lane - o >= head) v = vo + v;
    }
    if (head < 0) v = prefix + v;
    const float up = __shfl_up_sync(kFull, v, 1);
    const float excl = lane ? up : prefix;
    carry = __shfl_sync(kFull, v, 31);
    if (any) sc.y[first_row] = excl + first;
    __syncwarp();
    for (int r = lane; r < nrows; r += 32) a.out[t0.x + r] = sc.y[r];
    if (lane < IPT) sc.bits[lane] = 0u;
    __syncwarp();
  }

  // the share whose split entries start at wbase (tpc + 1 of them): per tile,
  // gather it, load the next tile's atoms (in flight while it is reduced),
  // reduce it
  __device__ __forceinline__ int2 walk(size_t wbase, int tpc, float& carry) {
    WarpSplits spl{a.splits + wbase, tpc + 1};
    const int32_t* sm = XB ? a.split_m + wbase : nullptr;
    int2 c0 = spl.get(0);
    const int ntiles = num_tiles(c0, __ldg(a.splits + wbase + tpc));
    carry = 0.f;
    int c_cur[IPT], vb_cur[IPT];  // atoms of the next tile to gather
    int2 c1 = c0;
    int e_cur = 0;
    if (ntiles > 0) {
      c1 = spl.get(1);
      load_atoms(c0, c1, c_cur, vb_cur);
      e_cur = load_ends(c0, c1);
    }
    for (int k = 0; k < ntiles; ++k) {
      float xg[IPT], vv[IPT];
      gather_tile(sm + k, c0, c1, c_cur, vb_cur, xg, vv);
      int2 c2 = c1;
      int e_next = 0;
      if (k + 1 < ntiles) {
        c2 = spl.get(k + 2);
        load_atoms(c1, c2, c_cur, vb_cur);
        e_next = load_ends(c1, c2);
      }
      reduce_tile(c0, c1, e_cur, xg, vv, carry);
      e_cur = e_next;
      c0 = c1;
      c1 = c2;
    }
    return c0;
  }
};

// Work unit u of a warp kernel is done: its carry slot is written and every
// row store of the unit is fenced.  For each run the unit takes part in (as a
// member, or as the unit that closes the run's row) count it in; the last of
// the run's participants to arrive adds the run's carries, in unit order, to
// the row (whose stored value already holds the closing unit's part) and
// resets the count for the next launch.  Called by one thread.
__device__ __forceinline__ void settle_unit_runs(const MpArgs& a, int u) {
  const int2 ur = __ldg(a.unit_runs + u);
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int r = k == 0 ? ur.x : ur.y;
    if (r < 0) continue;
    const int4 d = __ldg(a.runs + r);
    if (atomicAdd(a.run_cnt + r, 1u) + 1u != (unsigned)d.w) continue;
    __threadfence();
    float sum = 0.f;
    for (int q = d.x; q <= d.y; ++q) sum += __ldcg(a.carry_val + q);
    float* py = a.out + d.z;
    __stcg(py, __ldcg(py) + sum);
    a.run_cnt[r] = 0u;
  }
}

// Merge-path SpMV with warps as the workers and the fix-up of Sec. 5.2.1
// done inside the launch.  The plan's split table gives every warp worker an
// equal share of rows + atoms; a WORK UNIT is the 8 consecutive shares of one
// CTA.  After a unit, the CTA settles the rows split between its own warps (a
// segmented scan over the 8 warps' carries keyed by row) and leaves one
// carry; the last CTA to finish combines those in order.
template <int IPT, bool XB, bool PERM, bool VEC>
__global__ void __launch_bounds__(256, IPT <= 4 ? 5 : IPT <= 8 ? 4 : 2) mp_spmv_warp_kernel(MpArgs a) {
  constexpr int WPB = 8;
  __shared__ WarpScratch<IPT> sc_all[WPB];
  __shared__ float s_wv[WPB];
  __shared__ int s_wf[WPB];
  __shared__ float s_incl[256];
  __shared__ int s_last;
  __shared__ int s_crow[2][WPB];  // by unit parity: a warp may write its next unit's carry while
  __shared__ float s_cval[2][WPB];  // warp 0 still reads this unit's
  __shared__ int s_unit[2];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  WarpWalker<IPT, XB, PERM, VEC> walker(a, sc_all[warp]);
  // tables in waves come from batches: the forward (XB) or the transposed one
  // of dx (PERM); the single-matrix forward drops the wave logic
  constexpr bool kMayWave = XB || PERM;
  const int nwaves = kMayWave && a.waves ? a.num_waves : 1;
  const int upw = a.num_workers / WPB;  // work units per wave
  const int nunits = nwaves * upw;
  // Work unit u = the 8 consecutive warp shares (u mod upw) * 8 + warp of wave
  // u / upw.  With more units than CTAs the units are taken in order from a
  // counter: a CTA that finishes early takes the next open unit, and in a
  // batch all CTAs work on the earliest open shares, so the data in use spans
  // about one wave however long the batch.
  const bool dynamic = nunits > (int)gridDim.x;
  int u = blockIdx.x;
  for (int it = 0; u < nunits; ++it) {
    const int wave = u / upw;
    const int w = (u - wave * upw) * WPB + warp;
    int64_t ebase = 0;
    int tpc = a.tiles_per_cta;
    int row_end = a.num_tiles;
    if (kMayWave && a.waves) {
      ebase = a.waves[wave].entry_base;
      tpc = a.waves[wave].tpc;
      row_end = a.waves[wave].row_end;
    }
    float carry;
    const int2 c_end = walker.walk((size_t)ebase + (size_t)w * (tpc + 1), tpc, carry);
    if (lane == 0) {
      s_crow[it & 1][warp] = c_end.x < row_end ? c_end.x : -1;
      s_cval[it & 1][warp] = carry;
    }
    if (threadIdx.x == 0) s_unit[it & 1] = dynamic ? (int)gridDim.x + (int)atomicAdd(a.ticket + 1, 1u) : nunits;
    if (a.runs) __threadfence();  // this warp's row stores, before the unit's runs are counted in
    __syncthreads();
    // a run that a later warp of this CTA closed is added to its row, the run
    // left open by the last warp becomes the unit's carry-out
    if (warp == 0) {
      const int row = lane < WPB ? s_crow[it & 1][lane] : -5;
      float v = lane < WPB ? s_cval[it & 1][lane] : 0.f;
#pragma unroll
      for (int o = 1; o < WPB; o <<= 1) {
        const float vo = __shfl_up_sync(kFull, v, o, WPB);
        const int ro = __shfl_up_sync(kFull, row, o, WPB);
        if ((lane & (WPB - 1)) >= o && ro == row) v = vo + v;
      }
      const int nrow = __shfl_down_sync(kFull, row, 1, WPB);
      if (lane < WPB - 1 && row >= 0 && nrow != row) {
        float* py = a.out + row;
        __stcg(py, __ldcg(py) + v);
      }
      if (lane == WPB - 1) {
        a.carry_row[u] = row;
        a.carry_val[u] = v;
      }
      if (a.runs) {
        __threadfence();
        __syncwarp();
        if (lane == 0) settle_unit_runs(a, u);
      }
    }
    u = s_unit[it & 1];
  }
  if (a.runs) {
    // every run is settled by its last participant; the unit counter goes back to 0
    if (dynamic && cta_ticket(a, &s_last) && threadIdx.x == 0) {
      a.ticket[0] = 0u;
      a.ticket[1] = 0u;
    }
    return;
  }
  // rows split between units, all waves at once (a wave's rows are never
  // touched by a later wave, and the slots of all waves are in row order)
  if (cta_ticket(a, &s_last)) last_cta_fixup<256>(a, nunits, s_wv, s_wf, s_incl);
}

// Look-back record of share p: (flag << 32) | float bits of its partial sum,
// flag = (epoch << 1) | FINAL; one 64-bit store publishes both halves.
__device__ __forceinline__ void publish_record(unsigned long long* rec, unsigned epoch, bool final_, float v) {
  const unsigned long long w =
      ((unsigned long long)((epoch << 1) | (final_ ? 1u : 0u)) << 32) | (unsigned long long)__float_as_uint(v);
  *reinterpret_cast<volatile unsigned long long*>(rec) = w;
}

// Sum of the partial sums that shares before `s` hold of the row open at s's
// start: lane l reads record s - 1 - l (32 shares per window); the nearest
// FINAL record (or share 0) ends the run.  Waits, bounded, until every record
// up to that one carries this launch's epoch; adds the run with a fixed
// butterfly per window and the windows in order.  Returns false if a wait
// gave up (after max_spins polls).
__device__ __forceinline__ bool look_back(const unsigned long long* records, int s, unsigned epoch, float& total,
                                          long long max_spins = kLookbackSpins) {
  const int lane = threadIdx.x & 31;
  total = 0.f;
  for (int base = s - 1; base >= 0; base -= 32) {
    const int p = base - lane;
    unsigned long long w = 0;
    bool ready = p < 0;
    unsigned term = 0;
    int j = 31;
    for (long long spin = 0;; ++spin) {
      if (!ready) {
        w = *reinterpret_cast<volatile const unsigned long long*>(records + p);
        ready = (unsigned)(w >> 33) == epoch;
      }
      term = __ballot_sync(kFull, p < 0 || (ready && (((w >> 32) & 1ull) || p == 0)));
      j = term ? __ffs(term) - 1 : 31;
      const unsigned need = (2u << j) - 1u;  // lanes 0..j
      if ((__ballot_sync(kFull, ready) & need) == need) break;
      if (spin > max_spins) return false;
      __nanosleep(64);
    }
    float v = (lane <= j && p >= 0) ? __uint_as_float((unsigned)w) : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    total += v;
    if (term) break;
  }
  return true;
}

// Merge-path SpMV with warps as the workers on dynamically taken shares and
// the carries resolved by a decoupled look-back (no block barrier, no fix-up
// pass).  The plan cuts the rows + atoms into num_workers shares of whole warp
// tiles in merge order, large first and down to tiles_per_share tiles at the
// end (guided sizes: each share about 4/5 of the remaining work of one warp),
// so that the warps finish together.  A warp takes its next share from a
// counter two tiles before the end of the current one, loads that share's
// first tile while it reduces its last one, and walks tile after tile with
// the WarpWalker.  At a share's end it publishes the partial sum of the row
// left open there, FINAL if the share holds a row end (the open row then
// started inside it), PARTIAL if the share lies inside one row.  A share that
// closes a row adds, one share later, the partial sums its predecessors hold
// of its first row (look_back) to that row.  Every sum has a fixed order, so
// results do not depend on timing; every share is taken by a running warp and
// no share waits on a later one, so the waits end (and are bounded all the
// same: a wait that gives up sets the timeout bit of the status word).
// Records carry the launch's epoch (ticket[2]), which the last CTA to finish
// advances, so they need no reset between launches.
template <int IPT, bool XB, bool PERM, bool VEC>
__global__ void __launch_bounds__(256, IPT <= 4 ? LB_LOOKBACK_IPT4_CTAS : IPT <= 8 ? 4 : 2) mp_spmv_lookback_kernel(MpArgs a) {
  constexpr int WPB = 8;
  constexpr int kNarrow = 4;  // predecessors one lane walks before the warp-wide window takes over
  __shared__ WarpScratch<IPT> sc_all[WPB];
  __shared__ int s_pend[WPB][32];  // shares whose first row waits for its predecessors' sums
  __shared__ int s_last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  WarpWalker<IPT, XB, PERM, VEC, true, true> wk(a, sc_all[warp]);
  const unsigned epoch = *reinterpret_cast<volatile unsigned*>(a.ticket + 2);
  auto add_to_first_row = [&](int p, float total) {
    float* py = a.out + __ldg(&a.share_head[p].x);
    __stcg(py, __ldcg(py) + total);
  };
  // the first row of share p gets its predecessors' sums: the warp-wide window
  auto resolve = [&](int p) {
    float total;
    if (!look_back(a.records, p, epoch, total) && lane == 0 && a.status) atomicOr(a.status, kDevErrTimeout);
    if (lane == 0) add_to_first_row(p, total);
  };
  // The pending shares of this warp (all of whose predecessors' records are
  // published or being published): each lane walks back from one of them
  // through the records, nearest first, adding the partial sums up to the
  // nearest FINAL one (or share 0); a run longer than kNarrow records goes to
  // the warp-wide window instead.  Which of the two a share takes depends only
  // on the data, and every share goes through this same code whether its list
  // is resolved because it is full or because the warp has no shares left, so
  // the order of every sum is fixed by the plan.
  auto resolve_pending = [&](int npend) {
    bool wide = false;
    if (lane < npend) {
      const int p = s_pend[warp][lane];
      float total = 0.f;
      bool done = false, gave_up = false;
      for (int q = p - 1, n = 0; q >= 0 && n < kNarrow && !done && !gave_up; --q, ++n) {
        unsigned long long w = 0;
        for (long long spin = 0;; ++spin) {
          w = *reinterpret_cast<volatile const unsigned long long*>(a.records + q);
          if ((unsigned)(w >> 33) == epoch) break;
          if (spin > kLookbackSpins) {
            gave_up = true;
            break;
          }
          __nanosleep(64);
        }
        if (gave_up) break;
        total += __uint_as_float((unsigned)w);
        done = ((w >> 32) & 1ull) || q == 0;
      }
      if (gave_up && a.status) atomicOr(a.status, kDevErrTimeout);
      if (done || gave_up) add_to_first_row(p, total);
      else wide = true;
    }
    for (unsigned m = __ballot_sync(kFull, wide); m; m &= m - 1) resolve(s_pend[warp][__ffs(m) - 1]);
    __syncwarp();
  };
  int npend = 0;

  int s = 0;
  if (lane == 0) s = (int)atomicAdd(a.ticket + 1, 1u);
  s = __shfl_sync(kFull, s, 0);
  // the current tile starts at split entry e (e_last: the share's last tile)
  int e = 0, e_last = 0;
  int2 c0 = make_int2(0, 0), c1 = c0;
  int c_cur[IPT], vb_cur[IPT];
  int e_cur = 0;
  if (s < a.num_workers) {
    e = (int)__ldg(a.share_ent + s);
    e_last = (int)__ldg(a.share_ent + s + 1) - 2;
    const int4 h = __ldg(a.share_head + s);
    c0 = make_int2(h.x, h.y);
    c1 = make_int2(h.z, h.w);
    wk.load_atoms(c0, c1, c_cur, vb_cur);
    e_cur = wk.load_ends(c0, c1);
  }
  // split entries, 32 at a time in lane registers, by absolute index
  int chunk = -1;
  int2 creg = make_int2(0, 0);
  auto split_at = [&](int i) {
    if ((i >> 5) != chunk) {
      chunk = i >> 5;
      const int idx = (chunk << 5) + lane;
      creg = idx < a.num_entries ? __ldg(a.splits + idx) : make_int2(0, 0);
    }
    return make_int2(__shfl_sync(kFull, creg.x, i & 31), __shfl_sync(kFull, creg.y, i & 31));
  };
  float carry = 0.f;
  int next = 0;         // lane 0: the share after s, taken two tiles before its end
  bool taken = false;
  while (s < a.num_workers) {
    if (!taken && e + 1 >= e_last) {
      if (lane == 0) next = (int)atomicAdd(a.ticket + 1, 1u);
      taken = true;
    }
    float xg[IPT], vv[IPT];
    wk.gather_tile(XB ? a.split_m + e : nullptr, c0, c1, c_cur, vb_cur, xg, vv);
    const bool last = e == e_last;
    int2 c2 = c1;
    int e_next = 0;
    int sn = 0;
    if (!last) {
      c2 = split_at(e + 2);
      wk.load_atoms(c1, c2, c_cur, vb_cur);
      e_next = wk.load_ends(c1, c2);
    } else {
      sn = __shfl_sync(kFull, next, 0);
      if (sn < a.num_workers) {
        const int4 hn = __ldg(a.share_head + sn);
        wk.load_atoms(make_int2(hn.x, hn.y), make_int2(hn.z, hn.w), c_cur, vb_cur);
        e_next = wk.load_ends(make_int2(hn.x, hn.y), make_int2(hn.z, hn.w));
      }
    }
    wk.reduce_tile(c0, c1, e_cur, xg, vv, carry);
    e_cur = e_next;
    if (!last) {
      c0 = c1;
      c1 = c2;
      ++e;
      continue;
    }
    // share s is done; c1 is its end, its head holds its first row
    const bool has_end = c1.x > __ldg(&a.share_head[s].x);
    if (lane == 0 && s + 1 < a.num_workers) publish_record(a.records + s, epoch, has_end, carry);
    // resolved once the warp has no shares left (the records are published by then), one lane per
    // pending share; a full list is resolved at once, by the same code
    if (has_end && s > 0) {
      if (npend == 32) {
        resolve_pending(32);
        npend = 0;
      }
      if (lane == 0) s_pend[warp][npend] = s;
      ++npend;
      __syncwarp();
    }
    // on to share sn, its first tile already loading (head and entry base
    // read again: cached since the loads above)
    s = sn;
    if (s < a.num_workers) {
      e = (int)__ldg(a.share_ent + s);
      e_last = (int)__ldg(a.share_ent + s + 1) - 2;
      const int4 hn = __ldg(a.share_head + s);
      c0 = make_int2(hn.x, hn.y);
      c1 = make_int2(hn.z, hn.w);
    }
    carry = 0.f;
    taken = false;
  }
  resolve_pending(npend);
  // the last CTA to finish resets the share counter and advances the epoch
  if (cta_ticket(a, &s_last) && threadIdx.x == 0) {
    const unsigned e1 = (epoch + 1u) & 0x7fffffffu;
    a.ticket[1] = 0u;
    a.ticket[2] = e1 ? e1 : 1u;
    a.ticket[0] = 0u;
  }
}

// Warp-worker expand: the tile of every atom from the same row marks, then
// per atom either tile_of_atom[j] = tile or dvals[j] = dy[tile] * x[col[j]]
// (one correctly rounded FP32 product).  The tile of an atom is the row of
// the first marked slot at or after it (the row left open at the tile's end
// if there is none).
template <int IPT, bool XB, bool DVALS>
__global__ void __launch_bounds__(256) mp_expand_warp_kernel(MpArgs a) {
  constexpr int WPB = 8;
  __shared__ WarpScratch<IPT> sc_all[WPB];
  __shared__ int s_unit[2];
  __shared__ int s_last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  WarpScratch<IPT>& sc = sc_all[warp];
  if (lane < IPT) sc.bits[lane] = 0u;
  __syncwarp();
  const int s0 = lane * IPT;
  // the ntiles tiles of one share, split entries sp[0..ntiles], matrices sm;
  // a tile's column indices and first row ends are loaded one tile ahead and
  // its gathers issued before its row pass.  A lane's slots are whole 16-byte
  // vectors of the atom arrays (as in load_lane_atoms), so with col_idx
  // 16-byte aligned its indices come as int4 loads, and with the output
  // aligned a vector lying wholly inside the tile is stored as one 16-byte
  // store; the slots at the tile's two ends are stored one by one, since the
  // rest of their vector belongs to the neighbouring tiles.  (Power-law 1M,
  // dvals: 123 -> 100 us, the same products bit for bit.)
  const bool vec_idx = (reinterpret_cast<uintptr_t>(a.atoms.idx) & 15u) == 0;
  auto load_cols = [&](int2 t0, int2 t1, int (&c)[IPT]) {
    const int nnz = t1.y - t0.y, j0 = t0.y, off = j0 & 3;
    if (vec_idx) {
#pragma unroll
      for (int u = 0; u < IPT / 4; ++u) {
        const int l0 = s0 + 4 * u - off;
        const int64_t g4 = (int64_t)j0 + l0;
        if (l0 >= nnz) {
          c[4 * u] = c[4 * u + 1] = c[4 * u + 2] = c[4 * u + 3] = 0;
        } else if (g4 + 3 < a.num_atoms) {
          const int4 v = ld_stream(reinterpret_cast<const int4*>(a.atoms.idx + g4));
          c[4 * u] = v.x;
          c[4 * u + 1] = v.y;
          c[4 * u + 2] = v.z;
          c[4 * u + 3] = v.w;
        } else {
#pragma unroll
          for (int e = 0; e < 4; ++e) c[4 * u + e] = g4 + e < a.num_atoms ? ld_stream(a.atoms.idx + g4 + e) : 0;
        }
      }
    } else {
#pragma unroll
      for (int q = 0; q < IPT; ++q) {
        const int l = s0 + q - off;
        c[q] = (unsigned)l < (unsigned)nnz ? ld_stream(a.atoms.idx + j0 + l) : 0;
      }
    }
  };
  const bool vec_out = DVALS ? (reinterpret_cast<uintptr_t>(a.dvals) & 15u) == 0
                             : (reinterpret_cast<uintptr_t>(a.tile_of_atom) & 15u) == 0;
  auto expand_share = [&](const int2* sp, const int32_t* sm, int ntiles) {
    int2 c0 = __ldg(sp);
    int2 c1 = ntiles > 0 ? __ldg(sp + 1) : c0;
    int c_cur[IPT];
    if constexpr (DVALS) {
      if (ntiles > 0) load_cols(c0, c1, c_cur);
    }
    int e_cur = ntiles > 0 && lane < c1.x - c0.x ? __ldg(a.rp + c0.x + 1 + lane) : 0;
    for (int k = 0; k < ntiles; ++k) {
      const int nrows = c1.x - c0.x, nnz = c1.y - c0.y, j0 = c0.y, off = j0 & 3;
      float xv[IPT];
      if constexpr (DVALS) {
        int m0 = 0, m1 = 0;
        int64_t xb0 = 0;
        if constexpr (XB) {
          m0 = __ldg(sm + k);
          m1 = __ldg(sm + k + 1);
          xb0 = __ldg(a.vec_base + m0);
        }
        // whether the launch validates column indices is tested once per tile (the same
        // answer for every warp), so an unvalidated launch gathers without a test per atom
        if (a.atoms.check <= 0) {
#pragma unroll
          for (int q = 0; q < IPT; ++q) {
            const int l = s0 + q - off;
            xv[q] = (unsigned)l < (unsigned)nnz
                        ? __ldg(a.atoms.vec + atom_xbase<XB>(a, m0, m1, xb0, (int64_t)j0 + l) + c_cur[q])
                        : 0.f;
          }
        } else {
#pragma unroll
          for (int q = 0; q < IPT; ++q) {
            const int l = s0 + q - off;
            xv[q] = (unsigned)l < (unsigned)nnz
                        ? a.atoms.gather(c_cur[q], atom_xbase<XB>(a, m0, m1, xb0, (int64_t)j0 + l))
                        : 0.f;
          }
        }
      }
      // next tile's columns and row ends, in flight while this one is expanded
      int2 c2 = c1;
      int e_next = 0;
      if (k + 1 < ntiles) {
        c2 = __ldg(sp + k + 2);
        if constexpr (DVALS) load_cols(c1, c2, c_cur);
        e_next = lane < c2.x - c1.x ? __ldg(a.rp + c1.x + 1 + lane) : 0;
      }
      int rows_q[IPT];
      if (nrows == 0) {
        // the tile lies inside one row: every atom is that row's
#pragma unroll
        for (int q = 0; q < IPT; ++q) rows_q[q] = c1.x;
      } else {
        warp_row_pass<IPT, false>(a.rp, c0.x, nrows, j0, off, 0.f, e_cur, sc);
        __syncwarp();
        const unsigned bits = (sc.bits[s0 >> 5] >> (s0 & 31)) & (IPT == 32 ? 0xffffffffu : ((1u << IPT) - 1u));
        // first marked slot of each later lane: suffix minimum over the lanes
        int fm = bits ? s0 + __ffs(bits) - 1 : INT_MAX;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int n = __shfl_down_sync(kFull, fm, o);
          if (lane + o < 32) fm = min(fm, n);
        }
        int nxt = __shfl_down_sync(kFull, fm, 1);
        if (lane == 31) nxt = INT_MAX;
#pragma unroll
        for (int q = IPT - 1; q >= 0; --q) {
          if ((bits >> q) & 1u) nxt = s0 + q;
          rows_q[q] = nxt == INT_MAX ? c1.x : c0.x + sc.endrow[nxt];
        }
      }
#pragma unroll
      for (int u = 0; u < IPT / 4; ++u) {
        const int l0 = s0 + 4 * u - off;
        if (vec_out && l0 >= 0 && l0 + 3 < nnz) {
          const int64_t j = (int64_t)j0 + l0;
          if constexpr (DVALS) {
            const float4 v = make_float4(__fmul_rn(__ldg(a.dy + rows_q[4 * u]), xv[4 * u]),
                                         __fmul_rn(__ldg(a.dy + rows_q[4 * u + 1]), xv[4 * u + 1]),
                                         __fmul_rn(__ldg(a.dy + rows_q[4 * u + 2]), xv[4 * u + 2]),
                                         __fmul_rn(__ldg(a.dy + rows_q[4 * u + 3]), xv[4 * u + 3]));
            __stcs(reinterpret_cast<float4*>(a.dvals + j), v);
          } else {
            *reinterpret_cast<int4*>(a.tile_of_atom + j) =
                make_int4(rows_q[4 * u], rows_q[4 * u + 1], rows_q[4 * u + 2], rows_q[4 * u + 3]);
          }
        } else {
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int q = 4 * u + e, l = l0 + e;
            if ((unsigned)l < (unsigned)nnz) {
              const int64_t j = (int64_t)j0 + l;
              if constexpr (DVALS) {
                __stcs(a.dvals + j, __fmul_rn(__ldg(a.dy + rows_q[q]), xv[q]));
              } else {
                a.tile_of_atom[j] = rows_q[q];
              }
            }
          }
        }
      }
      __syncwarp();
      if (lane < IPT) sc.bits[lane] = 0u;
      __syncwarp();
      c0 = c1;
      c1 = c2;
      e_cur = e_next;
    }
  };
  bool dynamic;
  if (a.share_ent) {
    // guided shares of the look-back table, taken by each warp from the counter
    dynamic = true;
    const int S = a.num_workers;
    int sh = 0;
    if (lane == 0) sh = (int)atomicAdd(a.ticket + 1, 1u);
    sh = __shfl_sync(kFull, sh, 0);
    while (sh < S) {
      const int64_t b0 = __ldg(a.share_ent + sh);
      const int nt = (int)(__ldg(a.share_ent + sh + 1) - b0) - 1;
      expand_share(a.splits + b0, XB ? a.split_m + b0 : nullptr, nt);
      if (lane == 0) sh = (int)atomicAdd(a.ticket + 1, 1u);
      sh = __shfl_sync(kFull, sh, 0);
    }
  } else {
    const int nwaves = a.waves ? a.num_waves : 1;
    const int upw = a.num_workers / WPB;
    const int nunits = nwaves * upw;
    // work units as in mp_spmv_warp_kernel, taken in order when there are more
    // than CTAs
    dynamic = nunits > (int)gridDim.x;
    int u = blockIdx.x;
    for (int it = 0; u < nunits; ++it) {
      const int wave = u / upw;
      const int w = (u - wave * upw) * WPB + warp;
      int64_t ebase = 0;
      int tpc = a.tiles_per_cta;
      if (a.waves) {
        ebase = a.waves[wave].entry_base;
        tpc = a.waves[wave].tpc;
      }
      const int2* sp = a.splits + (size_t)ebase + (size_t)w * (tpc + 1);
      const int32_t* sm = XB ? a.split_m + (size_t)ebase + (size_t)w * (tpc + 1) : nullptr;
      const int2 t0 = __ldg(sp);
      const int2 e1 = __ldg(sp + tpc);
      const int64_t share = (int64_t)(e1.x - t0.x) + (e1.y - t0.y);
      expand_share(sp, sm, (int)((share + a.items_per_tile - 1) / a.items_per_tile));
      if (dynamic) {
        if (threadIdx.x == 0) s_unit[it & 1] = (int)gridDim.x + (int)atomicAdd(a.ticket + 1, 1u);
        __syncthreads();
        u = s_unit[it & 1];
      } else {
        u = nunits;
      }
    }
  }
  // the last CTA to finish resets the counter for the next launch
  if (dynamic && cta_ticket(a, &s_last) && threadIdx.x == 0) {
    a.ticket[0] = 0u;
    a.ticket[1] = 0u;
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
      for (int k = k0; k < k1; ++k) part += at.product(k, 0);
      total += part;
    }
    out[t] = total;
  }
}

// Thread-mapped schedule with the atoms staged in shared memory (Sec. 4.2's
// thread-mapped loop; the staging is the shared-memory use of Sec. 5.2.3).
// A warp takes 32 consecutive tiles, one per lane.  When their atoms fit in
// the warp's CAP slots, the warp first copies them (column indices and values,
// or permutation entries for a transposed tile set) into shared memory --
// 16-byte asynchronous copies (cp.async, no register round trip, all in
// flight at once) when both arrays are 16-byte aligned, else coalesced plain
// loads -- then every lane walks its own tile there, so that gather k of the
// 32 lanes reads entry k of 32 neighbouring tiles: where neighbouring tiles
// touch neighbouring columns (banded and stencil matrices), one gather
// instruction then touches one or two lines of the dense vector instead of up
// to 32.  A warp whose tiles hold more atoms reads them straight from global
// memory.  Each lane sums its tile's atoms in order, in chunks of 256 whose
// partials are added in order (as the plain thread-mapped kernel does).
__device__ __forceinline__ void cp_async16(void* dst, const void* src, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

template <int CAP>
__global__ void __launch_bounds__(256) tm_staged_spmv_kernel(const int32_t* __restrict__ rp, int32_t num_tiles,
                                                             AtomView at, float* __restrict__ out) {
  constexpr int WPB = 8, CHUNK = 256;
  static_assert(CAP % 4 == 0, "the last 16-byte copy must end inside the slot");
  // CAP atoms plus up to 3 before the first one (copies start on a 16-byte boundary)
  __shared__ __align__(16) int s_idx[WPB][CAP + 4];
  __shared__ __align__(16) int s_val[WPB][CAP + 4];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int32_t* vsrc = at.perm ? at.perm : reinterpret_cast<const int32_t*>(at.val);
  const bool async = ((reinterpret_cast<uintptr_t>(at.idx) | reinterpret_cast<uintptr_t>(vsrc)) & 15u) == 0;
  const int num_atoms = __ldg(rp + num_tiles);
  const int64_t groups = ((int64_t)num_tiles + 31) / 32;
  for (int64_t g = (int64_t)blockIdx.x * WPB + warp; g < groups; g += (int64_t)gridDim.x * WPB) {
    const int64_t t = g * 32 + lane;
    const int64_t t_last = min((int64_t)num_tiles, g * 32 + 32);
    const int a0 = __ldg(rp + g * 32), a1 = __ldg(rp + t_last);
    const int b = t < num_tiles ? __ldg(rp + t) : a1;
    const int e = t < num_tiles ? __ldg(rp + t + 1) : a1;
    float total = 0.f;
    if (a1 - a0 <= CAP) {
      const int base = a0 & ~3;
      if (async) {
        // 16-byte chunks from the aligned start; a chunk at the end of the arrays copies only
        // what exists (the rest of its slot is zero-filled)
        const int nchunk = (a1 - base + 3) >> 2;
        for (int c = lane; c < nchunk; c += 32) {
          const int k = base + 4 * c;
          const int bytes = 4 * min(4, num_atoms - k);
          cp_async16(&s_idx[warp][4 * c], at.idx + k, bytes);
          cp_async16(&s_val[warp][4 * c], vsrc + k, bytes);
        }
        cp_async_wait_all();
      } else {
        for (int k = a0 + lane; k < a1; k += 32) {
          s_idx[warp][k - base] = ld_stream(at.idx + k);
          s_val[warp][k - base] = ld_stream(vsrc + k);
        }
      }
      __syncwarp();
      const int* si = s_idx[warp] - base;
      const int* sv = s_val[warp] - base;
      for (int k0 = b; k0 < e; k0 += CHUNK) {
        const int k1 = min(e, k0 + CHUNK);
        float part = 0.f;
        int k = k0;
        for (; k + 4 <= k1; k += 4) {
          const float g0 = at.gather(si[k], 0), g1 = at.gather(si[k + 1], 0), g2 = at.gather(si[k + 2], 0),
                      g3 = at.gather(si[k + 3], 0);
          float w0, w1, w2, w3;
          if (at.perm) {
            w0 = __ldg(at.val + sv[k]);
            w1 = __ldg(at.val + sv[k + 1]);
            w2 = __ldg(at.val + sv[k + 2]);
            w3 = __ldg(at.val + sv[k + 3]);
          } else {
            w0 = __int_as_float(sv[k]);
            w1 = __int_as_float(sv[k + 1]);
            w2 = __int_as_float(sv[k + 2]);
            w3 = __int_as_float(sv[k + 3]);
          }
          part += w0 * g0;
          part += w1 * g1;
          part += w2 * g2;
          part += w3 * g3;
        }
        for (; k < k1; ++k) part += (at.perm ? __ldg(at.val + sv[k]) : __int_as_float(sv[k])) * at.gather(si[k], 0);
        total += part;
      }
      __syncwarp();  // the slots are free again
    } else {
      for (int k0 = b; k0 < e; k0 += CHUNK) {
        const int k1 = min(e, k0 + CHUNK);
        float part = 0.f;
        for (int k = k0; k < k1; ++k) part += at.product(k, 0);
        total += part;
      }
    }
    if (t < num_tiles) out[t] = total;
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
        p = at.product(abase + aa, 0);
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
