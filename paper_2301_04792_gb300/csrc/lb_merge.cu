// Merge-path split tables and kernel launches, plus the thread-mapped and
// group-mapped launchers.
#include <algorithm>
#include <vector>

#include "lb_internal.h"
#include "lb_kernels.cuh"

namespace lbh {

void MpTable::release() {
  cudaFree(splits);
  cudaFree(d_diag);
  cudaFree(split_m);
  cudaFree(d_waves);
  d_waves = nullptr;
  num_waves = 1;
  cudaFree(carry_val);
  cudaFree(carry_row);
  cudaFree(ticket);
  cudaFree(share_ent);
  cudaFree(share_head);
  cudaFree(records);
  cudaFree(unit_runs);
  cudaFree(runs);
  cudaFree(run_cnt);
  unit_runs = nullptr;
  runs = nullptr;
  run_cnt = nullptr;
  num_runs = 0;
  share_ent = nullptr;
  share_head = nullptr;
  records = nullptr;
  splits = nullptr;
  d_diag = nullptr;
  split_m = nullptr;
  carry_val = nullptr;
  carry_row = nullptr;
  ticket = nullptr;
  built = false;
}

void BatchBases::release() {
  cudaFree(nnz_base);
  cudaFree(vec_base);
  nnz_base = vec_base = nullptr;
}

int device_sms(int device) {
  int n = 0;
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, device);
  return n > 0 ? n : 1;
}

// Diagonal of split-table entry e: CTA c = e / (tpc+1) owns the items
// [floor(c*items/grid), floor((c+1)*items/grid)) and its k-th tile starts
// k*items_per_tile items in (clamped to the share's end).
__host__ __device__ inline int64_t mp_diag(int64_t items, int grid, int tpc, int ipt_items, int64_t e) {
  const int64_t c = e / (tpc + 1), k = e % (tpc + 1);
  const int64_t b = c * items / grid, en = (c + 1) * items / grid;
  const int64_t d = b + k * (int64_t)ipt_items;
  return d < en ? d : en;
}

int64_t mp_diagonal(int64_t items, int grid, int tiles_per_cta, int items_per_tile, int64_t e) {
  return mp_diag(items, grid, tiles_per_cta, items_per_tile, e);
}

void mp_geometry(int64_t items, int grid_cap, int items_per_tile, int block, int* grid, int* tiles_per_cta) {
  // at least `block` items (one per thread) per CTA; at most grid_cap CTAs
  int64_t g = (items + block - 1) / block;
  if (g > grid_cap) g = grid_cap;
  if (g < 1) g = 1;
  const int64_t share = (items + g - 1) / g;
  int64_t tpc = (share + items_per_tile - 1) / items_per_tile;
  if (tpc < 1) tpc = 1;
  *grid = (int)g;
  *tiles_per_cta = (int)tpc;
}

// ------------------------------------------------------------ instantiations --

template <int IPT, bool XB, bool PERM>
static void* tma_fn() {
  return reinterpret_cast<void*>(lbk::mp_spmv_tma_kernel<kBlock, IPT, XB, PERM>);
}
template <int IPT, bool XB>
static void* plain_fn() {
  return reinterpret_cast<void*>(lbk::mp_spmv_plain_kernel<kBlock, IPT, XB>);
}
template <int IPT, bool XB, bool DV>
static void* expand_fn() {
  return reinterpret_cast<void*>(lbk::mp_expand_kernel<kBlock, IPT, XB, DV>);
}

template <int IPT, bool XB, bool PERM, bool VEC>
static void* warp_fn() {
  return reinterpret_cast<void*>(lbk::mp_spmv_warp_kernel<IPT, XB, PERM, VEC>);
}
template <int IPT, bool XB, bool PERM, bool VEC>
static void* lookback_fn() {
  return reinterpret_cast<void*>(lbk::mp_spmv_lookback_kernel<IPT, XB, PERM, VEC>);
}
template <int IPT>
static void* pick_lookback(bool xb, bool perm, bool vec) {
  if (vec) {
    if (xb) return perm ? lookback_fn<IPT, true, true, true>() : lookback_fn<IPT, true, false, true>();
    return perm ? lookback_fn<IPT, false, true, true>() : lookback_fn<IPT, false, false, true>();
  }
  if (xb) return perm ? lookback_fn<IPT, true, true, false>() : lookback_fn<IPT, true, false, false>();
  return perm ? lookback_fn<IPT, false, true, false>() : lookback_fn<IPT, false, false, false>();
}
static void* kernel_lookback(int ipt, bool xb, bool perm, bool vec) {
  switch (ipt) {
    case 4: return pick_lookback<4>(xb, perm, vec);
    case 8: return pick_lookback<8>(xb, perm, vec);
    case 16: return pick_lookback<16>(xb, perm, vec);
  }
  return nullptr;
}
template <int IPT, bool XB, bool DV>
static void* expand_warp_fn() {
  return reinterpret_cast<void*>(lbk::mp_expand_warp_kernel<IPT, XB, DV>);
}
template <int IPT>
static void* pick_warp(bool xb, bool perm, bool vec) {
  if (vec) {
    if (xb) return perm ? warp_fn<IPT, true, true, true>() : warp_fn<IPT, true, false, true>();
    return perm ? warp_fn<IPT, false, true, true>() : warp_fn<IPT, false, false, true>();
  }
  if (xb) return perm ? warp_fn<IPT, true, true, false>() : warp_fn<IPT, true, false, false>();
  return perm ? warp_fn<IPT, false, true, false>() : warp_fn<IPT, false, false, false>();
}
template <int IPT>
static void* pick_expand_warp(bool xb, bool dv) {
  if (xb) return dv ? expand_warp_fn<IPT, true, true>() : expand_warp_fn<IPT, true, false>();
  return dv ? expand_warp_fn<IPT, false, true>() : expand_warp_fn<IPT, false, false>();
}
static void* kernel_warp(int ipt, bool xb, bool perm, bool vec) {
  switch (ipt) {
    case 4: return pick_warp<4>(xb, perm, vec);
    case 8: return pick_warp<8>(xb, perm, vec);
    case 16: return pick_warp<16>(xb, perm, vec);
  }
  return nullptr;
}
static void* kernel_expand_warp(int ipt, bool xb, bool dv) {
  switch (ipt) {
    case 4: return pick_expand_warp<4>(xb, dv);
    case 8: return pick_expand_warp<8>(xb, dv);
    case 16: return pick_expand_warp<16>(xb, dv);
  }
  return nullptr;
}

template <int IPT>
static void* pick_tma(bool xb, bool perm) {
  if (xb) return perm ? tma_fn<IPT, true, true>() : tma_fn<IPT, true, false>();
  return perm ? tma_fn<IPT, false, true>() : tma_fn<IPT, false, false>();
}
template <int IPT>
static void* pick_plain(bool xb) {
  return xb ? plain_fn<IPT, true>() : plain_fn<IPT, false>();
}
template <int IPT>
static void* pick_expand(bool xb, bool dv) {
  if (xb) return dv ? expand_fn<IPT, true, true>() : expand_fn<IPT, true, false>();
  return dv ? expand_fn<IPT, false, true>() : expand_fn<IPT, false, false>();
}

static size_t tma_smem(int ipt) {
  switch (ipt) {
    case 4: return lbk::mp_smem_bytes<kBlock, 4>();
    case 8: return lbk::mp_smem_bytes<kBlock, 8>();
    default: return lbk::mp_smem_bytes<kBlock, 16>();
  }
}
static size_t plain_smem(int ipt) { return sizeof(float) * 3 * (size_t)kBlock * ipt; }
static size_t expand_smem(int ipt) { return sizeof(int) * 2 * (size_t)kBlock * ipt; }

static void* kernel_tma(int ipt, bool xb, bool perm) {
  switch (ipt) {
    case 4: return pick_tma<4>(xb, perm);
    case 8: return pick_tma<8>(xb, perm);
    case 16: return pick_tma<16>(xb, perm);
  }
  return nullptr;
}
static void* kernel_plain(int ipt, bool xb) {
  switch (ipt) {
    case 4: return pick_plain<4>(xb);
    case 8: return pick_plain<8>(xb);
    case 16: return pick_plain<16>(xb);
  }
  return nullptr;
}
static void* kernel_expand(int ipt, bool xb, bool dv) {
  switch (ipt) {
    case 4: return pick_expand<4>(xb, dv);
    case 8: return pick_expand<8>(xb, dv);
    case 16: return pick_expand<16>(xb, dv);
  }
  return nullptr;
}

// Every launch sets the dynamic shared-memory limit of its kernel first (cheap,
// and correct whichever device is current).
static cudaError_t launch(void* fn, int grid, size_t smem, cudaStream_t s, lbk::MpArgs* a) {
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  void* args[] = {a};
  return cudaLaunchKernel(fn, dim3(grid), dim3(kBlock), args, smem, s);
}

int occupancy_mp(int ipt, int variant) {
  void* fn = variant == 0   ? kernel_warp(ipt, false, false, true)
             : variant == 3 ? kernel_lookback(ipt, false, false, true)
             : variant == 1 ? kernel_plain(ipt, false)
                            : kernel_tma(ipt, false, false);
  if (!fn) return 1;
  const size_t smem = warp_workers(variant) ? 0 : variant == 1 ? plain_smem(ipt) : tma_smem(ipt);
  cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kBlock, smem) != cudaSuccess || occ < 1) occ = 1;
  return occ;
}

// ------------------------------------------------------------ split kernels --

__global__ void mp_splits_kernel(const int32_t* __restrict__ rp, int32_t R, int64_t N, int64_t items, int grid,
                                 int tpc, int ipt_items, int64_t entries, int2* out, int64_t* diag) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= entries) return;
  const int64_t d = mp_diag(items, grid, tpc, ipt_items, e);
  // smallest i in [max(0, d-N), min(d, R)] with i == min(d, R) or rp[i+1] > d-i-1
  int64_t lo = d - N > 0 ? d - N : 0;
  int64_t hi = d < R ? d : R;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if ((int64_t)__ldg(rp + mid + 1) > d - mid - 1) hi = mid;
    else lo = mid + 1;
  }
  out[e] = make_int2((int)lo, (int)(d - lo));
  if (diag) diag[e] = d;
}

// Splits of a waved table: entry e belongs to wave v (largest v with
// entry_base[v] <= e); inside the wave, worker w = local / (tpc+1) owns the
// items [floor(w*I/P), floor((w+1)*I/P)) of the wave's I items, tile k starts
// k*items_per_tile in.
__global__ void mp_splits_waves_kernel(const int32_t* __restrict__ rp, int32_t R, int64_t N,
                                       const int64_t* __restrict__ wave_begin, const lbk::WaveDesc* __restrict__ wd,
                                       int num_waves, int workers, int ipt_items, int64_t entries, int2* out,
                                       int64_t* diag) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= entries) return;
  int lo = 0, hi = num_waves - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (wd[mid].entry_base <= e) lo = mid;
    else hi = mid - 1;
  }
  const int v = lo;
  const int64_t local = e - wd[v].entry_base;
  const int tpc = wd[v].tpc;
  const int64_t w = local / (tpc + 1), k = local % (tpc + 1);
  const int64_t items = wave_begin[v + 1] - wave_begin[v];
  const int64_t b = wave_begin[v] + w * items / workers, en = wave_begin[v] + (w + 1) * items / workers;
  const int64_t d0 = b + k * (int64_t)ipt_items;
  const int64_t d = d0 < en ? d0 : en;
  int64_t lo2 = d - N > 0 ? d - N : 0;
  int64_t hi2 = d < R ? d : R;
  while (lo2 < hi2) {
    const int64_t mid = (lo2 + hi2) >> 1;
    if ((int64_t)__ldg(rp + mid + 1) > d - mid - 1) hi2 = mid;
    else lo2 = mid + 1;
  }
  out[e] = make_int2((int)lo2, (int)(d - lo2));
  diag[e] = d;
}

// matrix holding each split's atom: largest m with nnz_base[m] <= j (over all matrices)
__global__ void split_matrix_kernel(const int2* __restrict__ splits, int64_t entries,
                                    const int64_t* __restrict__ nnz_base, int num, int32_t* out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= entries) return;
  out[e] = lbk::find_matrix(nnz_base, 0, num - 1, (int64_t)splits[e].y);
}

// Split (i, d - i) of diagonal d: the smallest i in [max(0, d-N), min(d, R)]
// with i == min(d, R) or rp[i+1] > d-i-1 (a row end precedes the atom with the
// same index).
__device__ __forceinline__ int2 merge_split(const int32_t* __restrict__ rp, int32_t R, int64_t N, int64_t d) {
  int64_t lo = d - N > 0 ? d - N : 0;
  int64_t hi = d < R ? d : R;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if ((int64_t)__ldg(rp + mid + 1) > d - mid - 1) hi = mid;
    else lo = mid + 1;
  }
  return make_int2((int)lo, (int)(d - lo));
}

// Diagonal of the last merge-path point whose cost wr * i + j (i row ends, j
// atoms) does not exceed W: i is the largest row count with wr * i + rp[i] <= W,
// and j runs on through row i's atoms as far as W allows.
__device__ __forceinline__ int64_t weighted_point(const int32_t* __restrict__ rp, int32_t R, int64_t N, int64_t wr,
                                                  int64_t W) {
  int64_t lo = 0, hi = R;
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) >> 1;
    if (wr * mid + (int64_t)__ldg(rp + mid) <= W) lo = mid;
    else hi = mid - 1;
  }
  const int64_t jmax = lo < R ? (int64_t)__ldg(rp + lo + 1) : N;
  const int64_t j = W - wr * lo < jmax ? W - wr * lo : jmax;
  return lo + j;
}

// Splits of a table with row ends weighted wr in the shares: share c runs
// between the points of cost floor(c * T / S) and floor((c + 1) * T / S),
// T = wr * R + N, S = workers; its k-th tile starts k * items_per_tile rows +
// atoms past the share's first point (clamped to the share's end).
__global__ void mp_splits_weighted_kernel(const int32_t* __restrict__ rp, int32_t R, int64_t N, int wr, int workers,
                                          int tpc, int ipt_items, int64_t entries, int2* out, int64_t* diag) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= entries) return;
  const int64_t c = e / (tpc + 1), k = e % (tpc + 1);
  const int64_t total = (int64_t)wr * R + N;
  const int64_t b = weighted_point(rp, R, N, wr, c * total / workers);
  const int64_t en = weighted_point(rp, R, N, wr, (c + 1) * total / workers);
  const int64_t d0 = b + k * (int64_t)ipt_items;
  const int64_t d = d0 < en ? d0 : en;
  out[e] = merge_split(rp, R, N, d);
  diag[e] = d;
}

// Carry row of every work unit of a warp-worker table: the row open at the
// end of the unit's last share (its 8th warp's), -1 where none may be named
// (the end of a wave, or of the tile set).
__global__ void unit_carry_rows_kernel(const int2* __restrict__ splits, const lbk::WaveDesc* __restrict__ waves,
                                       int num_waves, int workers, int tpc, int32_t R, int32_t* out) {
  const int upw = workers / 8;
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= num_waves * upw) return;
  const int v = u / upw, k = u - v * upw;
  int64_t ebase = 0;
  int t = tpc;
  int32_t row_end = R;
  if (waves) {
    ebase = waves[v].entry_base;
    t = waves[v].tpc;
    row_end = waves[v].row_end;
  }
  const int2 e = splits[ebase + (int64_t)(k * 8 + 7) * (t + 1) + t];
  out[u] = e.x < row_end ? e.x : -1;
}

__global__ void mp_splits_at_kernel(const int32_t* __restrict__ rp, int32_t R, int64_t N,
                                    const int64_t* __restrict__ diag, int64_t entries, int2* out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < entries) out[e] = merge_split(rp, R, N, diag[e]);
}

// first two split entries of every share (one load for a warp that opens it)
__global__ void share_heads_kernel(const int2* __restrict__ splits, const int64_t* __restrict__ share_ent, int S,
                                   int4* head) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= S) return;
  const int64_t b = share_ent[q];
  const int2 c0 = splits[b];
  const int2 c1 = share_ent[q + 1] - b > 1 ? splits[b + 1] : c0;
  head[q] = make_int4(c0.x, c0.y, c1.x, c1.y);
}

// The look-back table (mp_variant 3): shares of whole warp tiles in merge
// order with guided sizes, each about four fifths of one warp's part of the work
// still left (rounded up to whole tiles, at most max_tiles_cap, at least
// min_tiles), so shares shrink to min_tiles towards the end and the warps,
// taking them in order, finish close together.  For batches the cap
// (kMaxShareTiles) keeps the shares in flight (warps x 8 tiles, about 10 M
// items on a 152-SM GPU) within a window of the merge path, so the batch is
// worked through in order and each matrix's vectors stay in L2 meanwhile.
constexpr int64_t kMaxShareTiles = 8;
static lb_status_t build_guided_table(MpTable& t, const int32_t* rp, int32_t R, int64_t N, int num_sms, int occ,
                                      int min_tiles, int64_t max_tiles_cap, const BatchBases* batch, cudaStream_t s) {
  constexpr int kWarps = kBlock / 32;
  const int64_t tile = t.items_per_tile;
  int64_t ctas = (t.items + kWarps * tile - 1) / (kWarps * tile);
  ctas = std::max<int64_t>(1, std::min<int64_t>(ctas, (int64_t)num_sms * occ));
  t.grid = (int)ctas;
  const int64_t P = ctas * kWarps;
  const int64_t mt = std::max(1, min_tiles);
  std::vector<int64_t> ent{0}, diag;
  int64_t d = 0, max_tiles = 1;
  while (d < t.items) {
    const int64_t rem = t.items - d;
    // 4/5 of a warp's part of what is left: most of the work goes in the first round of shares (fewer
    // shares, less look-back), the tail in ever smaller ones (single matrices: power-law IPT 4
    // 104 -> 97 us, R-MAT 249 -> 247 us against half of a warp's part; batches, capped, unchanged)
    int64_t tiles = std::min(max_tiles_cap, (4 * rem + 5 * P * tile - 1) / (5 * P * tile));
    tiles = std::max(mt, tiles);
    const int64_t len = std::min(rem, tiles * tile);
    tiles = (len + tile - 1) / tile;
    for (int64_t k = 0; k < tiles; ++k) diag.push_back(d + k * tile);
    d += len;
    diag.push_back(d);
    ent.push_back(ent.back() + tiles + 1);
    max_tiles = std::max(max_tiles, tiles);
  }
  if (diag.empty()) {  // no rows and no atoms: one empty share
    diag = {0, 0};
    ent.push_back(2);
  }
  const int64_t S = (int64_t)ent.size() - 1;
  if ((int64_t)diag.size() >= ((int64_t)1 << 31)) {  // the kernel indexes split entries with int
    set_error("merge-path: too many look-back split entries");
    return LB_ERR_UNSUPPORTED;
  }
  t.workers = (int)S;
  t.tiles_per_cta = (int)max_tiles;
  t.entries = (int64_t)diag.size();
  t.num_waves = 1;
  LB_CUDA_TRY(cudaMalloc(&t.splits, sizeof(int2) * (size_t)t.entries));
  LB_CUDA_TRY(cudaMalloc(&t.d_diag, sizeof(int64_t) * (size_t)t.entries));
  LB_CUDA_TRY(cudaMalloc(&t.share_ent, sizeof(int64_t) * (size_t)(S + 1)));
  LB_CUDA_TRY(cudaMalloc(&t.share_head, sizeof(int4) * (size_t)S));
  LB_CUDA_TRY(cudaMalloc(&t.records, sizeof(unsigned long long) * (size_t)S));
  LB_CUDA_TRY(cudaMalloc(&t.ticket, sizeof(unsigned) * 4));
  LB_CUDA_TRY(cudaMemcpyAsync(t.d_diag, diag.data(), sizeof(int64_t) * diag.size(), cudaMemcpyHostToDevice, s));
  LB_CUDA_TRY(cudaMemcpyAsync(t.share_ent, ent.data(), sizeof(int64_t) * ent.size(), cudaMemcpyHostToDevice, s));
  LB_CUDA_TRY(cudaMemsetAsync(t.records, 0, sizeof(unsigned long long) * (size_t)S, s));
  // ticket, counter, epoch (records hold (epoch << 1) | FINAL; 0 = never published), spare
  const unsigned init[4] = {0u, 0u, 1u, 0u};
  LB_CUDA_TRY(cudaMemcpyAsync(t.ticket, init, sizeof(init), cudaMemcpyHostToDevice, s));
  const unsigned eb = (unsigned)((t.entries + 255) / 256);
  mp_splits_at_kernel<<<eb, 256, 0, s>>>(rp, R, N, t.d_diag, t.entries, t.splits);
  LB_CUDA_TRY(cudaGetLastError());
  share_heads_kernel<<<(unsigned)((S + 255) / 256), 256, 0, s>>>(t.splits, t.share_ent, (int)S, t.share_head);
  LB_CUDA_TRY(cudaGetLastError());
  if (batch) {
    LB_CUDA_TRY(cudaMalloc(&t.split_m, sizeof(int32_t) * (size_t)t.entries));
    split_matrix_kernel<<<eb, 256, 0, s>>>(t.splits, t.entries, batch->nnz_base, batch->num, t.split_m);
    LB_CUDA_TRY(cudaGetLastError());
  }
  // the expand kernels take the same shares dynamically with their own occupancy
  int occ_e = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_e, kernel_expand_warp(t.ipt, true, true), kBlock, 0) !=
          cudaSuccess || occ_e < 1)
    occ_e = occ;
  t.expand_grid = (int)std::max<int64_t>(1, std::min<int64_t>((S + kWarps - 1) / kWarps, (int64_t)num_sms * occ_e));
  // the host vectors must outlive the copies
  LB_CUDA_TRY(cudaStreamSynchronize(s));
  t.built = true;
  return LB_OK;
}

// Runs of a warp-worker table (variant 0): consecutive work units whose
// carries name the same row r, followed by the unit that closes r (the unit
// after a maximal run never carries r itself, so it holds r's end).  Each unit
// is a member of at most one run and closes at most one.  Synchronises s.
static lb_status_t build_runs(MpTable& t, int32_t R, cudaStream_t s) {
  const int upw = t.workers / 8;
  const int64_t nunits = (int64_t)upw * t.num_waves;
  if (nunits < 1) return LB_OK;
  int32_t* d_rows = nullptr;
  LB_CUDA_TRY(cudaMalloc(&d_rows, sizeof(int32_t) * (size_t)nunits));
  unit_carry_rows_kernel<<<(unsigned)((nunits + 255) / 256), 256, 0, s>>>(
      t.splits, t.num_waves > 1 ? static_cast<const lbk::WaveDesc*>(t.d_waves) : nullptr, t.num_waves, t.workers,
      t.tiles_per_cta, R, d_rows);
  std::vector<int32_t> rows((size_t)nunits);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(rows.data(), d_rows, sizeof(int32_t) * rows.size(), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(d_rows);
  LB_CUDA_TRY(e);
  std::vector<int2> unit_runs((size_t)nunits, make_int2(-1, -1));
  std::vector<int4> runs;
  for (int64_t u = 0; u < nunits;) {
    if (rows[u] < 0) {
      ++u;
      continue;
    }
    int64_t b = u;
    while (b + 1 < nunits && rows[b + 1] == rows[u]) ++b;
    if (b + 1 >= nunits) {
      set_error("merge-path: a carry run without a closing unit");
      return LB_ERR_CUDA;
    }
    const int r = (int)runs.size();
    runs.push_back(make_int4((int)u, (int)b, rows[u], (int)(b - u + 2)));
    for (int64_t q = u; q <= b; ++q) unit_runs[q].x = r;
    unit_runs[b + 1].y = r;
    u = b + 1;
  }
  LB_CUDA_TRY(cudaMalloc(&t.unit_runs, sizeof(int2) * unit_runs.size()));
  LB_CUDA_TRY(cudaMalloc(&t.runs, sizeof(int4) * std::max<size_t>(1, runs.size())));
  LB_CUDA_TRY(cudaMalloc(&t.run_cnt, sizeof(unsigned) * std::max<size_t>(1, runs.size())));
  LB_CUDA_TRY(cudaMemcpyAsync(t.unit_runs, unit_runs.data(), sizeof(int2) * unit_runs.size(), cudaMemcpyHostToDevice, s));
  if (!runs.empty())
    LB_CUDA_TRY(cudaMemcpyAsync(t.runs, runs.data(), sizeof(int4) * runs.size(), cudaMemcpyHostToDevice, s));
  LB_CUDA_TRY(cudaMemsetAsync(t.run_cnt, 0, sizeof(unsigned) * std::max<size_t>(1, runs.size()), s));
  LB_CUDA_TRY(cudaStreamSynchronize(s));  // the host vectors must outlive the copies
  t.num_runs = (int)runs.size();
  return LB_OK;
}

lb_status_t build_mp_table(MpTable& t, const int32_t* rp, int32_t R, int64_t N, int ipt, int variant, int num_sms,
                           int ctas_per_sm, const BatchBases* batch, cudaStream_t s, const int64_t* item_prefix,
                           const int64_t* row_prefix, int num_mats, int wave_items, int units_per_cta,
                           int tiles_per_share, int row_weight) {
  t.release();
  t.row_weight = 1;
  if (!kernel_tma(ipt, false, false)) {
    set_error("items_per_thread must be 4, 8 or 16");
    return LB_ERR_UNSUPPORTED;
  }
  if (variant < 0 || variant > 3) {
    set_error("mp_variant must be 0, 1, 2 or 3");
    return LB_ERR_UNSUPPORTED;
  }
  t.ipt = ipt;
  t.variant = variant;
  t.items = (int64_t)R + N;
  t.num_tiles = R;
  const int occ = ctas_per_sm > 0 ? ctas_per_sm : occupancy_mp(ipt, variant);
  if (variant == 0) {
    // warps are the workers: 8 per CTA, at least 32 items (one per lane) each on average
    constexpr int kWarps = kBlock / 32;
    t.items_per_tile = 32 * ipt - 4;
    int64_t ctas = (t.items + kBlock - 1) / kBlock;
    if (ctas > (int64_t)num_sms * occ) ctas = (int64_t)num_sms * occ;
    if (ctas < 1) ctas = 1;
    t.grid = (int)ctas;
    // units_per_cta work units of 8 warp shares per CTA, never fewer than 32
    // items per warp share on average
    int64_t units = (int64_t)t.grid * std::max(1, units_per_cta);
    const int64_t max_units = std::max<int64_t>(t.grid, t.items / (32 * kWarps));
    if (units > max_units) units = max_units;
    t.workers = (int)(units * kWarps);
    // row ends weighted in the shares (single-matrix tables of variant 0 only): a share holds at most
    // its weighted size plus one row end's weight in rows + atoms
    if (variant == 0 && row_weight > 1 && !(item_prefix && row_prefix && num_mats > 1)) t.row_weight = row_weight;
    const int64_t share = t.row_weight > 1
                              ? ((int64_t)t.row_weight * R + N + t.workers - 1) / t.workers + t.row_weight
                              : (t.items + t.workers - 1) / t.workers;
    int64_t tpc = (share + t.items_per_tile - 1) / t.items_per_tile;
    t.tiles_per_cta = (int)(tpc < 1 ? 1 : tpc);
  } else if (variant == 3) {
    t.items_per_tile = 32 * ipt - 4;
    // shares capped in batches only: a single matrix's dense vector stays in
    // L2 however far apart the shares in flight are
    return build_guided_table(t, rp, R, N, num_sms, occ, tiles_per_share, num_mats > 1 ? kMaxShareTiles : 1 << 20,
                              batch, s);
  } else {
    // 4 items short of the CTA's thread slots: a tile's atoms start up to 3
    // slots into their 16-byte aligned window, and all of them must still fall
    // inside the BLOCK * IPT slots the threads cover
    t.items_per_tile = kBlock * ipt - 4;
    mp_geometry(t.items, num_sms * occ, t.items_per_tile, kBlock, &t.grid, &t.tiles_per_cta);
    t.workers = t.grid;
  }
  t.entries = (int64_t)t.workers * (t.tiles_per_cta + 1);
  // waves: runs of whole matrices, each big enough to give every worker a few
  // tiles, so that the whole GPU works on about one wave at a time and the
  // wave's dense vector stays in L2
  std::vector<int64_t> wave_begin, wave_rows;  // diagonal and first row of every wave boundary
  std::vector<lbk::WaveDesc> wd;
  if (variant == 0 && item_prefix && row_prefix && num_mats > 1) {
    const int64_t min_items =
        wave_items > 0 ? (int64_t)wave_items
                       : std::max<int64_t>((int64_t)4 << 20, (int64_t)t.grid * (kBlock / 32) * t.items_per_tile * 2);
    wave_begin.push_back(0);
    wave_rows.push_back(0);
    for (int m = 1; m < num_mats; ++m) {
      if (item_prefix[m] - wave_begin.back() >= min_items) {
        wave_begin.push_back(item_prefix[m]);
        wave_rows.push_back(row_prefix[m]);
      }
    }
    // a short last wave joins the one before it
    if (wave_begin.size() > 1 && t.items - wave_begin.back() < min_items / 2) {
      wave_begin.pop_back();
      wave_rows.pop_back();
    }
    wave_begin.push_back(t.items);
    wave_rows.push_back(R);
  }
  const int nw = wave_begin.size() > 2 ? (int)wave_begin.size() - 1 : 1;
  t.num_waves = nw;
  if (nw > 1) {
    int64_t base = 0;
    int max_tpc = 1;
    for (int v = 0; v < nw; ++v) {
      const int64_t iv = wave_begin[v + 1] - wave_begin[v];
      const int64_t share = (iv + t.workers - 1) / t.workers;
      int64_t tpc = (share + t.items_per_tile - 1) / t.items_per_tile;
      if (tpc < 1) tpc = 1;
      wd.push_back(lbk::WaveDesc{base, (int32_t)tpc, (int32_t)wave_rows[v + 1]});
      base += (int64_t)t.workers * (tpc + 1);
      max_tpc = std::max(max_tpc, (int)tpc);
    }
    t.entries = base;
    t.tiles_per_cta = max_tpc;
  }
  LB_CUDA_TRY(cudaMalloc(&t.splits, sizeof(int2) * (size_t)t.entries));
  LB_CUDA_TRY(cudaMalloc(&t.d_diag, sizeof(int64_t) * (size_t)t.entries));
  LB_CUDA_TRY(cudaMalloc(&t.carry_val, sizeof(float) * (size_t)t.workers * nw));
  LB_CUDA_TRY(cudaMalloc(&t.carry_row, sizeof(int32_t) * (size_t)t.workers * nw));
  LB_CUDA_TRY(cudaMalloc(&t.ticket, sizeof(unsigned) * 4));
  LB_CUDA_TRY(cudaMemsetAsync(t.ticket, 0, sizeof(unsigned) * 4, s));
  const int threads = 256;
  const unsigned blocks = (unsigned)((t.entries + threads - 1) / threads);
  if (nw > 1) {
    int64_t* d_begin = nullptr;
    LB_CUDA_TRY(cudaMalloc(&t.d_waves, sizeof(lbk::WaveDesc) * nw));
    LB_CUDA_TRY(cudaMalloc(&d_begin, sizeof(int64_t) * (nw + 1)));
    LB_CUDA_TRY(cudaMemcpyAsync(t.d_waves, wd.data(), sizeof(lbk::WaveDesc) * nw, cudaMemcpyHostToDevice, s));
    LB_CUDA_TRY(cudaMemcpyAsync(d_begin, wave_begin.data(), sizeof(int64_t) * (nw + 1), cudaMemcpyHostToDevice, s));
    mp_splits_waves_kernel<<<blocks, threads, 0, s>>>(rp, R, N, d_begin, static_cast<lbk::WaveDesc*>(t.d_waves),
                                                      nw, t.workers, t.items_per_tile, t.entries, t.splits,
                                                      t.d_diag);
    const cudaError_t e = cudaGetLastError();
    cudaStreamSynchronize(s);
    cudaFree(d_begin);
    LB_CUDA_TRY(e);
  } else if (t.row_weight > 1) {
    mp_splits_weighted_kernel<<<blocks, threads, 0, s>>>(rp, R, N, t.row_weight, t.workers, t.tiles_per_cta,
                                                         t.items_per_tile, t.entries, t.splits, t.d_diag);
    LB_CUDA_TRY(cudaGetLastError());
  } else {
    mp_splits_kernel<<<blocks, threads, 0, s>>>(rp, R, N, t.items, t.workers, t.tiles_per_cta, t.items_per_tile,
                                                t.entries, t.splits, t.d_diag);
    LB_CUDA_TRY(cudaGetLastError());
  }
  if (batch) {
    LB_CUDA_TRY(cudaMalloc(&t.split_m, sizeof(int32_t) * (size_t)t.entries));
    split_matrix_kernel<<<blocks, threads, 0, s>>>(t.splits, t.entries, batch->nnz_base, batch->num, t.split_m);
    LB_CUDA_TRY(cudaGetLastError());
  }
  // runs for tables of one static unit per CTA; with dynamic units (several per CTA, or waves) the
  // per-unit fences and counts cost more than the single fix-up pass of the last CTA (measured on
  // the power-law matrix with 8 units per CTA: 123 -> 135 us)
  if (variant == 0 && t.num_waves == 1 && t.workers / 8 == t.grid) LB_TRY(build_runs(t, R, s));
  t.built = true;
  return LB_OK;
}

// ----------------------------------------------------------------- launches --

static bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

static lbk::MpArgs make_args(const MpTable& t, const SpmvCall& c) {
  lbk::MpArgs a{};
  a.rp = c.rp;
  a.atoms = lbk::AtomView{c.idx, c.val, c.perm, c.vec, c.check, c.status};
  a.out = c.out;
  a.splits = t.splits;
  a.split_m = c.batch ? t.split_m : nullptr;
  a.nnz_base = c.batch ? c.batch->nnz_base : nullptr;
  a.vec_base = c.batch ? c.batch->vec_base : nullptr;
  a.tiles_per_cta = t.tiles_per_cta;
  a.num_ctas = t.grid;
  a.num_workers = t.workers;
  a.items_per_tile = t.items_per_tile;
  a.num_tiles = t.num_tiles;
  a.num_atoms = t.items - t.num_tiles;
  a.carry_val = t.carry_val;
  a.carry_row = t.carry_row;
  a.ticket = t.ticket;
  a.num_entries = (int32_t)t.entries;
  a.share_ent = t.share_ent;
  a.share_head = t.share_head;
  a.records = t.records;
  a.waves = static_cast<const lbk::WaveDesc*>(t.d_waves);
  a.num_waves = t.num_waves;
  a.status = c.status;
  a.unit_runs = t.unit_runs;
  a.runs = t.unit_runs ? t.runs : nullptr;
  a.run_cnt = t.run_cnt;
  return a;
}

lb_status_t launch_mp_spmv(const MpTable& t, const SpmvCall& c, cudaStream_t s) {
  if (!t.built) {
    set_error("merge-path table not built");
    return LB_ERR_INVALID_ARG;
  }
  if (t.items == 0) return LB_OK;
  if (c.batch && !t.split_m) {
    set_error("batched launch on a table without matrix indices");
    return LB_ERR_INVALID_ARG;
  }
  if (t.num_waves > 1 && !c.batch && !c.perm) {  // the forward kernels walk waves only when batched
    set_error("a table in waves needs a batched or transposed launch");
    return LB_ERR_INVALID_ARG;
  }
  lbk::MpArgs a = make_args(t, c);
  const bool xb = c.batch != nullptr;
  const bool perm = c.perm != nullptr;
  const bool vec_atoms = aligned16(c.idx) && (perm ? aligned16(c.perm) : aligned16(c.val));
  cudaError_t e;
  if (t.variant == 0) {
    e = launch(kernel_warp(t.ipt, xb, perm, vec_atoms), t.grid, 0, s, &a);
  } else if (t.variant == 3) {
    e = launch(kernel_lookback(t.ipt, xb, perm, vec_atoms), t.grid, 0, s, &a);
  } else if (t.variant == 2 && vec_atoms && aligned16(c.rp)) {
    e = launch(kernel_tma(t.ipt, xb, perm), t.grid, tma_smem(t.ipt), s, &a);
  } else {
    e = launch(kernel_plain(t.ipt, xb), t.grid, plain_smem(t.ipt), s, &a);
  }
  LB_CUDA_TRY(e);
  return LB_OK;
}

lb_status_t launch_mp_expand(const MpTable& t, const SpmvCall& c, const float* dy, float* dvals,
                             int32_t* tile_of_atom, cudaStream_t s) {
  if (!t.built) {
    set_error("merge-path table not built");
    return LB_ERR_INVALID_ARG;
  }
  if (t.items == 0) return LB_OK;
  lbk::MpArgs a = make_args(t, c);
  a.dy = dy;
  a.dvals = dvals;
  a.tile_of_atom = tile_of_atom;
  const bool xb = c.batch != nullptr && dvals != nullptr;
  if (t.variant == 3) {
    a.num_ctas = t.expand_grid;
    LB_CUDA_TRY(launch(kernel_expand_warp(t.ipt, xb, dvals != nullptr), t.expand_grid, 0, s, &a));
  } else if (warp_workers(t.variant))
    LB_CUDA_TRY(launch(kernel_expand_warp(t.ipt, xb, dvals != nullptr), t.grid, 0, s, &a));
  else
    LB_CUDA_TRY(launch(kernel_expand(t.ipt, xb, dvals != nullptr), t.grid, expand_smem(t.ipt), s, &a));
  return LB_OK;
}

constexpr int kStagedCap = 864;  // atoms a warp's 32 tiles may hold to be staged in shared memory (27 x 32)

// one wave of CTAs of the staged thread-mapped kernel (queried once per plan)
int tm_staged_grid(int num_sms) {
  int o = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, lbk::tm_staged_spmv_kernel<kStagedCap>, kBlock, 0) !=
          cudaSuccess ||
      o < 1)
    o = 1;
  return num_sms * o;
}

lb_status_t launch_tm_staged_spmv(const SpmvCall& c, int grid, cudaStream_t s) {
  if (c.num_tiles == 0) return LB_OK;
  // one warp per 32 tiles, grid-stride over the groups
  const int64_t groups = ((int64_t)c.num_tiles + 31) / 32;
  int64_t blocks = (groups + 7) / 8;
  if (blocks > grid) blocks = grid;
  if (blocks < 1) blocks = 1;
  lbk::tm_staged_spmv_kernel<kStagedCap><<<(unsigned)blocks, kBlock, 0, s>>>(
      c.rp, c.num_tiles, lbk::AtomView{c.idx, c.val, c.perm, c.vec, c.check, c.status}, c.out);
  LB_CUDA_TRY(cudaGetLastError());
  return LB_OK;
}

lb_status_t launch_tm_spmv(const SpmvCall& c, cudaStream_t s) {
  if (c.num_tiles == 0) return LB_OK;
  // Listing 3 launches ceil(rows / 256) blocks of 256 threads
  const int64_t blocks = ((int64_t)c.num_tiles + kBlock - 1) / kBlock;
  lbk::tm_spmv_kernel<kBlock><<<(unsigned)blocks, kBlock, 0, s>>>(
      c.rp, c.num_tiles, lbk::AtomView{c.idx, c.val, c.perm, c.vec, c.check, c.status}, c.out);
  LB_CUDA_TRY(cudaGetLastError());
  return LB_OK;
}

template <int G>
static void gm_launch(int64_t blocks, const SpmvCall& c, cudaStream_t s) {
  lbk::gm_spmv_kernel<kBlock, G><<<(unsigned)blocks, kBlock, 0, s>>>(
      c.rp, c.num_tiles, lbk::AtomView{c.idx, c.val, c.perm, c.vec, c.check, c.status}, c.out);
}

lb_status_t launch_gm_spmv(int group, const SpmvCall& c, int num_sms, cudaStream_t s) {
  if (c.num_tiles == 0) return LB_OK;
  // one chunk of `group` tiles per group, kBlock / group groups per block;
  // oversubscribed grid capped at 64 blocks per SM, grid-stride beyond that
  int64_t blocks = ((int64_t)c.num_tiles + kBlock - 1) / kBlock;
  const int64_t cap = (int64_t)num_sms * 64;
  if (blocks > cap) blocks = cap;
  switch (group) {
    case 4: gm_launch<4>(blocks, c, s); break;
    case 8: gm_launch<8>(blocks, c, s); break;
    case 16: gm_launch<16>(blocks, c, s); break;
    case 32: gm_launch<32>(blocks, c, s); break;
    case 64: gm_launch<64>(blocks, c, s); break;
    case 128: gm_launch<128>(blocks, c, s); break;
    case 256: gm_launch<256>(blocks, c, s); break;
    default:
      set_error("group size must be a power of two in [4, 256]");
      return LB_ERR_UNSUPPORTED;
  }
  LB_CUDA_TRY(cudaGetLastError());
  return LB_OK;
}

}  // namespace lbh
