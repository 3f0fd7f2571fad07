// Merge-path tables and kernel launches for single and batched tile sets,
// plus the thread-mapped and group-mapped launchers.
#include <algorithm>
#include <vector>

#include "lb_internal.h"
#include "lb_kernels.cuh"

namespace lbh {

void MpTable::release() {
  cudaFree(splits);
  cudaFree(d_diag);
  cudaFree(carry_val);
  cudaFree(carry_row);
  cudaFree(ticket);
  splits = nullptr;
  d_diag = nullptr;
  carry_val = nullptr;
  carry_row = nullptr;
  ticket = nullptr;
  built = false;
}

void BatchSet::release() {
  if (owns_rp) cudaFree(const_cast<int32_t*>(rp_cat));
  cudaFree(row_base);
  cudaFree(nnz_base);
  cudaFree(vec_base);
  cudaFree(diag_base);
  rp_cat = nullptr;
  row_base = nnz_base = vec_base = diag_base = nullptr;
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

template <int IPT, bool BATCH, bool VEC>
static cudaError_t set_mp_smem() {
  return cudaFuncSetAttribute(lbk::mp_spmv_kernel<kBlock, IPT, BATCH, VEC>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)lbk::mp_smem_bytes<kBlock, IPT>());
}

int occupancy_mp(int ipt, bool batch) {
  int occ = 0;
  cudaError_t e = cudaSuccess;
#define OCC_CASE(I)                                                                                   \
  case I:                                                                                             \
    if (batch) {                                                                                      \
      set_mp_smem<I, true, true>();                                                                   \
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, lbk::mp_spmv_kernel<kBlock, I, true, true>, \
                                                        kBlock, lbk::mp_smem_bytes<kBlock, I>());     \
    } else {                                                                                          \
      set_mp_smem<I, false, true>();                                                                  \
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, lbk::mp_spmv_kernel<kBlock, I, false, true>, \
                                                        kBlock, lbk::mp_smem_bytes<kBlock, I>());     \
    }                                                                                                 \
    break;
  switch (ipt) {
    OCC_CASE(4)
    OCC_CASE(8)
    OCC_CASE(16)
    default:
      break;
  }
#undef OCC_CASE
  if (e != cudaSuccess || occ < 1) occ = 1;
  return occ;
}

// ------------------------------------------------------------ split kernels --

__global__ void mp_splits_single_kernel(const int32_t* __restrict__ rp, int32_t R, int64_t N, int64_t items, int grid,
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
  diag[e] = d;
}

__global__ void mp_splits_batch_kernel(const int32_t* __restrict__ rp_cat, const int64_t* __restrict__ row_base,
                                       const int64_t* __restrict__ nnz_base, const int64_t* __restrict__ diag_base,
                                       int num, int64_t items, int grid, int tpc, int ipt_items, int64_t entries,
                                       lbk::Split64* out, int64_t* diag) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= entries) return;
  const int64_t d = mp_diag(items, grid, tpc, ipt_items, e);
  // matrix: largest m in [0, num-1] with diag_base[m] <= d
  int lo_m = 0, hi_m = num - 1;
  while (lo_m < hi_m) {
    const int mid = (lo_m + hi_m + 1) >> 1;
    if (diag_base[mid] <= d) lo_m = mid;
    else hi_m = mid - 1;
  }
  const int m = lo_m;
  const int64_t R = row_base[m + 1] - row_base[m];
  const int64_t N = nnz_base[m + 1] - nnz_base[m];
  const int64_t dl = d - diag_base[m];
  const int32_t* rp = rp_cat + row_base[m] + m;
  int64_t lo = dl - N > 0 ? dl - N : 0;
  int64_t hi = dl < R ? dl : R;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if ((int64_t)__ldg(rp + mid + 1) > dl - mid - 1) hi = mid;
    else lo = mid + 1;
  }
  lbk::Split64 s;
  s.i = row_base[m] + lo;
  s.j = nnz_base[m] + (dl - lo);
  s.m = m;
  s.pad = 0;
  out[e] = s;
  diag[e] = d;
}

static lb_status_t alloc_table(MpTable& t, size_t split_bytes) {
  LB_CUDA_TRY(cudaMalloc(&t.splits, split_bytes * (size_t)t.entries));
  LB_CUDA_TRY(cudaMalloc(&t.d_diag, sizeof(int64_t) * (size_t)t.entries));
  LB_CUDA_TRY(cudaMalloc(&t.carry_val, sizeof(float) * (size_t)t.grid));
  LB_CUDA_TRY(cudaMalloc(&t.carry_row, sizeof(int64_t) * (size_t)t.grid));
  LB_CUDA_TRY(cudaMalloc(&t.ticket, sizeof(unsigned)));
  LB_CUDA_TRY(cudaMemset(t.ticket, 0, sizeof(unsigned)));
  return LB_OK;
}

lb_status_t build_mp_table_single(MpTable& t, const int32_t* rp, int32_t R, int64_t N, int ipt, int num_sms,
                                  int ctas_per_sm, cudaStream_t s) {
  t.release();
  t.batch = false;
  t.ipt = ipt;
  t.items_per_tile = kBlock * ipt;
  t.items = (int64_t)R + N;
  const int occ = ctas_per_sm > 0 ? ctas_per_sm : occupancy_mp(ipt, false);
  mp_geometry(t.items, num_sms * occ, t.items_per_tile, kBlock, &t.grid, &t.tiles_per_cta);
  t.entries = (int64_t)t.grid * (t.tiles_per_cta + 1);
  LB_TRY(alloc_table(t, sizeof(int2)));
  const int threads = 256;
  const int64_t blocks = (t.entries + threads - 1) / threads;
  mp_splits_single_kernel<<<(unsigned)blocks, threads, 0, s>>>(rp, R, N, t.items, t.grid, t.tiles_per_cta,
                                                              t.items_per_tile, t.entries,
                                                              reinterpret_cast<int2*>(t.splits), t.d_diag);
  LB_CUDA_TRY(cudaGetLastError());
  t.built = true;
  return LB_OK;
}

lb_status_t build_mp_table_batch(MpTable& t, const BatchSet& b, int ipt, int num_sms, int ctas_per_sm,
                                 cudaStream_t s) {
  t.release();
  t.batch = true;
  t.ipt = ipt;
  t.items_per_tile = kBlock * ipt;
  t.items = b.total_rows + b.total_nnz;
  const int occ = ctas_per_sm > 0 ? ctas_per_sm : occupancy_mp(ipt, true);
  mp_geometry(t.items, num_sms * occ, t.items_per_tile, kBlock, &t.grid, &t.tiles_per_cta);
  t.entries = (int64_t)t.grid * (t.tiles_per_cta + 1);
  LB_TRY(alloc_table(t, sizeof(lbk::Split64)));
  const int threads = 256;
  const int64_t blocks = (t.entries + threads - 1) / threads;
  mp_splits_batch_kernel<<<(unsigned)blocks, threads, 0, s>>>(
      b.rp_cat, b.row_base, b.nnz_base, b.diag_base, b.num, t.items, t.grid, t.tiles_per_cta, t.items_per_tile,
      t.entries, reinterpret_cast<lbk::Split64*>(t.splits), t.d_diag);
  LB_CUDA_TRY(cudaGetLastError());
  t.built = true;
  return LB_OK;
}

// ----------------------------------------------------------------- launches --

static lbk::MpArgs make_args(const MpTable& t, const int32_t* rp, const BatchSet* b, int64_t num_tiles) {
  lbk::MpArgs a{};
  a.rp = b ? b->rp_cat : rp;
  a.row_base = b ? b->row_base : nullptr;
  a.nnz_base = b ? b->nnz_base : nullptr;
  a.vec_base = b ? b->vec_base : nullptr;
  a.splits = t.splits;
  a.tiles_per_cta = t.tiles_per_cta;
  a.num_ctas = t.grid;
  a.num_tiles = num_tiles;
  a.carry_val = t.carry_val;
  a.carry_row = t.carry_row;
  a.ticket = t.ticket;
  return a;
}

static bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

template <int IPT, bool BATCH, bool VEC>
static void mp_launch(const lbk::MpArgs& a, cudaStream_t s) {
  lbk::mp_spmv_kernel<kBlock, IPT, BATCH, VEC>
      <<<a.num_ctas, kBlock, lbk::mp_smem_bytes<kBlock, IPT>(), s>>>(a);
}

template <int IPT, bool BATCH>
static void mp_launch_v(const lbk::MpArgs& a, bool vec, cudaStream_t s) {
  static bool attr_set[2] = {false, false};
  if (!attr_set[vec]) {
    if (vec) set_mp_smem<IPT, BATCH, true>();
    else set_mp_smem<IPT, BATCH, false>();
    attr_set[vec] = true;
  }
  if (vec) mp_launch<IPT, BATCH, true>(a, s);
  else mp_launch<IPT, BATCH, false>(a, s);
}

lb_status_t launch_mp_spmv(const MpTable& t, const int32_t* rp, const BatchSet* b, const int32_t* idx,
                           const float* val, const int32_t* perm, const float* vec, float* out, int64_t num_tiles,
                           int32_t check_cols, int* status, cudaStream_t s) {
  if (!t.built) {
    set_error("merge-path table not built");
    return LB_ERR_INVALID_ARG;
  }
  if (t.items == 0) return LB_OK;
  lbk::MpArgs a = make_args(t, rp, b, num_tiles);
  a.atoms = lbk::AtomView{idx, val, perm, vec, check_cols, status};
  a.out = out;
  const bool v = aligned16(idx) && (perm ? aligned16(perm) : aligned16(val));
  const bool batch = b != nullptr;
  switch (t.ipt) {
    case 4:
      batch ? mp_launch_v<4, true>(a, v, s) : mp_launch_v<4, false>(a, v, s);
      break;
    case 8:
      batch ? mp_launch_v<8, true>(a, v, s) : mp_launch_v<8, false>(a, v, s);
      break;
    case 16:
      batch ? mp_launch_v<16, true>(a, v, s) : mp_launch_v<16, false>(a, v, s);
      break;
    default:
      set_error("items_per_thread must be 4, 8 or 16");
      return LB_ERR_UNSUPPORTED;
  }
  LB_CUDA_TRY(cudaGetLastError());
  return LB_OK;
}

template <int IPT, bool BATCH, bool DV>
static void ex_launch(const lbk::MpArgs& a, cudaStream_t s) {
  const size_t smem = sizeof(int) * 2 * kBlock * IPT;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(lbk::mp_expand_kernel<kBlock, IPT, BATCH, DV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    attr = true;
  }
  lbk::mp_expand_kernel<kBlock, IPT, BATCH, DV><<<a.num_ctas, kBlock, smem, s>>>(a);
}

template <int IPT>
static void ex_dispatch(const lbk::MpArgs& a, bool batch, bool dv, cudaStream_t s) {
  if (batch) dv ? ex_launch<IPT, true, true>(a, s) : ex_launch<IPT, true, false>(a, s);
  else dv ? ex_launch<IPT, false, true>(a, s) : ex_launch<IPT, false, false>(a, s);
}

lb_status_t launch_mp_expand(const MpTable& t, const int32_t* rp, const BatchSet* b, const int32_t* idx,
                             const float* x, const float* dy, float* dvals, int32_t* tile_of_atom,
                             int32_t check_cols, int* status, cudaStream_t s) {
  if (!t.built) {
    set_error("merge-path table not built");
    return LB_ERR_INVALID_ARG;
  }
  if (t.items == 0) return LB_OK;
  lbk::MpArgs a = make_args(t, rp, b, 0);
  a.atoms = lbk::AtomView{idx, nullptr, nullptr, x, check_cols, status};
  a.dy = dy;
  a.dvals = dvals;
  a.tile_of_atom = tile_of_atom;
  const bool dv = dvals != nullptr;
  switch (t.ipt) {
    case 4: ex_dispatch<4>(a, b != nullptr, dv, s); break;
    case 8: ex_dispatch<8>(a, b != nullptr, dv, s); break;
    case 16: ex_dispatch<16>(a, b != nullptr, dv, s); break;
    default:
      set_error("items_per_thread must be 4, 8 or 16");
      return LB_ERR_UNSUPPORTED;
  }
  LB_CUDA_TRY(cudaGetLastError());
  return LB_OK;
}

lb_status_t launch_tm_spmv(const int32_t* rp, int32_t R, const int32_t* idx, const float* val, const int32_t* perm,
                           const float* vec, float* out, int32_t check_cols, int* status, int num_sms,
                           cudaStream_t s) {
  if (R == 0) return LB_OK;
  // Listing 3 launches ceil(rows / 256) blocks of 256 threads
  const int64_t blocks = ((int64_t)R + kBlock - 1) / kBlock;
  (void)num_sms;
  lbk::tm_spmv_kernel<kBlock><<<(unsigned)blocks, kBlock, 0, s>>>(rp, R, lbk::AtomView{idx, val, perm, vec, check_cols, status}, out);
  LB_CUDA_TRY(cudaGetLastError());
  return LB_OK;
}

template <int G>
static void gm_launch(int64_t blocks, const int32_t* rp, int32_t R, const lbk::AtomView& at, float* out,
                      cudaStream_t s) {
  lbk::gm_spmv_kernel<kBlock, G><<<(unsigned)blocks, kBlock, 0, s>>>(rp, R, at, out);
}

lb_status_t launch_gm_spmv(int group, const int32_t* rp, int32_t R, const int32_t* idx, const float* val,
                           const int32_t* perm, const float* vec, float* out, int32_t check_cols, int* status,
                           int num_sms, cudaStream_t s) {
  if (R == 0) return LB_OK;
  // one chunk of `group` tiles per group, kBlock / group groups per block;
  // oversubscribed grid capped at 64 blocks per SM, grid-stride beyond that
  int64_t blocks = ((int64_t)R + kBlock - 1) / kBlock;
  const int64_t cap = (int64_t)num_sms * 64;
  if (blocks > cap) blocks = cap;
  const lbk::AtomView at{idx, val, perm, vec, check_cols, status};
  switch (group) {
    case 4: gm_launch<4>(blocks, rp, R, at, out, s); break;
    case 8: gm_launch<8>(blocks, rp, R, at, out, s); break;
    case 16: gm_launch<16>(blocks, rp, R, at, out, s); break;
    case 32: gm_launch<32>(blocks, rp, R, at, out, s); break;
    case 64: gm_launch<64>(blocks, rp, R, at, out, s); break;
    case 128: gm_launch<128>(blocks, rp, R, at, out, s); break;
    case 256: gm_launch<256>(blocks, rp, R, at, out, s); break;
    default:
      set_error("group size must be a power of two in [4, 256]");
      return LB_ERR_UNSUPPORTED;
  }
  LB_CUDA_TRY(cudaGetLastError());
  return LB_OK;
}

}  // namespace lbh
