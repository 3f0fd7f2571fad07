// C ABI: plans, single-matrix SpMV and its backward, status and host helpers.
#include <algorithm>
#include <cstring>
#include <string>

#include "lb_internal.h"

namespace lbh {

static thread_local std::string g_last_error;
void set_error(const std::string& msg) { g_last_error = msg; }

namespace {

__global__ void validate_offsets_kernel(const int32_t* __restrict__ rp, int32_t R, int64_t N, int* bad) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < R && __ldg(rp + i) > __ldg(rp + i + 1)) atomicOr(bad, 1);
  if (i == 0 && (__ldg(rp) != 0 || (int64_t)__ldg(rp + R) != N)) atomicOr(bad, 2);
}

__global__ void check_columns_kernel(const int32_t* __restrict__ ci, int64_t n, int32_t C, int* bad) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int c = __ldg(ci + i);
    if (c < 0 || c >= C) atomicOr(bad, 1);
  }
}

// Roofline probe: stream idx / vals as 16-byte vectors and gather x, nothing else.
__global__ void __launch_bounds__(256) probe_gather_kernel(const int4* __restrict__ idx, const float4* __restrict__ v,
                                                           const float* __restrict__ x, int64_t n4,
                                                           float* __restrict__ out) {
  float acc = 0.f;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += 2 * stride) {
    const int64_t k = i + stride;
    const int4 c0 = __ldcs(idx + i);
    const float4 w0 = __ldcs(v + i);
    int4 c1 = make_int4(0, 0, 0, 0);
    float4 w1 = make_float4(0.f, 0.f, 0.f, 0.f);
    if (k < n4) {
      c1 = __ldcs(idx + k);
      w1 = __ldcs(v + k);
    }
    acc += w0.x * __ldg(x + c0.x) + w0.y * __ldg(x + c0.y) + w0.z * __ldg(x + c0.z) + w0.w * __ldg(x + c0.w);
    if (k < n4)
      acc += w1.x * __ldg(x + c1.x) + w1.y * __ldg(x + c1.y) + w1.z * __ldg(x + c1.z) + w1.w * __ldg(x + c1.w);
  }
  out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

unsigned blocks_for(int64_t n, int threads, int64_t cap = 65536LL * 16) {
  int64_t b = (n + threads - 1) / threads;
  if (b > cap) b = cap;
  return (unsigned)(b < 1 ? 1 : b);
}

bool pow2_group(int g) { return g >= 4 && g <= 256 && (g & (g - 1)) == 0; }

}  // namespace

// Column indices must lie in [0, C) before the transpose's histogram uses them
// as addresses.  Returns LB_ERR_BAD_INPUT otherwise.  Synchronises s.
lb_status_t check_columns(const int32_t* ci, int64_t n, int32_t C, cudaStream_t s) {
  if (n == 0) return LB_OK;
  int* bad = nullptr;
  LB_CUDA_TRY(cudaMalloc(&bad, sizeof(int)));
  cudaMemsetAsync(bad, 0, sizeof(int), s);
  check_columns_kernel<<<blocks_for(n, 256), 256, 0, s>>>(ci, n, C, bad);
  int h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, bad, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(bad);
  if (e != cudaSuccess) {
    set_error(std::string("column check: ") + cudaGetErrorString(e));
    return LB_ERR_CUDA;
  }
  if (h) {
    set_error("column index outside [0, num_cols)");
    return LB_ERR_BAD_INPUT;
  }
  return LB_OK;
}

}  // namespace lbh

using namespace lbh;

static lb_plan_opts_t defaults(const lb_plan_opts_t* o) {
  lb_plan_opts_t d{};
  if (o) d = *o;
  if (d.items_per_thread == 0) d.items_per_thread = 8;
  if (d.group_size == 0) d.group_size = 32;
  if (d.units_per_cta == 0) d.units_per_cta = 1;
  if (d.tiles_per_share == 0) d.tiles_per_share = 1;
  if (d.items_per_thread_t == 0) d.items_per_thread_t = d.items_per_thread;
  return d;
}

static void free_transpose(lb_plan_s* p) {
  cudaFree(p->cp);
  cudaFree(p->riT);
  cudaFree(p->perm);
  p->cp = p->riT = p->perm = nullptr;
  p->mp_t.release();
  p->has_t = false;
}

extern "C" {

const char* lb_last_error(void) { return g_last_error.c_str(); }

int32_t lb_version(void) { return 10100; }

int32_t lb_probe_gather_grid(void) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  return 4 * device_sms(dev);
}

lb_status_t lb_probe_gather(const int32_t* idx, const float* vals, const float* x, int64_t n, float* out,
                            int32_t grid, void* stream) {
  if (!idx || !vals || !x || !out || n < 0 || (n & 3) || (reinterpret_cast<uintptr_t>(idx) & 15) ||
      (reinterpret_cast<uintptr_t>(vals) & 15)) {
    set_error("lb_probe_gather: need 16-byte aligned idx and vals and n % 4 == 0");
    return LB_ERR_INVALID_ARG;
  }
  if (grid <= 0) grid = lb_probe_gather_grid();
  if (grid <= 0) {
    set_error("lb_probe_gather: no device");
    return LB_ERR_CUDA;
  }
  probe_gather_kernel<<<grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(
      reinterpret_cast<const int4*>(idx), reinterpret_cast<const float4*>(vals), x, n / 4, out);
  LB_CUDA_TRY(cudaGetLastError());
  return LB_OK;
}

const char* lb_status_string(lb_status_t s) {
  switch (s) {
    case LB_OK: return "LB_OK";
    case LB_ERR_INVALID_ARG: return "LB_ERR_INVALID_ARG: invalid argument";
    case LB_ERR_CUDA: return "LB_ERR_CUDA: CUDA runtime error";
    case LB_ERR_OOM: return "LB_ERR_OOM: device allocation failed";
    case LB_ERR_UNSUPPORTED: return "LB_ERR_UNSUPPORTED: option not supported";
    case LB_ERR_TIMEOUT: return "LB_ERR_TIMEOUT: device wait timed out";
    case LB_ERR_BAD_INPUT: return "LB_ERR_BAD_INPUT: column index out of range";
  }
  return "unknown lb_status_t";
}

lb_schedule_t lb_heuristic_schedule(int32_t rows, int32_t cols, int64_t nnz) {
  // Sec. 6.2: merge-path unless (rows < alpha or cols < alpha) and nnz < beta,
  // alpha = 500, beta = 10000
  return ((rows < 500 || cols < 500) && nnz < 10000) ? LB_THREAD_MAPPED : LB_MERGE_PATH;
}

lb_status_t lb_merge_diagonals(int64_t items, int32_t grid, int32_t items_per_tile, int64_t* host_diag, size_t cap,
                               size_t* count, int32_t* tiles_per_cta) {
  if (items < 0 || grid < 1 || items_per_tile < 1) {
    set_error("lb_merge_diagonals: items >= 0, grid >= 1, items_per_tile >= 1");
    return LB_ERR_INVALID_ARG;
  }
  const int64_t share = (items + grid - 1) / grid;
  int64_t tpc = (share + items_per_tile - 1) / items_per_tile;
  if (tpc < 1) tpc = 1;
  const int64_t entries = (int64_t)grid * (tpc + 1);
  if (count) *count = (size_t)entries;
  if (tiles_per_cta) *tiles_per_cta = (int32_t)tpc;
  if (host_diag)
    for (int64_t e = 0; e < entries && (size_t)e < cap; ++e)
      host_diag[e] = mp_diagonal(items, grid, (int)tpc, items_per_tile, e);
  return LB_OK;
}

lb_status_t lb_plan_ex(lb_plan_t* out, const int32_t* tile_offsets, int32_t num_tiles, int32_t num_atoms,
                       lb_schedule_t schedule, const lb_plan_opts_t* opts, void* stream) {
  if (!out) {
    set_error("lb_plan: out is NULL");
    return LB_ERR_INVALID_ARG;
  }
  *out = nullptr;
  if (num_tiles < 0 || num_atoms < 0 || (num_tiles > 0 && !tile_offsets) || (num_tiles == 0 && num_atoms != 0)) {
    set_error("lb_plan: need num_tiles >= 0, num_atoms >= 0, tile_offsets for num_tiles > 0");
    return LB_ERR_INVALID_ARG;
  }
  if ((int)schedule < 0 || (int)schedule > (int)LB_AUTO) {
    set_error("lb_plan: unknown schedule");
    return LB_ERR_INVALID_ARG;
  }
  const lb_plan_opts_t o = defaults(opts);
  auto ipt_ok = [](int v) { return v == 4 || v == 8 || v == 16; };
  if (!ipt_ok(o.items_per_thread) || !ipt_ok(o.items_per_thread_t)) {
    set_error("lb_plan: items_per_thread and items_per_thread_t must be 4, 8 or 16");
    return LB_ERR_UNSUPPORTED;
  }
  if (o.num_cols < 0 || o.ctas_per_sm < 0) {
    set_error("lb_plan: num_cols and ctas_per_sm must be >= 0");
    return LB_ERR_INVALID_ARG;
  }
  if (o.row_weight < 0 || o.row_weight > 64) {
    set_error("lb_plan: row_weight must be in [0, 64]");
    return LB_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0;
  LB_CUDA_TRY(cudaGetDevice(&dev));
  lb_plan_s* p = new lb_plan_s();
  p->opts = o;
  p->device = dev;
  p->num_sms = device_sms(p->device);
  p->rp = tile_offsets;
  p->num_tiles = num_tiles;
  p->num_atoms = num_atoms;
  p->num_cols = o.num_cols;
  if (schedule == LB_AUTO)
    schedule = lb_heuristic_schedule(num_tiles, o.num_cols > 0 ? o.num_cols : num_tiles, num_atoms);
  p->schedule = schedule;
  p->group_size = schedule == LB_WARP_MAPPED ? 32 : schedule == LB_BLOCK_MAPPED ? kBlock : o.group_size;
  if (schedule == LB_THREAD_MAPPED && o.staged) p->tm_grid = tm_staged_grid(p->num_sms);
  if (schedule == LB_GROUP_MAPPED && !pow2_group(p->group_size)) {
    delete p;
    set_error("lb_plan: group_size must be a power of two in [4, 256]");
    return LB_ERR_UNSUPPORTED;
  }
  auto fail = [&](lb_status_t st) {
    lb_plan_destroy(p);
    return st;
  };
  cudaError_t e = cudaMalloc(&p->d_status, sizeof(int));
  if (e != cudaSuccess) {
    delete p;
    set_error(std::string("cudaMalloc: ") + cudaGetErrorString(e));
    return LB_ERR_OOM;
  }
  cudaMemsetAsync(p->d_status, 0, sizeof(int), s);
  if (o.validate && num_tiles > 0) {
    validate_offsets_kernel<<<blocks_for(num_tiles, 256, 1LL << 30), 256, 0, s>>>(tile_offsets, num_tiles,
                                                                                  num_atoms, p->d_status);
    int h = 0;
    e = cudaMemcpyAsync(&h, p->d_status, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      set_error(std::string("lb_plan validation: ") + cudaGetErrorString(e));
      return fail(LB_ERR_CUDA);
    }
    if (h) {
      set_error(h & 2 ? "lb_plan: tile_offsets[0] != 0 or tile_offsets[num_tiles] != num_atoms"
                      : "lb_plan: tile_offsets decrease");
      return fail(LB_ERR_INVALID_ARG);
    }
    cudaMemsetAsync(p->d_status, 0, sizeof(int), s);
  }
  // The forward merge-path table serves the merge-path schedule and, for every
  // schedule, the atom->tile walk used by dvals and lb_atom_tiles.
  lb_status_t st = build_mp_table(p->mp, tile_offsets, num_tiles, num_atoms, o.items_per_thread, o.mp_variant,
                                  p->num_sms, o.ctas_per_sm, nullptr, s, nullptr, nullptr, 0, 0,
                                  o.units_per_cta, o.tiles_per_share, o.row_weight);
  if (st != LB_OK) return fail(st);
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    set_error(std::string("lb_plan: ") + cudaGetErrorString(e));
    return fail(LB_ERR_CUDA);
  }
  *out = p;
  return LB_OK;
}

lb_status_t lb_plan(lb_plan_t* out, const int32_t* tile_offsets, int32_t num_tiles, int32_t num_atoms,
                    lb_schedule_t schedule) {
  return lb_plan_ex(out, tile_offsets, num_tiles, num_atoms, schedule, nullptr, nullptr);
}

void lb_plan_destroy(lb_plan_t p) {
  if (!p) return;
  p->mp.release();
  p->mm.release();
  cudaFree(p->mm_carry_row);
  cudaFree(p->mm_carry_val);
  free_transpose(p);
  p->bb.release();
  cudaFree(p->rp_global);
  cudaFree(p->d_status);
  delete p;
}

lb_status_t lb_plan_get_info(lb_plan_t p, lb_plan_info_t* info) {
  if (!p || !info) {
    set_error("lb_plan_get_info: NULL argument");
    return LB_ERR_INVALID_ARG;
  }
  std::memset(info, 0, sizeof(*info));
  info->schedule = p->schedule;
  info->num_tiles = p->num_tiles;
  info->num_cols = p->num_cols;
  info->num_atoms = p->num_atoms;
  info->block_threads = kBlock;
  info->items_per_tile = p->mp.items_per_tile;
  info->tiles_per_cta = p->mp.tiles_per_cta;
  info->num_workers = p->mp.workers;
  info->mp_variant = p->mp.variant;
  info->num_waves = p->mp.num_waves;
  info->num_waves_t = p->has_t ? p->mp_t.num_waves : 0;
  info->num_splits = p->mp.entries;
  info->group_size = p->group_size;
  info->num_sms = p->num_sms;
  info->has_transpose = p->has_t ? 1 : 0;
  const int64_t R = info->num_tiles;
  switch (p->schedule) {
    case LB_MERGE_PATH:
      info->grid = p->mp.grid;
      info->kernels_per_spmv = p->mp.items > 0 ? 1 : 0;
      break;
    case LB_THREAD_MAPPED:
      info->grid = p->tm_grid ? (int32_t)std::min<int64_t>(((R + 31) / 32 + 7) / 8, p->tm_grid)
                              : (int32_t)((R + kBlock - 1) / kBlock);
      info->kernels_per_spmv = R > 0 ? 1 : 0;
      break;
    default: {
      int64_t b = (R + kBlock - 1) / kBlock;
      if (b > (int64_t)p->num_sms * 64) b = (int64_t)p->num_sms * 64;
      info->grid = (int32_t)b;
      info->kernels_per_spmv = R > 0 ? 1 : 0;
    }
  }
  return LB_OK;
}

lb_status_t lb_plan_splits(lb_plan_t p, int32_t which, int64_t* host_diag, int32_t* host_ij, size_t cap,
                           size_t* count) {
  if (!p || (which != 0 && which != 1)) {
    set_error("lb_plan_splits: bad plan or table");
    return LB_ERR_INVALID_ARG;
  }
  const MpTable& t = which == 0 ? p->mp : p->mp_t;
  if (!t.built) {
    set_error("lb_plan_splits: table not built");
    return LB_ERR_INVALID_ARG;
  }
  if (count) *count = (size_t)t.entries;
  const size_t n = cap < (size_t)t.entries ? cap : (size_t)t.entries;
  if (n == 0) return LB_OK;
  if (host_diag) LB_CUDA_TRY(cudaMemcpy(host_diag, t.d_diag, sizeof(int64_t) * n, cudaMemcpyDeviceToHost));
  if (host_ij) LB_CUDA_TRY(cudaMemcpy(host_ij, t.splits, sizeof(int32_t) * 2 * n, cudaMemcpyDeviceToHost));
  return LB_OK;
}

lb_status_t lb_spmv(lb_plan_t p, const int32_t* col_idx, const float* vals, const float* x, float* y, void* stream) {
  if (!p || p->is_batch) {
    set_error("lb_spmv: NULL plan or batch plan (use lb_batch_spmv)");
    return LB_ERR_INVALID_ARG;
  }
  if (p->num_tiles == 0) return LB_OK;
  if (!y || (p->num_atoms > 0 && (!col_idx || !vals || !x))) {
    set_error("lb_spmv: NULL buffer");
    return LB_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  SpmvCall c{p->rp, p->num_tiles, col_idx, vals, nullptr, x, y, p->opts.validate ? p->num_cols : 0, p->d_status};
  switch (p->schedule) {
    case LB_THREAD_MAPPED:
      return p->tm_grid ? launch_tm_staged_spmv(c, p->tm_grid, s) : launch_tm_spmv(c, s);
    case LB_WARP_MAPPED:
    case LB_BLOCK_MAPPED:
    case LB_GROUP_MAPPED:
      return launch_gm_spmv(p->group_size, c, p->num_sms, s);
    case LB_MERGE_PATH:
      return launch_mp_spmv(p->mp, c, s);
    default:
      set_error("lb_spmv: unknown schedule");
      return LB_ERR_INVALID_ARG;
  }
}

lb_status_t lb_prepare_backward(lb_plan_t p, int32_t num_cols, const int32_t* col_idx, void* stream) {
  if (!p || p->is_batch || num_cols < 0 || (p->num_atoms > 0 && !col_idx)) {
    set_error("lb_prepare_backward: bad arguments");
    return LB_ERR_INVALID_ARG;
  }
  if (p->has_t && p->t_cols == num_cols) return LB_OK;
  if (num_cols == 0 && p->num_atoms > 0) {
    set_error("lb_prepare_backward: num_cols = 0 with atoms");
    return LB_ERR_INVALID_ARG;
  }
  free_transpose(p);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t N = p->num_atoms;
  LB_TRY(check_columns(col_idx, N, num_cols, s));
  LB_CUDA_TRY(cudaMalloc(&p->cp, sizeof(int32_t) * ((size_t)num_cols + 1)));
  LB_CUDA_TRY(cudaMalloc(&p->riT, sizeof(int32_t) * (size_t)(N > 0 ? N : 1)));
  LB_CUDA_TRY(cudaMalloc(&p->perm, sizeof(int32_t) * (size_t)(N > 0 ? N : 1)));
  int32_t* row_of = nullptr;
  LB_CUDA_TRY(cudaMalloc(&row_of, sizeof(int32_t) * (size_t)(N > 0 ? N : 1)));
  SpmvCall c{p->rp, p->num_tiles, nullptr, nullptr, nullptr, nullptr, nullptr, 0, nullptr};
  lb_status_t st = launch_mp_expand(p->mp, c, nullptr, nullptr, row_of, s);
  if (st == LB_OK) st = transpose_sort(col_idx, row_of, N, num_cols, p->cp, p->riT, p->perm, s);
  cudaStreamSynchronize(s);
  cudaFree(row_of);
  if (st != LB_OK) {
    free_transpose(p);
    return st;
  }
  st = build_mp_table(p->mp_t, p->cp, num_cols, N, p->opts.items_per_thread_t, p->opts.mp_variant, p->num_sms,
                      p->opts.ctas_per_sm, nullptr, s, nullptr, nullptr, 0, 0, p->opts.units_per_cta,
                      p->opts.tiles_per_share, p->opts.row_weight);
  if (st != LB_OK) {
    free_transpose(p);
    return st;
  }
  LB_CUDA_TRY(cudaStreamSynchronize(s));
  p->has_t = true;
  p->t_cols = num_cols;
  if (p->num_cols == 0) p->num_cols = num_cols;
  return LB_OK;
}

lb_status_t lb_plan_transpose(lb_plan_t p, int32_t* cp, int32_t* riT, int32_t* perm, void* stream) {
  if (!p || !p->has_t) {
    set_error("lb_plan_transpose: no transpose (call lb_prepare_backward)");
    return LB_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t N = p->num_atoms;
  if (cp) LB_CUDA_TRY(cudaMemcpyAsync(cp, p->cp, sizeof(int32_t) * ((size_t)p->t_cols + 1), cudaMemcpyDeviceToDevice, s));
  if (riT && N) LB_CUDA_TRY(cudaMemcpyAsync(riT, p->riT, sizeof(int32_t) * (size_t)N, cudaMemcpyDeviceToDevice, s));
  if (perm && N) LB_CUDA_TRY(cudaMemcpyAsync(perm, p->perm, sizeof(int32_t) * (size_t)N, cudaMemcpyDeviceToDevice, s));
  return LB_OK;
}

lb_status_t lb_spmv_backward(lb_plan_t p, int32_t num_cols, const int32_t* col_idx, const float* vals, const float* x,
                             const float* dy, float* dx, float* dvals, void* stream) {
  if (!p || p->is_batch) {
    set_error("lb_spmv_backward: NULL plan or batch plan");
    return LB_ERR_INVALID_ARG;
  }
  if ((dx || dvals) && p->num_tiles > 0 && !dy) {
    set_error("lb_spmv_backward: dy is NULL");
    return LB_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (dx) {
    if (!p->has_t || p->t_cols != num_cols) LB_TRY(lb_prepare_backward(p, num_cols, col_idx, stream));
    if (p->num_atoms > 0 && !vals) {
      set_error("lb_spmv_backward: vals is NULL");
      return LB_ERR_INVALID_ARG;
    }
    if (p->num_atoms == 0) {
      if (num_cols > 0) LB_CUDA_TRY(cudaMemsetAsync(dx, 0, sizeof(float) * (size_t)num_cols, s));
    } else {
      // dx = A^T dy: the plan's schedule over the transposed tile set (tiles = columns)
      SpmvCall c{p->cp, num_cols, p->riT, vals, p->perm, dy, dx, 0, p->d_status};
      switch (p->schedule) {
        case LB_THREAD_MAPPED:
          LB_TRY(p->tm_grid ? launch_tm_staged_spmv(c, p->tm_grid, s) : launch_tm_spmv(c, s));
          break;
        case LB_WARP_MAPPED:
        case LB_BLOCK_MAPPED:
        case LB_GROUP_MAPPED:
          LB_TRY(launch_gm_spmv(p->group_size, c, p->num_sms, s));
          break;
        default:
          LB_TRY(launch_mp_spmv(p->mp_t, c, s));
      }
    }
  }
  if (dvals && p->num_atoms > 0) {
    if (!col_idx || !x) {
      set_error("lb_spmv_backward: col_idx or x is NULL");
      return LB_ERR_INVALID_ARG;
    }
    SpmvCall c{p->rp, p->num_tiles, col_idx, nullptr, nullptr, x, nullptr, p->opts.validate ? p->num_cols : 0,
               p->d_status};
    LB_TRY(launch_mp_expand(p->mp, c, dy, dvals, nullptr, s));
  }
  return LB_OK;
}

lb_status_t lb_atom_tiles(lb_plan_t p, int32_t* tile_of_atom, void* stream) {
  if (!p || (!tile_of_atom && p->num_atoms > 0)) {
    set_error("lb_atom_tiles: NULL argument");
    return LB_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  SpmvCall c{p->rp, p->num_tiles, nullptr, nullptr, nullptr, nullptr, nullptr, 0, nullptr};
  return launch_mp_expand(p->mp, c, nullptr, nullptr, tile_of_atom, s);
}

lb_status_t lb_status(lb_plan_t p, void* stream) {
  if (!p) {
    set_error("lb_status: NULL plan");
    return LB_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int h = 0;
  LB_CUDA_TRY(cudaStreamSynchronize(s));
  LB_CUDA_TRY(cudaMemcpy(&h, p->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  LB_CUDA_TRY(cudaMemset(p->d_status, 0, sizeof(int)));
  if (h & 2) {
    set_error("a bounded wait in a kernel gave up (results of that call are invalid)");
    return LB_ERR_TIMEOUT;
  }
  if (h) {
    set_error("a validated kernel saw a column index outside [0, num_cols)");
    return LB_ERR_BAD_INPUT;
  }
  return LB_OK;
}

}  // extern "C"
