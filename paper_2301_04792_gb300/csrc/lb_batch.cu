// Batched tile sets: many CSR matrices run as one persistent merge-path launch
// over their block-diagonal concatenation.  At plan time the matrices' row
// offsets are made global (one offset array over all rows), so the merge path
// is the single-matrix one over sum(rows) + sum(nnz) items; each atom's
// column is offset by its matrix's first column, found from the split table's
// per-split matrix index.  The backward pass transposes the whole
// block-diagonal matrix at once (its transpose is the block-diagonal of the
// transposes) and keeps global row and atom indices, so dx needs no per-matrix
// lookups at all.
#include <cstring>
#include <string>
#include <vector>

#include "lb_internal.h"
#include "lb_kernels.cuh"

using namespace lbh;

namespace {

// global row offsets: rp_global[g] = nnz_base[m] + rp_cat[g + m] for row g of
// matrix m (rp_cat holds each matrix's rows[m] + 1 offsets back to back);
// rp_global[total_rows] = total_nnz
__global__ void global_offsets_kernel(const int32_t* __restrict__ rp_cat, const int64_t* __restrict__ row_base,
                                      const int64_t* __restrict__ nnz_base, int num, int64_t total_rows,
                                      int64_t total_nnz, int32_t* __restrict__ out, int* bad) {
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g <= total_rows;
       g += (int64_t)gridDim.x * blockDim.x) {
    if (g == total_rows) {
      out[g] = (int32_t)total_nnz;
      continue;
    }
    const int m = lbk::find_matrix(row_base, 0, num - 1, g);
    const int64_t v = nnz_base[m] + (int64_t)rp_cat[g + m];
    const int64_t lo = nnz_base[m], hi = nnz_base[m + 1];
    if (v < lo || v > hi) atomicOr(bad, 1);
    out[g] = (int32_t)v;
  }
}

// global column key of every atom: col + first column of its matrix; flags
// columns outside the matrix's [0, cols)
__global__ void global_keys_kernel(const int32_t* __restrict__ ci, const int64_t* __restrict__ nnz_base,
                                   const int64_t* __restrict__ col_base, int num, int64_t n, int32_t* __restrict__ keys,
                                   int* bad) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    const int m = lbk::find_matrix(nnz_base, 0, num - 1, j);
    const int c = __ldg(ci + j);
    const int64_t cb = __ldg(col_base + m), ce = __ldg(col_base + m + 1);
    if (c < 0 || cb + c >= ce) {
      atomicOr(bad, 1);
      keys[j] = (int32_t)cb;
    } else {
      keys[j] = (int32_t)(cb + c);
    }
  }
}

unsigned nblocks(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > 65536LL * 16) b = 65536LL * 16;
  return (unsigned)(b < 1 ? 1 : b);
}

lb_status_t read_flag(int* d, cudaStream_t s, int* h) {
  LB_CUDA_TRY(cudaMemcpyAsync(h, d, sizeof(int), cudaMemcpyDeviceToHost, s));
  LB_CUDA_TRY(cudaStreamSynchronize(s));
  return LB_OK;
}

void free_transpose(lb_plan_s* p) {
  cudaFree(p->cp);
  cudaFree(p->riT);
  cudaFree(p->perm);
  p->cp = p->riT = p->perm = nullptr;
  p->mp_t.release();
  p->has_t = false;
}

}  // namespace

extern "C" {

lb_status_t lb_batch_plan(lb_plan_t* out, int32_t num_mats, const int32_t* host_rows, const int32_t* host_cols,
                          const int64_t* host_nnz, const int32_t* rp_cat, const lb_plan_opts_t* opts, void* stream) {
  if (!out) {
    set_error("lb_batch_plan: out is NULL");
    return LB_ERR_INVALID_ARG;
  }
  *out = nullptr;
  if (num_mats < 1 || !host_rows || !host_cols || !host_nnz || !rp_cat) {
    set_error("lb_batch_plan: need num_mats >= 1 and non-NULL size arrays and rp_cat");
    return LB_ERR_INVALID_ARG;
  }
  std::vector<int64_t> rows(num_mats + 1, 0), nnz(num_mats + 1, 0), cols(num_mats + 1, 0);
  for (int m = 0; m < num_mats; ++m) {
    if (host_rows[m] < 0 || host_cols[m] < 0 || host_nnz[m] < 0 || (host_rows[m] == 0 && host_nnz[m] != 0)) {
      set_error("lb_batch_plan: bad size for matrix " + std::to_string(m));
      return LB_ERR_INVALID_ARG;
    }
    rows[m + 1] = rows[m] + host_rows[m];
    cols[m + 1] = cols[m] + host_cols[m];
    nnz[m + 1] = nnz[m] + host_nnz[m];
  }
  if (rows[num_mats] >= INT32_MAX || cols[num_mats] >= INT32_MAX || nnz[num_mats] >= INT32_MAX ||
      rows[num_mats] + nnz[num_mats] >= ((int64_t)1 << 32)) {
    set_error("lb_batch_plan: batch totals must stay below 2^31 rows, columns and atoms");
    return LB_ERR_UNSUPPORTED;
  }
  lb_plan_opts_t o{};
  if (opts) o = *opts;
  if (o.items_per_thread == 0) o.items_per_thread = 8;
  if (o.units_per_cta == 0) o.units_per_cta = 1;
  if (o.tiles_per_share == 0) o.tiles_per_share = 1;
  if (o.items_per_thread_t == 0) o.items_per_thread_t = o.items_per_thread;
  auto ipt_ok = [](int v) { return v == 4 || v == 8 || v == 16; };
  if (!ipt_ok(o.items_per_thread) || !ipt_ok(o.items_per_thread_t)) {
    set_error("lb_batch_plan: items_per_thread and items_per_thread_t must be 4, 8 or 16");
    return LB_ERR_UNSUPPORTED;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0;
  LB_CUDA_TRY(cudaGetDevice(&dev));
  lb_plan_s* p = new lb_plan_s();
  p->is_batch = true;
  p->device = dev;
  p->num_sms = device_sms(dev);
  p->schedule = LB_MERGE_PATH;
  p->opts = o;
  p->num_tiles = (int32_t)rows[num_mats];
  p->num_cols = (int32_t)cols[num_mats];
  p->num_atoms = nnz[num_mats];
  p->bb.num = num_mats;
  int64_t* d_rows = nullptr;
  int* bad = nullptr;
  lb_status_t st = LB_OK;
  auto fail = [&](lb_status_t e, const std::string& msg) {
    if (!msg.empty()) set_error(msg);
    cudaFree(d_rows);
    cudaFree(bad);
    lb_plan_destroy(p);
    return e;
  };
  const size_t bytes = sizeof(int64_t) * (num_mats + 1);
  if (cudaMalloc(&p->bb.nnz_base, bytes) != cudaSuccess || cudaMalloc(&p->bb.vec_base, bytes) != cudaSuccess ||
      cudaMalloc(&d_rows, bytes) != cudaSuccess || cudaMalloc(&bad, sizeof(int)) != cudaSuccess ||
      cudaMalloc(&p->d_status, sizeof(int)) != cudaSuccess ||
      cudaMalloc(&p->rp_global, sizeof(int32_t) * ((size_t)rows[num_mats] + 1)) != cudaSuccess)
    return fail(LB_ERR_OOM, "lb_batch_plan: device allocation failed");
  cudaMemcpyAsync(p->bb.nnz_base, nnz.data(), bytes, cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(p->bb.vec_base, cols.data(), bytes, cudaMemcpyHostToDevice, s);
  cudaMemcpyAsync(d_rows, rows.data(), bytes, cudaMemcpyHostToDevice, s);
  cudaMemsetAsync(bad, 0, sizeof(int), s);
  cudaMemsetAsync(p->d_status, 0, sizeof(int), s);
  global_offsets_kernel<<<nblocks(rows[num_mats] + 1), 256, 0, s>>>(rp_cat, d_rows, p->bb.nnz_base, num_mats,
                                                                    rows[num_mats], nnz[num_mats], p->rp_global, bad);
  int h = 0;
  st = read_flag(bad, s, &h);
  if (st != LB_OK) return fail(st, "");
  if (h) return fail(LB_ERR_INVALID_ARG, "lb_batch_plan: a matrix's offsets leave [0, nnz]");
  p->rp = p->rp_global;
  std::vector<int64_t> items(num_mats + 1);
  for (int m = 0; m <= num_mats; ++m) items[m] = rows[m] + nnz[m];
  st = build_mp_table(p->mp, p->rp_global, p->num_tiles, p->num_atoms, o.items_per_thread, o.mp_variant, p->num_sms,
                      o.ctas_per_sm, &p->bb, s, items.data(), rows.data(), num_mats, o.wave_items,
                      o.units_per_cta, o.tiles_per_share);
  if (st != LB_OK) return fail(st, "");
  if (cudaStreamSynchronize(s) != cudaSuccess) return fail(LB_ERR_CUDA, "lb_batch_plan: split kernel failed");
  cudaFree(d_rows);
  cudaFree(bad);
  *out = p;
  return LB_OK;
}

lb_status_t lb_batch_spmv(lb_plan_t p, const int32_t* col_cat, const float* vals_cat, const float* x_cat,
                          float* y_cat, void* stream) {
  if (!p || !p->is_batch) {
    set_error("lb_batch_spmv: not a batch plan");
    return LB_ERR_INVALID_ARG;
  }
  if (p->num_tiles == 0) return LB_OK;
  if (!y_cat || (p->num_atoms > 0 && (!col_cat || !vals_cat || !x_cat))) {
    set_error("lb_batch_spmv: NULL buffer");
    return LB_ERR_INVALID_ARG;
  }
  SpmvCall c{p->rp, p->num_tiles, col_cat, vals_cat, nullptr, x_cat, y_cat, 0, p->d_status, &p->bb};
  return launch_mp_spmv(p->mp, c, static_cast<cudaStream_t>(stream));
}

lb_status_t lb_batch_prepare_backward(lb_plan_t p, const int32_t* col_cat, void* stream) {
  if (!p || !p->is_batch || (p->num_atoms > 0 && !col_cat)) {
    set_error("lb_batch_prepare_backward: bad arguments");
    return LB_ERR_INVALID_ARG;
  }
  if (p->has_t) return LB_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t N = p->num_atoms;
  const int32_t C = p->num_cols;
  const size_t nb = sizeof(int32_t) * (size_t)(N > 0 ? N : 1);
  int32_t *keys = nullptr, *row_of = nullptr;
  int* bad = nullptr;
  auto cleanup = [&]() {
    cudaFree(keys);
    cudaFree(row_of);
    cudaFree(bad);
  };
  auto fail = [&](lb_status_t e, const std::string& msg) {
    if (!msg.empty()) set_error(msg);
    cleanup();
    free_transpose(p);
    return e;
  };
  if (cudaMalloc(&keys, nb) != cudaSuccess || cudaMalloc(&row_of, nb) != cudaSuccess ||
      cudaMalloc(&bad, sizeof(int)) != cudaSuccess || cudaMalloc(&p->cp, sizeof(int32_t) * ((size_t)C + 1)) ||
      cudaMalloc(&p->riT, nb) != cudaSuccess || cudaMalloc(&p->perm, nb) != cudaSuccess)
    return fail(LB_ERR_OOM, "lb_batch_prepare_backward: device allocation failed");
  cudaMemsetAsync(bad, 0, sizeof(int), s);
  lb_status_t st = LB_OK;
  if (N > 0) {
    global_keys_kernel<<<nblocks(N), 256, 0, s>>>(col_cat, p->bb.nnz_base, p->bb.vec_base, p->bb.num, N, keys, bad);
    int h = 0;
    st = read_flag(bad, s, &h);
    if (st != LB_OK) return fail(st, "");
    if (h) return fail(LB_ERR_BAD_INPUT, "lb_batch_prepare_backward: column index outside its matrix");
    SpmvCall c{p->rp, p->num_tiles, nullptr, nullptr, nullptr, nullptr, nullptr, 0, nullptr};
    st = launch_mp_expand(p->mp, c, nullptr, nullptr, row_of, s);
    if (st != LB_OK) return fail(st, "");
  }
  st = transpose_sort(keys, row_of, N, C, p->cp, p->riT, p->perm, s);
  if (st != LB_OK) return fail(st, "");
  cudaStreamSynchronize(s);
  cleanup();
  keys = row_of = nullptr;
  bad = nullptr;
  // the transposed batch: matrix m has cols[m] tiles and the same atoms
  const int num = p->bb.num;
  std::vector<int64_t> hc(num + 1), hn(num + 1), titems(num + 1);
  if (cudaMemcpy(hc.data(), p->bb.vec_base, sizeof(int64_t) * (num + 1), cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(hn.data(), p->bb.nnz_base, sizeof(int64_t) * (num + 1), cudaMemcpyDeviceToHost) != cudaSuccess)
    return fail(LB_ERR_CUDA, "lb_batch_prepare_backward: copy of matrix bases failed");
  for (int m = 0; m <= num; ++m) titems[m] = hc[m] + hn[m];
  st = build_mp_table(p->mp_t, p->cp, C, N, p->opts.items_per_thread_t, p->opts.mp_variant, p->num_sms,
                      p->opts.ctas_per_sm, nullptr, s, titems.data(), hc.data(), num, p->opts.wave_items,
                      p->opts.units_per_cta, p->opts.tiles_per_share);
  if (st != LB_OK) return fail(st, "");
  if (cudaStreamSynchronize(s) != cudaSuccess) return fail(LB_ERR_CUDA, "lb_batch_prepare_backward: sync failed");
  p->has_t = true;
  p->t_cols = C;
  return LB_OK;
}

lb_status_t lb_batch_spmv_backward(lb_plan_t p, const int32_t* col_cat, const float* vals_cat, const float* x_cat,
                                   const float* dy_cat, float* dx_cat, float* dvals_cat, void* stream) {
  if (!p || !p->is_batch) {
    set_error("lb_batch_spmv_backward: not a batch plan");
    return LB_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if ((dx_cat || dvals_cat) && p->num_tiles > 0 && !dy_cat) {
    set_error("lb_batch_spmv_backward: dy is NULL");
    return LB_ERR_INVALID_ARG;
  }
  if (dx_cat) {
    if (!p->has_t) LB_TRY(lb_batch_prepare_backward(p, col_cat, stream));
    if (p->num_atoms == 0) {
      if (p->num_cols > 0) LB_CUDA_TRY(cudaMemsetAsync(dx_cat, 0, sizeof(float) * (size_t)p->num_cols, s));
    } else {
      if (!vals_cat) {
        set_error("lb_batch_spmv_backward: vals is NULL");
        return LB_ERR_INVALID_ARG;
      }
      // transposed block-diagonal matrix with global row and atom indices
      SpmvCall c{p->cp, p->num_cols, p->riT, vals_cat, p->perm, dy_cat, dx_cat, 0, p->d_status};
      LB_TRY(launch_mp_spmv(p->mp_t, c, s));
    }
  }
  if (dvals_cat && p->num_atoms > 0) {
    if (!col_cat || !x_cat) {
      set_error("lb_batch_spmv_backward: col or x is NULL");
      return LB_ERR_INVALID_ARG;
    }
    SpmvCall c{p->rp, p->num_tiles, col_cat, nullptr, nullptr, x_cat, nullptr, 0, p->d_status, &p->bb};
    LB_TRY(launch_mp_expand(p->mp, c, dy_cat, dvals_cat, nullptr, s));
  }
  return LB_OK;
}

}  // extern "C"
