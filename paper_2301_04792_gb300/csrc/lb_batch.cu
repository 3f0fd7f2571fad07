// Batched tile sets: many CSR matrices run as one persistent merge-path launch
// over their block-diagonal concatenation (global int64 diagonals; each split
// records its matrix), plus the batched backward.
#include <cstring>
#include <string>
#include <vector>

#include "lb_internal.h"

namespace lbh {
lb_status_t check_columns(const int32_t* ci, int64_t n, int32_t C, cudaStream_t s);
}

using namespace lbh;

namespace {

__device__ __forceinline__ int largest_le(const int64_t* base, int n, int64_t g) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(base + mid) <= g) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// global column key of every atom: col + first column of its matrix; flags
// columns outside the matrix's [0, cols)
__global__ void global_keys_kernel(const int32_t* __restrict__ ci, const int64_t* __restrict__ nnz_base,
                                   const int64_t* __restrict__ col_base, int num, int64_t n, int32_t* __restrict__ keys,
                                   int* bad) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    const int m = largest_le(nnz_base, num, j);
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

// per-matrix CSC offsets from the global ones: entry q of the concatenation
// (cols[m] + 1 entries per matrix) = cp_global[col_base[m] + c] - nnz_base[m]
__global__ void local_offsets_kernel(const int32_t* __restrict__ cp_global, const int64_t* __restrict__ col_base,
                                     const int64_t* __restrict__ nnz_base, const int64_t* __restrict__ cat_base,
                                     int num, int64_t n, int32_t* __restrict__ out) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
    const int m = largest_le(cat_base, num, q);
    const int64_t c = q - cat_base[m];
    out[q] = (int32_t)((int64_t)cp_global[col_base[m] + c] - nnz_base[m]);
  }
}

// make rows and atom indices matrix-local
__global__ void localize_kernel(int32_t* __restrict__ riT, int32_t* __restrict__ perm,
                                const int64_t* __restrict__ nnz_base, const int64_t* __restrict__ row_base, int num,
                                int64_t n) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const int m = largest_le(nnz_base, num, p);
    riT[p] = (int32_t)((int64_t)riT[p] - row_base[m]);
    perm[p] = (int32_t)((int64_t)perm[p] - nnz_base[m]);
  }
}

unsigned nblocks(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > 65536LL * 16) b = 65536LL * 16;
  return (unsigned)(b < 1 ? 1 : b);
}

lb_status_t upload_bases(BatchSet& b, const std::vector<int64_t>& rows, const std::vector<int64_t>& nnz,
                         const std::vector<int64_t>& vec, cudaStream_t s) {
  const int n = b.num;
  std::vector<int64_t> diag(n + 1);
  for (int m = 0; m <= n; ++m) diag[m] = rows[m] + nnz[m];
  const size_t bytes = sizeof(int64_t) * (n + 1);
  LB_CUDA_TRY(cudaMalloc(&b.row_base, bytes));
  LB_CUDA_TRY(cudaMalloc(&b.nnz_base, bytes));
  LB_CUDA_TRY(cudaMalloc(&b.vec_base, bytes));
  LB_CUDA_TRY(cudaMalloc(&b.diag_base, bytes));
  LB_CUDA_TRY(cudaMemcpyAsync(b.row_base, rows.data(), bytes, cudaMemcpyHostToDevice, s));
  LB_CUDA_TRY(cudaMemcpyAsync(b.nnz_base, nnz.data(), bytes, cudaMemcpyHostToDevice, s));
  LB_CUDA_TRY(cudaMemcpyAsync(b.vec_base, vec.data(), bytes, cudaMemcpyHostToDevice, s));
  LB_CUDA_TRY(cudaMemcpyAsync(b.diag_base, diag.data(), bytes, cudaMemcpyHostToDevice, s));
  LB_CUDA_TRY(cudaStreamSynchronize(s));
  b.total_rows = rows[n];
  b.total_nnz = nnz[n];
  b.total_cols = vec[n];
  return LB_OK;
}

void free_batch_transpose(lb_plan_s* p) {
  p->bs_t.release();
  p->mp_t.release();
  cudaFree(p->perm_t_local);
  cudaFree(p->riT_local);
  p->perm_t_local = p->riT_local = nullptr;
  p->cp_cat_t = nullptr;  // owned by bs_t
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
    if (host_rows[m] < 0 || host_cols[m] < 0 || host_nnz[m] < 0 || host_nnz[m] > INT32_MAX ||
        (host_rows[m] == 0 && host_nnz[m] != 0)) {
      set_error("lb_batch_plan: bad size for matrix " + std::to_string(m));
      return LB_ERR_INVALID_ARG;
    }
    rows[m + 1] = rows[m] + host_rows[m];
    cols[m + 1] = cols[m] + host_cols[m];
    nnz[m + 1] = nnz[m] + host_nnz[m];
  }
  if (rows[num_mats] >= INT32_MAX || cols[num_mats] >= INT32_MAX || nnz[num_mats] >= INT32_MAX) {
    set_error("lb_batch_plan: batch totals must stay below 2^31 rows, columns and atoms");
    return LB_ERR_UNSUPPORTED;
  }
  lb_plan_opts_t o{};
  if (opts) o = *opts;
  if (o.items_per_thread == 0) o.items_per_thread = 8;
  if (o.items_per_thread != 4 && o.items_per_thread != 8 && o.items_per_thread != 16) {
    set_error("lb_batch_plan: items_per_thread must be 4, 8 or 16");
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
  p->bs.num = num_mats;
  p->bs.rp_cat = rp_cat;
  p->bs.owns_rp = false;
  lb_status_t st = upload_bases(p->bs, rows, nnz, cols, s);
  if (st == LB_OK) {
    if (cudaMalloc(&p->d_status, sizeof(int)) != cudaSuccess) st = LB_ERR_OOM;
    else cudaMemsetAsync(p->d_status, 0, sizeof(int), s);
  }
  if (st == LB_OK) st = build_mp_table_batch(p->mp, p->bs, o.items_per_thread, p->num_sms, o.ctas_per_sm, s);
  if (st == LB_OK && cudaStreamSynchronize(s) != cudaSuccess) {
    set_error("lb_batch_plan: split kernel failed");
    st = LB_ERR_CUDA;
  }
  if (st != LB_OK) {
    lb_plan_destroy(p);
    return st;
  }
  *out = p;
  return LB_OK;
}

lb_status_t lb_batch_spmv(lb_plan_t p, const int32_t* col_cat, const float* vals_cat, const float* x_cat,
                          float* y_cat, void* stream) {
  if (!p || !p->is_batch) {
    set_error("lb_batch_spmv: not a batch plan");
    return LB_ERR_INVALID_ARG;
  }
  if (p->bs.total_rows == 0) return LB_OK;
  if (!y_cat || (p->bs.total_nnz > 0 && (!col_cat || !vals_cat || !x_cat))) {
    set_error("lb_batch_spmv: NULL buffer");
    return LB_ERR_INVALID_ARG;
  }
  return launch_mp_spmv(p->mp, nullptr, &p->bs, col_cat, vals_cat, nullptr, x_cat, y_cat, p->bs.total_rows, 0,
                        p->d_status, static_cast<cudaStream_t>(stream));
}

lb_status_t lb_batch_prepare_backward(lb_plan_t p, const int32_t* col_cat, void* stream) {
  if (!p || !p->is_batch || (p->bs.total_nnz > 0 && !col_cat)) {
    set_error("lb_batch_prepare_backward: bad arguments");
    return LB_ERR_INVALID_ARG;
  }
  if (p->has_t) return LB_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const BatchSet& b = p->bs;
  const int64_t N = b.total_nnz;
  const int32_t C = (int32_t)b.total_cols;
  const int num = b.num;
  int32_t *keys = nullptr, *row_of = nullptr, *cp_global = nullptr, *bad = nullptr;
  int32_t* cp_cat = nullptr;
  const size_t nb = sizeof(int32_t) * (size_t)(N > 0 ? N : 1);
  auto cleanup = [&]() {
    cudaFree(keys);
    cudaFree(row_of);
    cudaFree(cp_global);
    cudaFree(bad);
  };
  lb_status_t st = LB_OK;
#define BT_TRY(call)                                                                   \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess) {                                                           \
      set_error(std::string(#call) + ": " + cudaGetErrorString(e_));                   \
      cleanup();                                                                       \
      cudaFree(cp_cat);                                                                \
      free_batch_transpose(p);                                                         \
      return e_ == cudaErrorMemoryAllocation ? LB_ERR_OOM : LB_ERR_CUDA;               \
    }                                                                                  \
  } while (0)
  BT_TRY(cudaMalloc(&keys, nb));
  BT_TRY(cudaMalloc(&row_of, nb));
  BT_TRY(cudaMalloc(&cp_global, sizeof(int32_t) * ((size_t)C + 1)));
  BT_TRY(cudaMalloc(&bad, sizeof(int)));
  BT_TRY(cudaMalloc(&p->riT_local, nb));
  BT_TRY(cudaMalloc(&p->perm_t_local, nb));
  BT_TRY(cudaMalloc(&cp_cat, sizeof(int32_t) * ((size_t)C + num)));
  BT_TRY(cudaMemsetAsync(bad, 0, sizeof(int), s));
  if (N > 0) {
    global_keys_kernel<<<nblocks(N), 256, 0, s>>>(col_cat, b.nnz_base, b.vec_base, num, N, keys, bad);
    BT_TRY(cudaGetLastError());
    int h = 0;
    BT_TRY(cudaMemcpyAsync(&h, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    BT_TRY(cudaStreamSynchronize(s));
    if (h) {
      set_error("lb_batch_prepare_backward: column index outside its matrix");
      cleanup();
      cudaFree(cp_cat);
      free_batch_transpose(p);
      return LB_ERR_BAD_INPUT;
    }
    st = launch_mp_expand(p->mp, nullptr, &p->bs, nullptr, nullptr, nullptr, nullptr, row_of, 0, nullptr, s);
  }
  if (st == LB_OK) st = transpose_sort(keys, row_of, N, C, cp_global, p->riT_local, p->perm_t_local, s);
  if (st != LB_OK) {
    cleanup();
    cudaFree(cp_cat);
    free_batch_transpose(p);
    return st;
  }
  // transposed batch: matrix m has cols[m] tiles and the same atom range
  std::vector<int64_t> h_rows(num + 1), h_nnz(num + 1), h_cols(num + 1), h_cat(num + 1);
  BT_TRY(cudaMemcpy(h_rows.data(), b.row_base, sizeof(int64_t) * (num + 1), cudaMemcpyDeviceToHost));
  BT_TRY(cudaMemcpy(h_nnz.data(), b.nnz_base, sizeof(int64_t) * (num + 1), cudaMemcpyDeviceToHost));
  BT_TRY(cudaMemcpy(h_cols.data(), b.vec_base, sizeof(int64_t) * (num + 1), cudaMemcpyDeviceToHost));
  for (int m = 0; m <= num; ++m) h_cat[m] = h_cols[m] + m;
  int64_t* d_cat = nullptr;
  BT_TRY(cudaMalloc(&d_cat, sizeof(int64_t) * (num + 1)));
  BT_TRY(cudaMemcpy(d_cat, h_cat.data(), sizeof(int64_t) * (num + 1), cudaMemcpyHostToDevice));
  const int64_t ncat = (int64_t)C + num;
  local_offsets_kernel<<<nblocks(ncat), 256, 0, s>>>(cp_global, b.vec_base, b.nnz_base, d_cat, num, ncat, cp_cat);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && N > 0) {
    localize_kernel<<<nblocks(N), 256, 0, s>>>(p->riT_local, p->perm_t_local, b.nnz_base, b.row_base, num, N);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(d_cat);
  BT_TRY(e);
  cleanup();
  keys = row_of = cp_global = bad = nullptr;
  p->bs_t.num = num;
  p->bs_t.rp_cat = cp_cat;
  p->bs_t.owns_rp = true;
  p->cp_cat_t = cp_cat;
  cp_cat = nullptr;
  st = upload_bases(p->bs_t, h_cols, h_nnz, h_rows, s);
  if (st == LB_OK)
    st = build_mp_table_batch(p->mp_t, p->bs_t, p->opts.items_per_thread, p->num_sms, p->opts.ctas_per_sm, s);
  if (st == LB_OK && cudaStreamSynchronize(s) != cudaSuccess) st = LB_ERR_CUDA;
  if (st != LB_OK) {
    free_batch_transpose(p);
    return st;
  }
#undef BT_TRY
  p->has_t = true;
  return LB_OK;
}

lb_status_t lb_batch_spmv_backward(lb_plan_t p, const int32_t* col_cat, const float* vals_cat, const float* x_cat,
                                   const float* dy_cat, float* dx_cat, float* dvals_cat, void* stream) {
  if (!p || !p->is_batch) {
    set_error("lb_batch_spmv_backward: not a batch plan");
    return LB_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if ((dx_cat || dvals_cat) && p->bs.total_rows > 0 && !dy_cat) {
    set_error("lb_batch_spmv_backward: dy is NULL");
    return LB_ERR_INVALID_ARG;
  }
  if (dx_cat) {
    if (!p->has_t) LB_TRY(lb_batch_prepare_backward(p, col_cat, stream));
    if (p->bs.total_nnz == 0) {
      if (p->bs.total_cols > 0) LB_CUDA_TRY(cudaMemsetAsync(dx_cat, 0, sizeof(float) * (size_t)p->bs.total_cols, s));
    } else {
      if (!vals_cat) {
        set_error("lb_batch_spmv_backward: vals is NULL");
        return LB_ERR_INVALID_ARG;
      }
      LB_TRY(launch_mp_spmv(p->mp_t, nullptr, &p->bs_t, p->riT_local, vals_cat, p->perm_t_local, dy_cat, dx_cat,
                            p->bs.total_cols, 0, p->d_status, s));
    }
  }
  if (dvals_cat && p->bs.total_nnz > 0) {
    if (!col_cat || !x_cat) {
      set_error("lb_batch_spmv_backward: col or x is NULL");
      return LB_ERR_INVALID_ARG;
    }
    LB_TRY(launch_mp_expand(p->mp, nullptr, &p->bs, col_cat, x_cat, dy_cat, dvals_cat, nullptr, 0, p->d_status, s));
  }
  return LB_OK;
}

}  // extern "C"
