// Other input formats as CSR tile sets (Sec. 4: a new format needs only its
// own atom and tile iterators).  COO: the tiles are the rows, so the tile
// offsets are the prefix-summed run lengths of the atoms' row ids and the
// atoms are placed by a stable counting sort on the row id.  CSC: the arrays
// are the CSR of A^T; the column of every atom comes from the merge-path
// atom-to-tile walk over the column offsets (lb_atom_tiles), and the same
// stable counting sort on the row id gives A's CSR with columns ascending in
// each row.  Both reuse the library's transpose sort.
#include <string>

#include "lb_internal.h"

using namespace lbh;

namespace {

__global__ void key_range_kernel(const int32_t* __restrict__ keys, int64_t n, int32_t limit, int* bad) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    if ((unsigned)keys[k] >= (unsigned)limit) atomicOr(bad, 1);
}

__global__ void gather_f32_kernel(const float* __restrict__ src, const int32_t* __restrict__ idx, int64_t n,
                                  float* __restrict__ out) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    out[k] = src[idx[k]];
}

unsigned blocks_for(int64_t n) {
  const int64_t b = (n + 255) / 256;
  return (unsigned)(b < 1 ? 1 : (b > 65535 ? 65535 : b));
}

struct Scratch {
  void* p = nullptr;
  ~Scratch() { cudaFree(p); }
};

// keys in [0, limit)? (synchronises)
lb_status_t keys_in_range(const int32_t* keys, int64_t n, int32_t limit, const char* what, cudaStream_t s) {
  if (n == 0) return LB_OK;
  Scratch bad;
  LB_CUDA_TRY(cudaMalloc(&bad.p, sizeof(int)));
  LB_CUDA_TRY(cudaMemsetAsync(bad.p, 0, sizeof(int), s));
  key_range_kernel<<<blocks_for(n), 256, 0, s>>>(keys, n, limit, static_cast<int*>(bad.p));
  LB_CUDA_TRY(cudaGetLastError());
  int h = 0;
  LB_CUDA_TRY(cudaMemcpyAsync(&h, bad.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  LB_CUDA_TRY(cudaStreamSynchronize(s));
  if (h) {
    set_error(std::string(what) + " outside [0, " + std::to_string(limit) + ")");
    return LB_ERR_INVALID_ARG;
  }
  return LB_OK;
}

// rp_out, col_out, val_out from the atoms sorted stably by `row`; `other` is
// each atom's column
lb_status_t sort_by_row(int32_t R, int64_t N, const int32_t* row, const int32_t* other, const float* vals,
                        int32_t* rp_out, int32_t* col_out, float* val_out, cudaStream_t s) {
  Scratch perm;
  if (N > 0) LB_CUDA_TRY(cudaMalloc(&perm.p, sizeof(int32_t) * (size_t)N));
  int32_t* pm = static_cast<int32_t*>(perm.p);
  LB_TRY(transpose_sort(row, other, N, R, rp_out, col_out, pm, s));
  if (N > 0) {
    gather_f32_kernel<<<blocks_for(N), 256, 0, s>>>(vals, pm, N, val_out);
    LB_CUDA_TRY(cudaGetLastError());
    LB_CUDA_TRY(cudaStreamSynchronize(s));
  }
  return LB_OK;
}

}  // namespace

extern "C" {

lb_status_t lb_coo_to_csr(int32_t num_rows, int32_t num_atoms, const int32_t* row_idx, const int32_t* col_idx,
                          const float* vals, int32_t* tile_offsets_out, int32_t* col_idx_out, float* vals_out,
                          void* stream) {
  if (num_rows < 0 || num_atoms < 0 || !tile_offsets_out ||
      (num_atoms > 0 && (!row_idx || !col_idx || !vals || !col_idx_out || !vals_out)) ||
      (num_rows == 0 && num_atoms > 0)) {
    set_error("lb_coo_to_csr: need sizes >= 0, rows for any atom, and buffers");
    return LB_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  LB_TRY(keys_in_range(row_idx, num_atoms, num_rows, "lb_coo_to_csr: a row id", s));
  return sort_by_row(num_rows, num_atoms, row_idx, col_idx, vals, tile_offsets_out, col_idx_out, vals_out, s);
}

lb_status_t lb_csc_to_csr(int32_t num_rows, int32_t num_cols, int32_t num_atoms, const int32_t* col_offsets,
                          const int32_t* row_idx, const float* vals, int32_t* tile_offsets_out, int32_t* col_idx_out,
                          float* vals_out, void* stream) {
  if (num_rows < 0 || num_cols < 0 || num_atoms < 0 || !tile_offsets_out || (num_cols > 0 && !col_offsets) ||
      (num_atoms > 0 && (!row_idx || !vals || !col_idx_out || !vals_out)) ||
      ((num_rows == 0 || num_cols == 0) && num_atoms > 0)) {
    set_error("lb_csc_to_csr: need sizes >= 0, rows and columns for any atom, and buffers");
    return LB_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  LB_TRY(keys_in_range(row_idx, num_atoms, num_rows, "lb_csc_to_csr: a row id", s));
  Scratch colof;
  if (num_atoms > 0) {
    // the column of every atom: the columns are the tiles of the CSC arrays
    lb_plan_opts_t o{};
    o.validate = 1;
    lb_plan_t plan = nullptr;
    LB_TRY(lb_plan_ex(&plan, col_offsets, num_cols, num_atoms, LB_MERGE_PATH, &o, s));
    struct Destroy {
      lb_plan_t p;
      ~Destroy() { lb_plan_destroy(p); }
    } guard{plan};
    LB_CUDA_TRY(cudaMalloc(&colof.p, sizeof(int32_t) * (size_t)num_atoms));
    LB_TRY(lb_atom_tiles(plan, static_cast<int32_t*>(colof.p), s));
  }
  return sort_by_row(num_rows, num_atoms, row_idx, static_cast<const int32_t*>(colof.p), vals, tile_offsets_out,
                     col_idx_out, vals_out, s);
}

}  // extern "C"
