// SpMM C = A B for a dense row-major B (Sec. 7, Listing 4: the SpMV loop with
// one more loop over the columns of B), on two of the paper's schedules:
//  - merge-path: a warp per share of rows + atoms (the split table of Sec.
//    5.2.1 with warp tiles), the lanes holding the columns of B; per tile the
//    atoms and row ends are staged in shared memory, every row of the tile is
//    summed over its atoms with four rows of B in flight, and the row left open
//    at the share's end is finished by a second launch that adds the partial
//    sums of each run of shares to the row that closes it, in share order;
//  - thread-mapped: Listing 4 as printed, one thread per row looping over the
//    columns of B and the row's atoms.
// Columns are processed in panels of up to 128 (four per lane).
#include <algorithm>
#include <string>

#include "lb_internal.h"
#include "lb_kernels.cuh"

using namespace lbh;

namespace {

constexpr int kPanel = 128;  // columns of B per launch
constexpr int kTileCap = 256;  // atoms / rows of a warp tile staged in shared memory (tiles hold 252 items)

struct SpmmArgs {
  const int32_t* rp;
  int32_t R;
  const int32_t* idx;
  const float* val;
  const float* B;  // panel's first column
  int64_t ldb;
  float* C;        // panel's first column
  int64_t ldc;
  int K;           // columns in the panel
  const int2* splits;
  int num_shares;
  int tpc;
  int items_per_tile;
  int32_t* carry_row;  // [num_shares]
  float* carry_val;    // [num_shares x kPanel]
};

template <int KB>
__global__ void __launch_bounds__(256) spmm_mp_kernel(SpmmArgs a) {
  constexpr int WPB = 8;
  __shared__ int s_ci[WPB][kTileCap];
  __shared__ float s_v[WPB][kTileCap];
  __shared__ int s_end[WPB][kTileCap];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int* ci_s = s_ci[warp];
  float* v_s = s_v[warp];
  int* end_s = s_end[warp];
  const int nwarps = gridDim.x * WPB;
  for (int s = blockIdx.x * WPB + warp; s < a.num_shares; s += nwarps) {
    const int2* sp = a.splits + (size_t)s * (a.tpc + 1);
    int2 c0 = __ldg(sp);
    const int2 e1 = __ldg(sp + a.tpc);
    const int ntiles = (int)(((int64_t)(e1.x - c0.x) + (e1.y - c0.y) + a.items_per_tile - 1) / a.items_per_tile);
    float carry[KB];
#pragma unroll
    for (int kb = 0; kb < KB; ++kb) carry[kb] = 0.f;
    for (int k = 0; k < ntiles; ++k) {
      const int2 c1 = __ldg(sp + k + 1);
      const int nnz = c1.y - c0.y, nrows = c1.x - c0.x;
      for (int i = lane; i < nnz; i += 32) {
        ci_s[i] = lbk::ld_stream(a.idx + c0.y + i);
        v_s[i] = lbk::ld_stream(a.val + c0.y + i);
      }
      for (int i = lane; i < nrows; i += 32) end_s[i] = __ldg(a.rp + c0.x + 1 + i) - c0.y;
      __syncwarp();
      int j = 0;
      // rows closing in the tile, then the row left open at its end (r == nrows)
      for (int r = 0; r <= nrows; ++r) {
        const int e = r < nrows ? end_s[r] : nnz;
        float p[KB];
#pragma unroll
        for (int kb = 0; kb < KB; ++kb) p[kb] = 0.f;
        int q = j;
        for (; q + 4 <= e; q += 4) {
          float bq[4][KB];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const float* brow = a.B + (int64_t)ci_s[q + u] * a.ldb;
#pragma unroll
            for (int kb = 0; kb < KB; ++kb) {
              const int col = lane + 32 * kb;
              bq[u][kb] = col < a.K ? __ldg(brow + col) : 0.f;
            }
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const float w = v_s[q + u];
#pragma unroll
            for (int kb = 0; kb < KB; ++kb) p[kb] += w * bq[u][kb];
          }
        }
        for (; q < e; ++q) {
          const float* brow = a.B + (int64_t)ci_s[q] * a.ldb;
          const float w = v_s[q];
#pragma unroll
          for (int kb = 0; kb < KB; ++kb) {
            const int col = lane + 32 * kb;
            p[kb] += w * (col < a.K ? __ldg(brow + col) : 0.f);
          }
        }
        if (r == 0) {  // the row open at the tile's start: the earlier tiles' partial sum in front
#pragma unroll
          for (int kb = 0; kb < KB; ++kb) p[kb] = carry[kb] + p[kb];
        }
        if (r < nrows) {
          float* crow = a.C + (int64_t)(c0.x + r) * a.ldc;
#pragma unroll
          for (int kb = 0; kb < KB; ++kb) {
            const int col = lane + 32 * kb;
            if (col < a.K) crow[col] = p[kb];
          }
        } else {
#pragma unroll
          for (int kb = 0; kb < KB; ++kb) carry[kb] = p[kb];
        }
        j = e;
      }
      __syncwarp();
      c0 = c1;
    }
    // the row left open at the share's end (none after the last row)
    if (lane == 0) a.carry_row[s] = c0.x < a.R ? c0.x : -1;
#pragma unroll
    for (int kb = 0; kb < KB; ++kb) {
      const int col = lane + 32 * kb;
      if (col < a.K) a.carry_val[(size_t)s * kPanel + col] = carry[kb];
    }
  }
}

// Rows split between shares: the first share of every run of shares that left
// the same row open adds the run's partial sums, in share order, to that row
// (which the share after the run has written).
template <int KB>
__global__ void __launch_bounds__(256) spmm_fixup_kernel(SpmmArgs a) {
  const int lane = threadIdx.x & 31;
  const int nwarps = gridDim.x * 8;
  for (int s = blockIdx.x * 8 + (threadIdx.x >> 5); s < a.num_shares; s += nwarps) {
    const int r = a.carry_row[s];
    if (r < 0 || (s > 0 && a.carry_row[s - 1] == r)) continue;
    float tot[KB];
#pragma unroll
    for (int kb = 0; kb < KB; ++kb) tot[kb] = 0.f;
    for (int t = s; t < a.num_shares && a.carry_row[t] == r; ++t) {
#pragma unroll
      for (int kb = 0; kb < KB; ++kb) {
        const int col = lane + 32 * kb;
        if (col < a.K) tot[kb] += a.carry_val[(size_t)t * kPanel + col];
      }
    }
    float* crow = a.C + (int64_t)r * a.ldc;
#pragma unroll
    for (int kb = 0; kb < KB; ++kb) {
      const int col = lane + 32 * kb;
      if (col < a.K) crow[col] = crow[col] + tot[kb];
    }
  }
}

// Listing 4 as printed: thread t takes row t (grid stride) and, for every
// column of B, sums the row's atoms in chunks of 256 added in order.
__global__ void __launch_bounds__(256) spmm_tm_kernel(const int32_t* __restrict__ rp, int32_t R,
                                                      const int32_t* __restrict__ idx, const float* __restrict__ val,
                                                      const float* __restrict__ B, int64_t ldb, float* __restrict__ C,
                                                      int64_t ldc, int K) {
  constexpr int CHUNK = 256;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < R; t += (int64_t)gridDim.x * blockDim.x) {
    const int b = __ldg(rp + t), e = __ldg(rp + t + 1);
    for (int col = 0; col < K; ++col) {
      float total = 0.f;
      for (int k0 = b; k0 < e; k0 += CHUNK) {
        const int k1 = min(e, k0 + CHUNK);
        float part = 0.f;
        for (int k = k0; k < k1; ++k) part += __ldg(val + k) * __ldg(B + (int64_t)__ldg(idx + k) * ldb + col);
        total += part;
      }
      C[t * ldc + col] = total;
    }
  }
}

int spmm_grid(int sms) {
  static int occ = 0;
  if (occ == 0) {
    int o = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, spmm_mp_kernel<4>, kBlock, 0) != cudaSuccess || o < 1) o = 1;
    occ = o;
  }
  return sms * occ;
}

template <int KB>
cudaError_t launch_panel(const SpmmArgs& a, int grid, cudaStream_t s) {
  spmm_mp_kernel<KB><<<grid, kBlock, 0, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  spmm_fixup_kernel<KB><<<std::max(1, std::min(grid, (a.num_shares + 7) / 8)), kBlock, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

extern "C" {

lb_status_t lb_prepare_spmm(lb_plan_t p, void* stream) {
  if (!p) {
    set_error("lb_prepare_spmm: NULL plan");
    return LB_ERR_INVALID_ARG;
  }
  if (p->is_batch) {
    set_error("lb_prepare_spmm: batch plans have no SpMM");
    return LB_ERR_UNSUPPORTED;
  }
  if (p->schedule != LB_MERGE_PATH || p->mm_ready) return LB_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // warp tiles of 252 items (items_per_thread 8), four static shares per warp
  LB_TRY(build_mp_table(p->mm, p->rp, p->num_tiles, p->num_atoms, 8, 0, p->num_sms, 0, nullptr, s, nullptr, nullptr,
                        0, 0, 4));
  const size_t shares = (size_t)p->mm.workers;
  cudaError_t e = cudaMalloc(&p->mm_carry_row, sizeof(int32_t) * shares);
  if (e == cudaSuccess) e = cudaMalloc(&p->mm_carry_val, sizeof(float) * shares * kPanel);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    p->mm.release();
    cudaFree(p->mm_carry_row);
    cudaFree(p->mm_carry_val);
    p->mm_carry_row = nullptr;
    p->mm_carry_val = nullptr;
    set_error(std::string("lb_prepare_spmm: ") + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? LB_ERR_OOM : LB_ERR_CUDA;
  }
  p->mm_ready = true;
  return LB_OK;
}

lb_status_t lb_spmm(lb_plan_t p, int32_t K, const int32_t* col_idx, const float* vals, const float* B, int64_t ldb,
                    float* C, int64_t ldc, void* stream) {
  if (!p) {
    set_error("lb_spmm: NULL plan");
    return LB_ERR_INVALID_ARG;
  }
  if (K < 0 || ldb < K || ldc < K || (p->num_tiles > 0 && K > 0 && !C) ||
      (p->num_atoms > 0 && K > 0 && (!col_idx || !vals || !B))) {
    set_error("lb_spmm: need K >= 0, ldb >= K, ldc >= K and buffers for nonzero sizes");
    return LB_ERR_INVALID_ARG;
  }
  if (p->is_batch) {
    set_error("lb_spmm: batch plans have no SpMM");
    return LB_ERR_UNSUPPORTED;
  }
  if (p->schedule != LB_MERGE_PATH && p->schedule != LB_THREAD_MAPPED) {
    set_error("lb_spmm: SpMM runs on merge-path and thread-mapped plans");
    return LB_ERR_UNSUPPORTED;
  }
  if (K == 0 || p->num_tiles == 0) return LB_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (p->schedule == LB_THREAD_MAPPED) {
    const int64_t blocks = ((int64_t)p->num_tiles + kBlock - 1) / kBlock;
    spmm_tm_kernel<<<(unsigned)blocks, kBlock, 0, s>>>(p->rp, p->num_tiles, col_idx, vals, B, ldb, C, ldc, K);
    LB_CUDA_TRY(cudaGetLastError());
    return LB_OK;
  }
  LB_TRY(lb_prepare_spmm(p, stream));
  const int grid = spmm_grid(p->num_sms);
  for (int col0 = 0; col0 < K; col0 += kPanel) {
    SpmmArgs a{};
    a.rp = p->rp;
    a.R = p->num_tiles;
    a.idx = col_idx;
    a.val = vals;
    a.B = B + col0;
    a.ldb = ldb;
    a.C = C + col0;
    a.ldc = ldc;
    a.K = std::min(kPanel, K - col0);
    a.splits = p->mm.splits;
    a.num_shares = p->mm.workers;
    a.tpc = p->mm.tiles_per_cta;
    a.items_per_tile = p->mm.items_per_tile;
    a.carry_row = p->mm_carry_row;
    a.carry_val = p->mm_carry_val;
    const int g = std::max(1, std::min(grid, (a.num_shares + 7) / 8));
    cudaError_t e = a.K <= 32 ? launch_panel<1>(a, g, s) : a.K <= 64 ? launch_panel<2>(a, g, s) : launch_panel<4>(a, g, s);
    LB_CUDA_TRY(e);
  }
  return LB_OK;
}

}  // extern "C"
