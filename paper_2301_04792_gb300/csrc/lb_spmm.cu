// SpMM C = A B for a dense row-major B (Sec. 7, Listing 4: the SpMV loop with
// one more loop over the columns of B), on two of the paper's schedules:
//  - merge-path: a warp per share of rows + atoms (the split table of Sec.
//    5.2.1 with warp tiles), the lanes holding the columns of B; per tile the
//    atoms and row ends are staged in shared memory and summed (with 16-byte
//    rows of B, by lane groups over contiguous runs of the tile's atoms; else
//    row by row with several rows of B in flight), and the row left open at
//    the share's end is finished by a second launch that adds the partial sums
//    of each run of shares to the row that closes it, in share order;
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
  constexpr int U = KB == 1 ? 16 : 8;  // rows of B in flight per lane
  __shared__ int s_ci[WPB][kTileCap];
  __shared__ float s_v[WPB][kTileCap];
  __shared__ int s_mark[WPB][kTileCap];   // row (local) that ends at this atom, -1 if none
  __shared__ int s_empty[WPB][kTileCap];  // rows (local, > 0) with no atoms in the tile
  __shared__ int s_nempty[WPB];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int* ci_s = s_ci[warp];
  float* v_s = s_v[warp];
  int* mark_s = s_mark[warp];
  int* empty_s = s_empty[warp];
  const int nwarps = gridDim.x * WPB;
  auto store_row = [&](int row, const float (&val)[KB]) {
    float* crow = a.C + (int64_t)row * a.ldc;
#pragma unroll
    for (int kb = 0; kb < KB; ++kb) {
      const int col = lane + 32 * kb;
      if (col < a.K) crow[col] = val[kb];
    }
  };
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
      // stage the tile's atoms; mark the atom each closing row ends at
      for (int i = lane; i < nnz; i += 32) {
        ci_s[i] = lbk::ld_stream(a.idx + c0.y + i);
        v_s[i] = lbk::ld_stream(a.val + c0.y + i);
        mark_s[i] = -1;
      }
      if (lane == 0) s_nempty[warp] = 0;
      __syncwarp();
      bool first_empty = false;  // row 0 closes at the tile's start with no atoms here
      for (int rb = 0; rb < nrows; rb += 32) {
        const int r = rb + lane;
        int e = 0, pe = 0;
        if (r < nrows) {
          e = __ldg(a.rp + c0.x + 1 + r) - c0.y;
          pe = r == 0 ? 0 : __ldg(a.rp + c0.x + r) - c0.y;
        }
        const bool has = r < nrows && e > pe;
        if (has) mark_s[e - 1] = r;
        const bool empty = r < nrows && !has;
        if (empty && r == 0) first_empty = true;
        const unsigned em = __ballot_sync(lbk::kFull, empty && r > 0);
        if (empty && r > 0) empty_s[s_nempty[warp] + __popc(em & ((1u << lane) - 1u))] = r;
        __syncwarp();
        if (lane == 0) s_nempty[warp] += __popc(em);
        __syncwarp();
      }
      first_empty = __any_sync(lbk::kFull, first_empty);
      if (first_empty) {  // its value is the earlier tiles' partial sum
        store_row(c0.x, carry);
#pragma unroll
        for (int kb = 0; kb < KB; ++kb) carry[kb] = 0.f;
      }
      {
        float zero[KB];
#pragma unroll
        for (int kb = 0; kb < KB; ++kb) zero[kb] = 0.f;
        const int ne = s_nempty[warp];
        for (int q = 0; q < ne; ++q) store_row(c0.x + empty_s[q], zero);
      }
      // the atoms in order, U rows of B in flight; a marked atom closes its row
      // (row 0 gets the earlier tiles' partial sum in front of its own)
      float p[KB];
#pragma unroll
      for (int kb = 0; kb < KB; ++kb) p[kb] = 0.f;
      for (int q0 = 0; q0 < nnz; q0 += U) {
        float bq[U][KB];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int q = q0 + u;
          const float* brow = a.B + (int64_t)(q < nnz ? ci_s[q] : 0) * a.ldb;
#pragma unroll
          for (int kb = 0; kb < KB; ++kb) {
            const int col = lane + 32 * kb;
            bq[u][kb] = (q < nnz && col < a.K) ? __ldg(brow + col) : 0.f;
          }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int q = q0 + u;
          if (q < nnz) {
            const float w = v_s[q];
#pragma unroll
            for (int kb = 0; kb < KB; ++kb) p[kb] += w * bq[u][kb];
            const int r = mark_s[q];
            if (r >= 0) {
              if (r == 0) {
#pragma unroll
                for (int kb = 0; kb < KB; ++kb) p[kb] = carry[kb] + p[kb];
              }
              store_row(c0.x + r, p);
#pragma unroll
              for (int kb = 0; kb < KB; ++kb) p[kb] = 0.f;
            }
          }
        }
      }
      // the row open at the tile's end: its partial joins the running sum
      if (nrows == 0) {
#pragma unroll
        for (int kb = 0; kb < KB; ++kb) carry[kb] = carry[kb] + p[kb];
      } else {
#pragma unroll
        for (int kb = 0; kb < KB; ++kb) carry[kb] = p[kb];
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

// The same shares with 16-byte rows of B: lane l holds columns 4 (l mod CL) ..
// 4 (l mod CL) + 3 of the panel, so a row of B is CL float4 loads, and the
// warp's G = 32 / CL lane groups split each tile's atoms into G contiguous
// runs, the way the SpMV warp walker splits them over its lanes: a group sums
// its run in atom order with U rows of B in flight and closes a row at each
// atom that ends one (marked in the row pass).  A row closed inside a group's
// run is stored at once; the first row a group closes, and the row left open
// at its run's end, are finished by a segmented scan over the groups in order
// with the running carry in front (Hillis-Steele steps, a fixed tree).  Every
// group keeps its gathers in flight whatever the rows' lengths, instead of one
// row's gathers at a time (power-law 1M: K = 8 437 -> 249 us, K = 32 649 ->
// 482 us, K = 128 unchanged at 1.54 ms, where B's rows come from HBM).  Needs
// B, C 16-byte aligned, ldb, ldc and the panel width multiples of 4.
template <int CL>
__global__ void __launch_bounds__(256) spmm_mp_vec_kernel(SpmmArgs a) {
  constexpr int WPB = 8;
  constexpr int G = 32 / CL;
  constexpr int U = 4;
  __shared__ int2 s_cv[WPB][kTileCap];
  __shared__ int s_mark[WPB][kTileCap];  // local row whose last atom this is, -1 if none
  __shared__ int s_end[WPB][kTileCap];   // local end (exclusive) of each row of the tile
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane / CL, col = 4 * (lane % CL);
  const bool active = col < a.K;
  int2* cv_s = s_cv[warp];
  int* mark_s = s_mark[warp];
  int* end_s = s_end[warp];
  const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
  auto add4 = [](float4 x, float4 y) { return make_float4(x.x + y.x, x.y + y.y, x.z + y.z, x.w + y.w); };
  auto shfl_up4 = [](float4 v, int d) {
    return make_float4(__shfl_up_sync(lbk::kFull, v.x, d), __shfl_up_sync(lbk::kFull, v.y, d),
                       __shfl_up_sync(lbk::kFull, v.z, d), __shfl_up_sync(lbk::kFull, v.w, d));
  };
  auto store4 = [&](int row, float4 v) {
    if (active) *reinterpret_cast<float4*>(a.C + (int64_t)row * a.ldc + col) = v;
  };
  const int nwarps = gridDim.x * WPB;
  for (int s = blockIdx.x * WPB + warp; s < a.num_shares; s += nwarps) {
    const int2* sp = a.splits + (size_t)s * (a.tpc + 1);
    int2 c0 = __ldg(sp);
    const int2 e1 = __ldg(sp + a.tpc);
    const int ntiles = (int)(((int64_t)(e1.x - c0.x) + (e1.y - c0.y) + a.items_per_tile - 1) / a.items_per_tile);
    float4 carry = zero;
    for (int k = 0; k < ntiles; ++k) {
      const int2 c1 = __ldg(sp + k + 1);
      const int nnz = c1.y - c0.y, nrows = c1.x - c0.x;
      for (int i = lane; i < nnz; i += 32) {
        cv_s[i] = make_int2(lbk::ld_stream(a.idx + c0.y + i), __float_as_int(lbk::ld_stream(a.val + c0.y + i)));
        mark_s[i] = -1;
      }
      for (int i = lane; i < nrows; i += 32) end_s[i] = __ldg(a.rp + c0.x + 1 + i) - c0.y;
      __syncwarp();
      // row pass: a row with atoms in the tile marks its last one; a row with none gets 0, or
      // the carry if it is the tile's first row (it closes where the tile starts)
      for (int r = lane; r < nrows; r += 32) {
        const int e = end_s[r], pe = r > 0 ? end_s[r - 1] : 0;
        if (e > pe) mark_s[e - 1] = r;
      }
      for (int r = g; r < nrows; r += G) {
        const int e = end_s[r], pe = r > 0 ? end_s[r - 1] : 0;
        if (e == pe) store4(c0.x + r, r == 0 ? carry : zero);
      }
      __syncwarp();
      // this group's run of atoms
      const int per = (nnz + G - 1) / G;
      const int qa = g * per, qb = min(nnz, qa + per);
      float4 acc = zero, head = zero;
      int first = -1;
      for (int q0 = qa; q0 < qb; q0 += U) {
        float4 bq[U];
        float w[U];
        int mk[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int q = q0 + u;
          w[u] = 0.f;
          mk[u] = -1;
          bq[u] = zero;
          if (q < qb) {
            const int2 cv = cv_s[q];
            w[u] = __int_as_float(cv.y);
            mk[u] = mark_s[q];
            if (active) bq[u] = __ldg(reinterpret_cast<const float4*>(a.B + (int64_t)cv.x * a.ldb + col));
          }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          acc.x += w[u] * bq[u].x;
          acc.y += w[u] * bq[u].y;
          acc.z += w[u] * bq[u].z;
          acc.w += w[u] * bq[u].w;
          if (mk[u] >= 0) {
            if (first < 0) {
              head = acc;
              first = mk[u];
            } else {
              store4(c0.x + mk[u], acc);
            }
            acc = zero;
          }
        }
      }
      // segmented scan over the groups: the partial sum of the row open at each group's end
      // (reset where a group closed a row), then the carry in front of the groups before the
      // first reset -- unless the tile's first row closed where the tile starts and took it
      const float4 cin = nrows > 0 && end_s[0] == 0 ? zero : carry;
      float4 v = acc;
      int f = first >= 0;
#pragma unroll
      for (int o = 1; o < G; o <<= 1) {
        const float4 vo = shfl_up4(v, o * CL);
        const int fo = __shfl_up_sync(lbk::kFull, f, o * CL);
        if (g >= o) {
          if (!f) v = add4(vo, v);
          f |= fo;
        }
      }
      if (!f) v = add4(cin, v);
      float4 in = shfl_up4(v, CL);
      if (g == 0) in = cin;
      if (first >= 0) store4(c0.x + first, add4(in, head));
      const int src = (G - 1) * CL + (lane % CL);
      carry = make_float4(__shfl_sync(lbk::kFull, v.x, src), __shfl_sync(lbk::kFull, v.y, src),
                          __shfl_sync(lbk::kFull, v.z, src), __shfl_sync(lbk::kFull, v.w, src));
      __syncwarp();
      c0 = c1;
    }
    if (lane == 0) a.carry_row[s] = c0.x < a.R ? c0.x : -1;
    if (g == 0 && active) *reinterpret_cast<float4*>(a.carry_val + (size_t)s * kPanel + col) = carry;
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

template <int KB>
int spmm_grid(int sms) {
  static int occ = 0;  // per instantiation
  if (occ == 0) {
    int o = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, spmm_mp_kernel<KB>, kBlock, 0) != cudaSuccess || o < 1) o = 1;
    occ = o;
  }
  return sms * occ;
}

template <int CL>
int spmm_vec_grid(int sms) {
  static int occ = 0;  // per instantiation
  if (occ == 0) {
    int o = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, spmm_mp_vec_kernel<CL>, kBlock, 0) != cudaSuccess || o < 1)
      o = 1;
    occ = o;
  }
  return sms * occ;
}

template <int CL>
cudaError_t launch_vec_panel(const SpmmArgs& a, int sms, cudaStream_t s) {
  const int grid = std::max(1, std::min(spmm_vec_grid<CL>(sms), (a.num_shares + 7) / 8));
  spmm_mp_vec_kernel<CL><<<grid, kBlock, 0, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // the fix-up reads the carries column by column (its layout is the same)
  spmm_fixup_kernel<CL <= 8 ? 1 : CL / 8><<<grid, kBlock, 0, s>>>(a);
  return cudaGetLastError();
}

template <int KB>
cudaError_t launch_panel(const SpmmArgs& a, int sms, cudaStream_t s) {
  const int grid = std::max(1, std::min(spmm_grid<KB>(sms), (a.num_shares + 7) / 8));
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
    const bool vec = ((reinterpret_cast<uintptr_t>(a.B) | reinterpret_cast<uintptr_t>(a.C)) & 15u) == 0 &&
                     (ldb & 3) == 0 && (ldc & 3) == 0 && (a.K & 3) == 0;
    cudaError_t e;
    if (vec) {
      const int cl = (a.K + 3) / 4;  // float4 lanes per row of the panel
      e = cl <= 2    ? launch_vec_panel<2>(a, p->num_sms, s)
          : cl <= 4  ? launch_vec_panel<4>(a, p->num_sms, s)
          : cl <= 8  ? launch_vec_panel<8>(a, p->num_sms, s)
          : cl <= 16 ? launch_vec_panel<16>(a, p->num_sms, s)
                     : launch_vec_panel<32>(a, p->num_sms, s);
    } else {
      e = a.K <= 32   ? launch_panel<1>(a, p->num_sms, s)
          : a.K <= 64 ? launch_panel<2>(a, p->num_sms, s)
                      : launch_panel<4>(a, p->num_sms, s);
    }
    LB_CUDA_TRY(e);
  }
  return LB_OK;
}

}  // extern "C"
