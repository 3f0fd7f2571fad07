// Single-source shortest paths (Sec. 7, Listing 5) on the group-mapped
// schedule: every iteration the frontier's vertices are the tiles and their
// out-edges the atoms; a group of G threads takes G frontier vertices,
// prefix-sums their degrees in shared memory and walks the flattened edges
// with stride G, finding each edge's vertex with get_tile (a binary search in
// the prefix, Sec. 5.2.3).  Each edge relaxes its head with an atomic minimum
// on the distance's bits (non-negative floats order like their bit patterns),
// issued without waiting for its result, eight edges per thread at a time.  A
// pass over the vertices then puts every vertex whose distance dropped in this
// iteration on the next frontier (its distance at the previous pass is kept
// beside it).  The host loops until the frontier is empty.  The distances are
// the least fixed point of dist[v] = min over edges (u, v) of fl32(dist[u] +
// w), whatever order the relaxations take, so they are deterministic.
#include <algorithm>
#include <cmath>
#include <string>
#include <utility>

#include "lb_internal.h"
#include "lb_kernels.cuh"

using namespace lbh;

namespace {

// every edge's head inside [0, V) and weight finite and non-negative
__global__ void sssp_check_edges_kernel(const int32_t* __restrict__ col, const float* __restrict__ w, int64_t E,
                                        int32_t V, int* bad) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < E; k += (int64_t)gridDim.x * blockDim.x) {
    const float x = w[k];
    if (!(x >= 0.f) || isinf(x) || (unsigned)col[k] >= (unsigned)V) atomicOr(bad, 1);
  }
}

__global__ void sssp_init_kernel(int* __restrict__ dist_bits, int* __restrict__ prev_bits, int32_t V,
                                 int32_t source, int32_t* front) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < V; v += (int64_t)gridDim.x * blockDim.x) {
    const int d = v == source ? 0 : 0x7f800000;  // +0, +inf
    dist_bits[v] = d;
    prev_bits[v] = d;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) front[0] = source;
}

template <int BLOCK, int G>
__global__ void __launch_bounds__(BLOCK) sssp_relax_kernel(const int32_t* __restrict__ rp,
                                                           const int32_t* __restrict__ col,
                                                           const float* __restrict__ w, int* dist_bits,
                                                           const int32_t* __restrict__ front, int32_t nfront) {
  constexpr int GPB = BLOCK / G;             // groups per block
  constexpr int WPG = G >= 32 ? G / 32 : 1;  // warps per group
  constexpr int SW = G < 32 ? G : 32;        // shuffle width
  constexpr int R = 8;                       // edges per thread in flight (4: R-MAT warps 31 ms, 8: 26 ms)
  __shared__ int s_pre[GPB][G + 1];
  __shared__ int s_base[GPB][G];
  __shared__ float s_dist[GPB][G];
  __shared__ int s_wsum[GPB][WPG];
  const int g = threadIdx.x / G;
  const int lane = threadIdx.x % G;
  const int sl = threadIdx.x % SW;
  const int wg = lane / 32;

  auto group_sync = [&]() {
    if constexpr (G <= 32) {
      __syncwarp();
    } else if constexpr (G == BLOCK) {
      __syncthreads();
    } else {
      asm volatile("bar.sync %0, %1;" ::"r"(g + 1), "r"(G) : "memory");
    }
  };

  for (int64_t bc = blockIdx.x; bc * GPB * G < nfront; bc += gridDim.x) {
    const int64_t t0 = (bc * GPB + g) * G;
    const int64_t t = t0 + lane;
    const int u = t < nfront ? front[t] : -1;
    int len = 0;
    if (u >= 0) {
      const int b = __ldg(rp + u);
      len = __ldg(rp + u + 1) - b;
      s_base[g][lane] = b;
      // a relaxed read: a distance lowered meanwhile puts u back on the next frontier
      s_dist[g][lane] = __int_as_float(__ldcg(dist_bits + u));
    }
    int wtotal;
    int ex = lbk::group_excl_scan_small<SW>(len, sl, wtotal);
    if constexpr (G > 32) {
      if (sl == 0) s_wsum[g][wg] = wtotal;
      group_sync();
      int before = 0;
      for (int q = 0; q < wg; ++q) before += s_wsum[g][q];
      ex += before;
    }
    s_pre[g][lane] = ex;
    if (lane == G - 1) s_pre[g][G] = ex + len;
    group_sync();
    const int total = s_pre[g][G];
    for (int a0 = lane; a0 < total; a0 += R * G) {
      int k[R], lo[R];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int aa = a0 + r * G;
        k[r] = -1;
        lo[r] = 0;
        if (aa < total) {
          int l = 0, hi = G - 1;  // get_tile: the largest tile whose prefix is <= aa
          while (l < hi) {
            const int mid = (l + hi + 1) >> 1;
            if (s_pre[g][mid] <= aa) l = mid;
            else hi = mid - 1;
          }
          lo[r] = l;
          k[r] = s_base[g][l] + (aa - s_pre[g][l]);
        }
      }
      int head[R];
      float wt[R];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        head[r] = k[r] >= 0 ? __ldg(col + k[r]) : 0;
        wt[r] = k[r] >= 0 ? __ldg(w + k[r]) : 0.f;
      }
      // block-wide groups first read the heads' distances (relaxed reads: distances only fall, so a
      // value read bounds the current one from above) and skip the minima that cannot lower them,
      // which R-MAT's hub vertices would otherwise draw by the thousand on one address (R-MAT,
      // groups of 256: 13.4 -> 11.0 ms); narrower groups measured slower with the extra read
      int cur[R];
#pragma unroll
      for (int r = 0; r < R; ++r) cur[r] = (G == BLOCK && k[r] >= 0) ? __ldcg(dist_bits + head[r]) : 0x7f800000;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const float nd = s_dist[g][lo[r]] + wt[r];
        if (k[r] >= 0 && (G != BLOCK || nd < __int_as_float(cur[r]))) atomicMin(dist_bits + head[r], __float_as_int(nd));
      }
    }
    group_sync();
  }
}

// The next frontier: every vertex whose distance dropped since the last pass,
// appended with one counter update per warp; its distance at this pass is kept.
__global__ void sssp_frontier_kernel(const int* __restrict__ dist_bits, int* __restrict__ prev_bits, int32_t V,
                                     int32_t* next, int32_t* next_count) {
  const int wl = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v0 = blockIdx.x * (int64_t)blockDim.x; v0 < V; v0 += stride) {
    const int64_t v = v0 + threadIdx.x;
    bool push = false;
    if (v < V) {
      const int d = __ldcg(dist_bits + v);
      if (d < prev_bits[v]) {
        prev_bits[v] = d;
        push = true;
      }
    }
    const unsigned m = __ballot_sync(lbk::kFull, push);
    if (m) {
      int base = 0;
      const int leader = __ffs(m) - 1;
      if (wl == leader) base = atomicAdd(next_count, __popc(m));
      base = __shfl_sync(lbk::kFull, base, leader);
      if (push) next[base + __popc(m & ((1u << wl) - 1u))] = (int32_t)v;
    }
  }
}

template <int G>
void relax_launch(int64_t blocks, const int32_t* rp, const int32_t* col, const float* w, int* dist_bits,
                  const int32_t* front, int32_t n, cudaStream_t s) {
  sssp_relax_kernel<kBlock, G><<<(unsigned)blocks, kBlock, 0, s>>>(rp, col, w, dist_bits, front, n);
}

}  // namespace

extern "C" {

lb_status_t lb_sssp(const int32_t* tile_offsets, int32_t num_vertices, int32_t num_edges, const int32_t* col_idx,
                    const float* weights, int32_t source, int32_t group_size, float* dist, int32_t* host_iterations,
                    void* stream) {
  if (host_iterations) *host_iterations = 0;
  const int G = group_size ? group_size : 32;
  if (num_vertices < 0 || num_edges < 0 || (num_vertices > 0 && (!tile_offsets || !dist)) ||
      (num_edges > 0 && (!col_idx || !weights)) || (num_vertices > 0 && (source < 0 || source >= num_vertices))) {
    set_error("lb_sssp: need sizes >= 0, buffers for nonzero sizes and 0 <= source < num_vertices");
    return LB_ERR_INVALID_ARG;
  }
  if (G < 4 || G > 256 || (G & (G - 1))) {
    set_error("lb_sssp: group_size must be a power of two in [4, 256]");
    return LB_ERR_UNSUPPORTED;
  }
  if (num_vertices == 0) return LB_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int V = num_vertices;
  int dev = 0;
  LB_CUDA_TRY(cudaGetDevice(&dev));
  const int sms = device_sms(dev);
  // scratch: the distances at the last frontier pass, two frontier lists, the next-frontier count and
  // the weight check
  void* buf = nullptr;
  const size_t vbytes = sizeof(int) * (size_t)V;
  LB_CUDA_TRY(cudaMalloc(&buf, 3 * vbytes + 256));
  struct Free {
    void* p;
    ~Free() { cudaFree(p); }
  } guard{buf};
  int* prev_bits = static_cast<int*>(buf);
  int32_t* lists[2] = {static_cast<int32_t*>(buf) + (size_t)V, static_cast<int32_t*>(buf) + 2 * (size_t)V};
  int32_t* counters = reinterpret_cast<int32_t*>(static_cast<char*>(buf) + 3 * vbytes);  // [0] next count, [1] bad
  LB_CUDA_TRY(cudaMemsetAsync(counters, 0, 256, s));
  if (num_edges > 0) {
    const unsigned wb = (unsigned)std::min<int64_t>(((int64_t)num_edges + 255) / 256, (int64_t)sms * 32);
    sssp_check_edges_kernel<<<wb, 256, 0, s>>>(col_idx, weights, num_edges, V, counters + 1);
    LB_CUDA_TRY(cudaGetLastError());
  }
  int* dist_bits = reinterpret_cast<int*>(dist);
  const unsigned ib = (unsigned)std::min<int64_t>(((int64_t)V + 255) / 256, (int64_t)sms * 32);
  sssp_init_kernel<<<ib, 256, 0, s>>>(dist_bits, prev_bits, V, source, lists[0]);
  LB_CUDA_TRY(cudaGetLastError());
  int bad = 0;
  LB_CUDA_TRY(cudaMemcpyAsync(&bad, counters + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
  LB_CUDA_TRY(cudaStreamSynchronize(s));
  if (bad) {
    set_error("lb_sssp: edge heads must lie in [0, num_vertices) and weights be finite and non-negative");
    return LB_ERR_INVALID_ARG;
  }
  int32_t n = 1;
  int cur = 0, it = 0;
  // Bellman-Ford bound: every iteration settles at least one more vertex
  while (n > 0) {
    if (it > V) {
      set_error("lb_sssp: frontier did not empty within num_vertices iterations");
      return LB_ERR_CUDA;
    }
    LB_CUDA_TRY(cudaMemsetAsync(counters, 0, sizeof(int32_t), s));
    const int gpb = kBlock / G;
    int64_t blocks = ((int64_t)n + (int64_t)gpb * G - 1) / ((int64_t)gpb * G);
    blocks = std::min<int64_t>(blocks, (int64_t)sms * 64);
    const int nx = 1 - cur;
    switch (G) {
      case 4: relax_launch<4>(blocks, tile_offsets, col_idx, weights, dist_bits, lists[cur], n, s); break;
      case 8: relax_launch<8>(blocks, tile_offsets, col_idx, weights, dist_bits, lists[cur], n, s); break;
      case 16: relax_launch<16>(blocks, tile_offsets, col_idx, weights, dist_bits, lists[cur], n, s); break;
      case 32: relax_launch<32>(blocks, tile_offsets, col_idx, weights, dist_bits, lists[cur], n, s); break;
      case 64: relax_launch<64>(blocks, tile_offsets, col_idx, weights, dist_bits, lists[cur], n, s); break;
      case 128: relax_launch<128>(blocks, tile_offsets, col_idx, weights, dist_bits, lists[cur], n, s); break;
      default: relax_launch<256>(blocks, tile_offsets, col_idx, weights, dist_bits, lists[cur], n, s); break;
    }
    LB_CUDA_TRY(cudaGetLastError());
    sssp_frontier_kernel<<<ib, 256, 0, s>>>(dist_bits, prev_bits, V, lists[nx], counters);
    LB_CUDA_TRY(cudaGetLastError());
    LB_CUDA_TRY(cudaMemcpyAsync(&n, counters, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    LB_CUDA_TRY(cudaStreamSynchronize(s));
    cur = nx;
    ++it;
  }
  if (host_iterations) *host_iterations = it;
  return LB_OK;
}

}  // extern "C"
