// CSR -> CSC transpose by a stable counting sort of the atoms by column, run on
// the device without floating point and without order-dependent atomics:
//   cp   = inclusive scan of a column histogram (integer atomics: the final
//          counts do not depend on their order),
//   perm = source atom of every CSC slot, from a stable LSD radix sort of the
//          (column, atom) pairs in 8-bit digits: per 4096-atom tile a digit
//          histogram, one exclusive scan over (digit, tile), then a stable
//          scatter in which each atom's rank among equal digits follows its
//          position (warp ranks from __match_any_sync, warps and rounds in
//          order),
//   riT  = row of the source atom, gathered from the atom->row map.
// Rows therefore ascend within every column and the result is bit-exact.
#include <algorithm>

#include "lb_internal.h"

namespace lbh {

namespace {

constexpr int kScanBlock = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanBlock * kScanItems;

constexpr int kRadixBlock = 256;
constexpr int kRadixItems = 16;
constexpr int kRadixTile = kRadixBlock * kRadixItems;
constexpr int kRadixWarps = kRadixBlock / 32;

__device__ __forceinline__ int block_incl_scan_int(int v, int* s_w) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int n = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += n;
  }
  if (lane == 31) s_w[warp] = v;
  __syncthreads();
  int before = 0;
  for (int w = 0; w < warp; ++w) before += s_w[w];
  __syncthreads();
  return v + before;
}

// per-tile totals
__global__ void scan_reduce_kernel(const int32_t* __restrict__ in, int64_t n, int32_t* __restrict__ sums) {
  __shared__ int s_w[kScanBlock / 32];
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  int acc = 0;
#pragma unroll
  for (int r = 0; r < kScanItems; ++r) {
    const int64_t i = base + (int64_t)r * kScanBlock + threadIdx.x;
    if (i < n) acc += in[i];
  }
  const int tot = block_incl_scan_int(acc, s_w);
  if (threadIdx.x == kScanBlock - 1) sums[blockIdx.x] = tot;
}

// scan of one tile (blocked: thread t owns items [t*16, t*16+16)) plus the tile's prefix
__global__ void scan_apply_kernel(const int32_t* __restrict__ in, int32_t* __restrict__ out, int64_t n,
                                  const int32_t* __restrict__ prefix, int inclusive) {
  __shared__ int s_w[kScanBlock / 32];
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int v[kScanItems];
  int acc = 0;
#pragma unroll
  for (int r = 0; r < kScanItems; ++r) {
    const int64_t i = base + r;
    v[r] = i < n ? in[i] : 0;
    acc += v[r];
  }
  const int incl = block_incl_scan_int(acc, s_w);
  int run = incl - acc + (prefix ? prefix[blockIdx.x] : 0);
#pragma unroll
  for (int r = 0; r < kScanItems; ++r) {
    const int64_t i = base + r;
    const int x = v[r];
    if (i < n) out[i] = inclusive ? run + x : run;
    run += x;
  }
}

__global__ void histogram_kernel(const int32_t* __restrict__ keys, int64_t n, int32_t* __restrict__ cnt) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(cnt + keys[i], 1);
}

__global__ void radix_upsweep_kernel(const int32_t* __restrict__ keys, int64_t n, int shift, int32_t* __restrict__ hist,
                                     int64_t ntiles) {
  __shared__ int s_cnt[256];
  s_cnt[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kRadixTile;
#pragma unroll 4
  for (int r = 0; r < kRadixItems; ++r) {
    const int64_t i = base + (int64_t)r * kRadixBlock + threadIdx.x;
    if (i < n) atomicAdd(&s_cnt[(keys[i] >> shift) & 255], 1);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = s_cnt[threadIdx.x];
}

// Stable scatter of one tile.  Warp w owns the tile's atoms w*512 + [0, 512),
// visited in 16 rounds of 32 consecutive atoms (so atom order is warp, round,
// lane order).  A first walk counts each warp's atoms per digit (peers from
// __match_any_sync, counts kept by the warp in shared memory, no block
// barrier); the counts give every (warp, digit) its offset inside the digit's
// run of the tile and every digit its start in the tile.  A second walk over
// the same atoms (keys kept in registers, values read now) ranks them again
// and places each at its slot of the tile, ordered by digit, in shared
// memory; the tile is then written out run by run, each digit's run to its
// global start, so the stores of neighbouring threads land on neighbouring
// addresses.
__global__ void __launch_bounds__(kRadixBlock, 4) radix_downsweep_kernel(
    const int32_t* __restrict__ keys_in, const int32_t* __restrict__ vals_in, int64_t n, int shift,
    const int32_t* __restrict__ hist_scan, int64_t ntiles, int32_t* __restrict__ keys_out,
    int32_t* __restrict__ vals_out) {
  constexpr int kPerWarp = 32 * kRadixItems;
  __shared__ int s_base[256];             // global start of each digit's run of this tile
  __shared__ int s_loc[256];              // start of each digit's run inside the tile
  __shared__ int s_cnt[kRadixWarps][256];  // a warp's atoms per digit, then its offset in the run
  __shared__ int s_w[kRadixWarps];
  __shared__ int2 s_kv[kRadixTile];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned lt = (1u << lane) - 1u;
  s_base[tid] = hist_scan[(int64_t)tid * ntiles + blockIdx.x];
#pragma unroll
  for (int w = 0; w < kRadixWarps; ++w) s_cnt[w][tid] = 0;
  __syncthreads();
  const int64_t tbase = (int64_t)blockIdx.x * kRadixTile;
  const int64_t wbase = tbase + (int64_t)warp * kPerWarp;
  int key[kRadixItems];
#pragma unroll
  for (int r = 0; r < kRadixItems; ++r) {
    const int64_t i = wbase + r * 32 + lane;
    const bool valid = i < n;
    key[r] = valid ? keys_in[i] : 0;
    const int d = valid ? ((key[r] >> shift) & 255) : 256;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    if (valid && __popc(peers & lt) == 0) s_cnt[warp][d] += __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // thread tid = digit: offsets of the warps inside the digit's run, and the run's start in the tile
  int tot = 0;
#pragma unroll
  for (int w = 0; w < kRadixWarps; ++w) {
    const int c = s_cnt[w][tid];
    s_cnt[w][tid] = tot;
    tot += c;
  }
  s_loc[tid] = block_incl_scan_int(tot, s_w) - tot;
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kRadixItems; ++r) {
    const int64_t i = wbase + r * 32 + lane;
    const bool valid = i < n;
    const int d = valid ? ((key[r] >> shift) & 255) : 256;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const int rank = __popc(peers & lt);
    const int off = valid ? s_cnt[warp][d] : 0;
    __syncwarp();
    if (valid) {
      s_kv[s_loc[d] + off + rank] = make_int2(key[r], vals_in ? vals_in[i] : (int)i);
      if (rank == 0) s_cnt[warp][d] = off + __popc(peers);
    }
    __syncwarp();
  }
  __syncthreads();
  const int64_t left = n - tbase;
  const int count = left < kRadixTile ? (int)left : kRadixTile;
  for (int p = tid; p < count; p += kRadixBlock) {
    const int2 kv = s_kv[p];
    const int d = (kv.x >> shift) & 255;
    const int pos = s_base[d] + (p - s_loc[d]);
    keys_out[pos] = kv.x;
    vals_out[pos] = kv.y;
  }
}

__global__ void gather_kernel(const int32_t* __restrict__ src, const int32_t* __restrict__ idx, int64_t n,
                              int32_t* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = src[idx[i]];
}

__global__ void iota_kernel(int32_t* out, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (int32_t)i;
}

unsigned grid_for(int64_t n, int threads) {
  int64_t b = (n + threads - 1) / threads;
  if (b > 65536 * 8) b = 65536 * 8;
  if (b < 1) b = 1;
  return (unsigned)b;
}

struct DevBuf {
  void* p = nullptr;
  ~DevBuf() { cudaFree(p); }
};

}  // namespace

namespace {

// entries of scratch a scan of n items needs: the tile totals of every level above the first
int64_t scan_scratch(int64_t n) {
  int64_t t = 0;
  while (n > kScanTile) {
    n = (n + kScanTile - 1) / kScanTile;
    t += n;
  }
  return t;
}

// scan of n items with the tile totals in caller scratch (scan_scratch(n) entries): launches only
void scan_into(const int32_t* in, int32_t* out, int64_t n, bool inclusive, int32_t* scratch, cudaStream_t s) {
  if (n <= 0) return;
  const int64_t tiles = (n + kScanTile - 1) / kScanTile;
  if (tiles == 1) {
    scan_apply_kernel<<<1, kScanBlock, 0, s>>>(in, out, n, nullptr, inclusive ? 1 : 0);
    return;
  }
  scan_reduce_kernel<<<(unsigned)tiles, kScanBlock, 0, s>>>(in, n, scratch);
  scan_into(scratch, scratch, tiles, false, scratch + tiles, s);
  scan_apply_kernel<<<(unsigned)tiles, kScanBlock, 0, s>>>(in, out, n, scratch, inclusive ? 1 : 0);
}

}  // namespace

lb_status_t device_scan(const int32_t* in, int32_t* out, int64_t n, bool inclusive, cudaStream_t s) {
  if (n <= 0) return LB_OK;
  const int64_t need = scan_scratch(n);
  DevBuf sums;
  if (need > 0) LB_CUDA_TRY(cudaMalloc(&sums.p, sizeof(int32_t) * (size_t)need));
  scan_into(in, out, n, inclusive, static_cast<int32_t*>(sums.p), s);
  LB_CUDA_TRY(cudaGetLastError());
  // `sums` is freed when this returns; make sure the kernels using it are done
  if (need > 0) LB_CUDA_TRY(cudaStreamSynchronize(s));
  return LB_OK;
}

// One device allocation holds the sort's key and value buffers, its digit histograms and the scans'
// tile totals; nothing synchronises until the sort is done.
lb_status_t transpose_sort(const int32_t* keys, const int32_t* row_of, int64_t N, int32_t C, int32_t* cp,
                           int32_t* riT, int32_t* perm, cudaStream_t s) {
  LB_CUDA_TRY(cudaMemsetAsync(cp, 0, sizeof(int32_t) * ((size_t)C + 1), s));
  if (N == 0) return LB_OK;
  int bits = 0;
  while (bits < 31 && ((int64_t)1 << bits) < (int64_t)C) ++bits;
  const int passes = (bits + 7) / 8;
  const int64_t ntiles = (N + kRadixTile - 1) / kRadixTile;
  const int64_t nhist = passes > 0 ? 256 * ntiles : 0;
  const int64_t nscan = std::max(scan_scratch(C), scan_scratch(nhist));
  const int64_t nsort = passes > 0 ? 4 * N : 0;
  DevBuf buf;
  LB_CUDA_TRY(cudaMalloc(&buf.p, sizeof(int32_t) * (size_t)std::max<int64_t>(1, nsort + nhist + nscan)));
  int32_t* base = static_cast<int32_t*>(buf.p);
  int32_t* kbuf[2] = {base, base + N};
  int32_t* vbuf[2] = {base + 2 * N, base + 3 * N};
  int32_t* hist = base + nsort;
  int32_t* scratch = hist + nhist;
  // cp: histogram of keys into cp[1..C], then inclusive scan
  histogram_kernel<<<grid_for(N, 256), 256, 0, s>>>(keys, N, cp + 1);
  scan_into(cp + 1, cp + 1, C, true, scratch, s);
  LB_CUDA_TRY(cudaGetLastError());
  if (passes == 0) {
    iota_kernel<<<grid_for(N, 256), 256, 0, s>>>(perm, N);
  } else {
    const int32_t* kin = keys;
    const int32_t* vin = nullptr;  // first pass: values are the atom indices
    for (int p = 0; p < passes; ++p) {
      const int shift = 8 * p;
      int32_t* kout = kbuf[p & 1];
      int32_t* vout = (p == passes - 1) ? perm : vbuf[p & 1];
      radix_upsweep_kernel<<<(unsigned)ntiles, kRadixBlock, 0, s>>>(kin, N, shift, hist, ntiles);
      scan_into(hist, hist, nhist, false, scratch, s);
      radix_downsweep_kernel<<<(unsigned)ntiles, kRadixBlock, 0, s>>>(kin, vin, N, shift, hist, ntiles, kout, vout);
      kin = kout;
      vin = vout;
    }
  }
  LB_CUDA_TRY(cudaGetLastError());
  gather_kernel<<<grid_for(N, 256), 256, 0, s>>>(row_of, perm, N, riT);
  LB_CUDA_TRY(cudaGetLastError());
  // `buf` is freed when this returns
  LB_CUDA_TRY(cudaStreamSynchronize(s));
  return LB_OK;
}

}  // namespace lbh
