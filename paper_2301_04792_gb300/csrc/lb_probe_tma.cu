// Roofline probe of the other gather path on sm_100-class GPUs: TMA row
// gathers (cp.async.bulk.tensor ... tile::gather4) of the dense vector into
// shared memory, for comparison with the plain load-unit gathers of
// lb_probe_gather.  Measurement only; no SpMV schedule uses it.
//
// The dense vector x is seen by the tensor map as rows of 8 floats (32 bytes,
// one L2 sector); a gather4 copies four such rows, chosen by row coordinate
// idx >> 3, into 128 bytes of shared memory, and the thread picks element
// idx & 7 of each.  A warp handles 128 atoms per step (an int4 of indices per
// lane), one gather4 per lane, into a ring of two 4 KB slots per warp whose
// completion is counted on one mbarrier per slot.  Every wait is bounded and
// reports kDevErrTimeout through `err` instead of hanging.
#include <cuda.h>

#include <cstring>
#include <mutex>
#include <string>

#include "lb_internal.h"
#include "lb_kernels.cuh"

using namespace lbh;

namespace {

constexpr int kTmaWarps = 8;    // warps per CTA
constexpr int kTmaStages = 2;   // ring slots per warp
constexpr int kSlotBytes = 32 * 128;
constexpr int kTmaSmem = kTmaWarps * kTmaStages * kSlotBytes;

__device__ __forceinline__ void gather4_rows(void* dst, const CUtensorMap* tm, int r0, int r1, int r2, int r3,
                                             uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile::gather4.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(lbk::smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(0), "r"(r0), "r"(r1), "r"(r2), "r"(r3), "r"(lbk::smem_u32(bar))
      : "memory");
}

// atoms [0, 128 * nchunks); the tensor map holds rows8 = floor(num_x / 8)
// rows of 8 floats; an index past them fetches row 0 and counts as 0, so no
// copy ever leaves the tensor
__global__ void __launch_bounds__(kTmaWarps * 32) probe_gather_tma_kernel(const __grid_constant__ CUtensorMap tm,
                                                                          const int4* __restrict__ idx,
                                                                          const float4* __restrict__ v,
                                                                          int64_t nchunks, int rows8,
                                                                          float* __restrict__ out, int* err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t bars[kTmaWarps][kTmaStages];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float* wbuf = reinterpret_cast<float*>(smem + (size_t)warp * kTmaStages * kSlotBytes);
  if (lane == 0) {
#pragma unroll
    for (int s = 0; s < kTmaStages; ++s) lbk::mbar_init(&bars[warp][s], 1);
    lbk::fence_mbar_init();
  }
  __syncwarp();
  const int64_t TW = (int64_t)gridDim.x * kTmaWarps;
  const int64_t gw = (int64_t)blockIdx.x * kTmaWarps + warp;
  int issued[kTmaStages], waited[kTmaStages];  // copies issued into / waited for in each slot
#pragma unroll
  for (int s = 0; s < kTmaStages; ++s) issued[s] = waited[s] = 0;
  auto issue = [&](int s, int4 c) {
    if (lane == 0) lbk::mbar_arrive_expect_tx(&bars[warp][s], kSlotBytes);
    __syncwarp();
    auto row = [&](int k) { return (k >> 3) < rows8 ? (k >> 3) : 0; };
    gather4_rows(wbuf + s * (kSlotBytes / 4) + lane * 32, &tm, row(c.x), row(c.y), row(c.z), row(c.w),
                 &bars[warp][s]);
    ++issued[s];
  };
  int4 cs[kTmaStages];
  float4 vs[kTmaStages];
#pragma unroll
  for (int s = 0; s < kTmaStages; ++s) {
    const int64_t c = gw + s * TW;
    if (c < nchunks) {
      cs[s] = lbk::ld_stream(idx + c * 32 + lane);
      vs[s] = lbk::ld_stream(v + c * 32 + lane);
      issue(s, cs[s]);
    }
  }
  float acc = 0.f;
  bool ok = true;
  for (int64_t base = gw; base < nchunks && ok; base += kTmaStages * TW) {
#pragma unroll
    for (int s = 0; s < kTmaStages; ++s) {
      const int64_t c = base + s * TW;
      if (c >= nchunks) break;
      if (!lbk::mbar_wait_bounded(&bars[warp][s], (uint32_t)(waited[s] & 1))) {
        if (lane == 0) atomicOr(err, lbk::kDevErrTimeout);
        ok = false;
        break;
      }
      ++waited[s];
      const float* slot = wbuf + s * (kSlotBytes / 4) + lane * 32;
      auto got = [&](int k, int q) { return (k >> 3) < rows8 ? slot[8 * q + (k & 7)] : 0.f; };
      acc += vs[s].x * got(cs[s].x, 0) + vs[s].y * got(cs[s].y, 1) + vs[s].z * got(cs[s].z, 2) +
             vs[s].w * got(cs[s].w, 3);
      __syncwarp();
      const int64_t cn = c + kTmaStages * TW;
      if (cn < nchunks) {
        cs[s] = lbk::ld_stream(idx + cn * 32 + lane);
        vs[s] = lbk::ld_stream(v + cn * 32 + lane);
        issue(s, cs[s]);
      }
    }
  }
  if (!ok) {
    // wind down: this warp's copies still in flight land before the CTA may leave
#pragma unroll
    for (int s = 0; s < kTmaStages; ++s)
      if (issued[s] > waited[s]) lbk::mbar_wait_bounded(&bars[warp][s], (uint32_t)(waited[s] & 1), 4 * lbk::kSpinLimit);
  }
  out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

std::mutex g_encode_mu;
EncodeTiledFn g_encode = nullptr;

lb_status_t encode_fn(EncodeTiledFn* fn) {
  std::lock_guard<std::mutex> lock(g_encode_mu);
  if (!g_encode) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        !p || q != cudaDriverEntryPointSuccess) {
      set_error("lb_probe_gather_tma: cuTensorMapEncodeTiled is not available");
      return LB_ERR_UNSUPPORTED;
    }
    g_encode = reinterpret_cast<EncodeTiledFn>(p);
  }
  *fn = g_encode;
  return LB_OK;
}

}  // namespace

extern "C" {

int32_t lb_probe_gather_tma_grid(void) {
  int dev = 0, occ = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaFuncSetAttribute(probe_gather_tma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kTmaSmem) !=
          cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, probe_gather_tma_kernel, kTmaWarps * 32, kTmaSmem) !=
          cudaSuccess)
    return 0;
  return occ * device_sms(dev);
}

lb_status_t lb_probe_gather_tma(const int32_t* idx, const float* vals, const float* x, int64_t n, int32_t num_x,
                                float* out, int32_t grid, int32_t* err, void* stream) {
  if (n < 0 || n % 128 != 0 || num_x < 8 || !idx || !vals || !x || !out || !err || grid < 0) {
    set_error("lb_probe_gather_tma: need n a multiple of 128, num_x >= 8 and non-NULL buffers");
    return LB_ERR_INVALID_ARG;
  }
  if (((reinterpret_cast<uintptr_t>(idx) | reinterpret_cast<uintptr_t>(vals) | reinterpret_cast<uintptr_t>(x)) &
       15u) != 0) {
    set_error("lb_probe_gather_tma: idx, vals and x must be 16-byte aligned");
    return LB_ERR_INVALID_ARG;
  }
  if (n == 0) return LB_OK;
  EncodeTiledFn enc = nullptr;
  LB_TRY(encode_fn(&enc));
  // x as rows of 8 floats; a trailing partial row is left out (indices there count as 0)
  CUtensorMap tm;
  std::memset(&tm, 0, sizeof(tm));
  cuuint64_t dims[2] = {8, (cuuint64_t)(num_x / 8)};
  cuuint64_t strides[1] = {32};
  cuuint32_t box[2] = {8, 1};
  cuuint32_t es[2] = {1, 1};
  if (enc(&tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(x), dims, strides, box, es,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS) {
    set_error("lb_probe_gather_tma: cuTensorMapEncodeTiled failed");
    return LB_ERR_CUDA;
  }
  if (grid == 0) grid = lb_probe_gather_tma_grid();
  if (grid <= 0) {
    set_error("lb_probe_gather_tma: no occupancy");
    return LB_ERR_CUDA;
  }
  LB_CUDA_TRY(cudaFuncSetAttribute(probe_gather_tma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kTmaSmem));
  probe_gather_tma_kernel<<<grid, kTmaWarps * 32, kTmaSmem, static_cast<cudaStream_t>(stream)>>>(
      tm, reinterpret_cast<const int4*>(idx), reinterpret_cast<const float4*>(vals), n / 128, num_x / 8, out, err);
  LB_CUDA_TRY(cudaGetLastError());
  return LB_OK;
}

}  // extern "C"
