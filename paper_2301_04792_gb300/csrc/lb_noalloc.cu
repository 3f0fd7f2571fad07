// Merge-path SpMV for callers that cannot allocate device memory.
//
// Some callers must not call cudaMalloc at all: allocator-free embedded or
// real-time loops that reserve all device memory up front (cudaMalloc may
// synchronise the device and take unbounded time), and hosts whose memory
// pool is owned by another framework and forbids a library from reserving its
// own blocks.  lb_spmv_noalloc serves them: it needs no plan object and
// allocates nothing.  Its scratch (the merge-path split table, one carry slot
// per warp worker and the fix-up ticket) lives in the fixed file-scope device
// array below, which every GPU that loads this library holds until the
// process exits.
#include <cstring>
#include <mutex>
#include <string>

#include "lb_internal.h"
#include "lb_kernels.cuh"

namespace lbh {
__global__ void mp_splits_kernel(const int32_t* __restrict__ rp, int32_t R, int64_t N, int64_t items, int grid,
                                 int tpc, int ipt_items, int64_t entries, int2* out, int64_t* diag);
}

using namespace lbh;

namespace {

// Scratch of lb_spmv_noalloc, shared by every call on a device: 8 MiB.
constexpr size_t kNoAllocBytes = size_t(8) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kIpt = 8;        // items per lane of the warp-worker kernel
constexpr int kMaxDevices = 64;

struct DeviceSetup {
  bool ready = false;
  unsigned char* base = nullptr;  // device address of g_noalloc_scratch on this device
  int sms = 0;
  int ctas_per_sm = 0;
};
std::mutex g_setup_mu;
DeviceSetup g_setup[kMaxDevices];

// Once per device, with that device current: the device address of the
// scratch array (the host-side name is only a stand-in), the SM count and the
// kernel's occupancy.  None of these calls allocates.
lb_status_t setup_device(int dev, DeviceSetup** out) {
  std::lock_guard<std::mutex> lock(g_setup_mu);
  DeviceSetup& d = g_setup[dev];
  if (!d.ready) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || ptr == nullptr) {
      set_error(std::string("lb_spmv_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
      return LB_ERR_CUDA;
    }
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, lbk::mp_spmv_warp_kernel<kIpt, false, false, true>,
                                                      kBlock, 0);
    // load every kernel the entry point launches now, not at its first launch
    cudaFuncAttributes fa;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, lbk::mp_spmv_warp_kernel<kIpt, false, false, false>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, mp_splits_kernel);
    if (e != cudaSuccess) {
      set_error(std::string("lb_spmv_noalloc: kernel set-up failed: ") + cudaGetErrorString(e));
      return LB_ERR_CUDA;
    }
    d.base = static_cast<unsigned char*>(ptr);
    d.sms = device_sms(dev);
    d.ctas_per_sm = occ > 0 ? occ : 1;
    d.ready = true;
  }
  *out = &d;
  return LB_OK;
}

size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

}  // namespace

extern "C" {

lb_status_t lb_spmv_noalloc(const int32_t* tile_offsets, int32_t num_tiles, int32_t num_atoms,
                            const int32_t* col_idx, const float* vals, const float* x, float* y, void* stream) {
  if (num_tiles < 0 || num_atoms < 0 || (num_tiles == 0 && num_atoms != 0)) {
    set_error("lb_spmv_noalloc: need num_tiles >= 0, num_atoms >= 0");
    return LB_ERR_INVALID_ARG;
  }
  if (num_tiles == 0) return LB_OK;
  if (!tile_offsets || !y || (num_atoms > 0 && (!col_idx || !vals || !x))) {
    set_error("lb_spmv_noalloc: NULL buffer");
    return LB_ERR_INVALID_ARG;
  }
  int dev = 0;
  LB_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("lb_spmv_noalloc: device index out of range");
    return LB_ERR_UNSUPPORTED;
  }
  DeviceSetup* d = nullptr;
  LB_TRY(setup_device(dev, &d));

  // geometry of the warp-worker merge path (same rule as a plan with
  // items_per_thread 8): 8 warps per CTA, up to SMs x occupancy CTAs
  const int64_t items = (int64_t)num_tiles + num_atoms;
  const int items_per_tile = 32 * kIpt - 4;
  int64_t ctas = (items + kBlock - 1) / kBlock;
  if (ctas > (int64_t)d->sms * d->ctas_per_sm) ctas = (int64_t)d->sms * d->ctas_per_sm;
  if (ctas < 1) ctas = 1;
  const int64_t workers = ctas * (kBlock / 32);
  const int64_t share = (items + workers - 1) / workers;
  int64_t tpc = (share + items_per_tile - 1) / items_per_tile;
  if (tpc < 1) tpc = 1;
  const int64_t entries = workers * (tpc + 1);

  // scratch layout: ticket | carry rows | carry values | splits (the diagonals are not kept)
  const size_t off_rows = 256;
  const size_t off_vals = round_up(off_rows + sizeof(int32_t) * (size_t)workers, 256);
  const size_t off_splits = round_up(off_vals + sizeof(float) * (size_t)workers, 256);
  const size_t need = off_splits + sizeof(int2) * (size_t)entries;
  if (need > kNoAllocBytes) {
    set_error("lb_spmv_noalloc: problem needs " + std::to_string(need) + " bytes of scratch, more than the " +
              std::to_string(kNoAllocBytes) + " the no-allocation entry point has (use lb_plan + lb_spmv)");
    return LB_ERR_UNSUPPORTED;
  }
  unsigned char* base = d->base;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the ticket and unit counter must start at zero; the array keeps the previous call's contents
  LB_CUDA_TRY(cudaMemsetAsync(base, 0, 2 * sizeof(unsigned), s));
  int2* splits = reinterpret_cast<int2*>(base + off_splits);
  const unsigned sblocks = (unsigned)((entries + 255) / 256);
  mp_splits_kernel<<<sblocks, 256, 0, s>>>(tile_offsets, num_tiles, num_atoms, items, (int)workers, (int)tpc,
                                           items_per_tile, entries, splits, nullptr);
  LB_CUDA_TRY(cudaGetLastError());

  lbk::MpArgs a{};
  a.rp = tile_offsets;
  a.atoms = lbk::AtomView{col_idx, vals, nullptr, x, 0, nullptr};
  a.out = y;
  a.splits = splits;
  a.tiles_per_cta = (int)tpc;
  a.num_ctas = (int)ctas;
  a.num_workers = (int)workers;
  a.items_per_tile = items_per_tile;
  a.num_tiles = num_tiles;
  a.num_atoms = num_atoms;
  a.carry_row = reinterpret_cast<int32_t*>(base + off_rows);
  a.carry_val = reinterpret_cast<float*>(base + off_vals);
  a.ticket = reinterpret_cast<unsigned*>(base);
  const bool vec = ((reinterpret_cast<uintptr_t>(col_idx) | reinterpret_cast<uintptr_t>(vals)) & 15u) == 0;
  if (vec)
    lbk::mp_spmv_warp_kernel<kIpt, false, false, true><<<(unsigned)ctas, kBlock, 0, s>>>(a);
  else
    lbk::mp_spmv_warp_kernel<kIpt, false, false, false><<<(unsigned)ctas, kBlock, 0, s>>>(a);
  LB_CUDA_TRY(cudaGetLastError());
  return LB_OK;
}

}  // extern "C"
