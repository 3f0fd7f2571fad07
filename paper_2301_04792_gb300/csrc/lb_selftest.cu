// Self-tests of the library's failure detection.  Each runs one of the bounded
// waits the kernels use on a condition that never comes true -- a look-back
// record that is never published, an mbarrier phase that never completes --
// and reports what the device recorded.  Nothing faults or hangs: the wait
// gives up after a few thousand polls, sets the timeout bit of the status
// word and the kernel returns, so the context stays usable.
#include <string>

#include "lb_internal.h"
#include "lb_kernels.cuh"

using namespace lbh;

namespace {

constexpr long long kSelftestSpins = 4096;

// share 1 looks back at share 0, whose record holds another launch's epoch
__global__ void lookback_unpublished_kernel(const unsigned long long* records, int* status) {
  float total;
  if (!lbk::look_back(records, 1, 7u, total, kSelftestSpins) && threadIdx.x == 0)
    atomicOr(status, lbk::kDevErrTimeout);
}

// a phase that expects two arrivals and gets one
__global__ void mbarrier_incomplete_kernel(int* status) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    lbk::mbar_init(&bar, 2);
    lbk::fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) lbk::mbar_arrive(&bar);
  __syncthreads();
  if (!lbk::mbar_wait_bounded(&bar, 0u, kSelftestSpins) && threadIdx.x == 0) atomicOr(status, lbk::kDevErrTimeout);
}

}  // namespace

extern "C" {

lb_status_t lb_selftest(int32_t which, void* stream) {
  if (which != 1 && which != 2) {
    set_error("lb_selftest: which must be 1 (look-back) or 2 (mbarrier)");
    return LB_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  void* buf = nullptr;  // status word, then two zeroed records
  LB_CUDA_TRY(cudaMalloc(&buf, 64));
  struct Free {
    void* p;
    ~Free() { cudaFree(p); }
  } guard{buf};
  int* status = static_cast<int*>(buf);
  auto* records = reinterpret_cast<unsigned long long*>(static_cast<char*>(buf) + 16);
  LB_CUDA_TRY(cudaMemsetAsync(buf, 0, 64, s));
  if (which == 1)
    lookback_unpublished_kernel<<<1, 32, 0, s>>>(records, status);
  else
    mbarrier_incomplete_kernel<<<1, 32, 0, s>>>(status);
  LB_CUDA_TRY(cudaGetLastError());
  int h = 0;
  LB_CUDA_TRY(cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, s));
  LB_CUDA_TRY(cudaStreamSynchronize(s));
  if (h & lbk::kDevErrTimeout) {
    set_error(which == 1 ? "lb_selftest: look-back wait gave up as designed"
                         : "lb_selftest: mbarrier wait gave up as designed");
    return LB_ERR_TIMEOUT;
  }
  return LB_OK;
}

}  // extern "C"
