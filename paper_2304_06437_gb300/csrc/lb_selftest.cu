// lb_selftest.cu -- exercises the bounded wait every kernel uses on its TMA
// mbarriers, on a barrier that can never complete, so the timeout path
// (status word, clean return) is tested without faulting or hanging a GPU.
#include <cuda_runtime.h>

#include "../../include/lb.h"
#include "lb_ptx.cuh"

namespace lbgb {

__global__ void selftest_wait_kernel(uint64_t limit_ns, int* status, unsigned long long* waited_ns) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 2);  // two arrivals expected, only one ever comes
    fence_barrier_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_arrive(&bar);
    const uint64_t t0 = global_timer_ns();
    const bool ok = mbar_wait_bounded(&bar, 0, limit_ns);
    *waited_ns = global_timer_ns() - t0;
    *status = ok ? LB_OK : LB_E_TIMEOUT;
    mbar_inval(&bar);
  }
}

}  // namespace lbgb

extern "C" int lb_selftest_timeout(int64_t limit_ns, int64_t* waited_ns) {
  if (limit_ns < 0 || limit_ns > 5000000000LL) return LB_E_INVAL;
  int* d_st = nullptr;
  unsigned long long* d_w = nullptr;
  if (cudaMalloc(&d_st, sizeof(int)) != cudaSuccess) return LB_E_NOMEM;
  if (cudaMalloc(&d_w, sizeof(unsigned long long)) != cudaSuccess) {
    cudaFree(d_st);
    return LB_E_NOMEM;
  }
  lbgb::selftest_wait_kernel<<<1, 32>>>(uint64_t(limit_ns), d_st, d_w);
  int st = LB_E_CUDA;
  unsigned long long w = 0;
  int rc = LB_OK;
  if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess ||
      cudaMemcpy(&st, d_st, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(&w, d_w, sizeof(w), cudaMemcpyDeviceToHost) != cudaSuccess)
    rc = LB_E_CUDA;
  cudaFree(d_st);
  cudaFree(d_w);
  if (rc != LB_OK) return rc;
  if (waited_ns) *waited_ns = int64_t(w);
  return st;
}
