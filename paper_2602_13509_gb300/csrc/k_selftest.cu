// Self-test of the bounded-wait mechanism every tensor-core kernel relies on.
//
// The kernel initialises an mbarrier that nothing will ever arrive at and waits on it
// with the same bounded wait (tc::mbar_wait) as the production kernels. The wait must
// give up after `limit` clock cycles, record the timeout in device memory and return,
// leaving the context usable. Nothing is copied asynchronously, so nothing is in flight.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/hsad.h"
#include "hsad_internal.h"
#include "tc_util.cuh"

namespace {
__global__ void bounded_wait_kernel(int32_t* flag, long long limit) {
  __shared__ __align__(8) uint64_t bar;
  const uint32_t b = hsad::tc::smem_u32(&bar);
  if (threadIdx.x == 0) {
    hsad::tc::mbar_init(b, 1);
    hsad::tc::mbar_init_fence();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const bool ok = hsad::tc::mbar_wait(b, 0, limit);  // no arrival: must time out
    *flag = ok ? 0 : 1;
  }
}
}  // namespace

extern "C" int hsad_selftest_bounded_wait(int32_t device, int64_t limit_cycles, int32_t* timed_out) {
  if (!timed_out || limit_cycles <= 0 || limit_cycles > 20000000000LL) return HSAD_E_INVALID;
  int prev = -1;
  cudaGetDevice(&prev);
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return HSAD_E_CUDA;
  }
  int32_t* d = nullptr;
  int rc = HSAD_OK;
  if (cudaMalloc(&d, 4) != cudaSuccess || cudaMemset(d, 0xff, 4) != cudaSuccess) {
    rc = HSAD_E_CUDA;
  } else {
    bounded_wait_kernel<<<1, 32>>>(d, (long long)limit_cycles);
    int32_t h = -1;
    if (cudaGetLastError() != cudaSuccess || cudaMemcpy(&h, d, 4, cudaMemcpyDeviceToHost) != cudaSuccess) {
      rc = HSAD_E_CUDA;
    } else {
      *timed_out = h;
      rc = h == 1 ? HSAD_E_TIMEOUT : HSAD_OK;
    }
  }
  cudaGetLastError();
  if (d) cudaFree(d);
  if (prev >= 0) cudaSetDevice(prev);
  return rc;
}
