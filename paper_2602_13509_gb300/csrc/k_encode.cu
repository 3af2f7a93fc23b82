// Transmit encoding (Sec. 3.4, "Data Transmission"): every score is sent as an IEEE-754
// half-precision value of its square root, normalised to the block's maximum:
//   code = binary16(sqrt(delta / delta_max)),
// in FP32 as the paper computes its scores (the division and square root correctly
// rounded, the default without fast-math) and rounded to nearest even. delta_max is the
// largest finite score of the block; NaN scores (lines not ready) give the NaN code 0x7E00,
// +Inf gives 0x7C00, and when no score is positive every finite score gives 0.
// Two grid-stride passes: the maximum (the bits of a non-negative float order like an
// unsigned integer, so atomicMax on the bits), then the codes.
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <map>
#include <mutex>

#include "hsad.h"
#include "hsad_internal.h"

namespace hsad {

namespace {
constexpr int TX_THREADS = 256;

__global__ void tx_max_kernel(const float* __restrict__ s, int64_t n, unsigned int* __restrict__ max_bits) {
  float mx = 0.f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float v = s[i];
    if (v > mx && v < INFINITY) mx = v;  // NaN compares false
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0 && mx > 0.f) atomicMax(max_bits, __float_as_uint(mx));
}

__global__ void tx_encode_kernel(const float* __restrict__ s, int64_t n, uint16_t* __restrict__ codes,
                                 const unsigned int* __restrict__ max_bits) {
  const float dmax = __uint_as_float(*max_bits);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float v = s[i];
    uint16_t c;
    if (isnan(v)) c = 0x7E00;
    else if (dmax > 0.f) c = __half_as_ushort(__float2half_rn(sqrtf(v / dmax)));
    else c = isinf(v) ? (uint16_t)0x7C00 : (uint16_t)0;
    codes[i] = c;
  }
}

unsigned grid_for(int64_t n) {
  int64_t b = (n + TX_THREADS - 1) / TX_THREADS;
  if (b > 152 * 8) b = 152 * 8;
  return (unsigned)(b < 1 ? 1 : b);
}
}  // namespace

cudaError_t launch_tx_max(const float* s, int64_t n, unsigned int* max_bits, cudaStream_t st, LaunchCounter* lc) {
  if (n <= 0) return cudaSuccess;
  tx_max_kernel<<<grid_for(n), TX_THREADS, 0, st>>>(s, n, max_bits);
  if (lc) lc->n += 1;
  return cudaGetLastError();
}

cudaError_t launch_tx_encode(const float* s, int64_t n, uint16_t* codes, const unsigned int* max_bits,
                             cudaStream_t st, LaunchCounter* lc) {
  if (n <= 0) return cudaSuccess;
  tx_encode_kernel<<<grid_for(n), TX_THREADS, 0, st>>>(s, n, codes, max_bits);
  if (lc) lc->n += 1;
  return cudaGetLastError();
}

}  // namespace hsad

extern "C" int hsad_encode_scores(const float* scores, int64_t n, uint16_t* codes, float* max_score,
                                  int32_t device, void* stream) {
  using namespace hsad;
  if (n < 0 || (n > 0 && (!scores || !codes))) return HSAD_E_INVALID;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return ndev <= 0 ? HSAD_E_CUDA : HSAD_E_INVALID;
  }
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != device) cudaSetDevice(device);
  // one 4-byte scratch per device, kept for the process; calls on a device run one at a time
  static std::mutex mu;
  static std::map<int, unsigned int*> scratch;
  std::lock_guard<std::mutex> g(mu);
  int rc = HSAD_OK;
  unsigned int*& mb = scratch[device];
  cudaStream_t st = (cudaStream_t)stream;
  if (!mb && cudaMalloc(&mb, sizeof(unsigned int)) != cudaSuccess) {
    mb = nullptr;
    rc = HSAD_E_NOMEM;
  }
  unsigned int bits = 0;
  if (rc == HSAD_OK &&
      (cudaMemsetAsync(mb, 0, sizeof(unsigned int), st) != cudaSuccess ||
       launch_tx_max(scores, n, mb, st, nullptr) != cudaSuccess ||
       launch_tx_encode(scores, n, codes, mb, st, nullptr) != cudaSuccess ||
       cudaMemcpyAsync(&bits, mb, sizeof(unsigned int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
       cudaStreamSynchronize(st) != cudaSuccess))
    rc = HSAD_E_CUDA;
  cudaGetLastError();
  if (rc == HSAD_OK && max_score) {
    float f;
    memcpy(&f, &bits, sizeof f);
    *max_score = f;
  }
  if (prev >= 0 && prev != device) cudaSetDevice(prev);
  return rc;
}
