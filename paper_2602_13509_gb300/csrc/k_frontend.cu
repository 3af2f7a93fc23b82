// Front end (Sec. 3.2, "Data Acquisition"): the out-of-specification raw bands are
// discarded and every `bin` consecutive kept bands are summed into one band:
//   out[p][b] = sum_{i < bin} raw[p][first + bin * b + i],   b = 0 .. bands - 1.
// 12-bit DN summed in integers: exact, and below 2^16 for bin <= 16.
// One thread per output value, consecutive threads on consecutive bands of a pixel, so a
// warp reads one contiguous run of a pixel's raw bands. Memory-bound: 2 raw_bands bytes read
// and 2 bands bytes written per pixel, once (every later kernel reads the binned lines).
#include <cuda_runtime.h>
#include <stdint.h>

#include "hsad.h"
#include "hsad_internal.h"

namespace hsad {

namespace {
__global__ void frontend_kernel(const uint16_t* __restrict__ raw, int64_t n_px, int raw_bands, int first, int bin,
                                int bands, uint16_t* __restrict__ out) {
  const int64_t total = n_px * bands;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = i / bands;
    const int b = (int)(i - p * bands);
    const uint16_t* src = raw + p * raw_bands + first + (int64_t)b * bin;
    uint32_t acc = 0;
    for (int k = 0; k < bin; ++k) acc += __ldg(src + k);
    out[i] = (uint16_t)acc;
  }
}
}  // namespace

cudaError_t launch_frontend(const uint16_t* raw, int64_t n_px, int raw_bands, int first, int bin, int bands,
                            uint16_t* out, cudaStream_t st, LaunchCounter* lc) {
  if (n_px <= 0) return cudaSuccess;
  int64_t blocks = (n_px * bands + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  frontend_kernel<<<(unsigned)blocks, 256, 0, st>>>(raw, n_px, raw_bands, first, bin, bands, out);
  if (lc) lc->n += 1;
  return cudaGetLastError();
}

}  // namespace hsad

extern "C" int hsad_frontend(const uint16_t* raw, int64_t n_pixels, int32_t raw_bands, int32_t band_first,
                             int32_t band_bin, int32_t bands, uint16_t* out, int32_t device, void* stream) {
  using namespace hsad;
  if (n_pixels < 0 || raw_bands < 1 || band_first < 0 || band_bin < 1 || band_bin > 16 || bands < 1 ||
      (int64_t)band_first + (int64_t)band_bin * bands > raw_bands || (n_pixels > 0 && (!raw || !out)))
    return HSAD_E_INVALID;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return ndev <= 0 ? HSAD_E_CUDA : HSAD_E_INVALID;
  }
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != device) cudaSetDevice(device);
  cudaStream_t st = (cudaStream_t)stream;
  int rc = HSAD_OK;
  if (launch_frontend(raw, n_pixels, raw_bands, band_first, band_bin, bands, out, st, nullptr) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    rc = HSAD_E_CUDA;
  cudaGetLastError();
  if (prev >= 0 && prev != device) cudaSetDevice(prev);
  return rc;
}
