// Front end (Sec. 3.2, "Data Acquisition"): the out-of-specification raw bands are
// discarded and every `bin` consecutive kept bands are summed into one band:
//   out[p][b] = sum_{i < bin} raw[p][first + bin * b + i],   b = 0 .. bands - 1.
// 12-bit DN summed in integers: exact, and below 2^16 for bin <= 16.
// One thread per output value, consecutive threads on consecutive bands of a pixel, so a
// warp reads one contiguous run of a pixel's raw bands (in band pairs where aligned). Memory-bound: 2 raw_bands bytes read
// and 2 bands bytes written per pixel, once (every later kernel reads the binned lines).
#include <cuda_runtime.h>
#include <stdint.h>

#include "hsad.h"
#include "hsad_internal.h"

namespace hsad {

namespace {
template <typename I, bool PAIRS>
__global__ void frontend_kernel(const uint16_t* __restrict__ raw, I total, int raw_bands, int first, int bin,
                                int bands, uint16_t* __restrict__ out) {
  for (I i = (I)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (I)gridDim.x * blockDim.x) {
    const I p = i / (I)bands;  // 32-bit division when the batch allows it
    const int b = (int)(i - p * (I)bands);
    const uint16_t* src = raw + (int64_t)p * raw_bands + first + (int64_t)b * bin;
    uint32_t acc = 0;
    if (PAIRS) {  // bin, first and raw_bands even: 4-byte loads of band pairs
      const uint32_t* w = (const uint32_t*)src;
      for (int k = 0; k < bin / 2; ++k) {
        const uint32_t v = __ldg(w + k);
        acc += (v & 0xffffu) + (v >> 16);
      }
    } else {
      for (int k = 0; k < bin; ++k) acc += __ldg(src + k);
    }
    out[i] = (uint16_t)acc;
  }
}
}  // namespace

cudaError_t launch_frontend(const uint16_t* raw, int64_t n_px, int raw_bands, int first, int bin, int bands,
                            uint16_t* out, cudaStream_t st, LaunchCounter* lc) {
  if (n_px <= 0) return cudaSuccess;
  const int64_t total = n_px * bands;
  int64_t blocks = (total + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  const bool pairs = bin % 2 == 0 && first % 2 == 0 && raw_bands % 2 == 0 && ((uintptr_t)raw & 3) == 0;
#define HSAD_FE(I, PR) \
  frontend_kernel<I, PR><<<(unsigned)blocks, 256, 0, st>>>(raw, (I)total, raw_bands, first, bin, bands, out)
  if (total < ((int64_t)1 << 31) - (int64_t)blocks * 256) {
    if (pairs) HSAD_FE(int32_t, true);
    else HSAD_FE(int32_t, false);
  } else {
    if (pairs) HSAD_FE(int64_t, true);
    else HSAD_FE(int64_t, false);
  }
#undef HSAD_FE
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
