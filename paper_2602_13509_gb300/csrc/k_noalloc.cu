// hsad_global_rx_noalloc: global RX of one device-resident cube without any device
// allocation.
//
// Some callers cannot allocate device memory at all: flight or embedded software
// that must not touch the allocator after start-up, code running under an external
// memory manager that owns the whole device pool, or plugins hosted by a process that
// forbids cudaMalloc on its streams. This entry point lets them score a cube with the
// same kernels as the context-based API while the library allocates nothing: the
// caller passes the cube and the output buffers, and every intermediate lives in the
// file-scope array g_noalloc_scratch below.
//
// g_noalloc_scratch is HSAD_NOALLOC_SCRATCH_BYTES (16 MiB) of device memory that every
// GPU which loads this library's module keeps until the process exits. Its device
// address is looked up once per device with cudaGetSymbolAddress (host code cannot use
// the symbol itself: on the host it names a stand-in, not device memory).
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <mutex>

#include "../../include/hsad.h"
#include "hsad_internal.h"

using namespace hsad;

#define HSAD_NOALLOC_SCRATCH_BYTES (16u << 20)

static __device__ __align__(256) unsigned char g_noalloc_scratch[HSAD_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void* g_scratch_ptr[kMaxDevices] = {};
// Status codes only: this entry point keeps no error string.
int noalloc_fail(int code, const char*) { return code; }

// Device address of the scratch array on the current device (set-up on first use).
void* scratch_address(int device) {
  std::lock_guard<std::mutex> g(g_setup_mu);
  if (!g_scratch_ptr[device]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    g_scratch_ptr[device] = p;
  }
  return g_scratch_ptr[device];
}

// Carves 256-byte aligned regions out of the scratch array.
struct Carve {
  char* base;
  size_t off = 0;
  template <typename T>
  T* take(size_t count) {
    T* p = (T*)(base + off);
    off += (count * sizeof(T) + 255) / 256 * 256;
    return p;
  }
};

size_t scratch_need(int64_t n, int W, int B) {
  const size_t Bp = (size_t)pad64(B);
  auto r = [](size_t b) { return (b + 255) / 256 * 256; };
  (void)W;
  return r(B * 4) + r(B * 4) + r(B * 8) + r((size_t)B * B * 8)  // c (int, float), S1, S2
         + 2 * r((size_t)n * B * 8)                                            // s1_line, m_line
         + 2 * r((size_t)B * B * 8)                                            // sigma, inv
         + r(Bp * Bp * 4) + r(Bp * 4) + r(4)                                   // wmat, y0, inv_s2
         + 2 * r((size_t)n * 4) + r(4);                                        // status, ring status, max
}

}  // namespace

extern "C" int hsad_global_rx_noalloc(const void* cube, int64_t n_lines, int32_t width, int32_t bands,
                                      int32_t in_dtype, int32_t precision, const float* gain,
                                      int32_t threshold_mode, float threshold, int32_t flags, float* scores,
                                      uint8_t* mask, void* stream, int32_t device) {
  if (n_lines == 0) {
    // start-up warm-up: only the one-time set-up of `device` (the module load that commits
    // the scratch array, and its address lookup), so that no later call pays for it
    if (device < 0 || device >= kMaxDevices) return noalloc_fail(HSAD_E_INVALID, "bad device");
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != device && cudaSetDevice(device) != cudaSuccess) {
      cudaGetLastError();
      return noalloc_fail(HSAD_E_CUDA, "cudaSetDevice failed");
    }
    const int rc = scratch_address(device) ? HSAD_OK : noalloc_fail(HSAD_E_CUDA, "cudaGetSymbolAddress failed");
    if (prev >= 0 && prev != device) cudaSetDevice(prev);
    return rc;
  }
  if (!cube || !scores || !mask) return noalloc_fail(HSAD_E_INVALID, "cube, scores and mask are required");
  if (n_lines < 1 || width < 1 || bands < 1 || bands > 512) return noalloc_fail(HSAD_E_INVALID, "bad sizes");
  if (n_lines > 0x7fffffff || (int64_t)width * bands > ((int64_t)1 << 31))
    return noalloc_fail(HSAD_E_INVALID, "cube too large");
  if (in_dtype != HSAD_U16 && in_dtype != HSAD_F32) return noalloc_fail(HSAD_E_INVALID, "bad in_dtype");
  if (precision < HSAD_FP32 || precision > HSAD_FP16) return noalloc_fail(HSAD_E_INVALID, "bad precision");
  if (threshold_mode != HSAD_ABS && threshold_mode != HSAD_REL) return noalloc_fail(HSAD_E_INVALID, "bad threshold_mode");
  if (!(threshold >= 0.f) || threshold > 3.0e38f) return noalloc_fail(HSAD_E_INVALID, "bad threshold");
  if (flags & ~HSAD_NORMALIZE_SCORES) return noalloc_fail(HSAD_E_INVALID, "unknown flags");
  if (device < 0 || device >= kMaxDevices) return noalloc_fail(HSAD_E_INVALID, "bad device");
  for (int b = 0; b < bands; ++b) {  // the gains cancel from Eq. 1: validated, not used
    const double g = gain ? (double)gain[b] : 1.0;
    if (!(g == g) || g == 0.0 || g > 1e308 || g < -1e308)
      return noalloc_fail(HSAD_E_INVALID, "gain must be finite and non-zero");
  }
  const size_t need = scratch_need(n_lines, width, bands);
  if (need > HSAD_NOALLOC_SCRATCH_BYTES)
    return noalloc_fail(HSAD_E_INVALID, "cube needs more scratch than the 16 MiB static array holds");

  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != device && cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return noalloc_fail(HSAD_E_CUDA, "cudaSetDevice failed");
  }
  int rc = HSAD_OK;
  do {
    char* base = (char*)scratch_address(device);
    if (!base) {
      rc = noalloc_fail(HSAD_E_CUDA, "cudaGetSymbolAddress of the scratch array failed");
      break;
    }
    const int W = width, B = bands;
    const int it = in_dtype == HSAD_U16 ? IN_U16 : IN_F32;
    const int pr = precision == HSAD_FP32 ? P_FP32 : (precision == HSAD_BF16 ? P_BF16 : P_FP16);
    const int64_t N = n_lines * (int64_t)W;
    const float tau = threshold > 0.f ? threshold
                                      : (threshold_mode == HSAD_ABS ? (float)(B + 6.0 * sqrt(2.0 * B)) : 0.f);
    cudaStream_t st = (cudaStream_t)stream;
    Carve cv{base};
    int32_t* c_int = cv.take<int32_t>(B);
    float* c_flt = cv.take<float>(B);
    double* s1 = cv.take<double>(B);
    double* s2 = cv.take<double>((size_t)B * B);
    double* s1_line = cv.take<double>((size_t)n_lines * B);
    double* m_line = cv.take<double>((size_t)n_lines * B);
    double* sigma = cv.take<double>((size_t)B * B);
    double* inv = cv.take<double>((size_t)B * B);
    void* wmat = cv.take<char>((size_t)pad64(B) * pad64(B) * 4);
    float* y0 = cv.take<float>(pad64(B));
    float* inv_s2 = cv.take<float>(1);
    int32_t* status = cv.take<int32_t>(n_lines);
    int32_t* ring_status = cv.take<int32_t>(n_lines);
    unsigned int* dmax = cv.take<unsigned int>(1);

    // every region below is written before it is read except S1 / S2 and the status
    // words, which are cleared here; the array keeps the previous call's contents
    LaunchCounter lc;
    cudaError_t e = cudaMemsetAsync(s1, 0, (size_t)B * 8, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(s2, 0, (size_t)B * B * 8, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, (size_t)n_lines * 4, st);
    if (e == cudaSuccess) e = launch_shift_init(cube, W, B, it, c_int, c_flt, st, &lc);
    if (e == cudaSuccess) e = launch_colsum(cube, n_lines, W, B, it, c_int, c_flt, s1_line, st, &lc);
    if (e == cudaSuccess)
      e = launch_prefix_mean(s1_line, m_line, s1, 0, W, (int)n_lines, B, 1, 0, status, st, &lc);
    if (e == cudaSuccess) e = launch_syrk_simt(cube, 1, N, B, it, c_int, c_flt, s2, 0, 1, st, &lc);
    if (e == cudaSuccess)
      e = launch_finalize_cov(s1, s2, N, B, sigma, m_line, (int64_t)B + 1, status, st, &lc);
    if (e == cudaSuccess)
      e = launch_factor(sigma, inv, m_line, 1, B, pr, wmat, y0, inv_s2, status, N, 0, 0, st, &lc);
    const bool rel = threshold_mode == HSAD_REL, norm = (flags & HSAD_NORMALIZE_SCORES) != 0;
    ScoreOut o;
    o.scores = scores;
    o.mask = mask;
    o.ring_status = ring_status;
    o.slot0 = 0;
    o.ring = n_lines;
    o.tau = tau;
    o.write_mask = (rel || norm) ? 0 : 1;
    if (e == cudaSuccess)
      e = launch_whiten_score_simt(cube, (int)n_lines, W, B, it, c_int, c_flt, pr, wmat, y0, inv_s2, status, 0,
                                   o, st, &lc);
    if (e == cudaSuccess && (rel || norm)) e = launch_cube_normalize(o, n_lines, W, rel ? 1 : 0, norm ? 1 : 0, dmax, st, &lc);
    int32_t cube_status = -1;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&cube_status, status, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      cudaGetLastError();
      rc = noalloc_fail(HSAD_E_CUDA, cudaGetErrorString(e));
      break;
    }
    if (cube_status == LS_NOT_PD) rc = noalloc_fail(HSAD_E_NOT_PD, "covariance not positive definite");
    else if (cube_status != LS_OK) rc = noalloc_fail(HSAD_E_NOT_READY, "fewer than bands + 1 pixels");
  } while (0);
  if (prev >= 0 && prev != device) cudaSetDevice(prev);
  return rc;
}
