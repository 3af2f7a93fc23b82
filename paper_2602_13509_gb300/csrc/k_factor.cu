// K4 + K5: FP64 Cholesky factorisation and triangular inverse of each line's
// covariance, and the whitening operand in the working precision.
//
// Eq. 1 (Sec. 3.3) needs Sigma^{-1}. With Sigma = L L^T (Cholesky, FP64) the score is
// delta = || L^{-1} (x - mu) ||^2. In the DN frame used by the statistics kernels the
// calibrated deviation is x - mu = D (x' - m), with x' = DN - c and m = mu_DN - c, so
//     y = G x' - G m,   G = L^{-1} D,   delta = || y ||^2.
// G is lower triangular. It is stored row-major ([n][k], n = output coordinate) as the
// K-major operand of the whitening contraction, scaled by a power of two s so that
// max |s G| is in [0.5, 1) (keeps FP16 in range; exact in every format), and
// delta = || s G x' - s G m ||^2 / s^2.
//   FP32 : one float plane.
//   FP16 / BF16 : hi plane = rn(sG), lo plane = rn(sG - hi): the two-term split keeps
//                 about 16 (BF16) or 22 (FP16) bits of G.
// y0 = s G m is formed from the rounded operand actually used, in FP64.
// A non-positive or non-finite pivot marks the line LS_NOT_PD; nothing traps.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "hsad_internal.h"

namespace hsad {

namespace {
constexpr int FT = 256;  // threads per factorisation CTA

template <int PREC>
struct WOut;
template <>
struct WOut<P_FP32> {
  __device__ static double store(void* w, int64_t plane, int64_t idx, double v) {
    const float f = (float)v;
    ((float*)w)[idx] = f;
    return (double)f;
  }
};
template <>
struct WOut<P_FP16> {
  __device__ static double store(void* w, int64_t plane, int64_t idx, double v) {
    const __half hi = __double2half(v);
    const __half lo = __double2half(v - (double)__half2float(hi));
    ((__half*)w)[idx] = hi;
    ((__half*)w)[plane + idx] = lo;
    return (double)__half2float(hi) + (double)__half2float(lo);
  }
};
template <>
struct WOut<P_BF16> {
  __device__ static double store(void* w, int64_t plane, int64_t idx, double v) {
    const __nv_bfloat16 hi = __double2bfloat16(v);
    const __nv_bfloat16 lo = __double2bfloat16(v - (double)__bfloat162float(hi));
    ((__nv_bfloat16*)w)[idx] = hi;
    ((__nv_bfloat16*)w)[plane + idx] = lo;
    return (double)__bfloat162float(hi) + (double)__bfloat162float(lo);
  }
};

__device__ double block_max(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = red[0];
    for (int i = 1; i < FT / 32; ++i) m = fmax(m, red[i]);
    red[0] = m;
  }
  __syncthreads();
  return red[0];
}
}  // namespace

template <int PREC>
__global__ void __launch_bounds__(FT) factor_kernel(double* __restrict__ sigma_all,
                                                    double* __restrict__ inv_all,
                                                    const double* __restrict__ m_all,
                                                    const double* __restrict__ dgain, int B,
                                                    void* __restrict__ wmat,
                                                    float* __restrict__ y0_all,
                                                    float* __restrict__ inv_s2_all,
                                                    int32_t* __restrict__ status) {
  const int t = blockIdx.x;
  if (status[t] != LS_OK) return;
  const int64_t BB = (int64_t)B * B;
  double* A = sigma_all + t * BB;
  double* Inv = inv_all + t * BB;
  const double* m = m_all + (int64_t)t * B;
  const int Bp = pad64(B);
  __shared__ double col[512];
  __shared__ double red[FT / 32];
  __shared__ int s_fail;
  __shared__ double s_l;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // ---- Cholesky (right-looking, lower triangle in place) -------------------------
  for (int j = 0; j < B; ++j) {
    if (tid == 0) {
      const double piv = A[(int64_t)j * B + j];
      const int fail = !(piv > 0.0) || !isfinite(piv);
      s_fail = fail;
      const double l = fail ? 1.0 : sqrt(piv);
      s_l = l;
      A[(int64_t)j * B + j] = l;
    }
    __syncthreads();
    if (s_fail) {
      if (tid == 0) status[t] = LS_NOT_PD;
      return;
    }
    const double ljj = s_l;
    for (int i = j + 1 + tid; i < B; i += FT) {
      const double v = A[(int64_t)i * B + j] / ljj;
      A[(int64_t)i * B + j] = v;
      col[i] = v;
    }
    __syncthreads();
    // trailing lower triangle: one warp per row, lanes along the row
    for (int i = j + 1 + warp; i < B; i += FT / 32) {
      const double ci = col[i];
      double* row = A + (int64_t)i * B;
      for (int k = j + 1 + lane; k <= i; k += 32) row[k] -= ci * col[k];
    }
    __syncthreads();
  }

  // ---- triangular inverse Inv = L^{-1} (lower) -------------------------------------
  // Thread owns columns c = tid and tid + FT; column c needs only its own earlier
  // entries, so no synchronisation is needed between rows. Entries above the
  // diagonal are stored as zeros so the k loop can start at the warp's first column.
  for (int i = 0; i < B; ++i) {
    const double* Li = A + (int64_t)i * B;
    const double lii = Li[i];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int c = tid + q * FT;
      const int kstart = (c & ~31);
      if (c >= B && kstart >= B) continue;
      double acc = (c == i) ? 1.0 : 0.0;
      if (kstart <= i) {
        for (int k = kstart; k < i; ++k) acc -= Li[k] * (c < B ? Inv[(int64_t)k * B + c] : 0.0);
      }
      if (c < B) Inv[(int64_t)i * B + c] = (c <= i) ? acc / lii : 0.0;
    }
  }
  __syncthreads();

  // ---- G = Inv D, power-of-two scale, cast, y0 ------------------------------------
  double mx = 0.0;
  for (int64_t e = tid; e < BB; e += FT) {
    const int k = (int)(e % B);
    mx = fmax(mx, fabs(Inv[e] * dgain[k]));
  }
  mx = block_max(mx, red);
  int ex = 0;
  frexp(mx, &ex);
  const double s = (mx > 0.0) ? ldexp(1.0, -ex) : 1.0;
  const int64_t plane = (int64_t)Bp * Bp;
  void* w = (char*)wmat + (size_t)t * plane * 4;  // 4 bytes per element pair in every format
  // one warp per output row n: write the row and accumulate y0[n] from the rounded values
  for (int n = warp; n < Bp; n += FT / 32) {
    double acc = 0.0;
    for (int k = lane; k < Bp; k += 32) {
      double v = 0.0;
      if (n < B && k <= n) v = Inv[(int64_t)n * B + k] * dgain[k] * s;
      const double r = WOut<PREC>::store(w, plane, (int64_t)n * Bp + k, v);
      if (n < B && k <= n) acc += r * m[k];
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) y0_all[(int64_t)t * Bp + n] = (n < B) ? (float)acc : 0.0f;
  }
  if (tid == 0) inv_s2_all[t] = (float)(1.0 / (s * s));
}

cudaError_t launch_factor(double* sigma, double* scratch, const double* m, const double* dgain,
                          int L, int B, int prec, void* wmat, float* y0, float* inv_s2,
                          int32_t* status, cudaStream_t st, LaunchCounter* lc) {
  if (L <= 0) return cudaSuccess;
  dim3 grid(L), block(FT);
  switch (prec) {
    case P_FP32:
      factor_kernel<P_FP32><<<grid, block, 0, st>>>(sigma, scratch, m, dgain, B, wmat, y0, inv_s2, status);
      break;
    case P_FP16:
      factor_kernel<P_FP16><<<grid, block, 0, st>>>(sigma, scratch, m, dgain, B, wmat, y0, inv_s2, status);
      break;
    default:
      factor_kernel<P_BF16><<<grid, block, 0, st>>>(sigma, scratch, m, dgain, B, wmat, y0, inv_s2, status);
      break;
  }
  if (lc) lc->n += 1;
  return cudaGetLastError();
}

}  // namespace hsad
