// Statistics kernels of the RX detector: centring shift, column sums, covariance
// rank-k update and the running (prefix) mean / covariance per line.
//
// Sec. 3.3 ("Detection Algorithm"): each band is a variable and each pixel a
// sample; mu is the per-band mean and Sigma the covariance of the statistics set.
// The data are shifted by an integer per-band value c (the rounded mean of the
// first line after a reset), so for uint16 input every sum below is an exact
// integer: s1 = sum (x - c), s2 = sum (x - c)(x - c)^T. The covariance then
// follows as Sigma = (S2 - S1 S1^T / N) / (N - 1) (N-1 sample covariance). The
// calibrated spectrum is D (DN - offset) (Sec. 3.2, radiometric correction), a per-band
// affine map under which Eq. 1 is invariant, so the statistics stay in the DN frame.
// With the per-line gain correction (Sec. 3.2: each line divided by its gain g_t before
// the calibration) the prefix kernels turn each line's exact sums into the sums of
// DN / g_t about c, in FP64.
#include <cuda_runtime.h>
#include <stdint.h>

#include "hsad_internal.h"

namespace hsad {

#define HSAD_LAUNCH_CHECK(lc) \
  do {                        \
    if (lc) (lc)->n += 1;     \
    return cudaGetLastError(); \
  } while (0)

// ---------------------------------------------------------------------------------
// K1a shift_init: c_b = rint(mean over the W pixels of one line).
template <typename In>
__global__ void shift_init_kernel(const In* __restrict__ line, int W, int B, int32_t* c_int,
                                  float* c_flt) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  double s = 0.0;
  for (int p = 0; p < W; ++p) s += (double)line[(int64_t)p * B + b];
  double mean = s / (double)W;
  if (c_int) c_int[b] = (int32_t)rint(mean);
  if (c_flt) c_flt[b] = isfinite(mean) ? (float)mean : 0.0f;
}

cudaError_t launch_shift_init(const void* line, int W, int B, int in_type, int32_t* c_int,
                              float* c_flt, cudaStream_t st, LaunchCounter* lc) {
  dim3 grid((B + 127) / 128), block(128);
  if (in_type == IN_U16)
    shift_init_kernel<uint16_t><<<grid, block, 0, st>>>((const uint16_t*)line, W, B, c_int, nullptr);
  else
    shift_init_kernel<float><<<grid, block, 0, st>>>((const float*)line, W, B, nullptr, c_flt);
  HSAD_LAUNCH_CHECK(lc);
}

// ---------------------------------------------------------------------------------
// K1b colsum: one CTA per line, threads over bands (coalesced along the band axis).
__global__ void colsum_u16_kernel(const uint16_t* __restrict__ x, int W, int B,
                                  const int32_t* __restrict__ c, double* __restrict__ s1) {
  const int64_t t = blockIdx.x;
  const uint16_t* line = x + t * (int64_t)W * B;
  for (int b = threadIdx.x; b < B; b += blockDim.x) {
    int64_t acc = 0;
    const int cb = c[b];
#pragma unroll 8
    for (int p = 0; p < W; ++p) acc += (int64_t)((int)line[(int64_t)p * B + b] - cb);
    s1[t * B + b] = (double)acc;
  }
}

__global__ void colsum_f32_kernel(const float* __restrict__ x, int W, int B,
                                  const float* __restrict__ c, double* __restrict__ s1) {
  const int64_t t = blockIdx.x;
  const float* line = x + t * (int64_t)W * B;
  for (int b = threadIdx.x; b < B; b += blockDim.x) {
    double acc = 0.0;
    const float cb = c[b];
    for (int p = 0; p < W; ++p) acc += (double)(line[(int64_t)p * B + b] - cb);
    s1[t * B + b] = acc;
  }
}

cudaError_t launch_colsum(const void* x, int64_t n_lines, int W, int B, int in_type,
                          const int32_t* c_int, const float* c_flt, double* s1, cudaStream_t st,
                          LaunchCounter* lc) {
  if (n_lines <= 0) return cudaSuccess;
  // one thread per band (B <= 512): one pass over the line's pixels
  dim3 grid((unsigned)n_lines), block((unsigned)((B + 31) / 32 * 32));
  if (in_type == IN_U16)
    colsum_u16_kernel<<<grid, block, 0, st>>>((const uint16_t*)x, W, B, c_int, s1);
  else
    colsum_f32_kernel<<<grid, block, 0, st>>>((const float*)x, W, B, c_flt, s1);
  HSAD_LAUNCH_CHECK(lc);
}

// ---------------------------------------------------------------------------------
// K2 (SIMT) syrk: 64 x 64 output tiles of the upper block triangle, 256 threads with
// 4 x 4 micro-tiles, pixels staged through shared memory 16 at a time.
// u16: (x - c) is an integer with |x - c| <= 4095, so each product is below 2^24 and
// 64 of them fit in int32; partial sums flush into int64 every 64 pixels (exact).
// f32: products of two floats are exact in FP64 and accumulate in FP64.
namespace {
constexpr int SY_T = 64, SY_K = 16;

template <typename In>
struct SyrkTraits;
template <>
struct SyrkTraits<uint16_t> {
  using Stage = int32_t;
  using Acc = int32_t;
  using Wide = long long;
  __device__ static Stage load(uint16_t v, const int32_t* ci, const float*, int b) {
    return (int32_t)v - ci[b];
  }
};
template <>
struct SyrkTraits<float> {
  using Stage = float;
  using Acc = double;
  using Wide = double;
  __device__ static Stage load(float v, const int32_t*, const float* cf, int b) { return v - cf[b]; }
};
}  // namespace

template <typename In>
__global__ void __launch_bounds__(256) syrk_simt_kernel(const In* __restrict__ x,
                                                        int64_t pix_per_group, int B,
                                                        const int32_t* __restrict__ c_int,
                                                        const float* __restrict__ c_flt,
                                                        double* __restrict__ out,
                                                        int64_t out_stride, int64_t pix_per_slice,
                                                        int accumulate) {
  using Tr = SyrkTraits<In>;
  using Stage = typename Tr::Stage;
  using Acc = typename Tr::Acc;
  using Wide = typename Tr::Wide;
  __shared__ Stage As[SY_K][SY_T];
  __shared__ Stage Bs[SY_K][SY_T];

  // decode the upper-triangle tile (ti <= tj)
  const int nt = (B + SY_T - 1) / SY_T;
  int tile = blockIdx.x, ti = 0;
  while (tile >= nt - ti) {
    tile -= nt - ti;
    ++ti;
  }
  const int tj = ti + tile;
  const int i0 = ti * SY_T, j0 = tj * SY_T;
  const int64_t g = blockIdx.y;
  const int64_t p_begin = (int64_t)blockIdx.z * pix_per_slice;
  int64_t p_end = p_begin + pix_per_slice;
  if (p_end > pix_per_group) p_end = pix_per_group;
  const In* xg = x + g * pix_per_group * (int64_t)B;

  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  Acc acc[4][4];
  Wide wide[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      acc[a][b] = 0;
      wide[a][b] = 0;
    }

  int since_flush = 0;
  for (int64_t p0 = p_begin; p0 < p_end; p0 += SY_K) {
    // stage 16 pixels x 64 bands of each operand; element e -> (pixel e/64, band e%64)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = threadIdx.x + q * 256;
      const int pp = e >> 6, bb = e & 63;
      const int64_t p = p0 + pp;
      Stage va = 0, vb = 0;
      if (p < p_end) {
        const In* row = xg + p * B;
        if (i0 + bb < B) va = Tr::load(row[i0 + bb], c_int, c_flt, i0 + bb);
        if (j0 + bb < B) vb = Tr::load(row[j0 + bb], c_int, c_flt, j0 + bb);
      }
      As[pp][bb] = va;
      Bs[pp][bb] = vb;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < SY_K; ++k) {
      Stage a[4], b[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        a[r] = As[k][ty * 4 + r];
        b[r] = Bs[k][tx * 4 + r];
      }
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int s = 0; s < 4; ++s) acc[r][s] += (Acc)a[r] * (Acc)b[s];
    }
    __syncthreads();
    since_flush += SY_K;
    if (since_flush >= 64) {
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          wide[r][s] += (Wide)acc[r][s];
          acc[r][s] = 0;
        }
      since_flush = 0;
    }
  }
  double* o = out + g * out_stride;
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const int i = i0 + ty * 4 + r, j = j0 + tx * 4 + s;
      if (i >= B || j >= B) continue;
      const double v = (double)(wide[r][s] + (Wide)acc[r][s]);
      if (accumulate) {
        atomicAdd(&o[(int64_t)i * B + j], v);
        if (ti != tj) atomicAdd(&o[(int64_t)j * B + i], v);
      } else {
        o[(int64_t)i * B + j] = v;
        if (ti != tj) o[(int64_t)j * B + i] = v;
      }
    }
}

cudaError_t launch_syrk_simt(const void* x, int64_t n_groups, int64_t pix_per_group, int B,
                             int in_type, const int32_t* c_int, const float* c_flt, double* out,
                             int64_t out_stride, int accumulate, cudaStream_t st,
                             LaunchCounter* lc) {
  if (n_groups <= 0 || pix_per_group <= 0) return cudaSuccess;
  const int nt = (B + SY_T - 1) / SY_T;
  const int tiles = nt * (nt + 1) / 2;
  // split large groups over pixel slices (only when accumulating)
  int64_t slices = 1, per = pix_per_group;
  if (accumulate) {
    const int64_t target = 1024;  // pixels per slice
    slices = (pix_per_group + target - 1) / target;
    if (slices > 65535) slices = 65535;
    per = (pix_per_group + slices - 1) / slices;
    per = (per + SY_K - 1) / SY_K * SY_K;
    slices = (pix_per_group + per - 1) / per;
  }
  dim3 grid(tiles, (unsigned)n_groups, (unsigned)slices), block(256);
  if (in_type == IN_U16)
    syrk_simt_kernel<uint16_t><<<grid, block, 0, st>>>((const uint16_t*)x, pix_per_group, B, c_int,
                                                       nullptr, out, out_stride, per, accumulate);
  else
    syrk_simt_kernel<float><<<grid, block, 0, st>>>((const float*)x, pix_per_group, B, nullptr,
                                                    c_flt, out, out_stride, per, accumulate);
  HSAD_LAUNCH_CHECK(lc);
}

// ---------------------------------------------------------------------------------
// K3a prefix_mean: thread per band walks the lines of the batch in order.
// EXCLUSIVE (inclusive = 0): line t uses the lines before it; INCLUSIVE: through it.
// One warp per band scans 32 lines at a time with shuffles (u16 sums are exact
// integers, so the scan order does not change them).
__global__ void prefix_mean_kernel(const double* __restrict__ s1_line, double* __restrict__ m_out,
                                   double* __restrict__ state_s1, int64_t n0_arg, int W, int L, int B,
                                   int inclusive, int64_t min_pixels, int32_t* __restrict__ status,
                                   const int64_t* __restrict__ n0_dev, const double* __restrict__ gain,
                                   const int32_t* __restrict__ c_int, double lam,
                                   const double* __restrict__ n_line) {
  const int64_t n0 = n0_dev ? *n0_dev : n0_arg;
  const int lane = threadIdx.x & 31;
  const int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const double lam_lane = lam == 1.0 ? 1.0 : pow(lam, (double)(lane + 1));
  if (b < B) {
    double carry = state_s1[b];
    for (int t0 = 0; t0 < L; t0 += 32) {
      const int t = t0 + lane;
      double v = t < L ? s1_line[(int64_t)t * B + b] : 0.0;
      if (gain && t < L) {  // sum of (DN / g - c) = (s1 + W e) / g, e = c (1 - g)
        const double* gt = gain + kGainStride * t;
        v = fma((double)W * (double)c_int[b], gt[3], v) * gt[1];
      }
      double x = v;
      if (lam == 1.0) {
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const double y = __shfl_up_sync(0xffffffffu, x, o);
          if (lane >= o) x += y;
        }
        const double incl = carry + x;
        const double run = inclusive ? incl : incl - v;
        if (t < L) {
          const int64_t n = n0 + (int64_t)(t + inclusive) * W;
          m_out[(int64_t)t * B + b] = n > 0 ? run / (double)n : 0.0;
        }
        carry = __shfl_sync(0xffffffffu, incl, 31);
      } else {
        // forgetting: incl_t = lam incl_{t-1} + v_t, a scan of the affine steps (the
        // partial sum of a lane o places back decays by lam^o)
        double lo = lam;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const double y = __shfl_up_sync(0xffffffffu, x, o);
          if (lane >= o) x = fma(lo, y, x);
          lo *= lo;
        }
        const double incl = fma(lam_lane, carry, x);  // carry decayed over lanes 0..lane
        const double prev = __shfl_up_sync(0xffffffffu, incl, 1);
        const double run = inclusive ? incl : (lane == 0 ? carry : prev);
        if (t < L) {
          const double n = n_line[t];
          m_out[(int64_t)t * B + b] = n > 0.0 ? run / n : 0.0;
        }
        carry = __shfl_sync(0xffffffffu, incl, min(31, L - 1 - t0));  // the last real line
      }
    }
    if (lane == 0) state_s1[b] = carry;
  }
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < L; t += gridDim.x * blockDim.x) {
    const int64_t n = n0 + (int64_t)(t + inclusive) * W;
    const bool few = n_line ? n_line[t] < (double)min_pixels : n < min_pixels;
    if (few && status[t] == LS_OK) status[t] = LS_NOT_READY;
  }
}

cudaError_t launch_prefix_mean(const double* s1_line, double* m_out, double* state_s1, int64_t n0,
                               int W, int L, int B, int inclusive, int64_t min_pixels,
                               int32_t* status, cudaStream_t st, LaunchCounter* lc, const int64_t* n0_dev,
                               const double* gain, const int32_t* c_int, double lam, const double* n_line) {
  if ((gain && !c_int) || (lam != 1.0 && !n_line)) return cudaErrorInvalidValue;
  prefix_mean_kernel<<<(B + 7) / 8, 256, 0, st>>>(s1_line, m_out, state_s1, n0, W, L, B, inclusive,
                                                  min_pixels, status, n0_dev, gain, c_int, lam, n_line);
  HSAD_LAUNCH_CHECK(lc);
}

__global__ void set_batch_desc_kernel(int64_t* desc, int64_t n_stats, int64_t slot1) {
  desc[0] = n_stats;
  desc[1] = slot1;
}

cudaError_t launch_set_batch_desc(int64_t* desc, int64_t n_stats, int64_t slot1, cudaStream_t st,
                                  LaunchCounter* lc) {
  set_batch_desc_kernel<<<1, 1, 0, st>>>(desc, n_stats, slot1);
  HSAD_LAUNCH_CHECK(lc);
}

// K3b prefix_cov: thread per lower-triangle entry walks the lines and replaces each
// line's s2 by the running sum S2_t (EXCLUSIVE: lines before t; INCLUSIVE: through t).
// One FP64 add per entry and line; the covariance itself is formed by the factor
// kernel, which reads each entry once anyway.
__global__ void prefix_cov_kernel(double* __restrict__ buf, double* __restrict__ state_s2, int L, int B,
                                  int inclusive, const double* __restrict__ gain,
                                  const double* __restrict__ s1_line, const int32_t* __restrict__ c_int, int W,
                                  double lam) {
  const int64_t BB = (int64_t)B * B;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= BB) return;
  const int i = (int)(e / B), j = (int)(e % B);
  if (j > i) return;
  double run = state_s2[e];
  constexpr int U = 8;  // lines whose loads are in flight together (32 measured slower)
  for (int t0 = 0; t0 < L; t0 += U) {
    double v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) v[u] = (t0 + u < L) ? buf[(int64_t)(t0 + u) * BB + e] : 0.0;
    if (gain) {
      // sum of (DN/g - c)_i (DN/g - c)_j = (s2 + s1_i e_j + e_i s1_j + W e_i e_j) / g^2
      const double ci = (double)c_int[i], cj = (double)c_int[j], wci = (double)W * ci;
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int t = t0 + u;
        if (t < L) {
          const double* gt = gain + kGainStride * t;
          const double h = gt[3];
          const double* s1 = s1_line + (int64_t)t * B;
          // h (s1_i c_j + c_i s1_j + W h c_i c_j)
          const double x = fma(s1[i], cj, fma(ci, s1[j], wci * h * cj));
          v[u] = fma(h, x, v[u]) * gt[2];
        }
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (t0 + u >= L) break;
      const double before = run;
      run = lam == 1.0 ? run + v[u] : fma(lam, run, v[u]);
      buf[(int64_t)(t0 + u) * BB + e] = inclusive ? run : before;
    }
  }
  state_s2[e] = run;
}

cudaError_t launch_prefix_cov(double* buf, double* state_s2, int L, int B, int inclusive, cudaStream_t st,
                              LaunchCounter* lc, const double* gain, const double* s1_line, const int32_t* c_int,
                              int W, double lam) {
  if (gain && (!s1_line || !c_int)) return cudaErrorInvalidValue;
  const int64_t BB = (int64_t)B * B;
  prefix_cov_kernel<<<(unsigned)((BB + 255) / 256), 256, 0, st>>>(buf, state_s2, L, B, inclusive, gain, s1_line,
                                                                  c_int, W, lam);
  HSAD_LAUNCH_CHECK(lc);
}

// Forgetting weight of a window after k more lines of W pixels, from n_prev:
// lam^k n_prev + W (1 - lam^k) / (1 - lam), the geometric sum by expm1 (no cancellation
// for lam near 1). The host uses the same function for the state it carries.
__host__ __device__ double forget_weight_hd(double n_prev, double lam, int W, int64_t k) {
  const double ll = log(lam);
  const double lk = exp((double)k * ll);
  return fma(lk, n_prev, (double)W * (expm1((double)k * ll) / expm1(ll)));
}

double forget_weight(double n_prev, double lam, int W, int64_t k) { return forget_weight_hd(n_prev, lam, W, k); }

__global__ void forget_n_kernel(double n_prev, double lam, int W, int L, int incl, double* __restrict__ n_line) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < L) n_line[t] = forget_weight_hd(n_prev, lam, W, (int64_t)(t + incl));
}

cudaError_t launch_forget_n(double n_prev, double lam, int W, int L, int incl, double* n_line, cudaStream_t st,
                            LaunchCounter* lc) {
  if (L <= 0) return cudaSuccess;
  forget_n_kernel<<<(L + 255) / 256, 256, 0, st>>>(n_prev, lam, W, L, incl, n_line);
  HSAD_LAUNCH_CHECK(lc);
}

// Per-line gain correction of a whitening launch: m'_t = g (m_f + c) - c in FP64 from the
// FP32 mean offset of line t's factor slot, and 1 / g^2.
__global__ void gain_mean_kernel(const double* __restrict__ gain, int B, const float* __restrict__ y0,
                                 const int32_t* __restrict__ c_int, int factor_stride, ScoreOut out,
                                 float* __restrict__ m_out, float* __restrict__ scale_out) {
  const int t = blockIdx.y;
  const int Bp = pad64(B);
  const int f = factor_slot(out, factor_stride, t);
  const double g = gain[kGainStride * t], q = gain[kGainStride * t + 2];
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < Bp; b += gridDim.x * blockDim.x) {
    float v = 0.f;
    if (b < B) {
      const double c = (double)c_int[b];
      v = (float)(fma(g, (double)y0[(int64_t)f * Bp + b] + c, -c));
    }
    m_out[(int64_t)t * Bp + b] = v;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) scale_out[t] = (float)q;
}

cudaError_t launch_gain_mean(const double* gain, int L, int B, const float* y0, const int32_t* c_int,
                             int factor_stride, ScoreOut out, float* m_out, float* scale_out, cudaStream_t st,
                             LaunchCounter* lc) {
  if (L <= 0) return cudaSuccess;
  gain_mean_kernel<<<dim3(1, L), 256, 0, st>>>(gain, B, y0, c_int, factor_stride, out, m_out, scale_out);
  HSAD_LAUNCH_CHECK(lc);
}

// K3c finalize_cov (cube mode): the cube's raw sums S2 (lower triangle, read from the
// lower triangle of the state) and m = S1 / N; the factor kernel forms Sigma from them.
__global__ void finalize_cov_kernel(const double* __restrict__ s1, const double* __restrict__ s2,
                                    int64_t n, int B,
                                    double* __restrict__ sigma, double* __restrict__ m,
                                    int64_t min_pixels, int32_t* __restrict__ status) {
  const int64_t BB = (int64_t)B * B;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= BB) return;
  const int i = (int)(e / B), j = (int)(e % B);
  if (j <= i) sigma[e] = s2[e];
  if (j == 0) m[i] = s1[i] / (double)n;
  if (e == 0) status[0] = (n >= min_pixels && n > 1) ? LS_OK : LS_NOT_READY;
}

cudaError_t launch_finalize_cov(const double* state_s1, const double* state_s2, int64_t n, int B, double* sigma, double* m, int64_t min_pixels,
                                int32_t* status, cudaStream_t st, LaunchCounter* lc) {
  const int64_t BB = (int64_t)B * B;
  finalize_cov_kernel<<<(unsigned)((BB + 255) / 256), 256, 0, st>>>(state_s1, state_s2, n,
                                                                    B, sigma, m, min_pixels, status);
  HSAD_LAUNCH_CHECK(lc);
}

// ---------------------------------------------------------------------------------
__global__ void check_finite_kernel(const float* __restrict__ x, int64_t n, int32_t* bad) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int found = 0;
  for (; i < n; i += stride) found |= !isfinite(x[i]);
  if (__syncthreads_or(found) && threadIdx.x == 0) atomicExch(bad, 1);
}

cudaError_t launch_check_finite(const float* x, int64_t n, int32_t* bad, cudaStream_t st,
                                LaunchCounter* lc) {
  if (n <= 0) return cudaSuccess;
  int64_t blocks = (n + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  check_finite_kernel<<<(unsigned)blocks, 256, 0, st>>>(x, n, bad);
  HSAD_LAUNCH_CHECK(lc);
}

}  // namespace hsad
