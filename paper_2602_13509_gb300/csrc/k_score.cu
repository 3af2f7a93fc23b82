// K6 (SIMT form) whitening + score, and K7 cube normalisation / threshold.
//
// Eq. 1 (Sec. 3.3): delta = (x - mu)^T Sigma^{-1} (x - mu) = || G x' - y0 ||^2 / s^2 with
// the whitening operand G, offset y0 and scale s built by the factor kernel. The
// contraction Y = X' G^T (pixels x bands times bands x bands, G lower triangular so the
// k loop of output tile n stops at the tile's last row) is followed in registers by the
// row norm, so Y is never written. The mask marks scores above the threshold
// (Sec. 3.3, last paragraph; strict ">").
//
// Operand terms per working precision (products exact in FP32, FP32 accumulation):
//   FP32 : x' (exact for uint16) times G (float)
//   FP16 : h(x') times G_hi, h(x') times G_lo           (h: round to FP16; integer input)
//          H times G_hi, H times G_lo, R times G_hi      (float input: H = h(x'), R = h(x' - H))
//   BF16 : H times G_hi, H times G_lo, R times G_hi      (x' = H + R, both exact in BF16:
//          integer input H = 64 rint(x'/64); float input H = bf16(x'), R = bf16(x' - H))
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "hsad_internal.h"

namespace hsad {

namespace {
constexpr int WS_P = 64, WS_N = 64, WS_K = 16;

template <typename In>
__device__ __forceinline__ float centred(In v, const int32_t* ci, const float* cf, int b);
template <>
__device__ __forceinline__ float centred<uint16_t>(uint16_t v, const int32_t* ci, const float*, int b) {
  // DN - c exactly: the bits of 1.5 * 2^23 + (DN - c) minus 1.5 * 2^23 (no conversion instruction)
  return __int_as_float(0x4B400000 + (int)v - ci[b]) - 12582912.0f;
}
template <>
__device__ __forceinline__ float centred<float>(float v, const int32_t*, const float* cf, int b) {
  return v - cf[b];
}

template <typename In, int PREC>
__device__ __forceinline__ void split_x(float x, float& a0, float& a1) {
  if (PREC == P_FP32) {
    a0 = x;
    a1 = 0.f;
  } else if (PREC == P_FP16) {
    a0 = __half2float(__float2half_rn(x));
    a1 = sizeof(In) == 4 ? __half2float(__float2half_rn(x - a0)) : 0.f;
  } else {
    if (sizeof(In) == 2) {
      const float h = 64.f * rintf(x * (1.f / 64.f));
      a0 = h;
      a1 = x - h;
    } else {
      const float h = __bfloat162float(__float2bfloat16_rn(x));
      a0 = h;
      a1 = __bfloat162float(__float2bfloat16_rn(x - h));
    }
  }
}

template <int PREC>
__device__ __forceinline__ void load_w(const void* w, int64_t plane, int64_t idx, float& b0, float& b1) {
  if (PREC == P_FP32) {
    b0 = ((const float*)w)[idx];
    b1 = 0.f;
  } else if (PREC == P_FP16) {
    b0 = __half2float(((const __half*)w)[idx]);
    b1 = __half2float(((const __half*)w)[plane + idx]);
  } else {
    b0 = __bfloat162float(((const __nv_bfloat16*)w)[idx]);
    b1 = __bfloat162float(((const __nv_bfloat16*)w)[plane + idx]);
  }
}
}  // namespace

template <typename In, int PREC>
__global__ void __launch_bounds__(256) whiten_score_kernel(
    const In* __restrict__ x, int W, int B, const int32_t* __restrict__ c_int,
    const float* __restrict__ c_flt, const void* __restrict__ wmat, const float* __restrict__ y0_all,
    const float* __restrict__ inv_s2_all, const int32_t* __restrict__ status, int factor_stride,
    ScoreOut out) {
  // two stages (double buffering) x two operand terms; rows padded by 4 floats: the
  // staging stores walk k fastest
  __shared__ __align__(16) float As[2][2][WS_K][WS_P + 4];
  __shared__ __align__(16) float Bs[2][2][WS_K][WS_N + 4];
  const int t = blockIdx.y;
  const int p0 = blockIdx.x * WS_P;
  const int f = factor_slot(out, factor_stride, t);
  const int64_t slot = (slot0_of(out) + t) % out.ring;
  const int st = status[f];
  if (blockIdx.x == 0 && threadIdx.x == 0) out.ring_status[slot] = st;
  if (st != LS_OK) {
    for (int p = p0 + threadIdx.x; p < p0 + WS_P && p < W; p += blockDim.x) {
      out.scores[slot * W + p] = __int_as_float(0x7fc00000);
      out.mask[slot * W + p] = 0;
    }
    return;
  }
  const int Bp = pad64(B);
  const int64_t plane = (int64_t)Bp * Bp;
  const void* w = (const char*)wmat + (size_t)f * plane * 4;
  const float* y0 = y0_all + (int64_t)f * Bp;
  const In* xl = x + (int64_t)t * W * B;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;

  // One step = (output block n0, k slice k0); G is lower triangular, so block n0 stops at
  // k = n0 + 64. The next step's operands are loaded into registers while the current
  // step computes from shared memory, then stored into the other stage.
  float ra0[4], ra1[4], rb0[4], rb1[4];
  auto load_step = [&](int n0s, int k0s) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = threadIdx.x + q * 256;
      const int rr = e >> 4, kk = e & 15;
      const int k = k0s + kk;
      float a0 = 0.f, a1 = 0.f, b0 = 0.f, b1 = 0.f;
      const int p = p0 + rr;
      if (p < W && k < B) {
        const float xc = centred<In>(xl[(int64_t)p * B + k], c_int, c_flt, k);
        split_x<In, PREC>(xc, a0, a1);
      }
      const int n = n0s + rr;
      if (n < B && k < Bp) load_w<PREC>(w, plane, (int64_t)n * Bp + k, b0, b1);
      ra0[q] = a0;
      ra1[q] = a1;
      rb0[q] = b0;
      rb1[q] = b1;
    }
  };
  auto store_step = [&](int buf) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = threadIdx.x + q * 256;
      const int rr = e >> 4, kk = e & 15;
      As[buf][0][kk][rr] = ra0[q];
      As[buf][1][kk][rr] = ra1[q];
      Bs[buf][0][kk][rr] = rb0[q];
      Bs[buf][1][kk][rr] = rb1[q];
    }
  };

  float dsum[4] = {0.f, 0.f, 0.f, 0.f};
  float acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int s2 = 0; s2 < 4; ++s2) acc[r][s2] = 0.f;
  int n0 = 0, k0 = 0, cur = 0;
  load_step(n0, k0);
  store_step(0);
  __syncthreads();
  while (n0 < B) {
    int nn = n0, nk = k0 + WS_K;
    const bool last_k = nk >= min(B, n0 + WS_N);
    if (last_k) {
      nn = n0 + WS_N;
      nk = 0;
    }
    const bool more = nn < B;
    if (more) load_step(nn, nk);
#pragma unroll
    for (int kk = 0; kk < WS_K; ++kk) {
      float a0[4], b0[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        a0[r] = As[cur][0][kk][ty * 4 + r];
        b0[r] = Bs[cur][0][kk][tx * 4 + r];
      }
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int s2 = 0; s2 < 4; ++s2) acc[r][s2] = fmaf(a0[r], b0[s2], acc[r][s2]);
      if (PREC != P_FP32) {
        float b1[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) b1[r] = Bs[cur][1][kk][tx * 4 + r];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int s2 = 0; s2 < 4; ++s2) acc[r][s2] = fmaf(a0[r], b1[s2], acc[r][s2]);
      }
      if (PREC == P_BF16 || (PREC == P_FP16 && sizeof(In) == 4)) {
        float a1[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) a1[r] = As[cur][1][kk][ty * 4 + r];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int s2 = 0; s2 < 4; ++s2) acc[r][s2] = fmaf(a1[r], b0[s2], acc[r][s2]);
      }
    }
    if (last_k) {  // block n0 complete: fold its outputs into the row norms
#pragma unroll
      for (int s2 = 0; s2 < 4; ++s2) {
        const int n = n0 + tx * 4 + s2;
        if (n < B) {
          const float yn = y0[n];
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            const float v = acc[r][s2] - yn;
            dsum[r] = fmaf(v, v, dsum[r]);
          }
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) acc[r][s2] = 0.f;
      }
    }
    if (more) store_step(cur ^ 1);
    __syncthreads();
    cur ^= 1;
    n0 = nn;
    k0 = nk;
  }
  // row norm: reduce over the 16 lanes sharing ty (lanes tx = 0..15 are contiguous)
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) dsum[r] += __shfl_xor_sync(0xffffffffu, dsum[r], o);
  if (tx == 0) {
    const float is2 = inv_s2_all[f];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int p = p0 + ty * 4 + r;
      if (p < W) {
        const float d = dsum[r] * is2;
        out.scores[slot * W + p] = d;
        if (out.write_mask) out.mask[slot * W + p] = d > out.tau ? 1 : 0;
      }
    }
  }
}

// FP32 form, larger register tiles: one CTA = 128 pixels x 64 outputs n, a thread 8 pixels
// x 4 outputs (32 FFMA per three shared-memory vector loads), k slices of 16 bands staged
// through two shared-memory buffers with the next slice prefetched into registers.
constexpr int WF_P = 128, WF_N = 64, WF_K = 16;

template <typename In>
__global__ void __launch_bounds__(256) whiten_fp32_kernel(
    const In* __restrict__ x, int W, int B, const int32_t* __restrict__ c_int, const float* __restrict__ c_flt,
    const float* __restrict__ wmat, const float* __restrict__ y0_all, const float* __restrict__ inv_s2_all,
    const int32_t* __restrict__ status, int factor_stride, ScoreOut out) {
  __shared__ __align__(16) float As[2][WF_K][WF_P + 4];
  __shared__ __align__(16) float Bs[2][WF_K][WF_N + 4];
  const int t = blockIdx.y;
  const int p0 = blockIdx.x * WF_P;
  const int f = factor_slot(out, factor_stride, t);
  const int64_t slot = (slot0_of(out) + t) % out.ring;
  const int st = status[f];
  if (blockIdx.x == 0 && threadIdx.x == 0) out.ring_status[slot] = st;
  if (st != LS_OK) {
    for (int p = p0 + threadIdx.x; p < p0 + WF_P && p < W; p += blockDim.x) {
      out.scores[slot * W + p] = __int_as_float(0x7fc00000);
      out.mask[slot * W + p] = 0;
    }
    return;
  }
  const int Bp = pad64(B);
  const float* g = wmat + (size_t)f * Bp * Bp;
  const float* y0 = y0_all + (int64_t)f * Bp;
  const In* xl = x + (int64_t)t * W * B;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;  // 4 outputs tx*4.., 8 pixels ty*8..

  float ra[8], rb[4];
  auto load_step = [&](int n0s, int k0s) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {  // pixels: 16 threads read 16 consecutive bands of one pixel
      const int e = threadIdx.x + q * 256;
      const int pr = e >> 4, kk = e & 15, k = k0s + kk, p = p0 + pr;
      ra[q] = (p < W && k < B) ? centred<In>(xl[(int64_t)p * B + k], c_int, c_flt, k) : 0.f;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = threadIdx.x + q * 256;
      const int nr = e >> 4, kk = e & 15, k = k0s + kk, n = n0s + nr;
      rb[q] = (n < B && k < Bp) ? g[(int64_t)n * Bp + k] : 0.f;
    }
  };
  auto store_step = [&](int buf) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int e = threadIdx.x + q * 256;
      As[buf][e & 15][e >> 4] = ra[q];
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = threadIdx.x + q * 256;
      Bs[buf][e & 15][e >> 4] = rb[q];
    }
  };

  float dsum[8];
  float acc[8][4];
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    dsum[r] = 0.f;
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = 0.f;
  }
  int n0 = 0, k0 = 0, cur = 0;
  load_step(n0, k0);
  store_step(0);
  __syncthreads();
  while (n0 < B) {  // G is lower triangular: block n0 stops at k = n0 + 64
    int nn = n0, nk = k0 + WF_K;
    const bool last_k = nk >= min(B, n0 + WF_N);
    if (last_k) {
      nn = n0 + WF_N;
      nk = 0;
    }
    const bool more = nn < B;
    if (more) load_step(nn, nk);
#pragma unroll
    for (int kk = 0; kk < WF_K; ++kk) {
      const float4 a0 = *(const float4*)&As[cur][kk][ty * 8];
      const float4 a1 = *(const float4*)&As[cur][kk][ty * 8 + 4];
      const float4 b = *(const float4*)&Bs[cur][kk][tx * 4];
      const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(av[r], bv[c], acc[r][c]);
    }
    if (last_k) {  // block n0 complete: fold its outputs into the row norms
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int n = n0 + tx * 4 + c;
        if (n < B) {
          const float yn = y0[n];
#pragma unroll
          for (int r = 0; r < 8; ++r) {
            const float v = acc[r][c] - yn;
            dsum[r] = fmaf(v, v, dsum[r]);
          }
        }
#pragma unroll
        for (int r = 0; r < 8; ++r) acc[r][c] = 0.f;
      }
    }
    if (more) store_step(cur ^ 1);
    __syncthreads();
    cur ^= 1;
    n0 = nn;
    k0 = nk;
  }
  // row norm: reduce over the 16 lanes sharing ty (lanes tx = 0..15 are contiguous)
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) dsum[r] += __shfl_xor_sync(0xffffffffu, dsum[r], o);
  if (tx == 0) {
    const float is2 = inv_s2_all[f];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int p = p0 + ty * 8 + r;
      if (p < W) {
        const float d = dsum[r] * is2;
        out.scores[slot * W + p] = d;
        if (out.write_mask) out.mask[slot * W + p] = d > out.tau ? 1 : 0;
      }
    }
  }
}

cudaError_t launch_whiten_score_simt(const void* x, int L, int W, int B, int in_type,
                                     const int32_t* c_int, const float* c_flt, int prec,
                                     const void* wmat, const float* y0, const float* inv_s2,
                                     const int32_t* status, int factor_stride, ScoreOut out,
                                     cudaStream_t st, LaunchCounter* lc) {
  if (L <= 0) return cudaSuccess;
  if (prec == P_FP32) {
    dim3 g2((W + WF_P - 1) / WF_P, L), b2(256);
    if (in_type == IN_U16)
      whiten_fp32_kernel<uint16_t><<<g2, b2, 0, st>>>((const uint16_t*)x, W, B, c_int, c_flt, (const float*)wmat, y0,
                                                      inv_s2, status, factor_stride, out);
    else
      whiten_fp32_kernel<float><<<g2, b2, 0, st>>>((const float*)x, W, B, c_int, c_flt, (const float*)wmat, y0,
                                                   inv_s2, status, factor_stride, out);
    if (lc) lc->n += 1;
    return cudaGetLastError();
  }
  dim3 grid((W + WS_P - 1) / WS_P, L), block(256);
#define HSAD_WS(IN, P)                                                                          \
  whiten_score_kernel<IN, P><<<grid, block, 0, st>>>((const IN*)x, W, B, c_int, c_flt, wmat, y0, \
                                                     inv_s2, status, factor_stride, out)
  if (in_type == IN_U16) {
    if (prec == P_FP32) HSAD_WS(uint16_t, P_FP32);
    else if (prec == P_FP16) HSAD_WS(uint16_t, P_FP16);
    else HSAD_WS(uint16_t, P_BF16);
  } else {
    if (prec == P_FP32) HSAD_WS(float, P_FP32);
    else if (prec == P_FP16) HSAD_WS(float, P_FP16);
    else HSAD_WS(float, P_BF16);
  }
#undef HSAD_WS
  if (lc) lc->n += 1;
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------
// K7: cube maximum (delta >= 0, so the float bit pattern orders like an unsigned int),
// then delta / max and the mask (REL: delta / max > tau; ABS: delta > tau).
__global__ void cube_max_kernel(ScoreOut out, int64_t n_lines, int W, unsigned int* dmax_bits) {
  const int64_t n = n_lines * W;
  float mx = 0.f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t line = i / W, p = i % W;
    const float v = out.scores[((slot0_of(out) + line) % out.ring) * W + p];
    if (v > mx) mx = v;  // NaN compares false
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) atomicMax(dmax_bits, __float_as_uint(mx));
}

__global__ void cube_norm_kernel(ScoreOut out, int64_t n_lines, int W, int rel, int normalize,
                                 const unsigned int* dmax_bits) {
  const float dmax = __uint_as_float(*dmax_bits);
  const int64_t n = n_lines * W;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t line = i / W, p = i % W;
    const int64_t at = ((slot0_of(out) + line) % out.ring) * W + p;
    const float v = out.scores[at];
    const float r = v / dmax;
    out.mask[at] = (rel ? (r > out.tau) : (v > out.tau)) ? 1 : 0;
    if (normalize) out.scores[at] = r;
  }
}

cudaError_t launch_cube_normalize(ScoreOut out, int64_t n_lines, int W, int rel, int normalize,
                                  unsigned int* dmax_bits, cudaStream_t st, LaunchCounter* lc) {
  if (n_lines <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(dmax_bits, 0, sizeof(unsigned int), st);
  if (e != cudaSuccess) return e;
  int64_t blocks = (n_lines * W + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  cube_max_kernel<<<(unsigned)blocks, 256, 0, st>>>(out, n_lines, W, dmax_bits);
  cube_norm_kernel<<<(unsigned)blocks, 256, 0, st>>>(out, n_lines, W, rel, normalize, dmax_bits);
  if (lc) lc->n += 2;
  return cudaGetLastError();
}

}  // namespace hsad
