// K6, triangular-solve form on the SIMT cores (FP32 working precision): y = L^{-1} (x' - m)
// by blocked forward substitution and delta = ||y||^2 (Eq. 1, Sec. 3.3).
//
// Same blocking as the tensor-core form: for the 64-band block k,
//   z_k = (x'_k - m_k) - sum_{j<k} L_kj y_j,   y_k = L_kk^{-1} z_k,
// with H (FP32) holding L_jk below the diagonal blocks and L_kk^{-1} on them, so block k is
// one pass over block row k of H: columns [0, 64k) against y, then the diagonal block
// against z. Left-looking: the CTA keeps v = x' - m of its 64 pixels for all bands in shared
// memory (band-major) and overwrites block k with z_k and then y_k; H is streamed through
// two shared-memory slices of 16 columns, the next slice prefetched into registers. A thread
// owns a 4 x 4 tile (4 consecutive pixels x bands tx, tx + 16, tx + 32, tx + 48 of the block:
// the slice is stored with those four bands side by side, one 16-byte load per column, and
// the tile's z / y rows are written as conflict-free 16-byte stores) and its pixels' partial
// row norms.
#include <cuda_runtime.h>
#include <stdint.h>

#include "hsad_internal.h"

namespace hsad {

namespace {
constexpr int TF_P = 64, TF_N = 64, TF_K = 16, TF_THREADS = 256;
constexpr int TF_YS = TF_P + 4;  // band-row stride of the pixel buffer (floats)

// acc[r][c] += y[p_r][c0 + kk] * H[n_c][c0 + kk] over one 16-column slice, for the first NC
// of the thread's four bands (the block's bands past B need no work: NC < 4 only in the
// last block)
template <int NC>
__device__ __forceinline__ void slice_fma(float (&acc)[4][4], const float* ysrow, const float* hs, int ty, int tx) {
#pragma unroll
  for (int kk = 0; kk < TF_K; ++kk) {
    const float4 a = *(const float4*)&ysrow[kk * TF_YS + ty * 4];
    const float av[4] = {a.x, a.y, a.z, a.w};
    float bv[4];
    if (NC == 4) {
      const float4 b = *(const float4*)&hs[kk * (TF_N + 4) + tx * 4];
      bv[0] = b.x;
      bv[1] = b.y;
      bv[2] = b.z;
      bv[3] = b.w;
    } else {
#pragma unroll
      for (int c = 0; c < NC; ++c) bv[c] = hs[kk * (TF_N + 4) + tx * 4 + c];
    }
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < NC; ++c) acc[r][c] = fmaf(av[r], bv[c], acc[r][c]);
  }
}

template <typename In>
__device__ __forceinline__ float centred_t(In v, const int32_t* ci, const float* cf, int b);
template <>
__device__ __forceinline__ float centred_t<uint16_t>(uint16_t v, const int32_t* ci, const float*, int b) {
  // DN - c exactly: the bits of 1.5 * 2^23 + (DN - c) minus 1.5 * 2^23 (no conversion instruction)
  return __int_as_float(0x4B400000 + (int)v - ci[b]) - 12582912.0f;
}
template <>
__device__ __forceinline__ float centred_t<float>(float v, const int32_t*, const float* cf, int b) {
  return v - cf[b];
}
}  // namespace

template <typename In>
__global__ void __launch_bounds__(TF_THREADS) whiten_trsm_simt_kernel(
    const In* __restrict__ x, int W, int B, const int32_t* __restrict__ c_int, const float* __restrict__ c_flt,
    const float* __restrict__ H_all, const float* __restrict__ m_all, const float* __restrict__ inv_s2_all,
    const int32_t* __restrict__ status, int factor_stride, ScoreOut out) {
  extern __shared__ __align__(16) float ys[];  // [Bp][TF_YS]: v, then z_k / y_k per block
  __shared__ __align__(16) float Hs[2][TF_K][TF_N + 4];
  const int t = blockIdx.y;
  const int p0 = blockIdx.x * TF_P;
  const int f = factor_slot(out, factor_stride, t);
  const int64_t slot = (slot0_of(out) + t) % out.ring;
  const int st = status[f];
  if (blockIdx.x == 0 && threadIdx.x == 0) out.ring_status[slot] = st;
  if (st != LS_OK) {
    for (int p = p0 + threadIdx.x; p < p0 + TF_P && p < W; p += blockDim.x) {
      out.scores[slot * W + p] = __int_as_float(0x7fc00000);
      out.mask[slot * W + p] = 0;
    }
    return;
  }
  const int Bp = pad64(B), nkb = Bp / TF_N;
  const int npx = min(TF_P, W - p0);
  const float* H = H_all + (size_t)f * Bp * Bp;
  // mean offset: the factor slot's, or the gain-corrected one of this line
  const float* m = out.m_line ? out.m_line + (int64_t)t * Bp : m_all + (int64_t)f * Bp;
  const In* xt = x + ((int64_t)t * W + p0) * B;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tx = tid & 15, ty = tid >> 4;  // bands tx + 16 c, pixels ty*4..

  // v = x' - m, band-major (pixel rows read coalesced; zeros outside the tile and past B)
  for (int r = warp; r < TF_P; r += TF_THREADS / 32)
    for (int n = lane; n < Bp; n += 32) {
      float v = 0.f;
      if (r < npx && n < B) v = centred_t<In>(xt[(int64_t)r * B + n], c_int, c_flt, n) - m[n];
      ys[n * TF_YS + r] = v;
    }

  // steps (k, c0): block row k of H, 16 columns at a time, c0 = 0 .. 64k + 48
  float rb[4];
  auto load_slice = [&](int k, int c0) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = tid + q * TF_THREADS;
      const int nr = e >> 4, kk = e & 15;
      rb[q] = H[(int64_t)(k * TF_N + nr) * Bp + c0 + kk];  // rows and columns < Bp (zero-padded)
    }
  };
  auto store_slice = [&](int buf) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = tid + q * TF_THREADS;
      const int nr = e >> 4;
      Hs[buf][e & 15][((nr & 15) << 2) | (nr >> 4)] = rb[q];  // band nr at lane nr % 16, slot nr / 16
    }
  };
  float acc[4][4];
  float dsum[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = 0.f;
  int k = 0, c0 = 0, cur = 0;
  load_slice(0, 0);
  store_slice(0);
  __syncthreads();
  while (k < nkb) {
    const int n0 = k * TF_N;
    int nk = k, nc = c0 + TF_K;
    const bool last = nc == n0 + TF_N;
    if (last) {
      nk = k + 1;
      nc = 0;
    }
    const bool more = nk < nkb;
    if (more) load_slice(nk, nc);
    if (c0 == n0) {
      // the diagonal block starts: z_k = v_k - sum_{j<k} L_kj y_j, in place
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        float4* yp = (float4*)&ys[(n0 + tx + 16 * c) * TF_YS + ty * 4];
        float4 v = *yp;
        v.x -= acc[0][c];
        v.y -= acc[1][c];
        v.z -= acc[2][c];
        v.w -= acc[3][c];
        *yp = v;
#pragma unroll
        for (int r = 0; r < 4; ++r) acc[r][c] = 0.f;
      }
      __syncthreads();
    }
    // columns past B are zero in H; band groups past B need no output
    if (c0 < B) {
      const int groups = min(4, (B - n0 + 15) >> 4);  // band groups of this block below B
      const float* ysrow = &ys[c0 * TF_YS];
      const float* hs = &Hs[cur][0][0];
      if (groups == 4) slice_fma<4>(acc, ysrow, hs, ty, tx);
      else if (groups == 3) slice_fma<3>(acc, ysrow, hs, ty, tx);
      else if (groups == 2) slice_fma<2>(acc, ysrow, hs, ty, tx);
      else slice_fma<1>(acc, ysrow, hs, ty, tx);
    }
    if (last) {
      // y_k = L_kk^{-1} z_k: replaces z_k once every thread has read it
      __syncthreads();
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        *(float4*)&ys[(n0 + tx + 16 * c) * TF_YS + ty * 4] = make_float4(acc[0][c], acc[1][c], acc[2][c], acc[3][c]);
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          dsum[r] = fmaf(acc[r][c], acc[r][c], dsum[r]);
          acc[r][c] = 0.f;
        }
      }
    }
    if (more) store_slice(cur ^ 1);
    __syncthreads();
    cur ^= 1;
    k = nk;
    c0 = nc;
  }
  // row norms: reduce over the 16 lanes sharing ty
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) dsum[r] += __shfl_xor_sync(0xffffffffu, dsum[r], o);
  if (tx == 0) {
    const float is2 = inv_s2_all[f], ls = out.line_scale ? out.line_scale[t] : 1.f;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int p = p0 + ty * 4 + r;
      if (p < W) {
        float d = dsum[r] * is2;
        if (out.line_scale) d *= ls;
        out.scores[slot * W + p] = d;
        if (out.write_mask) out.mask[slot * W + p] = d > out.tau ? 1 : 0;
      }
    }
  }
}

cudaError_t launch_whiten_trsm_simt(const void* x, int L, int W, int B, int in_type, const int32_t* c_int,
                                    const float* c_flt, const float* H, const float* m, const float* inv_s2,
                                    const int32_t* status, int factor_stride, ScoreOut out, cudaStream_t st,
                                    LaunchCounter* lc) {
  if (L <= 0) return cudaSuccess;
  const int smem = pad64(B) * TF_YS * (int)sizeof(float);
  dim3 grid((W + TF_P - 1) / TF_P, L), block(TF_THREADS);
  cudaError_t e;
  if (in_type == IN_U16) {
    e = cudaFuncSetAttribute(whiten_trsm_simt_kernel<uint16_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    whiten_trsm_simt_kernel<uint16_t><<<grid, block, smem, st>>>((const uint16_t*)x, W, B, c_int, c_flt, H, m,
                                                                 inv_s2, status, factor_stride, out);
  } else {
    e = cudaFuncSetAttribute(whiten_trsm_simt_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    whiten_trsm_simt_kernel<float><<<grid, block, smem, st>>>((const float*)x, W, B, c_int, c_flt, H, m, inv_s2,
                                                              status, factor_stride, out);
  }
  if (lc) lc->n += 1;
  return cudaGetLastError();
}

}  // namespace hsad
