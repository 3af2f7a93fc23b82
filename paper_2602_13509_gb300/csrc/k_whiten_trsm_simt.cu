// K6, triangular-solve form on the SIMT cores (FP32 working precision): y = L^{-1} (x' - m)
// by blocked forward substitution and delta = ||y||^2 (Eq. 1, Sec. 3.3).
//
// Same blocking as the tensor-core form: for the 64-band block k,
//   z_k = (x'_k - m_k) - sum_{j<k} L_kj y_j,   y_k = L_kk^{-1} z_k,
// with H (FP32, stored column-major: H_T[c][n] = H[n][c]) holding L_jk below the diagonal
// blocks and L_kk^{-1} on them. Each block is two FFMA contractions over 128 pixels:
// Z_k = V_k - Y_{<k} H_k,<k^T (K = 64 k) and Y_k = Z_k H_kk^T (K = 64). A thread owns
// 8 pixels x 4 bands of the 128 x 64 output tile. The K operand slices (32 bands of y for
// the 128 pixels, 32 rows of H_T for the block's 64 bands) stream through a double-buffered
// shared-memory ring filled by cp.async, one barrier per 32-band slice. The y of earlier
// blocks are kept in a per-CTA scratch slot in global memory (band-major [Bp][128], about
// 57 KB at B = 448 per resident CTA, L2-resident) instead of shared memory, so that two CTAs
// fit on an SM; the kernel is persistent, each CTA looping over (line, 128-pixel tile)
// items with its own slot.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "hsad_internal.h"

namespace hsad {

namespace {
constexpr int T2_P = 128, T2_N = 64, T2_K = 32, T2_THREADS = 256;
constexpr int T2_YS = T2_P + 4;  // row stride (floats) of the pixel-major rows in shared memory
constexpr int T2_HS = T2_N + 4;  // row stride of the H slice
constexpr int T2_SMEM = (2 * T2_K * T2_YS + 2 * T2_K * T2_HS + T2_N * T2_YS) * 4;

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

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

// acc[r][c] += A[kk][px 8 ty + r] * Hs[kk][band 4 tx + c] over one K slice of 32
__device__ __forceinline__ void slice_fma(float (&acc)[8][4], const float* As, const float* Hs, int ty, int tx) {
#pragma unroll
  for (int kk = 0; kk < T2_K; ++kk) {
    const float4 a0 = *(const float4*)&As[kk * T2_YS + ty * 8];
    const float4 a1 = *(const float4*)&As[kk * T2_YS + ty * 8 + 4];
    const float4 b = *(const float4*)&Hs[kk * T2_HS + tx * 4];
    const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
    const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(av[r], bv[c], acc[r][c]);
  }
}
}  // namespace

template <typename In>
__global__ void __launch_bounds__(T2_THREADS, 2) whiten_trsm_simt_kernel(
    const In* __restrict__ x, int L, int W, int B, const int32_t* __restrict__ c_int, const float* __restrict__ c_flt,
    const float* __restrict__ H_all, const float* __restrict__ m_all, const float* __restrict__ inv_s2_all,
    const int32_t* __restrict__ status, int factor_stride, ScoreOut out, float* __restrict__ yscratch) {
  extern __shared__ __align__(16) float sm[];
  float* Ys = sm;                          // [2][T2_K][T2_YS]  y (or z) slices, pixel-major rows
  float* Hs = Ys + 2 * T2_K * T2_YS;       // [2][T2_K][T2_HS]  H_T slices
  float* Vs = Hs + 2 * T2_K * T2_HS;       // [T2_N][T2_YS]     v_k, then z_k, of the block
  const int Bp = pad64(B), nkb = Bp / T2_N;
  const int tiles = (W + T2_P - 1) / T2_P;
  const int64_t items = (int64_t)L * tiles;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  float* Yg = yscratch + (size_t)blockIdx.x * Bp * T2_P;  // this CTA's slot, [Bp][T2_P]

  for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
    const int t = (int)(it / tiles);
    const int p0 = (int)(it % tiles) * T2_P;
    const int f = factor_slot(out, factor_stride, t);
    const int64_t slot = (slot0_of(out) + t) % out.ring;
    const int st = status[f];
    if (p0 == 0 && tid == 0) out.ring_status[slot] = st;
    if (st != LS_OK) {
      for (int p = p0 + tid; p < p0 + T2_P && p < W; p += T2_THREADS) {
        out.scores[slot * W + p] = __int_as_float(0x7fc00000);
        out.mask[slot * W + p] = 0;
      }
      continue;  // uniform for the CTA
    }
    const int npx = min(T2_P, W - p0);
    const float* HT = H_all + (size_t)f * Bp * Bp;
    const float* m = out.m_line ? out.m_line + (int64_t)t * Bp : m_all + (int64_t)f * Bp;
    const In* xt = x + ((int64_t)t * W + p0) * B;
    float dsum[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};

    for (int k = 0; k < nkb; ++k) {
      const int n0 = k * T2_N;
      // v_k = x' - m for the block's bands, pixel-major rows (zeros outside the tile and past B)
      for (int e = tid; e < T2_N * T2_P; e += T2_THREADS) {
        const int px = e / T2_N, n = e % T2_N;  // consecutive threads: consecutive bands of a pixel
        float v = 0.f;
        if (px < npx && n0 + n < B) v = centred_t<In>(xt[(int64_t)px * B + n0 + n], c_int, c_flt, n0 + n) - m[n0 + n];
        Vs[n * T2_YS + px] = v;
      }
      float acc[8][4];
#pragma unroll
      for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = 0.f;
      // slices: s < 2k over the earlier blocks' y (scratch), then 2 over the diagonal block (z)
      const int nsl = 2 * k + 2;
      auto issue = [&](int sidx, int buf) {
        const int c0 = sidx * T2_K;  // band offset of the slice's K rows
        float* hd = Hs + buf * T2_K * T2_HS;
        for (int e = tid; e < T2_K * (T2_N / 4); e += T2_THREADS) {  // 32 rows x 16 chunks of H_T
          const int kk = e >> 4, ch = e & 15;
          cp_async16(hd + kk * T2_HS + ch * 4, HT + (size_t)(c0 + kk) * Bp + n0 + ch * 4);
        }
        if (sidx < 2 * k) {
          float* yd = Ys + buf * T2_K * T2_YS;
          for (int e = tid; e < T2_K * (T2_P / 4); e += T2_THREADS) {  // 32 rows x 32 chunks of y
            const int kk = e >> 5, ch = e & 31;
            cp_async16(yd + kk * T2_YS + ch * 4, Yg + (size_t)(c0 + kk) * T2_P + ch * 4);
          }
        }
        cp_async_commit();
      };
      issue(0, 0);
      for (int sidx = 0; sidx < nsl; ++sidx) {
        const int buf = sidx & 1;
        cp_async_wait_all();
        if (sidx == 2 * k) {
          // the diagonal block starts: z_k = v_k - sum_{j<k} L_kj y_j into Vs
          __syncthreads();  // v_k written by every thread
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const int n = tx * 4 + c;
#pragma unroll
            for (int r = 0; r < 8; ++r) {
              Vs[n * T2_YS + ty * 8 + r] -= acc[r][c];
              acc[r][c] = 0.f;
            }
          }
        }
        __syncthreads();  // slice sidx landed for everyone; the other buffer is free
        if (sidx + 1 < nsl) issue(sidx + 1, buf ^ 1);
        const float* As = sidx < 2 * k ? Ys + buf * T2_K * T2_YS : Vs + (sidx - 2 * k) * T2_K * T2_YS;
        slice_fma(acc, As, Hs + buf * T2_K * T2_HS, ty, tx);
      }
      // y_k: to this CTA's scratch (band-major) for the next blocks, and into the row norms
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int n = n0 + tx * 4 + c;
        float4* yp = (float4*)(Yg + (size_t)n * T2_P + ty * 8);
        yp[0] = make_float4(acc[0][c], acc[1][c], acc[2][c], acc[3][c]);
        yp[1] = make_float4(acc[4][c], acc[5][c], acc[6][c], acc[7][c]);
#pragma unroll
        for (int r = 0; r < 8; ++r) dsum[r] = fmaf(acc[r][c], acc[r][c], dsum[r]);
      }
      __threadfence();  // the scratch writes are visible to the next block's async copies (L2)
      __syncthreads();
    }
    // row norms: reduce over the 16 lanes sharing ty (a half-warp)
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int o = 8; o > 0; o >>= 1) dsum[r] += __shfl_xor_sync(0xffffffffu, dsum[r], o);
    if (tx == 0) {
      const float is2 = inv_s2_all[f], ls = out.line_scale ? out.line_scale[t] : 1.f;
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const int p = p0 + ty * 8 + r;
        if (p < W) {
          float d = dsum[r] * is2;
          if (out.line_scale) d *= ls;
          out.scores[slot * W + p] = d;
          if (out.write_mask) out.mask[slot * W + p] = d > out.tau ? 1 : 0;
        }
      }
    }
  }
}

int whiten_trsm_simt_slots() {
  static int n = [] {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 152;
    return 2 * sms;
  }();
  return n;
}

size_t whiten_trsm_simt_scratch_bytes(int B) { return (size_t)whiten_trsm_simt_slots() * pad64(B) * T2_P * 4; }

cudaError_t launch_whiten_trsm_simt(const void* x, int L, int W, int B, int in_type, const int32_t* c_int,
                                    const float* c_flt, const float* H, const float* m, const float* inv_s2,
                                    const int32_t* status, int factor_stride, ScoreOut out, float* yscratch,
                                    cudaStream_t st, LaunchCounter* lc) {
  if (L <= 0) return cudaSuccess;
  const int64_t items = (int64_t)L * ((W + T2_P - 1) / T2_P);
  const int grid = (int)std::min<int64_t>(items, whiten_trsm_simt_slots());
  cudaError_t e;
  if (in_type == IN_U16) {
    e = cudaFuncSetAttribute(whiten_trsm_simt_kernel<uint16_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, T2_SMEM);
    if (e != cudaSuccess) return e;
    whiten_trsm_simt_kernel<uint16_t><<<grid, T2_THREADS, T2_SMEM, st>>>(
        (const uint16_t*)x, L, W, B, c_int, c_flt, H, m, inv_s2, status, factor_stride, out, yscratch);
  } else {
    e = cudaFuncSetAttribute(whiten_trsm_simt_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, T2_SMEM);
    if (e != cudaSuccess) return e;
    whiten_trsm_simt_kernel<float><<<grid, T2_THREADS, T2_SMEM, st>>>((const float*)x, L, W, B, c_int, c_flt, H, m,
                                                                       inv_s2, status, factor_stride, out, yscratch);
  }
  if (lc) lc->n += 1;
  return cudaGetLastError();
}

}  // namespace hsad
