// K6, triangular-solve form (BF16 working precision, uint16 input): the whitened vector
// y = L^{-1} (x' - m) by blocked forward substitution on the tensor cores, and the score
// delta = ||y||^2 (Eq. 1, Sec. 3.3) read out of tensor memory.
//
// With S = L L^T the DN-frame covariance, delta = (x' - m)^T S^{-1} (x' - m) = ||y||^2 with
// L y = x' - m. The bands are cut into 64-band blocks; for block k
//   z_k = (x'_k - m_k) - sum_{j<k} L_kj y_j,   y_k = L_kk^{-1} z_k.
// The factor kernel leaves H (BF16 hi / lo planes) with H_jk = L_jk below the diagonal
// blocks and H_kk = L_kk^{-1} on them, so that every step is one contraction with H.
// Right-looking: once y_k is known, the contributions L_jk y_k of every later block j are
// accumulated in that block's tensor-memory columns, block k + 1 first, so that the
// converters can form z_{k+1} while the remaining updates run.
//
// One CTA scores 128 pixels of one line; tensor memory holds a 128 x Bp FP32 matrix whose
// 64-column block k holds first the accumulated sum for z_k and then y_k.
//   warps 0-3          one pixel (TMEM lane) each: z_k = v_k - acc_k in FP32, split into
//                      NT BF16 terms (hi + lo, or hi + mid + lo) and written as the A
//                      operand; y_k read back, its square summed into the score, split and
//                      written as the A operand of the updates. v = x' - m in FP32; the pixel's raw values of block k + 1
//                      are loaded into registers while block k is solved.
//   warp 4 (one lane)  TMA: the 64 x 64 blocks (j, k), j >= k, of the NT planes of H in
//                      the order the MMAs use them, through a ring of up to 10 stages
//                      (the whole solve streams ~(Bp/64)^2/2 blocks of 16 KB per CTA from
//                      L2, so the ring depth sets how much of that latency is hidden).
//   warp 5 (one lane)  tcgen05.mma (M = 128, N = 64, K = 16), FP32 accumulation in TMEM;
//                      NT = 2 (BF16 working precision): a0 h0 + a0 h1 + a1 h0, the terms
//                      above 2^-16 of the product; NT = 3 (FP32 working precision, both
//                      operands exact three-term splits of their FP32 values): the six terms
//                      a_t h_u with t + u <= 2, dropping those of order 2^-24 and below, the
//                      rounding of an FP32 product.
// Every wait is bounded; a timeout sets *err and the CTA drains its copies and exits.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>

#include "hsad_internal.h"
#include "tc_util.cuh"

namespace hsad {

namespace {
constexpr int TS_M = 128, TS_KB = 64, TS_MAX_STAGES = 10;
// converter warps: TMEM lane group (w & 3, 32 pixels) x half (w >> 2) of each 64-band block
constexpr int TS_CW = 8, TS_CONV = 32 * TS_CW;
constexpr int TS_TMA_WARP = TS_CW, TS_MMA_WARP = TS_CW + 1, TS_THREADS = 32 * (TS_CW + 2);
constexpr uint32_t TS_BLK = TS_M * TS_KB * 2;  // one 128 x 64 16-bit operand block: 16 KB
constexpr uint32_t TS_HALF = 64 * TS_KB * 2;   // one 64 x 64 16-bit block of H: 8 KB
constexpr uint32_t TS_BAR = 256;
constexpr uint32_t TS_SMEM_MAX = 227 * 1024;

__host__ __device__ inline uint32_t ts_cols(int Bp) {
  uint32_t c = 32;
  while (c < (uint32_t)Bp) c <<= 1;
  return c;
}
// shared memory after 1024-byte alignment: Z (nt planes), Y (nt planes), ring of stages of
// nt 64 x 64 blocks of H, {c, m} per band, barriers
__host__ __device__ inline uint32_t ts_smem(int Bp, int stages, int nt) {
  return 1024 + 2 * nt * TS_BLK + (uint32_t)stages * nt * TS_HALF + (uint32_t)Bp * 8 + TS_BAR;
}

__device__ __forceinline__ uint32_t bf16x2_bits(__nv_bfloat162 v) { return *(const uint32_t*)&v; }

// hi = bf16(z), lo = bf16(z - hi) for a pair of values; returns the two packed words
__device__ __forceinline__ void split2(float z0, float z1, uint32_t& hi, uint32_t& lo) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(z0, z1);
  const float h0 = __low2float(h), h1 = __high2float(h);
  hi = bf16x2_bits(h);
  lo = bf16x2_bits(__floats2bfloat162_rn(z0 - h0, z1 - h1));
}
// hi = bf16(z), mid = bf16(z - hi), lo = bf16(z - hi - mid): an exact split of an FP32 value
// (each difference is exact in FP32) for a pair of values
__device__ __forceinline__ void split3(float z0, float z1, uint32_t& hi, uint32_t& mid, uint32_t& lo) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(z0, z1);
  const float r0 = z0 - __low2float(h), r1 = z1 - __high2float(h);
  const __nv_bfloat162 m = __floats2bfloat162_rn(r0, r1);
  hi = bf16x2_bits(h);
  mid = bf16x2_bits(m);
  lo = bf16x2_bits(__floats2bfloat162_rn(r0 - __low2float(m), r1 - __high2float(m)));
}
// the term pairs (a_t, h_u) of one block product
template <int NT>
struct Terms;
template <>
struct Terms<2> {
  static constexpr int n = 3;
  __device__ static int a(int i) { return i == 2 ? 1 : 0; }
  __device__ static int h(int i) { return i == 1 ? 1 : 0; }
};
template <>
struct Terms<3> {
  static constexpr int n = 6;  // (0,0) (0,1) (1,0) (0,2) (1,1) (2,0)
  __device__ static int a(int i) { return i == 2 || i == 4 ? 1 : i == 5 ? 2 : 0; }
  __device__ static int h(int i) { return i == 1 || i == 4 ? 1 : i == 3 ? 2 : 0; }
};
// the NT-term split of 8 values (one 16-byte row chunk per plane) into plane base p
template <int NT>
__device__ __forceinline__ void store_split(uint8_t* p, uint32_t off, const float* v) {
  uint32_t w[NT][4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    if constexpr (NT == 2) split2(v[2 * j], v[2 * j + 1], w[0][j], w[1][j]);
    else split3(v[2 * j], v[2 * j + 1], w[0][j], w[1][j], w[2][j]);
  }
#pragma unroll
  for (int t = 0; t < NT; ++t) *(uint4*)(p + t * TS_BLK + off) = make_uint4(w[t][0], w[t][1], w[t][2], w[t][3]);
}
}  // namespace

template <int NT>
__global__ void __launch_bounds__(TS_THREADS, 1) whiten_trsm_kernel(
    const uint16_t* __restrict__ x, int W, int B, const int32_t* __restrict__ c_int,
    const __grid_constant__ CUtensorMap hmap, const float* __restrict__ m_all,
    const float* __restrict__ inv_s2_all, const int32_t* __restrict__ status, int factor_stride, ScoreOut out,
    int32_t* __restrict__ err, long long limit, int stages) {
  const int t = blockIdx.y;
  const int p0 = blockIdx.x * TS_M;
  const int f = factor_slot(out, factor_stride, t);
  const int64_t slot = (slot0_of(out) + t) % out.ring;
  const int st = status[f];
  if (blockIdx.x == 0 && threadIdx.x == 0) out.ring_status[slot] = st;
  if (st != LS_OK) {
    for (int p = p0 + threadIdx.x; p < p0 + TS_M && p < W; p += blockDim.x) {
      out.scores[slot * W + p] = __int_as_float(0x7fc00000);
      out.mask[slot * W + p] = 0;
    }
    return;
  }
  const int Bp = pad64(B), nkb = Bp / TS_KB;
  const int npx = min(TS_M, W - p0);
  const uint32_t tcols = ts_cols(Bp);
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = tc::align1024(smem_raw);
  constexpr uint32_t STAGE = NT * TS_HALF;   // the NT planes of one 64 x 64 block of H
  uint8_t* sZ = sm;                          // z_k: NT term blocks
  uint8_t* sY = sZ + NT * TS_BLK;            // y_k: NT term blocks
  uint8_t* sR = sY + NT * TS_BLK;            // ring: [stage][plane][64 x 64]
  // per band n: {bits of 1.5 * 2^23 - c_n, m_n} (zero past B), read as one 16-byte load per
  // two bands
  int2* cmS = (int2*)(sR + stages * STAGE);
  uint64_t* bars = (uint64_t*)(cmS + Bp);
  uint32_t* tslot = (uint32_t*)(bars + 2 * TS_MAX_STAGES + 8);
  const uint32_t b_full = tc::smem_u32(bars), b_empty = b_full + 8 * TS_MAX_STAGES;
  const uint32_t z_full = b_empty + 8 * TS_MAX_STAGES, y_full = z_full + 8, ya_full = y_full + 8;
  const uint32_t acc_full = ya_full + 8, done = acc_full + 8;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint16_t* xt = x + ((int64_t)t * W + p0) * B;  // the tile's 128 x B values are contiguous

  if (tid == 0) {
    for (int s = 0; s < stages; ++s) {
      tc::mbar_init(b_full + 8 * s, 1);
      tc::mbar_init(b_empty + 8 * s, 1);
    }
    tc::mbar_init(z_full, TS_CONV);
    tc::mbar_init(y_full, 1);
    tc::mbar_init(ya_full, TS_CONV);
    tc::mbar_init(acc_full, 1);
    tc::mbar_init(done, 1);
    tc::mbar_init_fence();
  }
  // mean offset: the factor slot's, or the gain-corrected one of this line
  const float* mf = out.m_line ? out.m_line + (int64_t)t * Bp : m_all + (int64_t)f * Bp;
  for (int n = tid; n < Bp; n += TS_THREADS)
    cmS[n] = make_int2(0x4B400000 - (n < B ? c_int[n] : 0), __float_as_int(n < B ? mf[n] : 0.f));
  if (warp == TS_MMA_WARP) tc::tmem_alloc(tc::smem_u32(tslot), tcols);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = *tslot;
  bool ok = true;

  if (warp == TS_TMA_WARP) {
    // ---------------- TMA: blocks (j, k) of H, j = k .. nkb - 1, k = 0 .. nkb - 1 ----------
    if (lane == 0) {
      // the tile's raw values (contiguous) into L2 at once: the converters then read each
      // block's values from L2 instead of DRAM (a hint; 16-byte aligned part only)
      const uintptr_t a0 = ((uintptr_t)xt + 15) & ~(uintptr_t)15;
      const uintptr_t a1 = ((uintptr_t)(xt + (int64_t)npx * B)) & ~(uintptr_t)15;
      if (a1 > a0)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a0), "r"((uint32_t)(a1 - a0)) : "memory");
      int it = 0;
      for (int k = 0; k < nkb && ok; ++k)
        for (int j = k; j < nkb && ok; ++j, ++it) {
          const int s = it % stages;
          const uint32_t use = (uint32_t)(it / stages);
          if (!tc::mbar_wait(b_empty + 8 * s, (use & 1) ^ 1, limit)) {
            ok = false;
            break;
          }
          tc::mbar_arrive_expect_tx(b_full + 8 * s, STAGE);
          const uint32_t dst = tc::smem_u32(sR + s * STAGE);
          const int row = (f * NT) * Bp + j * TS_KB;
#pragma unroll
          for (int pl = 0; pl < NT; ++pl)
            tc::tma_load_2d(dst + pl * TS_HALF, &hmap, k * TS_KB, row + pl * Bp, b_full + 8 * s);
        }
      // drain: every copy issued here has landed before the CTA may exit
      const int issued = it;
      for (int s = 0; s < stages && s < issued; ++s) {
        const int last = issued - 1 - ((issued - 1 - s) % stages);
        if (!tc::mbar_wait(b_full + 8 * s, (uint32_t)(last / stages) & 1, limit)) ok = false;
      }
      if (!ok) atomicExch(err, 1);
    }
  } else if (warp == TS_MMA_WARP) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      const uint32_t idesc = tc::idesc_f16(1, TS_M, 64);
      const uint64_t dz = tc::desc_sw128(tc::smem_u32(sZ)), dy = tc::desc_sw128(tc::smem_u32(sY));
      int it = 0;
      bool issued_any = false;
      for (int k = 0; k < nkb && ok; ++k) {
        if (!tc::mbar_wait(z_full, (uint32_t)(k & 1), limit)) { ok = false; break; }
        tc::fence_after_sync();
        for (int j = k; j < nkb; ++j, ++it) {
          if (j == k + 1) {  // y_k is in shared memory
            if (!tc::mbar_wait(ya_full, (uint32_t)(k & 1), limit)) { ok = false; break; }
            tc::fence_after_sync();
          }
          const int s = it % stages;
          if (!tc::mbar_wait(b_full + 8 * s, (uint32_t)((it / stages) & 1), limit)) { ok = false; break; }
          tc::fence_after_sync();
          const uint32_t d = tbase + (uint32_t)(j * TS_KB);
          // descriptors by offset: the start-address field holds the shared address / 16 (all
          // of shared memory fits its 14 bits), so a 32-byte K step adds 2, a plane its size / 16
          const uint64_t da0 = j == k ? dz : dy, dh0 = tc::desc_sw128(tc::smem_u32(sR + s * STAGE));
#pragma unroll
          for (int term = 0; term < Terms<NT>::n; ++term) {
            const uint64_t da = da0 + (uint64_t)(Terms<NT>::a(term) * (TS_BLK >> 4));
            const uint64_t db = dh0 + (uint64_t)(Terms<NT>::h(term) * (TS_HALF >> 4));
#pragma unroll
            for (int ks = 0; ks < TS_KB / 16; ++ks) {
              // y_k overwrites block k; the updates of block j start at k = 0
              const bool first = term == 0 && ks == 0 && (j == k || k == 0);
              tc::mma_f16(d, da + 2 * ks, db + 2 * ks, idesc, first ? 0u : 1u);
            }
          }
          issued_any = true;
          tc::mma_commit(b_empty + 8 * s);
          if (j == k) tc::mma_commit(y_full);
          if (j == k + 1) tc::mma_commit(acc_full);
        }
      }
      if (issued_any) tc::mma_commit(done);
      else tc::mbar_arrive(done);
      if (!ok) atomicExch(err, 1);
      if (!tc::mbar_wait(done, 0, limit)) atomicExch(err, 1);  // MMAs finished before TMEM is freed
    }
  } else {
    // ---------------- converter warps: one pixel and 32 bands of each block each ----------------
    const int lg = warp & 3, hh = warp >> 2, cs = 32 * hh;
    const int r = 32 * lg + lane;
    const bool rv = r < npx;
    const uint32_t taddr = tbase + ((uint32_t)(lg * 32) << 16);
    // this pixel's raw values of bands [64 k + cs, 64 k + cs + 32) as 16 packed pairs (zero
    // past B and for pixels past the tile); 4-byte loads when every row starts 4-byte aligned
    const uint16_t* px = xt + (int64_t)r * B;
    const bool pairs = (B & 1) == 0 && ((uintptr_t)x & 3) == 0;
    uint32_t rw[16];
    auto load_raw = [&](int k) {
      const int nb = rv ? min(TS_KB, B - k * TS_KB) - cs : 0;
      const uint16_t* pk = px + k * TS_KB + cs;
      if (pairs) {
#pragma unroll
        for (int i = 0; i < 16; ++i) rw[i] = 2 * i < nb ? __ldg((const uint32_t*)pk + i) : 0u;
      } else {
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const uint32_t lo = 2 * i < nb ? __ldg(pk + 2 * i) : 0u;
          const uint32_t hi = 2 * i + 1 < nb ? __ldg(pk + 2 * i + 1) : 0u;
          rw[i] = lo | (hi << 16);
        }
      }
    };
    load_raw(0);
    float dsum = 0.f;
    for (int k = 0; k < nkb; ++k) {
      float a[32];
      if (k > 0) {
        if (ok && !tc::mbar_wait(acc_full, (uint32_t)((k - 1) & 1), limit)) ok = false;
        __syncwarp();
        tc::fence_after_sync();
        tc::tmem_ld32(taddr + (uint32_t)(k * TS_KB + cs), a);
      } else {
#pragma unroll
        for (int i = 0; i < 32; ++i) a[i] = 0.f;
      }
      // z_k = (x' - m) - acc, x' = DN - c exact in FP32: the bits of 1.5 * 2^23 + x' minus
      // 1.5 * 2^23 (integer add + float subtract, no conversion instruction). Bands past B
      // give 0 (raw 0, c = m = 0, acc 0); pixels past the tile give values never stored.
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const uint32_t w4[4] = {rw[4 * q], rw[4 * q + 1], rw[4 * q + 2], rw[4 * q + 3]};
        float zv[8];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int n = k * TS_KB + cs + 8 * q + 2 * j;
          const int4 cm = *(const int4*)&cmS[n];  // bands n, n + 1
          const float x0 = __int_as_float(cm.x + (int)(w4[j] & 0xffffu)) - 12582912.0f;
          const float x1 = __int_as_float(cm.z + (int)(w4[j] >> 16)) - 12582912.0f;
          zv[2 * j] = (x0 - __int_as_float(cm.y)) - a[8 * q + 2 * j];
          zv[2 * j + 1] = (x1 - __int_as_float(cm.w)) - a[8 * q + 2 * j + 1];
        }
        store_split<NT>(sZ, tc::sw128_offset(r, cs + 8 * q), zv);
      }
      tc::fence_proxy_async();
      tc::fence_before_sync();
      tc::mbar_arrive(z_full);
      if (k + 1 < nkb) load_raw(k + 1);  // in flight while y_k is computed
      // y_k: score, and the A operand of the updates of the later blocks
      if (ok && !tc::mbar_wait(y_full, (uint32_t)(k & 1), limit)) ok = false;
      __syncwarp();
      tc::fence_after_sync();
      tc::tmem_ld32(taddr + (uint32_t)(k * TS_KB + cs), a);
#pragma unroll
      for (int i = 0; i < 32; ++i) dsum = fmaf(a[i], a[i], dsum);
      if (k + 1 < nkb) {
#pragma unroll
        for (int q = 0; q < 4; ++q) store_split<NT>(sY, tc::sw128_offset(r, cs + 8 * q), a + 8 * q);
        tc::fence_proxy_async();
        tc::fence_before_sync();
        tc::mbar_arrive(ya_full);
      }
    }
    if (!ok) atomicExch(err, 1);
    // the two halves' sums of squares (NaN where a wait gave up)
    // sZ holds them: once `done` completes every MMA (the last ones waited for every
    // converter's z) has finished reading the operand blocks
    float* red = reinterpret_cast<float*>(sZ);
    const bool dn = tc::mbar_wait(done, 0, limit);
    tc::fence_after_sync();
    if (!ok || !dn) dsum = __int_as_float(0x7fc00000);
    red[hh * TS_M + r] = dsum;
    asm volatile("bar.sync 1, %0;" ::"n"(TS_CONV) : "memory");
    const int p = p0 + r;
    if (hh == 0 && p < W) {
      const float tot = red[r] + red[TS_M + r];
      float dlt = tot == tot ? tot * inv_s2_all[f] : __int_as_float(0x7fc00000);
      if (out.line_scale) dlt *= out.line_scale[t];
      out.scores[slot * W + p] = dlt;
      if (out.write_mask) out.mask[slot * W + p] = dlt > out.tau ? 1 : 0;
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == TS_MMA_WARP) {
    __syncwarp();
    tc::tmem_dealloc(tbase, tcols);
  }
}

int bf16_form(int B, int in_type, bool cube, bool force_inverse) {
  if (cube || force_inverse) return P_BF16;
  return in_type == IN_U16 && whiten_trsm_stages(B, 2) > 0 ? P_BF16T : P_BF16;
}

int fp32_form(int B, int in_type, bool cube, bool force_inverse, bool tc_factor) {
  if (cube || force_inverse) return P_FP32;
  if (tc_factor && in_type == IN_U16 && factor_tc_supported(B, P_FP32X) && whiten_trsm_stages(B, 3) > 0)
    return P_FP32X;
  return P_FP32T;
}

int whiten_trsm_stages(int B, int planes) {
  // no deeper than the blocks one CTA streams (small B: less shared memory, more CTAs per SM)
  const int nkb = pad64(B) / TS_KB, blocks = nkb * (nkb + 1) / 2;
  for (int s = std::min(TS_MAX_STAGES, blocks); s >= 1; --s)
    if (ts_smem(pad64(B), s, planes) <= TS_SMEM_MAX) return s;
  return 0;
}

cudaError_t launch_whiten_trsm(const uint16_t* x, int L, int W, int B, int prec, const int32_t* c_int,
                               const void* hmap, const float* m, const float* inv_s2, const int32_t* status,
                               int factor_stride, ScoreOut out, int32_t* err, cudaStream_t st, LaunchCounter* lc) {
  if (L <= 0) return cudaSuccess;
  const int Bp = pad64(B), nt = trsm_planes(prec);
  if (nt == 0) return cudaErrorInvalidValue;
  const int stages = whiten_trsm_stages(B, nt);
  if (stages == 0) return cudaErrorInvalidValue;
  const uint32_t smem = ts_smem(Bp, stages, nt);
  const long long limit = 4000000000LL;  // ~2 s of clock cycles
  auto kern = nt == 3 ? whiten_trsm_kernel<3> : whiten_trsm_kernel<2>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((W + TS_M - 1) / TS_M, L), block(TS_THREADS);
  kern<<<grid, block, smem, st>>>(x, W, B, c_int, *(const CUtensorMap*)hmap, m, inv_s2, status, factor_stride, out,
                                  err, limit, stages);
  if (lc) lc->n += 1;
  return cudaGetLastError();
}

}  // namespace hsad
