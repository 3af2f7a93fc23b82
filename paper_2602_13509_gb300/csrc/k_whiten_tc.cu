// K6 on the tensor cores (FP16 / BF16 working precision): whitening contraction
// Y = X' G^T with tcgen05.mma, G fed by TMA, X' converted on chip, and the row-norm
// score / threshold epilogue read straight out of tensor memory.
//
// Eq. 1 (Sec. 3.3): delta = || G (x - c) - y0 ||^2 / s^2 (see k_factor.cu for G, y0, s).
// One CTA scores one tile of 128 pixels of one line:
//   warp 4 (one lane)  copy engine: the tile's raw values (128 pixels x B bands are
//                      contiguous in the BIP layout) in one bulk copy when aligned and it
//                      fits, then 128 x 64 blocks (n, k) (two 64-row n blocks) of the hi
//                      and lo planes of G by TMA into a ring of 2 to 4 stages with the
//                      128-byte swizzle; only blocks with n-block >= k-block (G is lower
//                      triangular).
//   warps 0-3          convert the pixels' value - c of one 64-band block into the A
//                      operand (FP16: one plane; BF16: H = 64 rint(x'/64) and R = x' - H,
//                      both exact for integer input) in the same swizzled K-major layout,
//                      double buffered: a thread takes 8 consecutive bands of one pixel
//                      and writes them with one 16-byte store per plane (8 threads fill a
//                      128-byte row, conflict free); afterwards the same 128 threads are
//                      the epilogue, one pixel (TMEM lane) each.
//   warp 5 (one lane)  issues tcgen05.mma (M = 128, N = 128 or 64, K = 16) into a 128 x Bp FP32
//                      accumulator in TMEM: FP16 terms x'.G_hi + x'.G_lo (integer input),
//                      BF16 (and FP16 with float input) terms H.G_hi + H.G_lo + R.G_hi;
//                      commits free the smem stages.
// Every wait is bounded; a timeout sets *err and the CTA drains and exits.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "hsad_internal.h"
#include "tc_util.cuh"

namespace hsad {

namespace {
constexpr int WT_M = 128, WT_KB = 64, WT_NB = 64, WT_NPAIR = 128, WT_MAX_STAGES = 4, WT_THREADS = 192;
constexpr uint32_t A_TILE = WT_M * WT_KB * 2;     // 16 KB
constexpr uint32_t B_TILE = WT_NPAIR * WT_KB * 2; // 16 KB per plane: two 64-row blocks of n
constexpr uint32_t SMEM_A = 2 * 2 * A_TILE;       // 2 buffers x 2 operands
constexpr uint32_t SMEM_BAR = 128;
constexpr uint32_t SMEM_MAX = 227 * 1024;

__host__ __device__ inline uint32_t tmem_cols_for(int Bp) {
  uint32_t c = 32;
  while (c < (uint32_t)Bp) c <<= 1;
  return c;
}
__host__ __device__ inline uint32_t wt_y0_bytes(int Bp) { return ((uint32_t)Bp * 4 + 127) / 128 * 128; }
__host__ __device__ inline uint32_t wt_fixed_smem(int stages, int Bp) {
  return 1024 + SMEM_A + (uint32_t)stages * 2 * B_TILE + wt_y0_bytes(Bp) + SMEM_BAR;
}

template <typename In>
__device__ __forceinline__ float centred_tc(In v, const int32_t* ci, const float* cf, int k);
template <>
__device__ __forceinline__ float centred_tc<uint16_t>(uint16_t v, const int32_t* ci, const float*, int k) {
  return (float)((int)v - ci[k]);
}
template <>
__device__ __forceinline__ float centred_tc<float>(float v, const int32_t*, const float* cf, int k) {
  return v - cf[k];
}
}  // namespace

template <typename In, int PREC>
__global__ void __launch_bounds__(WT_THREADS, 1) whiten_tc_kernel(
    const In* __restrict__ x, int W, int B, const int32_t* __restrict__ c_int, const float* __restrict__ c_flt,
    const __grid_constant__ CUtensorMap gmap, const float* __restrict__ y0_all,
    const float* __restrict__ inv_s2_all, const int32_t* __restrict__ status, int factor_stride, ScoreOut out,
    int32_t* __restrict__ err, long long limit, int stages, int raw_tile) {
  const int t = blockIdx.y;
  const int p0 = blockIdx.x * WT_M;
  const int f = factor_slot(out, factor_stride, t);
  const int64_t slot = (slot0_of(out) + t) % out.ring;
  const int st = status[f];
  if (blockIdx.x == 0 && threadIdx.x == 0) out.ring_status[slot] = st;
  if (st != LS_OK) {
    for (int p = p0 + threadIdx.x; p < p0 + WT_M && p < W; p += blockDim.x) {
      out.scores[slot * W + p] = __int_as_float(0x7fc00000);
      out.mask[slot * W + p] = 0;
    }
    return;
  }
  const int Bp = pad64(B), nkb = Bp / WT_KB;
  const int npx = min(WT_M, W - p0);
  const uint32_t tcols = tmem_cols_for(Bp);
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = tc::align1024(smem_raw);
  uint8_t* sA = sm;                                  // [2 buf][2 op][128 x 64] swizzled
  uint8_t* sB = sm + SMEM_A;                         // [stage][2 plane][64 x 64] swizzled
  float* y0s = (float*)(sB + stages * 2 * B_TILE);
  uint64_t* bars = (uint64_t*)((uint8_t*)y0s + wt_y0_bytes(Bp));
  In* sRaw = (In*)((uint8_t*)bars + SMEM_BAR);       // raw tile [npx][B] when raw_tile
  uint32_t* tslot = (uint32_t*)(bars + 15);
  const uint32_t b_full = tc::smem_u32(bars), b_empty = b_full + 8 * WT_MAX_STAGES;
  const uint32_t a_full = b_empty + 8 * WT_MAX_STAGES, a_empty = a_full + 16, d_full = a_empty + 16;
  const uint32_t raw_full = d_full + 8;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const In* xl = x + (int64_t)t * W * B;

  if (tid == 0) {
    for (int s = 0; s < stages; ++s) {
      tc::mbar_init(b_full + 8 * s, 1);
      tc::mbar_init(b_empty + 8 * s, 1);
    }
    for (int a = 0; a < 2; ++a) {
      tc::mbar_init(a_full + 8 * a, WT_M);
      tc::mbar_init(a_empty + 8 * a, 1);
    }
    tc::mbar_init(d_full, 1);
    tc::mbar_init(raw_full, 1);
    tc::mbar_init_fence();
  }
  const float* y0 = y0_all + (int64_t)f * Bp;
  for (int n = tid; n < Bp; n += WT_THREADS) y0s[n] = y0[n];
  if (warp == 5) tc::tmem_alloc(tc::smem_u32(tslot), tcols);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = *tslot;
  bool ok = true;
  // terms: BF16 H.G_hi + H.G_lo + R.G_hi; FP16 x'.G_hi + x'.G_lo for integer input (x' exact
  // in FP16 up to 2048), and H.G_hi + H.G_lo + R.G_hi with x' = H + R (two FP16 values, 22
  // bits) for float input, whose centred values a single FP16 keeps to only 11 bits
  constexpr int NT = (PREC == P_BF16 || sizeof(In) == 4) ? 3 : 2;

  if (warp == 4) {
    // ---------------- copy engine: raw tile, then G blocks ----------------
    if (lane == 0) {
      bool raw_issued = false;
      if (raw_tile) {
        const uint32_t bytes = (uint32_t)npx * B * sizeof(In);
        tc::mbar_arrive_expect_tx(raw_full, bytes);
        tc::bulk_load(tc::smem_u32(sRaw), xl + (int64_t)p0 * B, bytes, raw_full);
        raw_issued = true;
      }
      int it = 0;
      for (int kb = 0; kb < nkb && ok; ++kb)
        for (int nb = kb; nb < nkb && ok; nb += 2, ++it) {
          const int s = it % stages;
          const uint32_t use = (uint32_t)(it / stages);
          if (!tc::mbar_wait(b_empty + 8 * s, (use & 1) ^ 1, limit)) { ok = false; break; }
          tc::mbar_arrive_expect_tx(b_full + 8 * s, 2 * B_TILE);
          const uint32_t dst = tc::smem_u32(sB + s * 2 * B_TILE);
          const int row = (f * 2) * Bp + nb * WT_NB;
          tc::tma_load_2d(dst, &gmap, kb * WT_KB, row, b_full + 8 * s);
          tc::tma_load_2d(dst + B_TILE, &gmap, kb * WT_KB, row + Bp, b_full + 8 * s);
        }
      // drain: every copy issued by this thread has landed before the CTA may exit
      const int issued = it;
      for (int s = 0; s < stages && s < issued; ++s) {
        const int last = issued - 1 - ((issued - 1 - s) % stages);
        const uint32_t use = (uint32_t)(last / stages);
        if (!tc::mbar_wait(b_full + 8 * s, use & 1, limit)) ok = false;
      }
      if (raw_issued && !tc::mbar_wait(raw_full, 0, limit)) ok = false;
      if (!ok) atomicExch(err, 1);
    }
  } else if (warp == 5) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      const uint32_t idesc2 = tc::idesc_f16(PREC == P_BF16 ? 1 : 0, WT_M, WT_NPAIR);
      const uint32_t idesc1 = tc::idesc_f16(PREC == P_BF16 ? 1 : 0, WT_M, WT_NB);
      int it = 0;
      bool issued_any = false;
      for (int kb = 0; kb < nkb && ok; ++kb) {
        const int ab = kb & 1;
        if (!tc::mbar_wait(a_full + 8 * ab, (uint32_t)((kb >> 1) & 1), limit)) { ok = false; break; }
        tc::fence_after_sync();
        const uint32_t a0 = tc::smem_u32(sA + (ab * 2 + 0) * A_TILE);
        const uint32_t a1 = tc::smem_u32(sA + (ab * 2 + 1) * A_TILE);
        for (int nb = kb; nb < nkb; nb += 2, ++it) {
          const uint32_t idesc = nb + 1 < nkb ? idesc2 : idesc1;
          const int s = it % stages;
          if (!tc::mbar_wait(b_full + 8 * s, (uint32_t)((it / stages) & 1), limit)) { ok = false; break; }
          tc::fence_after_sync();
          const uint32_t bhi = tc::smem_u32(sB + s * 2 * B_TILE), blo = bhi + B_TILE;
          const uint32_t d = tbase + (uint32_t)(nb * WT_NB);
#pragma unroll
          for (int term = 0; term < NT; ++term) {
            const uint32_t aop = (term == 2) ? a1 : a0;
            const uint32_t bop = (term == 1) ? blo : bhi;
#pragma unroll
            for (int ks = 0; ks < WT_KB / 16; ++ks) {
              const uint32_t acc = (kb == 0 && term == 0 && ks == 0) ? 0u : 1u;
              tc::mma_f16(d, tc::desc_sw128(aop + ks * 32), tc::desc_sw128(bop + ks * 32), idesc, acc);
            }
          }
          issued_any = true;
          tc::mma_commit(b_empty + 8 * s);
        }
        if (!ok) break;
        tc::mma_commit(a_empty + 8 * ab);
      }
      if (issued_any) tc::mma_commit(d_full);
      else tc::mbar_arrive(d_full);
      if (!ok) atomicExch(err, 1);
      // MMAs must be finished before the accumulator is freed
      if (!tc::mbar_wait(d_full, 0, limit)) atomicExch(err, 1);
    }
  } else {
    // ---------------- converters (warps 0-3) ----------------
    if (raw_tile && !tc::mbar_wait(raw_full, 0, limit)) {
      ok = false;
      atomicExch(err, 1);
    }
    // raw values of pixel r, band k: shared memory when staged, else global
    const In* src = raw_tile ? (const In*)sRaw : xl + (int64_t)p0 * B;
    // unit = (pixel row, 8 consecutive bands); thread tid takes units tid + 128 i, so its
    // band group kg = tid % 8 is the same in every unit
    const int kg = tid & 7;
    const bool vec = (sizeof(In) == 2) && (B % 8 == 0) && (((uintptr_t)src & 15) == 0);
    for (int kb = 0; kb < nkb; ++kb) {
      const int ab = kb & 1;
      if (!tc::mbar_wait(a_empty + 8 * ab, (uint32_t)(((kb >> 1) & 1) ^ 1), limit)) {
        ok = false;
        atomicExch(err, 1);
      }
      uint8_t* A0 = sA + (ab * 2 + 0) * A_TILE;
      uint8_t* A1 = sA + (ab * 2 + 1) * A_TILE;
      const int k0 = kb * WT_KB + kg * 8;
      if (ok) {
        if (sizeof(In) == 2) {
          // x' = DN - c as an exact float: the bits of 1.5 * 2^23 + x' minus 1.5 * 2^23
          int mc[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) mc[j] = 0x4B400000 - (k0 + j < B ? c_int[k0 + j] : 0);
          // 16-byte rows: issue this thread's 8 unit loads together (8 in flight per thread)
          uint4 qv[8];
          if (vec) {
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              const int r = (tid + WT_M * i) >> 3;
              qv[i] = (r < npx && k0 + 8 <= B) ? *(const uint4*)((const uint16_t*)src + (int64_t)r * B + k0)
                                               : make_uint4(0, 0, 0, 0);
            }
          }
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const int u = tid + WT_M * i;
            const int r = u >> 3;
            const bool rv = r < npx;
            int dn[8];
            if (vec && k0 + 8 <= B) {
              const uint32_t w[4] = {qv[i].x, qv[i].y, qv[i].z, qv[i].w};
#pragma unroll
              for (int j = 0; j < 4; ++j) {
                dn[2 * j] = (int)(w[j] & 0xffffu);
                dn[2 * j + 1] = (int)(w[j] >> 16);
              }
            } else {
#pragma unroll
              for (int j = 0; j < 8; ++j)
                dn[j] = (rv && k0 + j < B) ? (int)((const uint16_t*)src)[(int64_t)r * B + k0 + j] : 0;
            }
            uint32_t p0w[4], p1w[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              float v[2];
#pragma unroll
              for (int e = 0; e < 2; ++e) {
                const int jj = 2 * j + e;
                v[e] = (rv && k0 + jj < B) ? __int_as_float(mc[jj] + dn[jj]) - 12582912.0f : 0.f;
              }
              if (PREC == P_FP16) {
                const __half2 h2 = __floats2half2_rn(v[0], v[1]);
                p0w[j] = *(const uint32_t*)&h2;
              } else {
                // H = 64 rint(x'/64) (round to nearest even), R = x' - H: small integers times
                // powers of two, exact in BF16, whose bits are the float's top half
                float h[2], rr[2];
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                  h[e] = (__fmaf_rn(v[e], 1.f / 64.f, 12582912.0f) - 12582912.0f) * 64.f;
                  rr[e] = v[e] - h[e];
                }
                p0w[j] = __byte_perm(__float_as_uint(h[0]), __float_as_uint(h[1]), 0x7632);
                p1w[j] = __byte_perm(__float_as_uint(rr[0]), __float_as_uint(rr[1]), 0x7632);
              }
            }
            const uint32_t off = tc::sw128_offset(r, kg * 8);
            *(uint4*)(A0 + off) = make_uint4(p0w[0], p0w[1], p0w[2], p0w[3]);
            if (PREC != P_FP16) *(uint4*)(A1 + off) = make_uint4(p1w[0], p1w[1], p1w[2], p1w[3]);
          }
        } else {
          // float input: one value at a time (H = rn(v), R = rn(v - H) in BF16 or FP16)
          for (int u = tid; u < WT_M * 8; u += WT_M) {
            const int r = u >> 3;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              const int k = k0 + j;
              float v = 0.f;
              if (r < npx && k < B) v = centred_tc<In>(src[(int64_t)r * B + k], c_int, c_flt, k);
              const uint32_t off = tc::sw128_offset(r, kg * 8 + j);
              if (PREC == P_FP16) {
                const __half h = __float2half_rn(v);
                *(__half*)(A0 + off) = h;
                *(__half*)(A1 + off) = __float2half_rn(v - __half2float(h));
              } else {
                const float h = __bfloat162float(__float2bfloat16_rn(v));
                *(__nv_bfloat16*)(A0 + off) = __float2bfloat16_rn(h);
                *(__nv_bfloat16*)(A1 + off) = __float2bfloat16_rn(v - h);
              }
            }
          }
        }
      }
      tc::fence_proxy_async();
      tc::mbar_arrive(a_full + 8 * ab);
    }
    // ---------------- epilogue: one pixel per thread ----------------
    const bool dok = tc::mbar_wait(d_full, 0, limit);
    __syncwarp();
    tc::fence_after_sync();
    if (!dok) atomicExch(err, 1);
    const int p = p0 + tid;
    const uint32_t taddr = tbase + ((uint32_t)(warp * 32) << 16);
    float dsum = 0.f;
    for (int c0 = 0; c0 < Bp; c0 += 32) {
      float v[32];
      tc::tmem_ld32(taddr + (uint32_t)c0, v);
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int n = c0 + j;
        if (n < B) {
          const float dv = v[j] - y0s[n];
          dsum = fmaf(dv, dv, dsum);
        }
      }
    }
    if (p < W) {
      const float dlt = dok && ok ? dsum * inv_s2_all[f] : __int_as_float(0x7fc00000);
      out.scores[slot * W + p] = dlt;
      if (out.write_mask) out.mask[slot * W + p] = dlt > out.tau ? 1 : 0;
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 5) {
    __syncwarp();
    tc::tmem_dealloc(tbase, tcols);
  }
}

cudaError_t launch_whiten_tc(const void* x, int L, int W, int B, int in_type, const int32_t* c_int,
                             const float* c_flt, int prec, const void* gmap, const float* y0,
                             const float* inv_s2, const int32_t* status, int factor_stride, ScoreOut out,
                             int32_t* err, cudaStream_t st, LaunchCounter* lc) {
  if (L <= 0) return cudaSuccess;
  const CUtensorMap& map = *(const CUtensorMap*)gmap;
  dim3 grid((W + WT_M - 1) / WT_M, L), block(WT_THREADS);
  const long long limit = 4000000000LL;  // ~2 s of clock cycles
  // Raw-tile bulk copy: every tile start (line base and 128-pixel steps) and the last
  // partial tile must be 16-byte aligned in address and size, and the tile must fit.
  const int64_t esz = in_type == IN_U16 ? 2 : 4;
  const bool aligned = ((uintptr_t)x % 16 == 0) && (((int64_t)W * B * esz) % 16 == 0) &&
                       (((int64_t)(W % WT_M) * B * esz) % 16 == 0);
  const uint32_t rawb = (uint32_t)(((int64_t)WT_M * B * esz + 127) / 128 * 128);
  // the deepest G ring that leaves room for the raw tile; else read the pixels from global
  int stages = WT_MAX_STAGES, raw_tile = 0;
  if (aligned)
    for (int sg = WT_MAX_STAGES; sg >= 2 && !raw_tile; --sg)
      if (wt_fixed_smem(sg, pad64(B)) + rawb <= SMEM_MAX) {
        raw_tile = 1;
        stages = sg;
      }
  const uint32_t smem = wt_fixed_smem(stages, pad64(B)) + (raw_tile ? rawb : 0);
  cudaError_t e = cudaSuccess;
#define HSAD_WT(IN, P)                                                                                  \
  do {                                                                                                  \
    e = cudaFuncSetAttribute(whiten_tc_kernel<IN, P>, cudaFuncAttributeMaxDynamicSharedMemorySize,      \
                             (int)smem);                                                                \
    if (e != cudaSuccess) return e;                                                                     \
    whiten_tc_kernel<IN, P><<<grid, block, smem, st>>>((const IN*)x, W, B, c_int, c_flt, map, y0, inv_s2, \
                                                       status, factor_stride, out, err, limit, stages,    \
                                                       raw_tile);                                        \
  } while (0)
  if (in_type == IN_U16) {
    if (prec == P_FP16) HSAD_WT(uint16_t, P_FP16);
    else HSAD_WT(uint16_t, P_BF16);
  } else {
    if (prec == P_FP16) HSAD_WT(float, P_FP16);
    else HSAD_WT(float, P_BF16);
  }
#undef HSAD_WT
  if (lc) lc->n += 1;
  return cudaGetLastError();
}

}  // namespace hsad
