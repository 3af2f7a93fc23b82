// K4 + K5 on the tensor cores for streamed statistics (the triangular-solve form with the
// float-float factor): the same factorisation as factor_kernel, S = L L^T of each line's
// DN-frame covariance with the inverses of L's 64 x 64 diagonal blocks (Eq. 1, Sec. 3.3:
// delta = ||L^{-1}(x' - m)||^2), reorganised so that its O(B^3) part, the trailing
// updates, runs as tcgen05 contractions.
//
// Blocked right-looking Cholesky in 64-column panels, one launch per step for a whole
// batch of lines:
//   tcf_form_kernel      S = (S2 - n m m^T) / (n - 1) as float-float, in place;
//   tcf_diag_kernel(k)   one CTA per line: the 64 x 64 diagonal block factored and inverted
//                        together (float-float, right-looking, pivots by a Newton step), the
//                        whitening operand's diagonal block written (L_kk^{-1});
//   tcf_trsm_kernel(k)   one CTA per line: the rows below solved as L_ik = A_ik L_kk^{-T}
//                        (float-float product with the inverse), written to the whitening
//                        operand, and every row split into six signed base-256 digits with a
//                        per-row power of two: L_ik[r][c] = 2^e_r sum_t d_t[r][c] 256^-(t+1)
//                        up to 2^e_r 256^-6 / 2 (the error-free splitting of Ozaki et al.,
//                        2012, with BF16 digits: every digit is an integer of magnitude <= 256,
//                        exact in BF16);
//   tcf_update_kernel(k) A_ij -= sum_c L_ic L_jc over the trailing lower triangle in
//                        128 x 64 tiles: for each digit level l = t + u <= 5 the products
//                        d_t(i) d_u(j)^T are summed by tcgen05.mma (BF16 in, FP32 in TMEM).
//                        Digit products are integers below 2^16 and a 64-term level sum of up
//                        to six such products stays below 2^24, so every level sum is exact;
//                        the epilogue combines the six levels in float-float, scales by
//                        2^(e_i + e_j - 16) and subtracts from A (float-float).
// The digit levels past 5 (and the last digit's remainder) are dropped: a relative error of
// about 2^-45 of the row scales per update, the order of float-float's 2^-48 (a CPU
// emulation of this update on a 1024 x 448 stream covariance: score error 2e-12; at
// condition number 1e10: 5e-7). Operand slices live in the context's inverse scratch
// ([6][Bp + 64][64] BF16 per line, 128-byte swizzled rows, then the exponents and the
// diagonal block's float-float inverse, from the first 1024-byte boundary of the line's
// slot), which is large enough from B = 192 on.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "factor_kernel.cuh"
#include "hsad_internal.h"
#include "tc_util.cuh"

namespace hsad {

namespace {

constexpr int TP_T = 256;          // threads of the panel kernel
constexpr int DS = 65;             // padded row stride (8-byte slots) of the 64 x 64 blocks in shared memory
constexpr int NDIG = 6;            // base-256 digits per value
constexpr int TU_M = 128, TU_N = 64, TU_K = 64;
constexpr int TU_T = 160;          // 4 epilogue warps + 1 copy / MMA warp
constexpr uint32_t TU_A_PLANE = TU_M * TU_K * 2;   // 16 KB
constexpr uint32_t TU_B_PLANE = TU_N * TU_K * 2;   // 8 KB
constexpr int TU_AS = TU_N + 1;    // row stride (float2) of the staged trailing tile
constexpr uint32_t TU_TILE = TU_M * TU_AS * 8;
constexpr uint32_t TU_SMEM = 1024 + NDIG * (TU_A_PLANE + TU_B_PLANE) + TU_TILE + 256 + 64;

// Byte layout of one line's slice region (in the inverse scratch): NDIG planes of
// (Bp + 64) rows x 128 bytes, then (Bp + 64) int32 exponents.
__host__ __device__ inline size_t plane_bytes(int Bp) { return (size_t)(Bp + 64) * 128; }
// the diagonal block's inverse X (float-float, [64][64]) follows the exponents
__host__ __device__ inline size_t xinv_offset(int Bp) { return NDIG * plane_bytes(Bp) + (size_t)(Bp + 64) * 4; }
__host__ __device__ inline size_t slice_region_bytes(int Bp) { return xinv_offset(Bp) + 64 * 64 * 8; }
constexpr int TD_T = 128;            // threads per line of the diagonal-block kernel
constexpr int TRI64 = 64 * 65 / 2;   // a packed 64 x 64 lower triangle
__host__ __device__ constexpr int tri(int r) { return r * (r + 1) / 2; }

// Line t's slice region: its inverse-scratch slot rounded up to 1024 bytes (bulk copies
// and the swizzled operand tiles need aligned rows).
__host__ __device__ inline uint8_t* slice_base(uint8_t* all, size_t stride, int t) {
  return (uint8_t*)(((uintptr_t)(all + (size_t)t * stride) + 1023) & ~(uintptr_t)1023);
}

using fk::ff_fms;
using fk::ff_mul;
using fk::ff_norm;

__device__ __forceinline__ double ffd(float2 v) { return (double)v.x + (double)v.y; }
__device__ __forceinline__ float2 dff(double d) {
  const float h = __double2float_rn(d);
  return make_float2(h, __double2float_rn(d - (double)h));
}
// a - b in float-float (two-sum of the high words, low words added, renormalised)
__device__ __forceinline__ float2 ff_sub(float2 a, float2 b) {
  const float s = __fsub_rn(a.x, b.x);
  const float z = __fsub_rn(s, a.x);
  const float e = __fadd_rn(__fsub_rn(a.x, __fsub_rn(s, z)), __fsub_rn(-b.x, z));
  return ff_norm(s, __fadd_rn(e, __fsub_rn(a.y, b.y)));
}

__device__ __forceinline__ bool skip_line(const int32_t* status, int t, int every, int q_off) {
  return status[t] != LS_OK || (every > 1 && (q_off + t) % every != 0);
}

}  // namespace

// ---- covariance -----------------------------------------------------------------------
namespace {
// A double holding an integer of magnitude below 2^53 (the exact covariance sums of uint16
// input) as a float-float pair, by integer operations on its bits only (the FP64 pipe
// issues at 1/64 of the FP32 rate here). Returns false for any other value.
__device__ __forceinline__ bool int_double_to_ff(double v, float2& out) {
  const long long bits = __double_as_longlong(v);
  const int ex = (int)((bits >> 52) & 0x7ff) - 1075;  // v = mant * 2^ex
  if (v == 0.0) {
    out = make_float2(0.f, 0.f);
    return true;
  }
  if (ex > 0 || ex < -52) return false;
  const long long mant = (bits & 0xFFFFFFFFFFFFFLL) | 0x10000000000000LL;
  const long long ival = mant >> (-ex);
  if ((ival << (-ex)) != mant) return false;  // a fractional part
  // ival < 2^53: a = ival >> 24 (< 2^29) rounded to 24 significant bits, b = the rest
  long long a = ival >> 24;
  int sh = 0;
  while ((a >> sh) >= (1LL << 24)) ++sh;
  const long long ar = sh ? ((a + (1LL << (sh - 1))) >> sh) << sh : a;
  const float fa = ldexpf((float)(int)(ar >> sh), 24 + sh);  // exact: < 2^24 significant bits
  const float fb = (float)(int)(ival - (ar << 24));         // |.| < 2^29: rounded only past 2^48
  const float h = __fadd_rn(fa, fb);
  const float z = __fsub_rn(h, fa);
  const float l = __fadd_rn(__fsub_rn(fa, __fsub_rn(h, z)), __fsub_rn(fb, z));
  out = (bits < 0) ? make_float2(-h, -l) : make_float2(h, l);
  return true;
}
}  // namespace

// S = (S2 - n m m^T) / (n - 1), lower triangle, in place as float-float: one warp per row.
// Integer sums (uint16 input without gains or forgetting) take the float-float route
// (exact split of S2, n m_i m_j and the scale as float-float products); any other value
// is formed in FP64 and split.
__global__ void tcf_form_kernel(double* __restrict__ sigma_all, const double* __restrict__ m_all, int B,
                                const int32_t* __restrict__ status, int64_t n0_arg, int W, int incl,
                                const int64_t* __restrict__ n0_dev, int every, int q_off,
                                const double* __restrict__ n_line) {
  const int t = blockIdx.y, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (skip_line(status, t, every, q_off)) return;  // the same for the whole block
  const int i = blockIdx.x * 8 + warp;
  const double* m = m_all + (int64_t)t * B;
  // the means as float-float pairs, once per block (FP64 conversions are slow here)
  __shared__ float2 mf[512];
  const int jmax = min(B, blockIdx.x * 8 + 8);
  for (int j = threadIdx.x; j < jmax; j += blockDim.x) mf[j] = dff(m[j]);
  __syncthreads();
  if (i >= B) return;
  const int64_t n = (n0_dev ? *n0_dev : n0_arg) + (int64_t)(t + incl) * W;
  const double nn = n_line ? n_line[t] : (double)n, inv_nm1 = 1.0 / (nn - 1.0);
  double* row = sigma_all + (int64_t)t * B * B + (int64_t)i * B;
  float2* row2 = reinterpret_cast<float2*>(row);
  const double nmi = nn * m[i];
  const float2 nmi_f = dff(nmi), sc_f = dff(inv_nm1);
  for (int j0 = 0; j0 <= i; j0 += 128) {
    double v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {  // four independent loads per lane
      const int j = j0 + lane + 32 * u;
      v[u] = j <= i ? row[j] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int j = j0 + lane + 32 * u;
      if (j > i) continue;
      float2 s2;
      if (int_double_to_ff(v[u], s2)) {
        const float2 p = ff_mul(nmi_f, mf[j]);
        row2[j] = ff_mul(ff_sub(s2, p), sc_f);
      } else {
        row2[j] = dff(inv_nm1 * fma(-nmi, m[j], v[u]));
      }
    }
  }
}

// ---- diagonal block -----------------------------------------------------------------------
// One CTA of TD_T threads per line: the 64 x 64 diagonal block of panel k, as packed lower
// triangles in shared memory, factored and inverted together, right-looking, a column at a
// time: the pivot l = sqrt(A_jj) and r = 1 / l (float-float Newton step from the FP32 rsqrt
// seed, computed by every thread), column j of L = A_.j r, row j of X = R_j. r (R: the
// running right-hand sides, I at the start), then the rank-1 updates A_ic -= L_ij L_cj
// (j < c <= i) and R_ic -= L_ij X_jc (i > j, c <= j) over the flattened trapezoid of rows
// j + 1 .. kb - 1. Writes X (float-float, [64][64]) to the line's slice region for the
// triangular solve, and the whitening operand's diagonal block (L_kk^{-1}).
template <int PREC>
__global__ void __launch_bounds__(TD_T) tcf_diag_kernel(double* __restrict__ sigma_all,
                                                        uint8_t* __restrict__ slice_all, size_t slice_stride,
                                                        const double* __restrict__ m_all, int B, int k,
                                                        int32_t* __restrict__ status, int every, int q_off,
                                                        void* __restrict__ wmat, float* __restrict__ y0_all,
                                                        float* __restrict__ inv_s2_all) {
  __shared__ float2 Dg[TRI64];  // L_kk, packed: (i, c) at tri(i) + c
  __shared__ float2 X[TRI64];   // R, then X = L_kk^{-1}, packed
  __shared__ uint8_t row_of[TRI64];
  const int t = blockIdx.x, tid = threadIdx.x;
  if (skip_line(status, t, every, q_off)) return;  // the same for the whole CTA
  const int Bp = pad64(B), p = 64 * k, kb = min(64, B - p);
  const float2* A = reinterpret_cast<const float2*>(sigma_all + (int64_t)t * B * B);
  uint8_t* sl = slice_base(slice_all, slice_stride, t);
  float2* Xg = reinterpret_cast<float2*>(sl + xinv_offset(Bp));
  const int64_t plane = (int64_t)Bp * Bp;
  void* w = (char*)wmat + (size_t)t * plane * 4;
  if (k == 0) {  // the means of the triangular-solve form and the unit score scale
    for (int n = tid; n < Bp; n += TD_T) y0_all[(int64_t)t * Bp + n] = n < B ? (float)m_all[(int64_t)t * B + n] : 0.f;
    if (tid == 0) inv_s2_all[t] = 1.0f;
  }
  for (int e = tid; e < TRI64; e += TD_T) {
    int i = (int)((sqrtf(8.f * e + 1.f) - 1.f) * 0.5f);
    while (tri(i + 1) <= e) ++i;
    while (tri(i) > e) --i;
    const int c = e - tri(i);
    row_of[e] = (uint8_t)i;
    Dg[e] = i < kb ? A[(int64_t)(p + i) * B + p + c] : make_float2(0.f, 0.f);
    X[e] = make_float2(i == c ? 1.f : 0.f, 0.f);
  }
  __syncthreads();
  for (int j = 0; j < kb; ++j) {
    const float2 a = Dg[tri(j) + j];
    if (!(a.x > 0.f) || !isfinite(a.x)) {  // the same value in every thread
      if (tid == 0) status[t] = LS_NOT_PD;
      return;
    }
    // r = 1 / sqrt(a): FP32 seed, one Newton step r += r (1 - a r^2) / 2 in float-float (the
    // seed's relative error, below 2^-22, squares to below 2^-44: the order of the six-digit
    // updates' 2^-45); l = a r
    float2 r = make_float2(rsqrtf(a.x), 0.f);
    {
      const float2 ee = ff_sub(make_float2(1.f, 0.f), ff_mul(a, ff_mul(r, r)));
      r = ff_sub(r, ff_mul(r, make_float2(-0.5f * ee.x, -0.5f * ee.y)));
    }
    __syncthreads();  // every thread has read the pivot
    // column j of L below the pivot, row j of X
    const int nl = kb - 1 - j;
    if (tid < nl) {
      const int i = j + 1 + tid;
      Dg[tri(i) + j] = ff_mul(Dg[tri(i) + j], r);
    } else if (tid - nl <= j) {
      const int c = tid - nl;
      X[tri(j) + c] = ff_mul(X[tri(j) + c], r);
    } else if (tid == 127) {
      Dg[tri(j) + j] = ff_mul(a, r);
    }
    __syncthreads();
    // rank-1 update of rows j + 1 .. kb - 1: X columns c <= j, L columns c > j
    const int e0 = tri(j + 1), e1 = tri(kb);
    for (int e = e0 + tid; e < e1; e += TD_T) {
      const int i = row_of[e], c = e - tri(i);
      const bool inx = c <= j;
      float2* base = inx ? X : Dg;
      const float2 lij = Dg[tri(i) + j];
      const float2 y = inx ? X[tri(j) + c] : Dg[tri(c) + j];
      float2 v = base[e];
      ff_fms(v.x, v.y, lij, y);
      base[e] = ff_norm(v.x, v.y);
    }
    __syncthreads();
  }
  // X for the triangular solve (full 64 x 64, zero above the diagonal and past kb) and the
  // operand's diagonal block, threads on consecutive addresses
  constexpr bool TR = PREC == P_FP32T;
  for (int e = tid; e < 64 * 64; e += TD_T) {
    const int i = e >> 6, c = e & 63;
    Xg[e] = (c <= i && i < kb) ? X[tri(i) + c] : make_float2(0.f, 0.f);
  }
  for (int e = tid; e < 64 * 64; e += TD_T) {
    const int n = TR ? e & 63 : e >> 6, c = TR ? e >> 6 : e & 63;  // row n, column c of the block
    const int64_t idx = fk::h_index<PREC>(p + n, p + c, Bp);
    if (c <= n && n < kb) fk::WOut<PREC>::store(w, plane, idx, fk::ArFF::to_f(X[tri(n) + c]));
    else fk::WOut<PREC>::zero(w, plane, idx);
  }
}

// ---- rows below the diagonal block ----------------------------------------------------------
// One CTA per line: L_ik = A_ik X^T for the 64-row chunks below panel k's diagonal block
// (float-float products with the inverse from the diagonal-block kernel), written to the
// whitening operand and split into six base-256 digits with a per-row power of two.
template <int PREC>
__global__ void __launch_bounds__(TP_T, 3) tcf_trsm_kernel(double* __restrict__ sigma_all,
                                                           uint8_t* __restrict__ slice_all, size_t slice_stride,
                                                           int B, int k, const int32_t* __restrict__ status,
                                                           int every, int q_off, void* __restrict__ wmat) {
  const int t = blockIdx.x;
  if (skip_line(status, t, every, q_off)) return;  // the same for the whole CTA
  extern __shared__ __align__(16) float2 psm[];
  float2* Ch = psm;             // [64][DS] a chunk of 64 rows below: A_ik, then L_ik
  float2* Iv = Ch + 64 * DS;    // [64][DS] X = L_kk^{-1}
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int Bp = pad64(B), p = 64 * k, kb = min(64, B - p);
  float2* A = reinterpret_cast<float2*>(sigma_all + (int64_t)t * B * B);
  uint8_t* sl = slice_base(slice_all, slice_stride, t);
  int32_t* expo = reinterpret_cast<int32_t*>(sl + NDIG * plane_bytes(Bp));
  const float2* Xg = reinterpret_cast<const float2*>(sl + xinv_offset(Bp));
  const int64_t plane = (int64_t)Bp * Bp;
  void* w = (char*)wmat + (size_t)t * plane * 4;
  constexpr bool TR = PREC == P_FP32T;  // transposed operand: consecutive threads on consecutive rows n
  for (int e = tid; e < 64 * 64; e += TP_T) Iv[(e >> 6) * DS + (e & 63)] = Xg[e];
  __syncthreads();

  // ---- rows below: L_ik = A_ik L_kk^{-T}, written to the operand and split into digits ----
  const int tr = tid >> 4, tcg = tid & 15;  // rows 4 tr .. 4 tr + 3, columns 4 tcg .. 4 tcg + 3
  for (int c0 = p + 64; c0 < Bp; c0 += 64) {
    for (int e = tid; e < 64 * 64; e += TP_T) {
      const int r = e >> 6, c = e & 63;
      Ch[r * DS + c] = (c0 + r < B && c < kb) ? A[(int64_t)(c0 + r) * B + p + c] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    float s[4][4], cc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) s[a][b] = cc[a][b] = 0.f;
    const int qmax = min(kb, 4 * tcg + 4);  // X[c][q] = 0 for q > c
    for (int q = 0; q < qmax; ++q) {
      float2 av[4], xv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        av[a] = Ch[(4 * tr + a) * DS + q];
        const float2 x = Iv[(4 * tcg + a) * DS + q];  // X[c][q]: zero for q > c
        xv[a] = make_float2(-x.x, -x.y);
      }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) ff_fms(s[a][b], cc[a][b], av[a], xv[b]);  // s += A X^T
    }
    __syncthreads();  // every thread has read Ch
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) Ch[(4 * tr + a) * DS + 4 * tcg + b] = ff_norm(s[a][b], cc[a][b]);
    __syncthreads();
    // the operand's rows c0 .. c0 + 63 of block column k
    for (int e = tid; e < 64 * 64; e += TP_T) {
      const int r = TR ? e & 63 : e >> 6, c = TR ? e >> 6 : e & 63;
      const int64_t idx = fk::h_index<PREC>(c0 + r, p + c, Bp);
      if (c0 + r < B && c < kb) fk::WOut<PREC>::store(w, plane, idx, fk::ArFF::to_f(Ch[r * DS + c]));
      else fk::WOut<PREC>::zero(w, plane, idx);
    }
    // digits: one warp per row, two columns per lane
    for (int r = warp; r < 64; r += TP_T / 32) {
      const int row = c0 + r;
      float2 v[2] = {Ch[r * DS + lane], Ch[r * DS + lane + 32]};
      float mx = fmaxf(fabsf(v[0].x), fabsf(v[1].x));
      for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      int e = 0;
      if (mx > 0.f) frexpf(mx, &e);  // |value| <= mx < 2^e
      if (lane == 0) expo[row] = e;
      const float sc = ldexpf(1.f, -e);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        float xh = __fmul_rn(v[h].x, sc), xl = __fmul_rn(v[h].y, sc);  // exact: a power of two
        const int col = lane + 32 * h;
        const uint32_t off = tc::sw128_offset(row, col);
#pragma unroll
        for (int d = 0; d < NDIG; ++d) {
          xh = __fmul_rn(xh, 256.f);
          xl = __fmul_rn(xl, 256.f);
          const float dg = rintf(xh);
          const float2 rem = ff_norm(__fsub_rn(xh, dg), xl);  // xh - dg is exact
          xh = rem.x;
          xl = rem.y;
          *(__nv_bfloat16*)(sl + d * plane_bytes(Bp) + off) = __float2bfloat16_rn(dg);  // |dg| <= 256: exact
        }
      }
    }
    __syncthreads();  // before the next chunk overwrites Ch
  }
}

// ---- trailing update on the tensor cores ------------------------------------------------
__global__ void __launch_bounds__(TU_T, 1) tcf_update_kernel(double* __restrict__ sigma_all,
                                                             uint8_t* __restrict__ slice_all,
                                                             size_t slice_stride, int B, int k,
                                                             const int32_t* __restrict__ status, int every,
                                                             int q_off, int32_t* __restrict__ err,
                                                             long long limit) {
  const int t = blockIdx.y;
  const int Bp = pad64(B), r0 = 64 * (k + 1);
  const int nbr = (Bp - r0 + TU_M - 1) / TU_M, nbc = (Bp - r0) / TU_N;
  // tile index -> (row tile a, column block b <= 2a + 1)
  int a = 0, b = blockIdx.x;
  for (; a < nbr; ++a) {
    const int cnt = min(2 * a + 2, nbc);
    if (b < cnt) break;
    b -= cnt;
  }
  if (a >= nbr || skip_line(status, t, every, q_off)) return;  // uniform for the CTA
  extern __shared__ uint8_t usm_raw[];
  uint8_t* sm = (uint8_t*)(((uintptr_t)usm_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = sm;                                  // NDIG planes of 128 x 64 BF16 (swizzled)
  uint8_t* sB = sm + NDIG * TU_A_PLANE;              // NDIG planes of 64 x 64 BF16
  float2* As = (float2*)(sB + NDIG * TU_B_PLANE);   // the trailing tile A[i0 ..][j0 ..], [128][TU_AS]
  uint64_t* bars = (uint64_t*)((uint8_t*)As + TU_TILE);
  uint32_t* tslot = (uint32_t*)(bars + 4);
  int* ej = (int*)(bars + 8);                        // exponents of the 64 columns
  const uint32_t full = tc::smem_u32(bars), done = full + 8;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint8_t* sl = slice_base(slice_all, slice_stride, t);
  const int32_t* expo = reinterpret_cast<const int32_t*>(sl + NDIG * plane_bytes(Bp));
  const int i0 = r0 + TU_M * a, j0 = r0 + TU_N * b;

  if (tid == 0) {
    tc::mbar_init(full, 1);
    tc::mbar_init(done, 1);
    tc::mbar_init_fence();
  }
  if (tid < 64) ej[tid] = expo[j0 + tid];
  if (warp == 4) tc::tmem_alloc(tc::smem_u32(tslot), 512);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = *tslot;
  bool ok = true;

  if (warp == 4) {
    if (lane == 0) {
      tc::mbar_arrive_expect_tx(full, NDIG * (TU_A_PLANE + TU_B_PLANE));
      for (int d = 0; d < NDIG; ++d) {
        tc::bulk_load(tc::smem_u32(sA + d * TU_A_PLANE), sl + d * plane_bytes(Bp) + (size_t)i0 * 128, TU_A_PLANE,
                      full);
        tc::bulk_load(tc::smem_u32(sB + d * TU_B_PLANE), sl + d * plane_bytes(Bp) + (size_t)j0 * 128, TU_B_PLANE,
                      full);
      }
      if (!tc::mbar_wait(full, 0, limit)) ok = false;
      tc::fence_after_sync();
      if (ok) {
        const uint32_t idesc = tc::idesc_f16(1, TU_M, TU_N);
        // level l = t + u accumulates d_t(rows i) d_u(rows j)^T into columns 64 l .. 64 l + 63
        for (int l = 0; l < NDIG; ++l)
          for (int dt = 0; dt <= l; ++dt) {
            const uint32_t aop = tc::smem_u32(sA + dt * TU_A_PLANE), bop = tc::smem_u32(sB + (l - dt) * TU_B_PLANE);
#pragma unroll
            for (int ks = 0; ks < TU_K / 16; ++ks)
              tc::mma_f16(tbase + (uint32_t)(64 * l), tc::desc_sw128(aop + ks * 32), tc::desc_sw128(bop + ks * 32),
                          idesc, (dt > 0 || ks > 0) ? 1u : 0u);
          }
        tc::mma_commit(done);
      } else {
        tc::mbar_arrive(done);
        atomicExch(err, 1);
        tc::mbar_wait(full, 0, limit);  // copies still in flight land before the CTA may exit
      }
    }
  } else {
    // epilogue warps: stage the trailing tile (coalesced rows, while the digits load and the
    // MMAs run), then one tile row per thread (= its TMEM lane), then store it back coalesced
    float2* A = reinterpret_cast<float2*>(sigma_all + (int64_t)t * B * B);
    // 16 rows per round: 32 independent loads in flight per lane
    for (int r0w = warp * 32; r0w < warp * 32 + 32; r0w += 16) {
      float2 v[16][2];
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int i = i0 + r0w + q;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int j = j0 + lane + 32 * h;
          v[q][h] = (i < B && j < B && j <= i) ? A[(int64_t)i * B + j] : make_float2(0.f, 0.f);
        }
      }
#pragma unroll
      for (int q = 0; q < 16; ++q)
#pragma unroll
        for (int h = 0; h < 2; ++h) As[(r0w + q) * TU_AS + lane + 32 * h] = v[q][h];
    }
    const bool dok = tc::mbar_wait(done, 0, limit);
    __syncwarp();
    tc::fence_after_sync();
    if (!dok) atomicExch(err, 1);
    const int row = 32 * warp + lane, i = i0 + row;
    const int ei = expo[i];  // i < Bp + 64: the region's exponent rows
    const uint32_t taddr = tbase + ((uint32_t)(32 * warp) << 16);
    for (int c0 = 0; c0 < TU_N; c0 += 16) {
      float lev[NDIG][16];
#pragma unroll
      for (int l = 0; l < NDIG; ++l) tc::tmem_ld16(taddr + (uint32_t)(64 * l + c0), lev[l]);
      if (dok && i < B) {
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          const int j = j0 + c0 + c;
          if (j <= i && j < B) {
            // sum_l S_l 2^(-8 l) in float-float (each term an exact FP32 integer times a power of two)
            float hs = lev[0][c], hc = 0.f;
#pragma unroll
            for (int l = 1; l < NDIG; ++l) {
              const float p = __fmul_rn(lev[l][c], ldexpf(1.f, -8 * l));
              const float s2 = __fadd_rn(hs, p);
              const float z = __fsub_rn(s2, hs);
              hc = __fadd_rn(hc, __fadd_rn(__fsub_rn(hs, __fsub_rn(s2, z)), __fsub_rn(p, z)));
              hs = s2;
            }
            const float sc = ldexpf(1.f, ei + ej[c0 + c] - 16);
            const float2 upd = ff_norm(__fmul_rn(hs, sc), __fmul_rn(hc, sc));
            As[row * TU_AS + c0 + c] = ff_sub(As[row * TU_AS + c0 + c], upd);
          }
        }
      }
    }
    __syncwarp();  // the warp's 32 rows are complete
    if (dok) {
      for (int r = warp * 32; r < warp * 32 + 32; ++r) {
        const int i2 = i0 + r;
        for (int c = lane; c < TU_N; c += 32) {
          const int j = j0 + c;
          if (i2 < B && j < B && j <= i2) A[(int64_t)i2 * B + j] = As[r * TU_AS + c];
        }
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 4) {
    __syncwarp();
    tc::tmem_dealloc(tbase, 512);
  }
}

bool factor_tc_supported(int B, int prec) { return is_trsm(prec) && B >= 192; }

// Steps: 0 forms the covariance; then per panel k the diagonal block, and, for every panel
// but the last, the rows below and the trailing update: 1 + 3 nb - 2 launches.
int factor_tc_steps(int B) { return 3 * (pad64(B) / 64) - 1; }
int factor_tc_step_kind(int step) { return step == 0 ? 0 : 1 + (step - 1) % 3; }

cudaError_t launch_factor_tc_step(int step, double* sigma, double* scratch, const double* m, int L, int B, int prec,
                                  void* wmat, float* y0, float* inv_s2, int32_t* status, int64_t n0, int W,
                                  int incl, cudaStream_t st, LaunchCounter* lc, const int64_t* n0_dev, int every,
                                  int q_off, const double* n_line, int32_t* err) {
  if (L <= 0) return cudaSuccess;
  if (!factor_tc_supported(B, prec) || step < 0 || step >= factor_tc_steps(B)) return cudaErrorInvalidValue;
  const int Bp = pad64(B);
  const size_t stride = (size_t)B * B * 8;  // the inverse scratch per line holds the slices
  if (slice_region_bytes(Bp) + 1024 > stride) return cudaErrorInvalidValue;
  uint8_t* slices = reinterpret_cast<uint8_t*>(scratch);
  cudaError_t e = cudaSuccess;
  const int kind = factor_tc_step_kind(step), k = (step - 1) / 3;
  if (kind == 0) {
    tcf_form_kernel<<<dim3((B + 7) / 8, L), 256, 0, st>>>(sigma, m, B, status, n0, W, incl, n0_dev, every, q_off,
                                                           n_line);
  } else if (kind == 1) {
    auto diag = prec == P_BF16T ? tcf_diag_kernel<P_BF16T> : tcf_diag_kernel<P_FP32T>;
    diag<<<L, TD_T, 0, st>>>(sigma, slices, stride, m, B, k, status, every, q_off, wmat, y0, inv_s2);
  } else if (kind == 2) {
    const size_t psmem = (size_t)2 * 64 * DS * sizeof(float2);
    auto trsm = prec == P_BF16T ? tcf_trsm_kernel<P_BF16T> : tcf_trsm_kernel<P_FP32T>;
    e = cudaFuncSetAttribute(trsm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psmem);
    if (e != cudaSuccess) return e;
    trsm<<<L, TP_T, psmem, st>>>(sigma, slices, stride, B, k, status, every, q_off, wmat);
  } else {
    const long long limit = 4000000000LL;  // ~2 s of clock cycles
    e = cudaFuncSetAttribute(tcf_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TU_SMEM);
    if (e != cudaSuccess) return e;
    const int r0 = 64 * (k + 1), nbr = (Bp - r0 + TU_M - 1) / TU_M, nbc = (Bp - r0) / TU_N;
    int tiles = 0;
    for (int a = 0; a < nbr; ++a) tiles += (2 * a + 2 < nbc) ? 2 * a + 2 : nbc;
    tcf_update_kernel<<<dim3(tiles, L), TU_T, TU_SMEM, st>>>(sigma, slices, stride, B, k, status, every, q_off, err,
                                                               limit);
  }
  if (lc) lc->n += 1;
  return cudaGetLastError();
}

}  // namespace hsad
