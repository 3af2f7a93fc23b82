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

#include <algorithm>

#include "factor_kernel.cuh"
#include "hsad_internal.h"
#include "tc_util.cuh"

namespace hsad {

namespace {

constexpr int NDIG = 6;            // base-256 digits per value
constexpr int TU_M = 128, TU_N = 64, TU_K = 64;
constexpr uint32_t TU_A_PLANE = TU_M * TU_K * 2;   // 16 KB
constexpr uint32_t TU_B_PLANE = TU_N * TU_K * 2;   // 8 KB
constexpr int TU_AS = TU_N + 1;    // row stride (float2) of the staged trailing tile
// the update and panel kernels: 16 epilogue warps (TMEM lane group w & 3 x 16-column quarter
// w >> 2) and one copy / MMA warp
constexpr int UP_EW = 16, UP_MW = UP_EW, UP_T = 32 * (UP_EW + 1);
constexpr uint32_t TU_TILE = TU_M * TU_AS * 8;
constexpr uint32_t TU_SMEM = 1024 + NDIG * (TU_A_PLANE + TU_B_PLANE) + TU_TILE + 256 + 64;

// Byte layout of one line's slice region (in the inverse scratch): NDIG planes of
// (Bp + 64) rows x 128 bytes, then (Bp + 64) int32 exponents.
__host__ __device__ inline size_t plane_bytes(int Bp) { return (size_t)(Bp + 64) * 128; }
// then the digits of the diagonal block's inverse X (NDIG planes of [64][64] BF16, swizzled
// like the panel rows) and X's 64 row exponents
__host__ __device__ inline size_t xdig_offset(int Bp) { return NDIG * plane_bytes(Bp) + (size_t)(Bp + 64) * 4; }
constexpr uint32_t XDIG_BYTES = NDIG * TU_B_PLANE + 64 * 4;
__host__ __device__ inline size_t slice_region_bytes(int Bp) { return xdig_offset(Bp) + XDIG_BYTES; }
constexpr int TD_T = 256;            // threads per line of the diagonal-block kernel
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

// The six signed base-256 digits of v * sc (|v * sc| < 1): v * sc = sum_d dg[d] 256^-(d+1)
// up to 256^-6 / 2; every digit an integer of magnitude <= 256 (exact in BF16).
__device__ __forceinline__ void split_digits(float2 v, float sc, float (&dg)[NDIG]) {
  float xh = __fmul_rn(v.x, sc), xl = __fmul_rn(v.y, sc);  // exact: a power of two
#pragma unroll
  for (int d = 0; d < NDIG; ++d) {
    xh = __fmul_rn(xh, 256.f);
    xl = __fmul_rn(xl, 256.f);
    dg[d] = rintf(xh);
    const float2 rem = ff_norm(__fsub_rn(xh, dg[d]), xl);  // xh - dg is exact
    xh = rem.x;
    xl = rem.y;
  }
}
// Exponent e with |v| <= mx < 2^e (0 for an all-zero row): the biased exponent field of mx
// minus 126 (frexp's exponent for normal mx; -126, still a bound, for subnormal mx).
__device__ __forceinline__ int row_exponent(float mx) {
  return mx > 0.f ? ((__float_as_int(mx) >> 23) & 0xff) - 126 : 0;
}
// 2^e as a float: the exponent field directly where 2^e is a normal float.
__device__ __forceinline__ float pow2f(int e) {
  return (e >= -126 && e <= 127) ? __int_as_float((e + 127) << 23) : ldexpf(1.f, e);
}
__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&h);
}
// 2^(-16) sum_l S_l 256^-l in float-float times 2^e: the digit levels (exact FP32 integers)
// of one accumulator column combined.
template <int W>
__device__ __forceinline__ float2 combine_levels(const float (&lev)[NDIG][W], int c, int e) {
  constexpr float kLevel[NDIG] = {1.f, 0x1p-8f, 0x1p-16f, 0x1p-24f, 0x1p-32f, 0x1p-40f};
  float hs = lev[0][c], hc = 0.f;
#pragma unroll
  for (int l = 1; l < NDIG; ++l) {
    const float p = __fmul_rn(lev[l][c], kLevel[l]);
    const float s2 = __fadd_rn(hs, p);
    const float z = __fsub_rn(s2, hs);
    hc = __fadd_rn(hc, __fadd_rn(__fsub_rn(hs, __fsub_rn(s2, z)), __fsub_rn(p, z)));
    hs = s2;
  }
  const float sc = pow2f(e - 16);
  return ff_norm(__fmul_rn(hs, sc), __fmul_rn(hc, sc));
}

// Eight consecutive operand values as NP BF16 planes (hi / lo, or hi / mid / lo: each the
// BF16 rounding of the FP32 remainder of the ones before), one 16-byte store per plane.
template <int NP>
__device__ __forceinline__ void store_planes8(__nv_bfloat16* w, int64_t plane, int64_t idx, const float (&f)[8]) {
  uint32_t pk[NP][4];
#pragma unroll
  for (int h = 0; h < 4; ++h) {
    const __nv_bfloat162 hi = __floats2bfloat162_rn(f[2 * h], f[2 * h + 1]);
    const float r0 = f[2 * h] - __low2float(hi), r1 = f[2 * h + 1] - __high2float(hi);
    const __nv_bfloat162 m = __floats2bfloat162_rn(r0, r1);
    pk[0][h] = *reinterpret_cast<const uint32_t*>(&hi);
    pk[1][h] = *reinterpret_cast<const uint32_t*>(&m);
    if constexpr (NP == 3) {
      const __nv_bfloat162 lo = __floats2bfloat162_rn(r0 - __low2float(m), r1 - __high2float(m));
      pk[2][h] = *reinterpret_cast<const uint32_t*>(&lo);
    }
  }
#pragma unroll
  for (int q = 0; q < NP; ++q)
    *reinterpret_cast<uint4*>(w + q * plane + idx) = make_uint4(pk[q][0], pk[q][1], pk[q][2], pk[q][3]);
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

// ---- running sums and covariance formation in one pass ---------------------------------
// Streamed statistics without gains or forgetting: the prefix over a batch's lines of the
// integer sums (S2 of lines so far, FP64, exact) and the formation of each line's covariance
// from it, (S2 - n m m^T) / (n - 1) as float-float, by one thread per lower-triangle entry
// walking the lines, so that the FP64 prefix is never written and re-read. The per-line
// float-float means, n m and 1 / (n - 1) come from a small pass first (FP64 conversions
// are slow here): ffm[t] = {m_0 .. m_B-1, n m_0 .. n m_B-1, 1 / (n - 1)}.
__global__ void tcf_form_prep_kernel(const double* __restrict__ m_all, int L, int B, int64_t n0_arg, int W,
                                     int incl, const int64_t* __restrict__ n0_dev, float2* __restrict__ ffm) {
  const int t = blockIdx.y, i = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= L) return;
  const double nn = (double)((n0_dev ? *n0_dev : n0_arg) + (int64_t)(t + incl) * W);
  float2* f = ffm + (int64_t)t * (2 * B + 1);
  if (i < B) {
    const double mi = m_all[(int64_t)t * B + i];
    f[i] = dff(mi);
    f[B + i] = dff(nn * mi);
  }
  if (i == 0) f[2 * B] = dff(1.0 / (nn - 1.0));
}

// A double (normal in FP32's range, or zero) as a float-float pair by integer operations on
// its bits (the FP64 pipe, and FP64 -> FP32 conversion, issue at 1/64 of the FP32 rate
// here): hi = the value truncated to 24 significant bits (exact), lo = the remaining 29 bits
// rounded to FP32, a relative error below 2^-47 of the value.
__device__ __forceinline__ float2 double_to_ff_bits(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const int ex = (int)((b >> 52) & 0x7ff) - 1023;
  if (((b >> 52) & 0x7ff) == 0 || ex < -126) return make_float2(0.f, 0.f);
  const unsigned int sign = (unsigned int)(b >> 32) & 0x80000000u;
  const unsigned long long mant = b & 0xFFFFFFFFFFFFFULL;
  const float hi = __uint_as_float(sign | ((unsigned int)(ex + 127) << 23) | (unsigned int)(mant >> 29));
  float lo = (float)(int)(mant & 0x1FFFFFFFULL) * pow2f(ex - 52);  // exact scaling (or flush below FP32's range)
  lo = sign ? -lo : lo;
  return make_float2(hi, lo);
}

// The batch's lines are cut into S segments of `len` lines so that S threads share each
// entry's walk: a first pass sums each segment (but the last) per entry, the second starts
// each segment from the state plus the sums of the segments before it. The sums are exact
// integers below 2^53 in FP64, so the running values do not depend on the segmentation.
__device__ __forceinline__ int tri_row(int q) {
  int i = (int)((sqrtf(8.f * (float)q + 1.f) - 1.f) * 0.5f);
  while (tri(i + 1) <= q) ++i;
  while (tri(i) > q) --i;
  return i;
}

__global__ void tcf_segsum_kernel(const double* __restrict__ buf, int L, int B, int len,
                                  double* __restrict__ segsum) {
  const int nq = B * (B + 1) / 2;
  const int q = blockIdx.x * blockDim.x + threadIdx.x, sg = blockIdx.y;
  if (q >= nq) return;
  const int i = tri_row(q), j = q - tri(i);
  const int64_t BB = (int64_t)B * B, e = (int64_t)i * B + j;
  const int t1 = min(L, (sg + 1) * len);
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  int t = sg * len;
  for (; t + 4 <= t1; t += 4)
#pragma unroll
    for (int u = 0; u < 4; ++u) acc[u] += buf[(int64_t)(t + u) * BB + e];
  for (; t < t1; ++t) acc[0] += buf[(int64_t)t * BB + e];
  segsum[(int64_t)sg * nq + q] = (acc[0] + acc[1]) + (acc[2] + acc[3]);
}

__global__ void tcf_prefix_form_kernel(double* __restrict__ buf, double* __restrict__ state_s2, int L, int B,
                                       int inclusive, const float2* __restrict__ ffm, int nseg, int len,
                                       const double* __restrict__ segsum) {
  const int64_t BB = (int64_t)B * B;
  const int nq = B * (B + 1) / 2;
  const int q = blockIdx.x * blockDim.x + threadIdx.x, sg = blockIdx.y;  // entry q = tri(i) + j
  if (q >= nq) return;
  const int i = tri_row(q), j = q - tri(i);
  const int64_t e = (int64_t)i * B + j;
  double run = state_s2[e];
  for (int s2 = 0; s2 < sg; ++s2) run += segsum[(int64_t)s2 * nq + q];
  const int tb = sg * len, te = min(L, tb + len);
  constexpr int U = 8;  // lines whose loads are in flight together
  for (int t0 = tb; t0 < te; t0 += U) {
    double v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) v[u] = (t0 + u < te) ? buf[(int64_t)(t0 + u) * BB + e] : 0.0;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int t = t0 + u;
      if (t >= te) break;
      const double before = run;
      run += v[u];
      const double S = inclusive ? run : before;
      const float2* f = ffm + (int64_t)t * (2 * B + 1);
      const float2 out = ff_mul(ff_sub(double_to_ff_bits(S), ff_mul(f[B + i], f[j])), f[2 * B]);
      reinterpret_cast<float2*>(buf)[(int64_t)t * BB + e] = out;
    }
  }
  if (sg == nseg - 1) state_s2[e] = run;
}

// ---- diagonal block -----------------------------------------------------------------------
// One CTA of TD_T threads per line: the 64 x 64 diagonal block of panel k, as packed lower
// triangles in shared memory, factored and inverted together, right-looking, a column at a
// time: the pivot l = sqrt(A_jj) and r = 1 / l (float-float Newton step from the FP32 rsqrt
// seed, computed by one thread), column j of L = A_.j r, row j of X = R_j. r (R: the
// running right-hand sides, I at the start), then the rank-1 updates A_ic -= L_ij L_cj
// (j < c <= i) and R_ic -= L_ij X_jc (i > j, c <= j) over the flattened trapezoid of rows
// j + 1 .. kb - 1. Writes X's digits (per-row power of two, six base-256 digits) to the
// line's slice region for the triangular solve, and the operand's diagonal block (L_kk^{-1}).
template <int PREC>
__global__ void __launch_bounds__(TD_T) tcf_diag_kernel(double* __restrict__ sigma_all,
                                                        uint8_t* __restrict__ slice_all, size_t slice_stride,
                                                        const double* __restrict__ m_all, int B, int k,
                                                        int32_t* __restrict__ status, int every, int q_off,
                                                        void* __restrict__ wmat, float* __restrict__ y0_all,
                                                        float* __restrict__ inv_s2_all) {
  __shared__ float2 S[2 * TRI64];  // L_kk then R (later X = L_kk^{-1}), packed: (i, c) at tri(i) + c
  __shared__ uint8_t row_of[TRI64];
  __shared__ float2 rs;            // 1 / l_jj of the current column
  __shared__ int not_pd;
  float2* Dg = S;
  float2* X = S + TRI64;
  const int t = blockIdx.x, tid = threadIdx.x;
  if (skip_line(status, t, every, q_off)) return;  // the same for the whole CTA
  const int Bp = pad64(B), p = 64 * k, kb = min(64, B - p);
  const float2* A = reinterpret_cast<const float2*>(sigma_all + (int64_t)t * B * B);
  uint8_t* sl = slice_base(slice_all, slice_stride, t);
  uint8_t* xd = sl + xdig_offset(Bp);
  int32_t* xe = reinterpret_cast<int32_t*>(xd + NDIG * TU_B_PLANE);
  const int64_t plane = (int64_t)Bp * Bp;
  void* w = (char*)wmat + (size_t)t * plane * wmat_elem_bytes(PREC);
  if (k == 0) {  // the means of the triangular-solve form and the unit score scale
    for (int n = tid; n < Bp; n += TD_T) y0_all[(int64_t)t * Bp + n] = n < B ? (float)m_all[(int64_t)t * B + n] : 0.f;
    if (tid == 0) inv_s2_all[t] = 1.0f;
  }
  if (tid == 0) not_pd = 0;
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
    if (tid < 32) {  // the pivot, by one warp: r = 1 / sqrt(a), l_jj = a r
      const float2 a = Dg[tri(j) + j];
      if (!(a.x > 0.f) || !isfinite(a.x)) {
        if (tid == 0) not_pd = 1;
      } else if (tid == 0) {
        // FP32 seed, one Newton step r += r (1 - a r^2) / 2 in float-float (the seed's relative
        // error, below 2^-22, squares to below 2^-44: the order of the six-digit updates' 2^-45)
        float2 r = make_float2(rsqrtf(a.x), 0.f);
        const float2 ee = ff_sub(make_float2(1.f, 0.f), ff_mul(a, ff_mul(r, r)));
        r = ff_sub(r, ff_mul(r, make_float2(-0.5f * ee.x, -0.5f * ee.y)));
        rs = r;
        Dg[tri(j) + j] = ff_mul(a, r);  // read by nobody during this step
      }
    }
    __syncthreads();
    if (not_pd) {  // the same value in every thread
      if (tid == 0) status[t] = LS_NOT_PD;
      return;
    }
    const float2 r = rs;
    // column j of L below the pivot, row j of X
    const int nl = kb - 1 - j;
    if (tid < nl) {
      const int i = j + 1 + tid;
      Dg[tri(i) + j] = ff_mul(Dg[tri(i) + j], r);
    } else if (tid - nl <= j) {
      const int c = tid - nl;
      X[tri(j) + c] = ff_mul(X[tri(j) + c], r);
    }
    __syncthreads();
    // rank-1 update of rows j + 1 .. kb - 1: X columns c <= j, L columns c > j (one shared
    // array indexed by offset, so that every access is a shared-memory one)
    const int e0 = tri(j + 1), e1 = tri(kb);
    for (int e = e0 + tid; e < e1; e += TD_T) {
      const int i = row_of[e], c = e - tri(i);
      const bool inx = c <= j;
      const int off = inx ? TRI64 : 0;
      const float2 lij = S[tri(i) + j];
      const float2 y = S[inx ? TRI64 + tri(j) + c : tri(c) + j];
      float2 v = S[off + e];
      ff_fms(v.x, v.y, lij, y);
      S[off + e] = ff_norm(v.x, v.y);
    }
    __syncthreads();
  }
  // X for the triangular solve, where rows lie below: per row c an exponent and six digit
  // planes of X[c][q] (zero above the diagonal), the B operand of the tensor-core solve
  constexpr bool TR = PREC == P_FP32T;
  if (p + 64 < Bp) {
    __shared__ int xe_s[64];
    if (tid < 64) {
      float mx = 0.f;
      for (int q = 0; q <= tid && tid < kb; ++q) mx = fmaxf(mx, fabsf(X[tri(tid) + q].x));
      const int e = row_exponent(mx);
      xe_s[tid] = e;
      xe[tid] = e;
    }
    __syncthreads();
    for (int it = tid; it < 64 * 8; it += TD_T) {  // (row c, 8-column group g)
      const int c = it >> 3, g = it & 7;
      const float sc = pow2f(-xe_s[c]);
      uint32_t pk[NDIG][4];
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        float d0[NDIG], d1[NDIG];
        const int q0 = 8 * g + 2 * h;
        split_digits((q0 <= c && c < kb) ? X[tri(c) + q0] : make_float2(0.f, 0.f), sc, d0);
        split_digits((q0 + 1 <= c && c < kb) ? X[tri(c) + q0 + 1] : make_float2(0.f, 0.f), sc, d1);
#pragma unroll
        for (int d = 0; d < NDIG; ++d) pk[d][h] = pack_bf16x2(d0[d], d1[d]);
      }
#pragma unroll
      for (int d = 0; d < NDIG; ++d)
        *reinterpret_cast<uint4*>(xd + d * TU_B_PLANE + c * 128 + (((g ^ c) & 7) << 4)) =
            make_uint4(pk[d][0], pk[d][1], pk[d][2], pk[d][3]);
    }
  }
  // the operand's diagonal block, threads on consecutive addresses
  for (int e = tid; e < 64 * 64; e += TD_T) {
    const int n = TR ? e & 63 : e >> 6, c = TR ? e >> 6 : e & 63;  // row n, column c of the block
    const int64_t idx = fk::h_index<PREC>(p + n, p + c, Bp);
    if (c <= n && n < kb) fk::WOut<PREC>::store(w, plane, idx, fk::ArFF::to_f(X[tri(n) + c]));
    else fk::WOut<PREC>::zero(w, plane, idx);
  }
}

// ---- rows below the diagonal block on the tensor cores -------------------------------------
// L_ik = A_ik X^T for a 128-row tile of the rows below panel k's diagonal block (grid: row
// tiles x lines; 16 epilogue warps + 1 copy / MMA warp, like the update): the tile's rows of A
// (float-float) are split into six digits with a per-row power of two straight into the
// swizzled A operand while X's digits arrive by one bulk copy; the 21 digit-product MMAs sum
// each level exactly in TMEM (the update's bound: a 64-term level sum stays below 2^24); the
// epilogue combines the levels per row (one row per thread), writes the row to the whitening
// operand, and splits it again into six digits for the trailing updates.
constexpr uint32_t TT_SMEM = 1024 + NDIG * (TU_A_PLANE + TU_B_PLANE) + 256 + 128 * 4 + 4 * 128 * 4 + 64;
template <int PREC>
__global__ void __launch_bounds__(UP_T, 1) tcf_trsm_kernel(double* __restrict__ sigma_all,
                                                           uint8_t* __restrict__ slice_all, size_t slice_stride,
                                                           int B, int k, const int32_t* __restrict__ status,
                                                           int every, int q_off, void* __restrict__ wmat,
                                                           int32_t* __restrict__ err, long long limit) {
  const int t = blockIdx.y;
  const int Bp = pad64(B), p = 64 * k, i0 = p + 64 + TU_M * blockIdx.x;
  if (i0 >= Bp || skip_line(status, t, every, q_off)) return;  // uniform for the CTA
  extern __shared__ uint8_t tsm_raw[];
  uint8_t* sm = tc::align1024(tsm_raw);
  uint8_t* sA = sm;                          // NDIG planes of 128 x 64 BF16 (swizzled); later the L rows
  uint8_t* sX = sm + NDIG * TU_A_PLANE;      // NDIG planes of 64 x 64 BF16, then X's 64 row exponents
  const int* fx = (const int*)(sX + NDIG * TU_B_PLANE);
  int* ea = (int*)(sX + XDIG_BYTES);         // exponents of the tile's rows of A
  float* rmax = (float*)(ea + 128);          // [4][128] row maxima of the four column quarters of L
  uint64_t* bars = (uint64_t*)(rmax + 512);
  uint32_t* tslot = (uint32_t*)(bars + 4);
  const uint32_t full = tc::smem_u32(bars), done = full + 8;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  uint8_t* sl = slice_base(slice_all, slice_stride, t);
  int32_t* expo = reinterpret_cast<int32_t*>(sl + NDIG * plane_bytes(Bp));

  if (tid == 0) {
    tc::mbar_init(full, 1);
    tc::mbar_init(done, 1);
    tc::mbar_init_fence();
  }
  if (warp == UP_MW) tc::tmem_alloc(tc::smem_u32(tslot), 512);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = *tslot;
  const float2* A = reinterpret_cast<const float2*>(sigma_all + (int64_t)t * B * B);

  if (warp == UP_MW) {
    if (lane == 0) {
      tc::mbar_arrive_expect_tx(full, XDIG_BYTES);
      tc::bulk_load(tc::smem_u32(sX), sl + xdig_offset(Bp), XDIG_BYTES, full);
    }
  } else {
    // the A operand: rows of the tile split into digits (8 rows per warp, lanes across the
    // 64 columns: coalesced loads, conflict-free 2-byte stores within a swizzled row)
    for (int rr = warp * 8; rr < warp * 8 + 8; rr += 8) {
      float2 v[8][2];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int i = i0 + rr + q;
#pragma unroll
        for (int h = 0; h < 2; ++h)
          v[q][h] = i < B ? A[(int64_t)i * B + p + lane + 32 * h] : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        float mx = fmaxf(fabsf(v[q][0].x), fabsf(v[q][1].x));
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        const int e = row_exponent(mx);
        if (lane == 0) ea[rr + q] = e;
        const float sc = pow2f(-e);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          float dg[NDIG];
          split_digits(v[q][h], sc, dg);
          const uint32_t off = tc::sw128_offset(rr + q, lane + 32 * h);
#pragma unroll
          for (int d = 0; d < NDIG; ++d) *(__nv_bfloat16*)(sA + d * TU_A_PLANE + off) = __float2bfloat16_rn(dg[d]);
        }
      }
    }
    tc::fence_proxy_async();  // the digits written by these threads, visible to the tensor cores
  }
  __syncthreads();
  bool ok = true;
  if (warp == UP_MW) {
    if (lane == 0) {
      if (!tc::mbar_wait(full, 0, limit)) ok = false;
      tc::fence_after_sync();
      if (ok) {
        const uint32_t idesc = tc::idesc_f16(1, TU_M, TU_N);
        // descriptors by offset: a plane adds its size / 16, a 32-byte K step 2
        const uint64_t dA = tc::desc_sw128(tc::smem_u32(sA)), dB = tc::desc_sw128(tc::smem_u32(sX));
        for (int l = 0; l < NDIG; ++l)
          for (int dt = 0; dt <= l; ++dt) {
            const uint64_t da = dA + (uint64_t)(dt * (TU_A_PLANE >> 4)), db = dB + (uint64_t)((l - dt) * (TU_B_PLANE >> 4));
#pragma unroll
            for (int ks = 0; ks < TU_K / 16; ++ks)
              tc::mma_f16(tbase + (uint32_t)(64 * l), da + 2 * ks, db + 2 * ks, idesc, (dt > 0 || ks > 0) ? 1u : 0u);
          }
        tc::mma_commit(done);
      } else {
        tc::mbar_arrive(done);
        atomicExch(err, 1);
        tc::mbar_wait(full, 0, limit);  // a copy still in flight lands before the CTA may exit
      }
    }
  } else {
    const bool dok = tc::mbar_wait(done, 0, limit);
    __syncwarp();
    tc::fence_after_sync();
    if (!dok) atomicExch(err, 1);
    // thread (TMEM lane group lg, column quarter ch): row 32 lg + lane, columns 16 ch .. 16 ch + 15
    const int lg = warp & 3, ch = warp >> 2, cs = 16 * ch;
    const int row = 32 * lg + lane, i = i0 + row;
    const int ei = ea[row];
    const uint32_t taddr = tbase + ((uint32_t)(32 * lg) << 16);
    float2* Ls = reinterpret_cast<float2*>(sA) + row * TU_AS;  // this thread's row (the MMAs are done)
    float mx = 0.f;
    for (int c0 = cs; c0 < cs + 16; c0 += 8) {
      float lev[NDIG][8];
#pragma unroll
      for (int l = 0; l < NDIG; ++l) tc::tmem_ld8(taddr + (uint32_t)(64 * l + c0), lev[l]);
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const float2 v = (dok && i < B) ? combine_levels(lev, c, ei + fx[c0 + c]) : make_float2(0.f, 0.f);
        Ls[c0 + c] = v;
        mx = fmaxf(mx, fabsf(v.x));
      }
    }
    rmax[ch * 128 + row] = mx;
    asm volatile("bar.sync 1, %0;" ::"n"(32 * UP_EW) : "memory");  // the epilogue warps only
    mx = fmaxf(fmaxf(rmax[row], rmax[128 + row]), fmaxf(rmax[256 + row], rmax[384 + row]));
    if (dok && i < Bp) {
      // the whitening operand's rows (zero past B)
      const int64_t plane = (int64_t)Bp * Bp;
      void* w = (char*)wmat + (size_t)t * plane * wmat_elem_bytes(PREC);
      if constexpr (PREC == P_FP32T) {  // transposed: consecutive threads on consecutive rows
        for (int c = cs; c < cs + 16; ++c)
          fk::WOut<PREC>::store(w, plane, fk::h_index<PREC>(i, p + c, Bp), fk::ArFF::to_f(Ls[c]));
      } else {  // BF16 planes, row-major: this thread's row in 16-byte pieces
        __nv_bfloat16* wb = (__nv_bfloat16*)w;
        for (int g = 2 * ch; g < 2 * ch + 2; ++g) {
          float f[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) f[j] = fk::ArFF::to_f(Ls[8 * g + j]);
          store_planes8<trsm_planes(PREC)>(wb, plane, fk::h_index<PREC>(i, p + 8 * g, Bp), f);
        }
      }
      // the row's digits for the trailing updates: 16-byte stores into the swizzled planes
      const int e = row_exponent(mx);
      if (ch == 0) expo[i] = e;
      const float sc = pow2f(-e);
      for (int g = 2 * ch; g < 2 * ch + 2; ++g) {
        uint32_t pk[NDIG][4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
          float d0[NDIG], d1[NDIG];
          split_digits(Ls[8 * g + 2 * h], sc, d0);
          split_digits(Ls[8 * g + 2 * h + 1], sc, d1);
#pragma unroll
          for (int d = 0; d < NDIG; ++d) pk[d][h] = pack_bf16x2(d0[d], d1[d]);
        }
#pragma unroll
        for (int d = 0; d < NDIG; ++d)
          *reinterpret_cast<uint4*>(sl + d * plane_bytes(Bp) + (size_t)i * 128 + (((g ^ i) & 7) << 4)) =
              make_uint4(pk[d][0], pk[d][1], pk[d][2], pk[d][3]);
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == UP_MW) {
    __syncwarp();
    tc::tmem_dealloc(tbase, 512);
  }
}

// ---- trailing update on the tensor cores ------------------------------------------------
__global__ void __launch_bounds__(UP_T, 1) tcf_update_kernel(double* __restrict__ sigma_all,
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
  uint8_t* sm = tc::align1024(usm_raw);
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
  if (warp == UP_MW) tc::tmem_alloc(tc::smem_u32(tslot), 512);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = *tslot;
  bool ok = true;

  if (warp == UP_MW) {
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
        const uint64_t dA = tc::desc_sw128(tc::smem_u32(sA)), dB = tc::desc_sw128(tc::smem_u32(sB));
        for (int l = 0; l < NDIG; ++l)
          for (int dt = 0; dt <= l; ++dt) {
            const uint64_t da = dA + (uint64_t)(dt * (TU_A_PLANE >> 4)), db = dB + (uint64_t)((l - dt) * (TU_B_PLANE >> 4));
#pragma unroll
            for (int ks = 0; ks < TU_K / 16; ++ks)
              tc::mma_f16(tbase + (uint32_t)(64 * l), da + 2 * ks, db + 2 * ks, idesc, (dt > 0 || ks > 0) ? 1u : 0u);
          }
        tc::mma_commit(done);
      } else {
        tc::mbar_arrive(done);
        atomicExch(err, 1);
        tc::mbar_wait(full, 0, limit);  // copies still in flight land before the CTA may exit
      }
    }
  } else {
    // epilogue warps: each stages its 32 rows x 16 columns of the trailing tile (two rows of
    // 128 contiguous bytes per load instruction, while the digits load and the MMAs run),
    // then takes one row (= its TMEM lane) of those columns per thread, then stores them
    // back the way it loaded them
    float2* A = reinterpret_cast<float2*>(sigma_all + (int64_t)t * B * B);
    const int lg = warp & 3, cq = warp >> 2, cs = 16 * cq;
    {
      const int rr = lane >> 4, cc = cs + (lane & 15);
      float2 v[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int i = i0 + 32 * lg + 2 * q + rr, j = j0 + cc;
        v[q] = (i < B && j < B && j <= i) ? A[(int64_t)i * B + j] : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int q = 0; q < 16; ++q) As[(32 * lg + 2 * q + rr) * TU_AS + cc] = v[q];
    }
    const bool dok = tc::mbar_wait(done, 0, limit);
    __syncwarp();
    tc::fence_after_sync();
    if (!dok) atomicExch(err, 1);
    const int row = 32 * lg + lane, i = i0 + row;
    const int ei = expo[i];  // i < Bp + 64: the region's exponent rows
    const uint32_t taddr = tbase + ((uint32_t)(32 * lg) << 16);
    for (int c0 = cs; c0 < cs + 16; c0 += 8) {
      float lev[NDIG][8];
#pragma unroll
      for (int l = 0; l < NDIG; ++l) tc::tmem_ld8(taddr + (uint32_t)(64 * l + c0), lev[l]);
      if (dok && i < B) {
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const int j = j0 + c0 + c;
          if (j <= i && j < B) {
            const float2 upd = combine_levels(lev, c, ei + ej[c0 + c]);
            As[row * TU_AS + c0 + c] = ff_sub(As[row * TU_AS + c0 + c], upd);
          }
        }
      }
    }
    __syncwarp();  // the warp's 32 rows x 16 columns are complete
    if (dok) {
      const int rr = lane >> 4, cc = cs + (lane & 15);
#pragma unroll 4
      for (int q = 0; q < 16; ++q) {
        const int r = 32 * lg + 2 * q + rr, i2 = i0 + r, j = j0 + cc;
        if (i2 < B && j < B && j <= i2) A[(int64_t)i2 * B + j] = As[r * TU_AS + cc];
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == UP_MW) {
    __syncwarp();
    tc::tmem_dealloc(tbase, 512);
  }
}

bool factor_tc_supported(int B, int prec) { return is_trsm(prec) && B >= 192; }

// Steps: 0 forms the covariance; then per panel k the diagonal block, and, for every panel
// but the last, the rows below and the trailing update: 1 + 3 nb - 2 launches.
int factor_tc_steps(int B) { return 3 * (pad64(B) / 64) - 1; }
int factor_tc_step_kind(int step) { return step == 0 ? 0 : 1 + (step - 1) % 3; }

constexpr int kSegMax = 32;  // segments of the prefix pass
__host__ __device__ inline size_t ffm_bytes(int L, int B) {
  return ((size_t)L * (2 * B + 1) * sizeof(float2) + 255) / 256 * 256;
}
size_t tcf_form_scratch_bytes(int L, int B) {
  return ffm_bytes(L, B) + (size_t)kSegMax * (B * (B + 1) / 2) * sizeof(double);
}

cudaError_t launch_tcf_prefix_form(double* buf, double* state_s2, int L, int B, int inclusive, const double* m,
                                   int64_t n0, int W, int incl, const int64_t* n0_dev, float2* ffm,
                                   cudaStream_t st, LaunchCounter* lc) {
  if (L <= 0) return cudaSuccess;
  tcf_form_prep_kernel<<<dim3((B + 127) / 128, L), 128, 0, st>>>(m, L, B, n0, W, incl, n0_dev, ffm);
  if (lc) lc->n += 1;
  const int nq = B * (B + 1) / 2;
  // segments so that the walk is spread over about 600 k threads (four per FP32 lane of the
  // GPU), of at least 32 lines each
  int nseg = (int)std::min<int64_t>({(int64_t)kSegMax, std::max<int64_t>(1, L / 32), (600000 + nq - 1) / nq});
  nseg = std::max(nseg, 1);
  const int len = (L + nseg - 1) / nseg;
  nseg = (L + len - 1) / len;
  double* segsum = reinterpret_cast<double*>(reinterpret_cast<char*>(ffm) + ffm_bytes(L, B));
  const unsigned gx = (unsigned)((nq + 255) / 256);
  if (nseg > 1) {
    tcf_segsum_kernel<<<dim3(gx, nseg - 1), 256, 0, st>>>(buf, L, B, len, segsum);
    if (lc) lc->n += 1;
  }
  tcf_prefix_form_kernel<<<dim3(gx, nseg), 256, 0, st>>>(buf, state_s2, L, B, inclusive, ffm, nseg, len, segsum);
  if (lc) lc->n += 1;
  return cudaGetLastError();
}

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
    auto diag = prec == P_BF16T   ? tcf_diag_kernel<P_BF16T>
                : prec == P_FP32X ? tcf_diag_kernel<P_FP32X>
                                  : tcf_diag_kernel<P_FP32T>;
    diag<<<L, TD_T, 0, st>>>(sigma, slices, stride, m, B, k, status, every, q_off, wmat, y0, inv_s2);
  } else if (kind == 2) {
    const long long limit = 4000000000LL;  // ~2 s of clock cycles
    auto trsm = prec == P_BF16T   ? tcf_trsm_kernel<P_BF16T>
                : prec == P_FP32X ? tcf_trsm_kernel<P_FP32X>
                                  : tcf_trsm_kernel<P_FP32T>;
    e = cudaFuncSetAttribute(trsm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TT_SMEM);
    if (e != cudaSuccess) return e;
    const int tiles = (Bp - 64 * (k + 1) + TU_M - 1) / TU_M;
    trsm<<<dim3(tiles, L), UP_T, TT_SMEM, st>>>(sigma, slices, stride, B, k, status, every, q_off, wmat, err, limit);
  } else {
    const long long limit = 4000000000LL;  // ~2 s of clock cycles
    e = cudaFuncSetAttribute(tcf_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TU_SMEM);
    if (e != cudaSuccess) return e;
    const int r0 = 64 * (k + 1), nbr = (Bp - r0 + TU_M - 1) / TU_M, nbc = (Bp - r0) / TU_N;
    int tiles = 0;
    for (int a = 0; a < nbr; ++a) tiles += (2 * a + 2 < nbc) ? 2 * a + 2 : nbc;
    tcf_update_kernel<<<dim3(tiles, L), UP_T, TU_SMEM, st>>>(sigma, slices, stride, B, k, status, every, q_off, err,
                                                               limit);
  }
  if (lc) lc->n += 1;
  return cudaGetLastError();
}

}  // namespace hsad
