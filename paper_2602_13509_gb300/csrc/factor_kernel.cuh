// K4 + K5: Cholesky factorisation and triangular inverse of each line's covariance, and
// the whitening operand in the working precision (device code and launch templates;
// included by the translation units that instantiate it, one per arithmetic and working
// precision, so that they compile in parallel).
//
// Eq. 1 (Sec. 3.3) needs Sigma^{-1}. In the DN frame used by the statistics kernels the
// calibrated deviation is x - mu = D (x' - m), with x' = DN - c, m = mu_DN - c and D the
// per-band calibration gains, and Sigma = D S D with S the DN-frame covariance, so
//     delta = (x' - m)^T S^{-1} (x' - m) = || L^{-1} (x' - m) ||^2,   S = L L^T:
// the gains cancel and the factor works on S alone. The covariance is formed in FP64, and
// so are the 16 x 16 diagonal blocks with their pivots. The panel solves, the O(B^3)
// register-tiled updates (Cholesky trailing update, inverse block rows) and the inverse's
// forward substitutions run in the arithmetic AR:
//   ArFF  float-float (pairs of FP32 values, about 48 significant bits): FP64 issues at
//         1/64 of the FP32 rate on this part, so this is the fast form;
//   ArF64 FP64 throughout (53 bits).
// With G = L^{-1} the score is delta = || G x' - G m ||^2.
// G is lower triangular. It is stored row-major ([n][k], n = output coordinate) as the
// K-major operand of the whitening contraction, scaled by a power of two s so that
// max |s G| is in [0.5, 1) (keeps FP16 in range; exact in every format), and
// delta = || s G x' - s G m ||^2 / s^2.
//   FP32 : one float plane.
//   FP16 / BF16 : hi plane = rn(sG), lo plane = rn(sG - hi): the two-term split keeps
//                 about 16 (BF16) or 22 (FP16) bits of G.
// y0 = s G m is formed from the rounded operand actually used, in FP64.
// A non-positive or non-finite pivot marks the line LS_NOT_PD; nothing traps.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <mutex>
#include <utility>

#include "hsad_internal.h"

namespace hsad {
namespace fk {

constexpr int FT_CLUSTER = 256;  // threads per factorisation CTA in a cluster
constexpr int NB = 16;           // Cholesky panel width = inverse block height
constexpr int PS = NB + 1;       // padded panel row stride (8-byte slots): rows fall in different banks

__host__ __device__ inline int smem_slots(int B) { return B * PS; }

// Store one element of the whitening operand, given in FP32, and return the value actually
// stored (the sum of the stored planes, exact in FP32): the hi / lo split keeps 16 (BF16)
// or 22 (FP16) of its 24 bits.
template <int PREC>
struct WOut;
template <>
struct WOut<P_FP32> {
  __device__ static float store(void* w, int64_t, int64_t idx, float f) {
    ((float*)w)[idx] = f;
    return f;
  }
  __device__ static void zero(void* w, int64_t, int64_t idx) { ((float*)w)[idx] = 0.f; }
};
template <>
struct WOut<P_FP16> {
  __device__ static float store(void* w, int64_t plane, int64_t idx, float f) {
    const __half hi = __float2half_rn(f);
    const float hf = __half2float(hi);
    const __half lo = __float2half_rn(f - hf);
    ((__half*)w)[idx] = hi;
    ((__half*)w)[plane + idx] = lo;
    return hf + __half2float(lo);
  }
  __device__ static void zero(void* w, int64_t plane, int64_t idx) {
    ((uint16_t*)w)[idx] = 0;
    ((uint16_t*)w)[plane + idx] = 0;
  }
};
template <>
struct WOut<P_BF16> {
  __device__ static float store(void* w, int64_t plane, int64_t idx, float f) {
    const __nv_bfloat16 hi = __float2bfloat16_rn(f);
    const float hf = __bfloat162float(hi);
    const __nv_bfloat16 lo = __float2bfloat16_rn(f - hf);
    ((__nv_bfloat16*)w)[idx] = hi;
    ((__nv_bfloat16*)w)[plane + idx] = lo;
    return hf + __bfloat162float(lo);
  }
  __device__ static void zero(void* w, int64_t plane, int64_t idx) {
    ((uint16_t*)w)[idx] = 0;
    ((uint16_t*)w)[plane + idx] = 0;
  }
};
template <>
struct WOut<P_BF16T> : WOut<P_BF16> {};
template <>
struct WOut<P_FP32T> : WOut<P_FP32> {};
// three BF16 planes hi / mid / lo: an exact split of the FP32 value (each remainder is exact
// in FP32 and holds at most 16, then 8, significant bits)
template <>
struct WOut<P_FP32X> {
  __device__ static float store(void* w, int64_t plane, int64_t idx, float f) {
    const __nv_bfloat16 hi = __float2bfloat16_rn(f);
    const float r = f - __bfloat162float(hi);
    const __nv_bfloat16 mid = __float2bfloat16_rn(r);
    ((__nv_bfloat16*)w)[idx] = hi;
    ((__nv_bfloat16*)w)[plane + idx] = mid;
    ((__nv_bfloat16*)w)[2 * plane + idx] = __float2bfloat16_rn(r - __bfloat162float(mid));
    return f;
  }
  __device__ static void zero(void* w, int64_t plane, int64_t idx) {
    const __nv_bfloat16 z = __float2bfloat16_rn(0.f);
    ((__nv_bfloat16*)w)[idx] = z;
    ((__nv_bfloat16*)w)[plane + idx] = z;
    ((__nv_bfloat16*)w)[2 * plane + idx] = z;
  }
};

// Element (n, k) of the triangular-solve operand H: row n = output band (n-major) for the
// tensor-core form, whose TMA boxes are K-major rows; column k major (transposed) for the
// FP32 SIMT form, whose K-slices then load as contiguous rows.
template <int PREC>
__host__ __device__ __forceinline__ int64_t h_index(int n, int k, int Bp) {
  return PREC == P_FP32T ? (int64_t)k * Bp + n : (int64_t)n * Bp + k;
}

template <int FT>
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

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// CL == 1: block barrier. CL > 1: cluster barrier with release / acquire ordering.
template <int CL>
__device__ __forceinline__ void csync() {
  if (CL == 1) {
    __syncthreads();
  } else {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
  }
}
// A double in the shared memory of CTA `rank` of this cluster.
__device__ __forceinline__ double ld_remote(const double* local, int rank) {
  uint32_t laddr = (uint32_t)__cvta_generic_to_shared(local), raddr;
  double v;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(raddr) : "r"(laddr), "r"(rank));
  asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(raddr) : "memory");
  return v;
}

// ---- float-float: a value is an unevaluated pair hi + lo of FP32 numbers (about 48
// significant bits; FP32's exponent range), stored as a float2 in an 8-byte slot.
// s + c -= x y: the product's rounding error from an FMA (Dekker's two-product, with the
// hi x lo cross terms; lo x lo is below the format's precision), the sum's rounding error
// from Knuth's two-sum, both errors gathered in c (compensated dot product, Ogita, Rump
// and Oishi 2005). Explicitly rounded operations: the compiler may not fuse or reorder.
__device__ __forceinline__ void ff_fms(float& s, float& c, float2 x, float2 y) {
  const float p = __fmul_rn(x.x, y.x);
  float e = __fmaf_rn(x.x, y.x, -p);
  e = __fmaf_rn(x.x, y.y, e);
  e = __fmaf_rn(x.y, y.x, e);
  const float t = __fsub_rn(s, p);
  const float z = __fsub_rn(t, s);
  const float q = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(-p, z));
  s = t;
  c = __fsub_rn(__fadd_rn(c, q), e);
}
// a b in float-float (two-product with the cross terms), renormalised by fast two-sum
// (the error term is below half an ulp of the product).
__device__ __forceinline__ float2 ff_mul(float2 a, float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  float e = __fmaf_rn(a.x, b.x, -p);
  e = __fmaf_rn(a.x, b.y, e);
  e = __fmaf_rn(a.y, b.x, e);
  const float h = __fadd_rn(p, e);
  return make_float2(h, __fsub_rn(e, __fsub_rn(h, p)));
}
// The pair renormalised (two-sum: c may exceed s after cancellation).
__device__ __forceinline__ float2 ff_norm(float s, float c) {
  const float h = __fadd_rn(s, c);
  const float z = __fsub_rn(h, s);
  return make_float2(h, __fadd_rn(__fsub_rn(s, __fsub_rn(h, z)), __fsub_rn(c, z)));
}

struct ArFF {
  using T = float2;
  struct Acc {
    float s, c;
  };
  static constexpr bool kFP64 = false;
  __device__ static T from_d(double d) {
    const float h = __double2float_rn(d);
    return make_float2(h, __double2float_rn(d - (double)h));  // d - h is exact in FP64
  }
  __device__ static double to_d(T v) { return (double)v.x + (double)v.y; }
  __device__ static Acc acc(T v) { return Acc{v.x, v.y}; }
  __device__ static void fms(Acc& a, T x, T y) { ff_fms(a.s, a.c, x, y); }
  __device__ static T fin(Acc a) { return ff_norm(a.s, a.c); }
  __device__ static T mul(T a, T b) { return ff_mul(a, b); }
  __device__ static float to_f(T v) { return __fadd_rn(v.x, v.y); }  // nearest FP32 to hi + lo
  __device__ static T zero() { return make_float2(0.f, 0.f); }
  __device__ static T one() { return make_float2(1.f, 0.f); }
};

struct ArF64 {
  using T = double;
  struct Acc {
    double s;
  };
  static constexpr bool kFP64 = true;
  __device__ static T from_d(double d) { return d; }
  __device__ static double to_d(T v) { return v; }
  __device__ static Acc acc(T v) { return Acc{v}; }
  __device__ static void fms(Acc& a, T x, T y) { a.s = fma(-x, y, a.s); }
  __device__ static T fin(Acc a) { return a.s; }
  __device__ static T mul(T a, T b) { return a * b; }
  __device__ static float to_f(T v) { return __double2float_rn(v); }
  __device__ static T zero() { return 0.0; }
  __device__ static T one() { return 1.0; }
};

// Global loads of data other CTAs of the cluster may have written: through L2.
template <int CL, typename T>
__device__ __forceinline__ T ldg_c(const T* p) {
  return CL == 1 ? *p : __ldcg(p);
}

// One row of L21 = A21 L11^{-T} (forward substitution against the panel's factored
// diagonal block L11 and the reciprocals of its pivots): each element takes its updates in
// column order, then the pivot's reciprocal.
template <typename AR>
__device__ __forceinline__ void row_solve(typename AR::T (&v)[NB], const typename AR::T* L11,
                                          const typename AR::T* rdg, int kb) {
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    if (j < kb) {
      typename AR::Acc a = AR::acc(v[j]);
#pragma unroll
      for (int q = 0; q < j; ++q) AR::fms(a, v[q], L11[j * PS + q]);
      v[j] = AR::mul(AR::fin(a), rdg[j]);
    }
  }
}

// Trailing update of panel p: A[i][k] -= sum_j P[i][j] P[k][j] for p + kb <= k <= i < B,
// in TS x TS register tiles over the lower triangle (same operations per element for any
// TS). A and the panel rows below its diagonal block (P, rows p.., kb columns, in shared
// memory) are in AR's format.
template <typename AR, int CL, int TS>
__device__ __forceinline__ void trailing_update(typename AR::T* A, const typename AR::T* P, int B, int p, int kb,
                                                int rows, int gtid, int gthreads) {
  using T = typename AR::T;
  const int mt = (rows - kb + TS - 1) / TS;
  const int ntiles = mt * (mt + 1) / 2;
  for (int idx = gtid; idx < ntiles; idx += gthreads) {
    int ti = (int)((sqrtf(8.f * (float)idx + 1.f) - 1.f) * 0.5f);
    while (ti * (ti + 1) / 2 > idx) --ti;
    while ((ti + 1) * (ti + 2) / 2 <= idx) ++ti;
    const int tk = idx - ti * (ti + 1) / 2;
    const int r0 = kb + TS * ti, c0 = kb + TS * tk;  // panel-relative
    typename AR::Acc acc[TS][TS];
#pragma unroll
    for (int a = 0; a < TS; ++a)
#pragma unroll
      for (int b = 0; b < TS; ++b) {
        const int r = r0 + a, cc = c0 + b;
        acc[a][b] = AR::acc((r < rows && cc <= r) ? ldg_c<CL>(A + (int64_t)(p + r) * B + p + cc) : AR::zero());
      }
    for (int j = 0; j < kb; ++j) {
      T x[TS], y[TS];
#pragma unroll
      for (int a = 0; a < TS; ++a) {
        x[a] = (r0 + a < rows) ? P[(r0 + a) * PS + j] : AR::zero();
        y[a] = (c0 + a < rows) ? P[(c0 + a) * PS + j] : AR::zero();
      }
#pragma unroll
      for (int a = 0; a < TS; ++a)
#pragma unroll
        for (int b = 0; b < TS; ++b) AR::fms(acc[a][b], x[a], y[b]);
    }
#pragma unroll
    for (int a = 0; a < TS; ++a)
#pragma unroll
      for (int b = 0; b < TS; ++b) {
        const int r = r0 + a, cc = c0 + b;
        if (r < rows && cc <= r) A[(int64_t)(p + r) * B + p + cc] = AR::fin(acc[a][b]);
      }
  }
}

// Inverse update of block row p: R_j -= L_jp X_p for the rows below the block (panel-
// relative kb..rows) and the columns c < ncols, in TS x TS register tiles.
template <typename AR, int CL, int TS>
__device__ __forceinline__ void inverse_update(typename AR::T* R, const typename AR::T* P, int B, int p, int kb,
                                               int rows, int cbase, int ncols, int gtid, int gthreads) {
  using T = typename AR::T;
  const int mt = (rows - kb + TS - 1) / TS, nct = (ncols - cbase + TS - 1) / TS;
  for (int idx = gtid; idx < mt * nct; idx += gthreads) {
    const int tr = idx / nct, tcx = idx - tr * nct;
    const int j0 = kb + TS * tr, c0 = cbase + TS * tcx;  // j0 panel-relative row, c0 column
    typename AR::Acc acc[TS][TS];
#pragma unroll
    for (int a = 0; a < TS; ++a)
#pragma unroll
      for (int b = 0; b < TS; ++b)
        acc[a][b] = AR::acc((j0 + a < rows && c0 + b < ncols) ? ldg_c<CL>(R + (int64_t)(p + j0 + a) * B + c0 + b)
                                                               : AR::zero());
    for (int q = 0; q < kb; ++q) {
      T l[TS], xq[TS];
#pragma unroll
      for (int a = 0; a < TS; ++a) l[a] = (j0 + a < rows) ? P[(j0 + a) * PS + q] : AR::zero();
#pragma unroll
      for (int b = 0; b < TS; ++b)
        xq[b] = (c0 + b < ncols) ? ldg_c<CL>(R + (int64_t)(p + q) * B + c0 + b) : AR::zero();
#pragma unroll
      for (int a = 0; a < TS; ++a)
#pragma unroll
        for (int b = 0; b < TS; ++b) AR::fms(acc[a][b], l[a], xq[b]);
    }
#pragma unroll
    for (int a = 0; a < TS; ++a)
#pragma unroll
      for (int b = 0; b < TS; ++b)
        if (j0 + a < rows && c0 + b < ncols) R[(int64_t)(p + j0 + a) * B + c0 + b] = AR::fin(acc[a][b]);
  }
}

// One CTA per line. Sigma (full B x B, lower triangle used) is factored in place in
// global memory with a blocked right-looking Cholesky: the NB-column panel is staged in
// shared memory and factored there (its diagonal block by one warp in FP64, the rows
// below by one thread each), and the trailing lower triangle is updated with 4 x 4
// register tiles (NB multiply-subtracts per element loaded and stored). The inverse
// X = L^{-1} (all of it, or only its 64 x 64 diagonal blocks in the triangular-solve form)
// is built NB rows at a time, fused into the same loop: the contribution of earlier block
// rows is a register-tiled product, and the within-block forward substitution runs per
// column, each thread owning whole columns, so it needs no synchronisation.
// CL = 1: one CTA per line (throughput: many lines in flight). CL > 1: the CTAs of a
// thread-block cluster share one line (latency: few lines). Each CTA then factors every
// diagonal block redundantly in its own shared memory, the updates and the final cast
// are spread over all CL x FT threads, steps are separated by cluster barriers
// (release / acquire), and data written by other CTAs is read through L2 (ld.global.cg).
// MB: CTAs per SM the register allocation is sized for (a one-CTA-per-line launch of 128
// threads fits 4 at <= 128 registers or 5 at <= 96; 256 threads fit 2).
template <typename AR, int PREC, int CL, int FT, int MB = (CL == 1 ? 512 / FT : 1)>
__global__ void __launch_bounds__(FT, MB) factor_kernel(double* __restrict__ sigma_all,
                                                       double* __restrict__ inv_all,
                                                       const double* __restrict__ m_all, int B,
                                                       void* __restrict__ wmat,
                                                       float* __restrict__ y0_all,
                                                       float* __restrict__ inv_s2_all,
                                                       int32_t* __restrict__ status, int64_t n0_arg, int W,
                                                       int incl, const int64_t* __restrict__ n0_dev,
                                                       int every, int q_off,
                                                       const double* __restrict__ n_line) {
  using T = typename AR::T;
  const int t = blockIdx.x / CL;
  if (status[t] != LS_OK) return;  // same for every CTA of the cluster
  if (every > 1 && (q_off + t) % every != 0) return;  // not a snapshot of the cadence
  const int64_t BB = (int64_t)B * B;
  double* A = sigma_all + t * BB;                            // raw sums in, then Sigma and L in AR's format
  T* A2 = reinterpret_cast<T*>(A);
  T* Inv = reinterpret_cast<T*>(inv_all + t * BB);           // the inverse
  const double* m = m_all + (int64_t)t * B;
  const int Bp = pad64(B);
  extern __shared__ double smem[];
  __shared__ double red[FT / 32];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int rank = CL > 1 ? (int)cluster_rank() : 0;
  // cluster-wide warp and thread indices: warps are dealt round-robin over the CTAs and
  // a work list is cut into warp-sized pieces, so that any prefix of it (a shrinking
  // trailing matrix) runs as full warps spread over every CTA of the cluster
  const int gwarp = rank + CL * warp, gwarps = CL * (FT / 32);
  const int gtid = gwarp * 32 + lane, gthreads = CL * FT;

  // ---- covariance from the raw sums (lower triangle, in place) ----------------------
  // The DN-frame covariance S_ij = (S2_ij - n m_i m_j) / (n - 1), n = pixels in this
  // line's window, in FP64, stored in AR's format. The calibration gains cancel from
  // Eq. 1: with x - mu = D (x' - m) and Sigma = D S D, delta = (x' - m)^T S^{-1} (x' - m).
  constexpr bool TRSM = is_trsm(PREC);
  {
    // pixels in the window, or their forgetting weight (n_line: one value per line)
    const int64_t n = (n0_dev ? *n0_dev : n0_arg) + (int64_t)(t + incl) * W;
    const double nn = n_line ? n_line[t] : (double)n, inv_nm1 = 1.0 / (nn - 1.0);
    for (int i = gwarp; i < B; i += gwarps) {
      const double nmi = nn * m[i];
      double* row = A + (int64_t)i * B;
      for (int j = lane; j <= i; j += 32) {
        const double v = inv_nm1 * fma(-nmi, m[j], row[j]);
        A2[(int64_t)i * B + j] = AR::from_d(v);
      }
    }
    // the inverse is built in place of R = I (entries above the diagonal stay zero)
    for (int64_t e = gtid; e < BB; e += gthreads)
      Inv[e] = ((int)(e / B) == (int)(e % B)) ? AR::one() : AR::zero();
    csync<CL>();
  }

  // ---- blocked Cholesky (right-looking, lower triangle in place) -------------------
  // panel: element (r, j) = A[p + r][p + j] at r * PS + j in AR's format (Pf); the kb x kb
  // diagonal block is factored in FP64 (P, the same 8-byte slots) and then converted
  double* P = smem;
  T* Pf = reinterpret_cast<T*>(smem);
  __shared__ T rdg[NB];  // 1 / L[p + j][p + j] of the current panel
  __shared__ int notpd;  // a non-positive pivot in the diagonal block
  if (tid == 0) notpd = 0;
  __syncthreads();
  for (int p = 0; p < B; p += NB) {
    const int kb = min(NB, B - p), rows = B - p;
    // One warp factors the kb x kb diagonal block of the panel (in a cluster every CTA
    // does, with the same values everywhere, so a non-positive pivot exits every CTA
    // alike); the rows below it are then solved one per thread: by the CTA in shared
    // memory, or once across the cluster and gathered by every CTA.
    const int frows = CL == 1 ? rows : kb;
    for (int e = tid; e < frows * kb; e += FT) {
      const int r = e / kb, j = e - r * kb;
      const T v = ldg_c<CL>(A2 + (int64_t)(p + r) * B + p + j);
      if (r < kb) P[r * PS + j] = AR::to_d(v);
      else Pf[r * PS + j] = v;
    }
    __syncthreads();
    {
      // the kb x kb diagonal block: one warp, column by column, warp-level syncs only
      // (pivot, reciprocal, column scaled by it, rank-1 update of the block's remainder)
      if (warp == 0) {
        bool bad = false;
        for (int j = 0; j < kb; ++j) {
          const double piv = P[j * PS + j];
          if (!(piv > 0.0) || !isfinite(piv)) {  // same value in every lane
            if (lane == 0) notpd = 1;
            bad = true;
            break;
          }
          const double l = sqrt(piv);
          const double rl = 1.0 / l;
          for (int r = j + 1 + lane; r < kb; r += 32) P[r * PS + j] *= rl;
          __syncwarp();
          if (lane == 0) {
            P[j * PS + j] = l;
            rdg[j] = AR::from_d(rl);
          }
          const int nc = kb - j - 1;
          for (int e = lane; e < nc * nc; e += 32) {
            const int r = j + 1 + e / nc, k = j + 1 + e % nc;
            if (k <= r) P[r * PS + k] = fma(-P[r * PS + j], P[k * PS + j], P[r * PS + k]);
          }
          __syncwarp();
        }
        if (!bad && !AR::kFP64) {  // the factored block to AR's format, in place (lower triangle)
          for (int e = lane; e < kb * kb; e += 32) {
            const int r = e / kb, j = e - r * kb;
            if (j <= r) Pf[r * PS + j] = AR::from_d(P[r * PS + j]);
          }
        }
      }
      __syncthreads();
      if (notpd) {  // the same in every CTA of the cluster: uniform exit
        if (tid == 0) status[t] = LS_NOT_PD;
        return;
      }
    }
    if (CL == 1) {
      // L21 = A21 L11^{-T} in shared memory, one thread per row: forward substitution in
      // the order of a column-by-column sweep (each element takes its updates in column
      // order, then the pivot's reciprocal)
      for (int r = kb + tid; r < rows; r += FT) {
        T v[NB];
#pragma unroll
        for (int j = 0; j < NB; ++j) v[j] = j < kb ? Pf[r * PS + j] : AR::zero();
        row_solve<AR>(v, Pf, rdg, kb);
#pragma unroll
        for (int j = 0; j < NB; ++j)
          if (j < kb) Pf[r * PS + j] = v[j];
      }
      __syncthreads();
    }
    if (CL > 1) {
      // L21 = A21 L11^{-T}: the same forward substitution as the one-CTA form (bitwise
      // the same factor), rows spread over the cluster
      for (int r = kb + gtid; r < rows; r += gthreads) {
        T v[NB];
        const T* arow = A2 + (int64_t)(p + r) * B + p;
#pragma unroll
        for (int j = 0; j < NB; ++j) v[j] = j < kb ? ldg_c<CL>(arow + j) : AR::zero();
        row_solve<AR>(v, Pf, rdg, kb);
        T* wrow = A2 + (int64_t)(p + r) * B + p;
#pragma unroll
        for (int j = 0; j < NB; ++j)
          if (j < kb) wrow[j] = v[j];
      }
      csync<CL>();
      for (int e = tid; e < (rows - kb) * kb; e += FT) {
        const int r = kb + e / kb, j = e - (r - kb) * kb;
        Pf[r * PS + j] = ldg_c<CL>(A2 + (int64_t)(p + r) * B + p + j);
      }
      __syncthreads();
    }
    for (int e = tid; e < frows * kb; e += FT) {
      const int r = e / kb, j = e - r * kb;
      if (r >= j && rank == 0) A2[(int64_t)(p + r) * B + p + j] = Pf[r * PS + j];
    }
    // trailing update: A[i][k] -= sum_j P[i][j] P[k][j] for p + kb <= k <= i < B. A cluster
    // switches to 2 x 2 tiles once the 4 x 4 tiles of a phase no longer cover all of its
    // threads (late panels), so that every SM sub-partition of the cluster has work.
    const int mrem = rows - kb;
    if (mrem > 0) {
      const int mt4 = (mrem + 3) >> 2;
      if (CL > 1 && mt4 * (mt4 + 1) / 2 < gthreads)
        trailing_update<AR, CL, 2>(A2, Pf, B, p, kb, rows, gtid, gthreads);
      else
        trailing_update<AR, CL, 4>(A2, Pf, B, p, kb, rows, gtid, gthreads);
    }
    // ---- triangular inverse, block row p, fused into the Cholesky step ----------------
    // X = L^{-1} is built right-looking in place of R = I: once panel p is factored, block
    // row p of X is X_p = L_pp^{-1} R_p (forward substitution, one thread per column, in
    // this phase next to the trailing update), and every later block row takes the rank-kb
    // update R_j -= L_jp X_p (next phase, register tiles). R_p has received the
    // updates of every earlier block row, and the operations per element run in the same
    // order as in a separate inverse sweep after the whole factorisation.
    T* R = Inv;
    {
      // triangular-solve form: only the inverses of the 64 x 64 diagonal blocks of L
      const int cbase = TRSM ? p / 64 * 64 : 0;
      const int irows = TRSM ? min(B, cbase + 64) - p : rows;  // panel-relative row limit
      const int imrem = irows - kb;
      const int ncols = p + kb;
      for (int c = cbase + gtid; c < ncols; c += gthreads) {
        T xr[NB];
#pragma unroll
        for (int r = 0; r < NB; ++r) {
          xr[r] = AR::zero();
          if (r < kb) {
            typename AR::Acc a = AR::acc(ldg_c<CL>(R + (int64_t)(p + r) * B + c));
#pragma unroll
            for (int q = 0; q < r; ++q) AR::fms(a, Pf[r * PS + q], xr[q]);
            xr[r] = AR::mul(AR::fin(a), rdg[r]);
            R[(int64_t)(p + r) * B + c] = xr[r];
          }
        }
      }
      csync<CL>();  // the trailing update of A and X_p are complete cluster-wide
      if (imrem > 0) {
        if (CL > 1 && ((imrem + 3) >> 2) * ((ncols - cbase + 3) >> 2) < gthreads)
          inverse_update<AR, CL, 2>(R, Pf, B, p, kb, irows, cbase, ncols, gtid, gthreads);
        else
          inverse_update<AR, CL, 4>(R, Pf, B, p, kb, irows, cbase, ncols, gtid, gthreads);
      }
      csync<CL>();  // panel p done: next panel (and its shared-memory buffer) may start
    }
  }

  if (TRSM) {
    // ---- triangular-solve operand H (BF16 hi / lo or FP32): H_ij = L_ij below the diagonal
    // 64 x 64 blocks, H_ii = L_ii^{-1}; y0 = m (the whitening forms x' - m in FP32); no scale
    const int64_t plane = (int64_t)Bp * Bp;
    void* w = (char*)wmat + (size_t)t * plane * 4;
    // (u, v) = (row n, column k), or (column k, row n) for the transposed FP32 layout, so
    // that the lanes of a warp write consecutive addresses
    constexpr bool TR = PREC == P_FP32T;
    for (int u = gwarp; u < Bp; u += gwarps) {
      for (int v = lane; v < Bp; v += 32) {
        const int n = TR ? v : u, k = TR ? u : v;
        const int64_t idx = h_index<PREC>(n, k, Bp);
        if (n < B && k <= n) {
          const T* src = ((n >> 6) == (k >> 6)) ? Inv : A2;
          WOut<PREC>::store(w, plane, idx, AR::to_f(ldg_c<CL>(src + (int64_t)n * B + k)));
        } else {
          WOut<PREC>::zero(w, plane, idx);
        }
      }
      if (lane == 0) y0_all[(int64_t)t * Bp + u] = (u < B) ? (float)m[u] : 0.0f;
    }
    if (gtid == 0) inv_s2_all[t] = 1.0f;
    if (CL > 1) csync<CL>();  // no CTA leaves while others may still read its shared memory
    return;
  }
  // ---- G = L^{-1} of the DN-frame covariance, power-of-two scale, cast, y0 ----------
  float mxf = 0.f;
  for (int n = gwarp; n < B; n += gwarps)  // X is lower triangular
    for (int k = lane; k <= n; k += 32) mxf = fmaxf(mxf, fabsf(AR::to_f(ldg_c<CL>(Inv + (int64_t)n * B + k))));
  double mx = block_max<FT>((double)mxf, red);
  if (CL > 1) {  // maximum over the cluster: read every CTA's partial from its shared memory
    csync<CL>();
    for (int r = 0; r < CL; ++r) mx = fmax(mx, ld_remote(&red[0], r));
  }
  int ex = 0;
  frexp(mx, &ex);
  const double s = (mx > 0.0) ? ldexp(1.0, -ex) : 1.0;
  const float sf = (float)s;  // a power of two within FP32's range (mx is an FP32 value)
  const int64_t plane = (int64_t)Bp * Bp;
  void* w = (char*)wmat + (size_t)t * plane * 4;  // 4 bytes per element pair in every format
  // one warp per output row n: write the row and accumulate y0[n] from the rounded values
  for (int n = gwarp; n < Bp; n += gwarps) {
    double acc = 0.0;
    for (int k = lane; k < Bp; k += 32) {
      const int64_t idx = (int64_t)n * Bp + k;
      if (n < B && k <= n) {
        const float r =
            WOut<PREC>::store(w, plane, idx, __fmul_rn(AR::to_f(ldg_c<CL>(Inv + (int64_t)n * B + k)), sf));
        acc = fma((double)r, m[k], acc);
      } else {
        WOut<PREC>::zero(w, plane, idx);
      }
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) y0_all[(int64_t)t * Bp + n] = (n < B) ? (float)acc : 0.0f;
  }
  if (gtid == 0) inv_s2_all[t] = (float)(1.0 / (s * s));
  if (CL > 1) csync<CL>();  // no CTA leaves while others may still read its shared memory
}

// ---- launch templates -------------------------------------------------------------------

// How many clusters of CL factor CTAs the device can run at once (queried once per
// device and shared-memory size; 0 if none fits).
template <typename AR, int PREC, int CL, int FT = FT_CLUSTER, int MB = (CL == 1 ? 512 / FT : 1)>
int cluster_capacity(size_t smem) {
  static std::mutex mu;
  static std::map<std::pair<int, size_t>, int> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> g(mu);
  const auto key = std::make_pair(dev, smem);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  int n = 0;
  bool ok = cudaFuncSetAttribute(factor_kernel<AR, PREC, CL, FT, MB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem) == cudaSuccess;
  if (ok && CL > 8)
    ok = cudaFuncSetAttribute(factor_kernel<AR, PREC, CL, FT, MB>, cudaFuncAttributeNonPortableClusterSizeAllowed,
                              1) == cudaSuccess;
  if (ok) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CL);
    cfg.blockDim = dim3(FT);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cudaOccupancyMaxActiveClusters(&n, factor_kernel<AR, PREC, CL, FT, MB>, &cfg) != cudaSuccess) n = 0;
  }
  cudaGetLastError();
  cache[key] = n;
  return n;
}

template <typename AR, int PREC, int CL, int FT = FT_CLUSTER, int MB = (CL == 1 ? 512 / FT : 1)>
cudaError_t launch_t(const FactorArgs& a) {
  const size_t smem = (size_t)smem_slots(a.B) * sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(factor_kernel<AR, PREC, CL, FT, MB>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (CL > 8) {
    e = cudaFuncSetAttribute(factor_kernel<AR, PREC, CL, FT, MB>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)a.L * CL);
  cfg.blockDim = dim3(FT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = a.st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  // a non-portable size: launch only where the device can place such a cluster
  if (CL > 8 && cluster_capacity<AR, PREC, CL, FT, MB>(smem) <= 0) return cudaErrorInvalidConfiguration;
  return cudaLaunchKernelEx(&cfg, factor_kernel<AR, PREC, CL, FT, MB>, a.sigma, a.scratch, a.m, a.B, a.wmat, a.y0,
                            a.inv_s2, a.status, a.n0, a.W, a.incl, a.n0_dev, a.every, a.q_off, a.n_line);
}

// Resident one-CTA-per-line factor CTAs on the whole device (SMs x CTAs per SM), cached.
template <typename AR, int PREC, int FT, int MB>
int wave_slots_t(size_t smem) {
  static std::mutex mu;
  static std::map<std::pair<int, size_t>, int> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> g(mu);
  const auto key = std::make_pair(dev, smem);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  int per_sm = 0, sms = 0;
  if (cudaFuncSetAttribute(factor_kernel<AR, PREC, 1, FT, MB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, factor_kernel<AR, PREC, 1, FT, MB>, FT, smem) !=
          cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    per_sm = 0;
  cudaGetLastError();
  return cache[key] = per_sm * sms;
}

}  // namespace fk

// The three entry points one (arithmetic, working precision) translation unit defines.
#define HSAD_FACTOR_INSTANCE(AR, PREC, SUFFIX)                                                          \
  cudaError_t factor_launch_##SUFFIX(int cl, int ft, const FactorArgs& a) {                            \
    switch (cl) {                                                                                       \
      case 16: {                                                                                        \
        const cudaError_t e = fk::launch_t<AR, PREC, 16>(a);                                            \
        if (e != cudaErrorInvalidConfiguration) return e;                                               \
        return fk::launch_t<AR, PREC, 8>(a);                                                            \
      }                                                                                                 \
      case 8: return fk::launch_t<AR, PREC, 8>(a);                                                      \
      case 4: return fk::launch_t<AR, PREC, 4>(a);                                                      \
      case 2: return fk::launch_t<AR, PREC, 2>(a);                                                      \
      default:                                                                                          \
        if (ft == 96) return fk::launch_t<AR, PREC, 1, 128, 5>(a); /* 128 threads sized for 5 per SM */ \
        if (ft == 128) return fk::launch_t<AR, PREC, 1, 128>(a);                                        \
        return fk::launch_t<AR, PREC, 1, 256>(a);                                                       \
    }                                                                                                   \
  }                                                                                                     \
  int factor_capacity_##SUFFIX(int cl, size_t smem) {                                                   \
    switch (cl) {                                                                                       \
      case 16: return fk::cluster_capacity<AR, PREC, 16>(smem);                                         \
      case 8: return fk::cluster_capacity<AR, PREC, 8>(smem);                                           \
      case 4: return fk::cluster_capacity<AR, PREC, 4>(smem);                                           \
      case 2: return fk::cluster_capacity<AR, PREC, 2>(smem);                                           \
      default: return 0;                                                                                \
    }                                                                                                   \
  }                                                                                                     \
  int factor_wave_slots_##SUFFIX(int ft, size_t smem) {                                                 \
    if (ft == 96) return fk::wave_slots_t<AR, PREC, 128, 5>(smem);                                      \
    if (ft == 128) return fk::wave_slots_t<AR, PREC, 128, 4>(smem);                                     \
    return fk::wave_slots_t<AR, PREC, 256, 2>(smem);                                                    \
  }

}  // namespace hsad
