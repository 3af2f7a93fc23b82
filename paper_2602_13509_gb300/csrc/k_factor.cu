// K4 + K5: Cholesky factorisation and triangular inverse of each line's covariance, and
// the whitening operand in the working precision.
//
// Eq. 1 (Sec. 3.3) needs Sigma^{-1}. In the DN frame used by the statistics kernels the
// calibrated deviation is x - mu = D (x' - m), with x' = DN - c, m = mu_DN - c and D the
// per-band calibration gains, and Sigma = D S D with S the DN-frame covariance, so
//     delta = (x' - m)^T S^{-1} (x' - m) = || L^{-1} (x' - m) ||^2,   S = L L^T:
// the gains cancel and the factor works on S alone. Arithmetic: the covariance is formed
// in FP64, and so are the 16 x 16 diagonal blocks with their pivots; the panel solves,
// the O(B^3) register-tiled updates (Cholesky trailing update, inverse block rows) and the
// inverse's forward substitutions run in float-float (pairs of FP32 values, about 48
// significant bits), as FP64 issues at 1/64 of the FP32 rate here. With G = L^{-1} the
// score is delta = || G x' - G m ||^2.
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
#include <stdlib.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <utility>
#include <vector>

#include "hsad_internal.h"

namespace hsad {

namespace {
constexpr int FT_CLUSTER = 256;  // threads per factorisation CTA in a cluster

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
struct WOut<P_BF16T>;
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
}  // namespace

constexpr int NB = 16;      // Cholesky panel width = inverse block height
constexpr int PS = NB + 1;  // padded panel row stride (doubles): rows fall in different banks

__host__ __device__ inline int factor_smem_doubles(int B) { return B * PS; }

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

// The factorisation runs in float-float arithmetic: a value is an unevaluated pair hi + lo
// of FP32 numbers (about 48 significant bits; FP32's exponent range), stored as a float2
// in the 8 bytes of a double. FP64 issues at 1/64 of the FP32 rate on this part, while
// one float-float multiply-subtract costs 12 FP32 operations. The covariance, the 16 x 16
// diagonal blocks and their pivots stay in FP64.
__device__ __forceinline__ double ff_to_d(float2 v) { return (double)v.x + (double)v.y; }
__device__ __forceinline__ float2 d_to_ff(double d) {
  const float h = __double2float_rn(d);
  return make_float2(h, __double2float_rn(d - (double)h));  // d - h is exact in FP64
}
// Global loads of data other CTAs of the cluster may have written: through L2.
template <int CL>
__device__ __forceinline__ float2 ldg_c2(const float2* p) {
  return CL == 1 ? *p : __ldcg(p);
}
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
// The FP32 value nearest to hi + lo.
__device__ __forceinline__ float ff_f(float2 v) { return __fadd_rn(v.x, v.y); }
// The pair renormalised (two-sum: c may exceed s after cancellation).
__device__ __forceinline__ float2 ff_norm(float s, float c) {
  const float h = __fadd_rn(s, c);
  const float z = __fsub_rn(h, s);
  return make_float2(h, __fadd_rn(__fsub_rn(s, __fsub_rn(h, z)), __fsub_rn(c, z)));
}

// One row of L21 = A21 L11^{-T} (forward substitution against the panel's factored
// diagonal block L11 and the reciprocals of its pivots), float-float: each element takes
// its updates in column order, then the pivot's reciprocal.
__device__ __forceinline__ void row_solve(float2 (&v)[NB], const float2* L11, const float2* rdg, int kb) {
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    if (j < kb) {
      float s = v[j].x, c = v[j].y;
#pragma unroll
      for (int q = 0; q < j; ++q) ff_fms(s, c, v[q], L11[j * PS + q]);
      v[j] = ff_mul(ff_norm(s, c), rdg[j]);
    }
  }
}

// Trailing update of panel p: A[i][k] -= sum_j P[i][j] P[k][j] for p + kb <= k <= i < B,
// in TS x TS register tiles over the lower triangle (same operations per element for any
// TS). A and the panel rows below its diagonal block (P, rows p.., kb columns, in shared
// memory) are float-float.
template <int CL, int TS>
__device__ __forceinline__ void trailing_update(float2* A, const float2* P, int B, int p, int kb, int rows, int gtid,
                                                int gthreads) {
  const int mt = (rows - kb + TS - 1) / TS;
  const int ntiles = mt * (mt + 1) / 2;
  for (int idx = gtid; idx < ntiles; idx += gthreads) {
    int ti = (int)((sqrtf(8.f * (float)idx + 1.f) - 1.f) * 0.5f);
    while (ti * (ti + 1) / 2 > idx) --ti;
    while ((ti + 1) * (ti + 2) / 2 <= idx) ++ti;
    const int tk = idx - ti * (ti + 1) / 2;
    const int r0 = kb + TS * ti, c0 = kb + TS * tk;  // panel-relative
    float s[TS][TS], c[TS][TS];
#pragma unroll
    for (int a = 0; a < TS; ++a)
#pragma unroll
      for (int b = 0; b < TS; ++b) {
        const int r = r0 + a, cc = c0 + b;
        const float2 v =
            (r < rows && cc <= r) ? ldg_c2<CL>(A + (int64_t)(p + r) * B + p + cc) : make_float2(0.f, 0.f);
        s[a][b] = v.x;
        c[a][b] = v.y;
      }
    for (int j = 0; j < kb; ++j) {
      float2 x[TS], y[TS];
#pragma unroll
      for (int a = 0; a < TS; ++a) {
        x[a] = (r0 + a < rows) ? P[(r0 + a) * PS + j] : make_float2(0.f, 0.f);
        y[a] = (c0 + a < rows) ? P[(c0 + a) * PS + j] : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int a = 0; a < TS; ++a)
#pragma unroll
        for (int b = 0; b < TS; ++b) ff_fms(s[a][b], c[a][b], x[a], y[b]);
    }
#pragma unroll
    for (int a = 0; a < TS; ++a)
#pragma unroll
      for (int b = 0; b < TS; ++b) {
        const int r = r0 + a, cc = c0 + b;
        if (r < rows && cc <= r) A[(int64_t)(p + r) * B + p + cc] = ff_norm(s[a][b], c[a][b]);
      }
  }
}

// Inverse update of block row p: R_j -= L_jp X_p for the rows below the block (panel-
// relative kb..rows) and the columns c < ncols, in TS x TS register tiles, float-float.
template <int CL, int TS>
__device__ __forceinline__ void inverse_update(float2* R, const float2* P, int B, int p, int kb, int rows, int cbase,
                                               int ncols, int gtid, int gthreads) {
  const int mt = (rows - kb + TS - 1) / TS, nct = (ncols - cbase + TS - 1) / TS;
  for (int idx = gtid; idx < mt * nct; idx += gthreads) {
    const int tr = idx / nct, tcx = idx - tr * nct;
    const int j0 = kb + TS * tr, c0 = cbase + TS * tcx;  // j0 panel-relative row, c0 column
    float s[TS][TS], c[TS][TS];
#pragma unroll
    for (int a = 0; a < TS; ++a)
#pragma unroll
      for (int b = 0; b < TS; ++b) {
        const float2 v = (j0 + a < rows && c0 + b < ncols) ? ldg_c2<CL>(R + (int64_t)(p + j0 + a) * B + c0 + b)
                                                           : make_float2(0.f, 0.f);
        s[a][b] = v.x;
        c[a][b] = v.y;
      }
    for (int q = 0; q < kb; ++q) {
      float2 l[TS], xq[TS];
#pragma unroll
      for (int a = 0; a < TS; ++a) l[a] = (j0 + a < rows) ? P[(j0 + a) * PS + q] : make_float2(0.f, 0.f);
#pragma unroll
      for (int b = 0; b < TS; ++b)
        xq[b] = (c0 + b < ncols) ? ldg_c2<CL>(R + (int64_t)(p + q) * B + c0 + b) : make_float2(0.f, 0.f);
#pragma unroll
      for (int a = 0; a < TS; ++a)
#pragma unroll
        for (int b = 0; b < TS; ++b) ff_fms(s[a][b], c[a][b], l[a], xq[b]);
    }
#pragma unroll
    for (int a = 0; a < TS; ++a)
#pragma unroll
      for (int b = 0; b < TS; ++b)
        if (j0 + a < rows && c0 + b < ncols) R[(int64_t)(p + j0 + a) * B + c0 + b] = ff_norm(s[a][b], c[a][b]);
  }
}

// One CTA per line. Sigma (full B x B, lower triangle used) is factored in place in
// global memory with a blocked right-looking Cholesky: the NB-column panel is staged in
// shared memory and factored there (its diagonal block by one warp, the rows below by
// one thread each), and the trailing lower triangle is updated with 4 x 4 register tiles
// (NB float-float multiply-subtracts per element loaded and stored). The inverse
// X = L^{-1} (all of it, or only its
// 64 x 64 diagonal blocks in the triangular-solve form) is built NB rows at a time, fused
// into the same loop: the contribution of earlier block rows is a register-tiled product,
// and the within-block forward substitution runs per column, each thread owning whole
// columns, so it needs no synchronisation.
// CL = 1: one CTA per line (throughput: many lines in flight). CL > 1: the CTAs of a
// thread-block cluster share one line (latency: few lines). Each CTA then factors every
// diagonal block redundantly in its own shared memory, the updates and the final cast
// are spread over all CL x FT threads, steps are separated by cluster barriers
// (release / acquire), and data written by other CTAs is read through L2 (ld.global.cg).
// MB: CTAs per SM the register allocation is sized for (a one-CTA-per-line launch of 128
// threads fits 4 at <= 128 registers or 5 at <= 96; 256 threads fit 2).
template <int PREC, int CL, int FT, int MB = (CL == 1 ? 512 / FT : 1)>
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
  const int t = blockIdx.x / CL;
  if (status[t] != LS_OK) return;  // same for every CTA of the cluster
  if (every > 1 && (q_off + t) % every != 0) return;  // not a snapshot of the cadence
  const int64_t BB = (int64_t)B * B;
  double* A = sigma_all + t * BB;        // raw sums in, then Sigma and L as float-float
  float2* A2 = reinterpret_cast<float2*>(A);
  float2* Inv = reinterpret_cast<float2*>(inv_all + t * BB);  // the inverse, float-float
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
  // line's window, in FP64, stored float-float. The calibration gains cancel from Eq. 1:
  // with x - mu = D (x' - m) and Sigma = D S D, delta = (x' - m)^T S^{-1} (x' - m).
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
        A2[(int64_t)i * B + j] = d_to_ff(v);
      }
    }
    // the inverse is built in place of R = I (entries above the diagonal stay zero)
    for (int64_t e = gtid; e < BB; e += gthreads)
      Inv[e] = make_float2(((int)(e / B) == (int)(e % B)) ? 1.f : 0.f, 0.f);
    csync<CL>();
  }

  // ---- blocked Cholesky (right-looking, lower triangle in place) -------------------
  // panel: element (r, j) = A[p + r][p + j] at r * PS + j, float-float (Pf); the kb x kb
  // diagonal block is factored in FP64 (P, the same 8-byte slots) and then converted
  double* P = smem;
  float2* Pf = reinterpret_cast<float2*>(smem);
  __shared__ float2 rdg[NB];  // 1 / L[p + j][p + j] of the current panel
  __shared__ int notpd;       // a non-positive pivot in the diagonal block
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
      const float2 v = ldg_c2<CL>(A2 + (int64_t)(p + r) * B + p + j);
      if (r < kb) P[r * PS + j] = ff_to_d(v);
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
            rdg[j] = d_to_ff(rl);
          }
          const int nc = kb - j - 1;
          for (int e = lane; e < nc * nc; e += 32) {
            const int r = j + 1 + e / nc, k = j + 1 + e % nc;
            if (k <= r) P[r * PS + k] = fma(-P[r * PS + j], P[k * PS + j], P[r * PS + k]);
          }
          __syncwarp();
        }
        if (!bad) {  // the factored block to float-float, in place (lower triangle)
          for (int e = lane; e < kb * kb; e += 32) {
            const int r = e / kb, j = e - r * kb;
            if (j <= r) Pf[r * PS + j] = d_to_ff(P[r * PS + j]);
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
        float2 v[NB];
#pragma unroll
        for (int j = 0; j < NB; ++j) v[j] = j < kb ? Pf[r * PS + j] : make_float2(0.f, 0.f);
        row_solve(v, Pf, rdg, kb);
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
        float2 v[NB];
        const float2* arow = A2 + (int64_t)(p + r) * B + p;
#pragma unroll
        for (int j = 0; j < NB; ++j) v[j] = j < kb ? ldg_c2<CL>(arow + j) : make_float2(0.f, 0.f);
        row_solve(v, Pf, rdg, kb);
        float2* wrow = A2 + (int64_t)(p + r) * B + p;
#pragma unroll
        for (int j = 0; j < NB; ++j)
          if (j < kb) wrow[j] = v[j];
      }
      csync<CL>();
      for (int e = tid; e < (rows - kb) * kb; e += FT) {
        const int r = kb + e / kb, j = e - (r - kb) * kb;
        Pf[r * PS + j] = ldg_c2<CL>(A2 + (int64_t)(p + r) * B + p + j);
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
        trailing_update<CL, 2>(A2, Pf, B, p, kb, rows, gtid, gthreads);
      else
        trailing_update<CL, 4>(A2, Pf, B, p, kb, rows, gtid, gthreads);
    }
    // ---- triangular inverse, block row p, fused into the Cholesky step ----------------
    // X = L^{-1} is built right-looking in place of R = I: once panel p is factored, block
    // row p of X is X_p = L_pp^{-1} R_p (forward substitution, one thread per column, in
    // this phase next to the trailing update), and every later block row takes the rank-kb
    // update R_j -= L_jp X_p (next phase, register tiles). R_p has received the
    // updates of every earlier block row, and the operations per element run in the same
    // order as in a separate inverse sweep after the whole factorisation.
    float2* R = Inv;
    {
      // triangular-solve form: only the inverses of the 64 x 64 diagonal blocks of L
      const int cbase = TRSM ? p / 64 * 64 : 0;
      const int irows = TRSM ? min(B, cbase + 64) - p : rows;  // panel-relative row limit
      const int imrem = irows - kb;
      const int ncols = p + kb;
      for (int c = cbase + gtid; c < ncols; c += gthreads) {
        float2 xr[NB];
#pragma unroll
        for (int r = 0; r < NB; ++r) {
          xr[r] = make_float2(0.f, 0.f);
          if (r < kb) {
            const float2 v = ldg_c2<CL>(R + (int64_t)(p + r) * B + c);
            float sv = v.x, cv = v.y;
#pragma unroll
            for (int q = 0; q < r; ++q) ff_fms(sv, cv, Pf[r * PS + q], xr[q]);
            xr[r] = ff_mul(ff_norm(sv, cv), rdg[r]);
            R[(int64_t)(p + r) * B + c] = xr[r];
          }
        }
      }
      csync<CL>();  // the trailing update of A and X_p are complete cluster-wide
      if (imrem > 0) {
        if (CL > 1 && ((imrem + 3) >> 2) * ((ncols - cbase + 3) >> 2) < gthreads)
          inverse_update<CL, 2>(R, Pf, B, p, kb, irows, cbase, ncols, gtid, gthreads);
        else
          inverse_update<CL, 4>(R, Pf, B, p, kb, irows, cbase, ncols, gtid, gthreads);
      }
      csync<CL>();  // panel p done: next panel (and its shared-memory buffer) may start
    }
  }

  if (TRSM) {
    // ---- triangular-solve operand H (BF16 hi / lo or FP32): H_ij = L_ij below the diagonal
    // 64 x 64 blocks, H_ii = L_ii^{-1}; y0 = m (the whitening forms x' - m in FP32); no scale
    const int64_t plane = (int64_t)Bp * Bp;
    void* w = (char*)wmat + (size_t)t * plane * 4;
    for (int n = gwarp; n < Bp; n += gwarps) {
      for (int k = lane; k < Bp; k += 32) {
        const int64_t idx = (int64_t)n * Bp + k;
        if (n < B && k <= n) {
          const float2* src = ((n >> 6) == (k >> 6)) ? Inv : A2;
          WOut<PREC>::store(w, plane, idx, ff_f(ldg_c2<CL>(src + (int64_t)n * B + k)));
        } else {
          WOut<PREC>::zero(w, plane, idx);
        }
      }
      if (lane == 0) y0_all[(int64_t)t * Bp + n] = (n < B) ? (float)m[n] : 0.0f;
    }
    if (gtid == 0) inv_s2_all[t] = 1.0f;
    if (CL > 1) csync<CL>();  // no CTA leaves while others may still read its shared memory
    return;
  }
  // ---- G = L^{-1} of the DN-frame covariance, power-of-two scale, cast, y0 ----------
  float mxf = 0.f;
  for (int n = gwarp; n < B; n += gwarps)  // X is lower triangular
    for (int k = lane; k <= n; k += 32) mxf = fmaxf(mxf, fabsf(ff_f(ldg_c2<CL>(Inv + (int64_t)n * B + k))));
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
        const float r = WOut<PREC>::store(w, plane, idx, __fmul_rn(ff_f(ldg_c2<CL>(Inv + (int64_t)n * B + k)), sf));
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

namespace {

// How many clusters of CL factor CTAs the device can run at once (queried once per
// device, working precision, cluster size and shared-memory size; 0 if none fits).
template <int PREC, int CL, int FT = FT_CLUSTER, int MB = (CL == 1 ? 512 / FT : 1)>
int factor_cluster_capacity(size_t smem) {
  static std::mutex mu;
  static std::map<std::pair<int, size_t>, int> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> g(mu);
  const auto key = std::make_pair(dev, smem);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  int n = 0;
  bool ok = cudaFuncSetAttribute(factor_kernel<PREC, CL, FT, MB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem) == cudaSuccess;
  if (ok && CL > 8)
    ok = cudaFuncSetAttribute(factor_kernel<PREC, CL, FT, MB>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
         cudaSuccess;
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
    if (cudaOccupancyMaxActiveClusters(&n, factor_kernel<PREC, CL, FT, MB>, &cfg) != cudaSuccess) n = 0;
  }
  cudaGetLastError();
  cache[key] = n;
  return n;
}

template <int PREC, int CL, int FT = FT_CLUSTER, int MB = (CL == 1 ? 512 / FT : 1)>
cudaError_t launch_factor_t(double* sigma, double* scratch, const double* m, int L, int B,
                            void* wmat, float* y0, float* inv_s2, int32_t* status, int64_t n0, int W, int incl,
                            cudaStream_t st, const int64_t* n0_dev, int every, int q_off, const double* n_line) {
  const size_t smem = (size_t)factor_smem_doubles(B) * sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(factor_kernel<PREC, CL, FT, MB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  if (CL > 8) {
    e = cudaFuncSetAttribute(factor_kernel<PREC, CL, FT, MB>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)L * CL);
  cfg.blockDim = dim3(FT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = CL;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  // a non-portable size: launch only where the device can place such a cluster
  if (CL > 8 && factor_cluster_capacity<PREC, CL, FT, MB>(smem) <= 0) return cudaErrorInvalidConfiguration;
  return cudaLaunchKernelEx(&cfg, factor_kernel<PREC, CL, FT, MB>, sigma, scratch, m, B, wmat, y0, inv_s2, status,
                            n0, W, incl, n0_dev, every, q_off, n_line);
}

// Threads of a one-CTA-per-line factorisation: 128 threads with registers for 5 CTAs per
// SM (code 96; so that one CTA's barrier-bound panel step overlaps other CTAs' updates),
// 128 threads for 4 CTAs per SM (code 128), or 256 threads, 2 per SM. Measured on 4000
// lines of B = 270: 57.1, 57.6 and 66.6 ms. HSAD_FACTOR_THREADS = 96, 128 or 256 in the
// environment fixes it (tuning).
int factor_single_threads() {
  static const int n = [] {
    const char* v = getenv("HSAD_FACTOR_THREADS");
    const int c = v ? atoi(v) : 0;
    return (c == 96 || c == 128 || c == 256) ? c : 96;
  }();
  return n;
}

template <int PREC>
cudaError_t launch_factor_p(int cl, int ft, double* sigma, double* scratch, const double* m, int L,
                            int B, void* wmat, float* y0, float* inv_s2, int32_t* status, int64_t n0, int W,
                            int incl, cudaStream_t st, const int64_t* n0_dev, int every, int q_off, const double* n_line) {
  switch (cl) {
    case 16: {
      const cudaError_t e =
          launch_factor_t<PREC, 16>(sigma, scratch, m, L, B, wmat, y0, inv_s2, status, n0, W, incl, st, n0_dev, every, q_off, n_line);
      if (e != cudaErrorInvalidConfiguration) return e;
      return launch_factor_t<PREC, 8>(sigma, scratch, m, L, B, wmat, y0, inv_s2, status, n0, W, incl, st, n0_dev, every, q_off, n_line);
    }
    case 8: return launch_factor_t<PREC, 8>(sigma, scratch, m, L, B, wmat, y0, inv_s2, status, n0, W, incl, st, n0_dev, every, q_off, n_line);
    case 4: return launch_factor_t<PREC, 4>(sigma, scratch, m, L, B, wmat, y0, inv_s2, status, n0, W, incl, st, n0_dev, every, q_off, n_line);
    case 2: return launch_factor_t<PREC, 2>(sigma, scratch, m, L, B, wmat, y0, inv_s2, status, n0, W, incl, st, n0_dev, every, q_off, n_line);
    default:
      if (ft == 96)  // 128 threads sized for 5 CTAs per SM
        return launch_factor_t<PREC, 1, 128, 5>(sigma, scratch, m, L, B, wmat, y0, inv_s2, status, n0, W,
                                                incl, st, n0_dev, every, q_off, n_line);
      if (ft == 128)
        return launch_factor_t<PREC, 1, 128>(sigma, scratch, m, L, B, wmat, y0, inv_s2, status, n0, W, incl,
                                             st, n0_dev, every, q_off, n_line);
      return launch_factor_t<PREC, 1, 256>(sigma, scratch, m, L, B, wmat, y0, inv_s2, status, n0, W, incl, st, n0_dev, every, q_off, n_line);
  }
}

// CTAs per factorisation. A cluster shortens one factorisation (the trailing updates and
// the inverse are shared; each CTA still factors every 16-column panel), so few lines
// (latency) take the largest cluster of which the device can run one per line at once,
// and many lines (throughput) one CTA each.
// HSAD_FACTOR_CLUSTER = 1, 2, 4, 8 or 16 in the environment fixes the size (tuning).
template <int PREC>
int factor_cluster_size(int L, size_t smem) {
  static const int forced = [] {
    const char* v = getenv("HSAD_FACTOR_CLUSTER");
    const int c = v ? atoi(v) : 0;
    return (c == 1 || c == 2 || c == 4 || c == 8 || c == 16) ? c : 0;
  }();
  if (forced) return forced;
  if (L <= factor_cluster_capacity<PREC, 16>(smem)) return 16;
  if (L <= factor_cluster_capacity<PREC, 8>(smem)) return 8;
  if (L <= factor_cluster_capacity<PREC, 4>(smem)) return 4;
  if (L <= factor_cluster_capacity<PREC, 2>(smem)) return 2;
  return 1;
}

}  // namespace

// Measured launch shapes (hsad_autotune_factor): per (device, precision, B) a list of
// (largest batch size of the bucket, cluster size, threads of a one-CTA factorisation).
struct TunedShape {
  int max_lines, cl, ft;
  float ms;
};
std::mutex& tune_mu() {
  static std::mutex m;
  return m;
}
std::map<std::tuple<int, int, int>, std::vector<TunedShape>>& tune_table() {
  static std::map<std::tuple<int, int, int>, std::vector<TunedShape>> t;
  return t;
}
bool tuned_shape(int B, int prec, int L, int* cl, int* ft) {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> g(tune_mu());
  auto it = tune_table().find(std::make_tuple(dev, prec, B));
  if (it == tune_table().end() || it->second.empty()) return false;
  for (const auto& t : it->second)
    if (L <= t.max_lines) {
      *cl = t.cl;
      *ft = t.ft;
      return true;
    }
  return false;  // larger than every measured batch: the occupancy rule
}

namespace {
// Resident one-CTA-per-line factor CTAs on the whole device (SMs x CTAs per SM), cached.
template <int PREC, int FT, int MB>
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
  if (cudaFuncSetAttribute(factor_kernel<PREC, 1, FT, MB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
          cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, factor_kernel<PREC, 1, FT, MB>, FT, smem) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    per_sm = 0;
  cudaGetLastError();
  return cache[key] = per_sm * sms;
}
template <int PREC>
int wave_slots_p(int ft, size_t smem) {
  if (ft == 96) return wave_slots_t<PREC, 128, 5>(smem);
  if (ft == 128) return wave_slots_t<PREC, 128, 4>(smem);
  return wave_slots_t<PREC, 256, 2>(smem);
}
}  // namespace

int factor_wave_lines(int B, int prec) {
  const size_t smem = (size_t)factor_smem_doubles(B) * sizeof(double);
  const int ft = factor_single_threads();
  return prec == P_FP32    ? wave_slots_p<P_FP32>(ft, smem)
         : prec == P_FP16  ? wave_slots_p<P_FP16>(ft, smem)
         : prec == P_BF16T ? wave_slots_p<P_BF16T>(ft, smem)
         : prec == P_FP32T ? wave_slots_p<P_FP32T>(ft, smem)
                           : wave_slots_p<P_BF16>(ft, smem);
}

void factor_prepare(int B, int prec) {
  const size_t smem = (size_t)factor_smem_doubles(B) * sizeof(double);
#define HSAD_FP(P)                             \
  factor_cluster_capacity<P, 16>(smem);        \
  factor_cluster_capacity<P, 8>(smem);         \
  factor_cluster_capacity<P, 4>(smem);         \
  factor_cluster_capacity<P, 2>(smem)
  switch (prec) {
    case P_FP32: HSAD_FP(P_FP32); break;
    case P_FP16: HSAD_FP(P_FP16); break;
    case P_BF16T: HSAD_FP(P_BF16T); break;
    case P_FP32T: HSAD_FP(P_FP32T); break;
    default: HSAD_FP(P_BF16); break;
  }
#undef HSAD_FP
  factor_wave_lines(B, prec);
}

cudaError_t launch_factor(double* sigma, double* scratch, const double* m,
                          int L, int B, int prec, void* wmat, float* y0, float* inv_s2,
                          int32_t* status, int64_t n0, int W, int incl, cudaStream_t st, LaunchCounter* lc,
                          const int64_t* n0_dev, int every, int q_off, const double* n_line) {
  if (L <= 0) return cudaSuccess;
  const size_t smem = (size_t)factor_smem_doubles(B) * sizeof(double);
  int cl = 0, ft = 0;
  if (getenv("HSAD_FACTOR_CLUSTER") || getenv("HSAD_FACTOR_THREADS") || !tuned_shape(B, prec, L, &cl, &ft)) {
    cl = prec == P_FP32    ? factor_cluster_size<P_FP32>(L, smem)
         : prec == P_FP16  ? factor_cluster_size<P_FP16>(L, smem)
         : prec == P_BF16T ? factor_cluster_size<P_BF16T>(L, smem)
         : prec == P_FP32T ? factor_cluster_size<P_FP32T>(L, smem)
                           : factor_cluster_size<P_BF16>(L, smem);
    ft = factor_single_threads();
  }
  return launch_factor_shape(cl, ft, sigma, scratch, m, L, B, prec, wmat, y0, inv_s2, status, n0, W, incl,
                             st, lc, n0_dev, every, q_off, n_line);
}

cudaError_t launch_factor_shape(int cl, int ft, double* sigma, double* scratch, const double* m,
                                int L, int B, int prec, void* wmat, float* y0, float* inv_s2, int32_t* status,
                                int64_t n0, int W, int incl, cudaStream_t st, LaunchCounter* lc,
                                const int64_t* n0_dev, int every, int q_off, const double* n_line) {
  if (L <= 0) return cudaSuccess;
  cudaError_t e;
  switch (prec) {
    case P_FP32: e = launch_factor_p<P_FP32>(cl, ft, sigma, scratch, m, L, B, wmat, y0, inv_s2, status, n0, W, incl, st, n0_dev, every, q_off, n_line); break;
    case P_FP16: e = launch_factor_p<P_FP16>(cl, ft, sigma, scratch, m, L, B, wmat, y0, inv_s2, status, n0, W, incl, st, n0_dev, every, q_off, n_line); break;
    case P_BF16T: e = launch_factor_p<P_BF16T>(cl, ft, sigma, scratch, m, L, B, wmat, y0, inv_s2, status, n0, W, incl, st, n0_dev, every, q_off, n_line); break;
    case P_FP32T: e = launch_factor_p<P_FP32T>(cl, ft, sigma, scratch, m, L, B, wmat, y0, inv_s2, status, n0, W, incl, st, n0_dev, every, q_off, n_line); break;
    default: e = launch_factor_p<P_BF16>(cl, ft, sigma, scratch, m, L, B, wmat, y0, inv_s2, status, n0, W, incl, st, n0_dev, every, q_off, n_line); break;
  }
  if (lc) lc->n += 1;
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

namespace {
__global__ void tune_identity_kernel(double* sigma, int L, int B, double c) {
  const int64_t BB = (int64_t)B * B;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)L * BB;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = e % BB;
    sigma[e] = (k / B == k % B) ? c : 0.0;
  }
}
}  // namespace

// Time every launch shape of the factor kernel on L synthetic SPD problems (raw sums
// c * I, zero mean: every shape does the same arithmetic on any data) for each batch-size
// bucket and keep the fastest. Returns the number of buckets, or a negative status.
int factor_autotune(int B, int prec, int max_lines, float* report, int cap) {
  int dev = 0;
  cudaGetDevice(&dev);
  {
    std::lock_guard<std::mutex> g(tune_mu());
    auto it = tune_table().find(std::make_tuple(dev, prec, B));
    if (it != tune_table().end() && !it->second.empty() && it->second.back().max_lines >= max_lines) {
      const auto& v = it->second;
      for (int i = 0; i < (int)v.size() && i < cap && report; ++i) {
        report[4 * i] = (float)v[i].max_lines;
        report[4 * i + 1] = (float)v[i].cl;
        report[4 * i + 2] = (float)v[i].ft;
        report[4 * i + 3] = v[i].ms;
      }
      return (int)v.size();
    }
  }
  std::vector<int> buckets;
  for (int b = 1; b < max_lines; b *= 2) buckets.push_back(b);
  buckets.push_back(max_lines);
  const int Lt = max_lines, Bp = pad64(B);
  const int64_t BB = (int64_t)B * B;
  double *sigma = nullptr, *inv = nullptr, *m = nullptr;
  float *y0 = nullptr, *inv_s2 = nullptr;
  int32_t* status = nullptr;
  void* wmat = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  bool ok = cudaMalloc(&sigma, (size_t)Lt * BB * 8) == cudaSuccess && cudaMalloc(&inv, (size_t)Lt * BB * 8) == cudaSuccess &&
            cudaMalloc(&m, (size_t)Lt * B * 8) == cudaSuccess &&
            cudaMalloc(&y0, (size_t)Lt * Bp * 4) == cudaSuccess && cudaMalloc(&inv_s2, (size_t)Lt * 4) == cudaSuccess &&
            cudaMalloc(&status, (size_t)Lt * 4) == cudaSuccess &&
            cudaMalloc(&wmat, (size_t)Lt * Bp * Bp * 4) == cudaSuccess &&
            cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess;
  std::vector<TunedShape> result;
  if (ok) {
    ok = cudaMemsetAsync(m, 0, (size_t)Lt * B * 8, st) == cudaSuccess && cudaStreamSynchronize(st) == cudaSuccess;
  }
  const size_t smem = (size_t)factor_smem_doubles(B) * sizeof(double);
  for (size_t bi = 0; ok && bi < buckets.size(); ++bi) {
    const int L = buckets[bi];
    std::vector<std::pair<int, int>> cands = {{1, 96}, {1, 128}, {1, 256}};
    const int cls[4] = {2, 4, 8, 16};
    for (int c : cls) {
      int capc = 0;
      switch (prec) {
        case P_FP32: capc = c == 2 ? factor_cluster_capacity<P_FP32, 2>(smem) : c == 4 ? factor_cluster_capacity<P_FP32, 4>(smem) : c == 8 ? factor_cluster_capacity<P_FP32, 8>(smem) : factor_cluster_capacity<P_FP32, 16>(smem); break;
        case P_FP16: capc = c == 2 ? factor_cluster_capacity<P_FP16, 2>(smem) : c == 4 ? factor_cluster_capacity<P_FP16, 4>(smem) : c == 8 ? factor_cluster_capacity<P_FP16, 8>(smem) : factor_cluster_capacity<P_FP16, 16>(smem); break;
        case P_BF16T: capc = c == 2 ? factor_cluster_capacity<P_BF16T, 2>(smem) : c == 4 ? factor_cluster_capacity<P_BF16T, 4>(smem) : c == 8 ? factor_cluster_capacity<P_BF16T, 8>(smem) : factor_cluster_capacity<P_BF16T, 16>(smem); break;
        case P_FP32T: capc = c == 2 ? factor_cluster_capacity<P_FP32T, 2>(smem) : c == 4 ? factor_cluster_capacity<P_FP32T, 4>(smem) : c == 8 ? factor_cluster_capacity<P_FP32T, 8>(smem) : factor_cluster_capacity<P_FP32T, 16>(smem); break;
        default: capc = c == 2 ? factor_cluster_capacity<P_BF16, 2>(smem) : c == 4 ? factor_cluster_capacity<P_BF16, 4>(smem) : c == 8 ? factor_cluster_capacity<P_BF16, 8>(smem) : factor_cluster_capacity<P_BF16, 16>(smem); break;
      }
      if (capc > 0 && L <= 2 * capc) cands.push_back({c, FT_CLUSTER});  // larger batches only queue
    }
    TunedShape best{L, 1, 128, 1e30f};
    for (const auto& cf : cands) {
      float tot = 0.f;
      for (int rep = 0; ok && rep < 4; ++rep) {  // one untimed run, then three timed
        tune_identity_kernel<<<256, 256, 0, st>>>(sigma, L, B, 1.0e6);
        ok = cudaMemsetAsync(status, 0, (size_t)L * 4, st) == cudaSuccess;
        cudaEventRecord(e0, st);
        if (launch_factor_shape(cf.first, cf.second, sigma, inv, m, L, B, prec, wmat, y0, inv_s2, status,
                                1000, 1, 0, st, nullptr, nullptr) != cudaSuccess)
          ok = false;
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) ok = false;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0) tot += ms;
      }
      if (ok && tot / 3.f < best.ms) best = TunedShape{L, cf.first, cf.second, tot / 3.f};
    }
    if (ok) result.push_back(best);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  cudaFree(sigma);
  cudaFree(inv);
  cudaFree(m);
  cudaFree(y0);
  cudaFree(inv_s2);
  cudaFree(status);
  cudaFree(wmat);
  cudaGetLastError();
  if (!ok) return -1;
  {
    std::lock_guard<std::mutex> g(tune_mu());
    tune_table()[std::make_tuple(dev, prec, B)] = result;
  }
  for (int i = 0; i < (int)result.size() && i < cap && report; ++i) {
    report[4 * i] = (float)result[i].max_lines;
    report[4 * i + 1] = (float)result[i].cl;
    report[4 * i + 2] = (float)result[i].ft;
    report[4 * i + 3] = result[i].ms;
  }
  return (int)result.size();
}

}  // namespace hsad
