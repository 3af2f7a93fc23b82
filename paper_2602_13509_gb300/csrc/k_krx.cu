// Subsampled kernel RX (Sec. 2.2, Table tab:results: the kernel RX of Kwon and Nasrabadi,
// 2005, with a random background subsample, Hidalgo et al., 2021) of one cube in device
// memory: hsad_krx.
//
// With m background pixels s_i (calibrated bands x_b = (v_b - offset_b) gain_b; offsets
// cancel from every distance), the Gaussian kernel k(x, y) = exp(-||x - y||^2 / c) and
// the centred Gram matrix K~ = H K H (H = I - 1 1^T / m), the score of a pixel r is
//     delta(r) = (m - 1) || (K~ + lam I)^{-1} H (k_r - kbar) ||^2,
// kbar = K 1 / m, lam = eps tr(K~) / m, c = the mean squared distance of distinct
// background pairs unless given. Steps:
//   background (FP64, once per call): gather the m samples, pairwise squared distances,
//     c, K = exp(-D / c), kbar, K~ + lam I (krx_center_kernel), its Cholesky factor and
//     X = L^{-1} (the factor kernel in FP64, explicit-inverse form), then
//     G = (K~ + lam I)^{-1} H = X^T X H and ybar = G kbar (krx_inverse_kernel), stored as
//     float-float pairs (G transposed, [j][i], for coalesced rows);
//   per pixel (krx_score_kernel, SIMT): squared distances to the m samples (exact
//     differences times the band's gain, FP32 partial sums of 8 bands gathered in
//     float-float), k = exp(-d / c) as a float-float pair (ff_exp_neg), y = G k - ybar
//     accumulated in float-float, and delta = (m - 1) ||y||^2 (FP32 squares, FP64 sum over
//     the outputs).
// The map k -> y amplifies rounding by up to kappa(K~ + lam I) (about 1e4 at eps = 1e-2):
// a CPU emulation with FP32 distances and FP32 accumulation of G k gave 1.7e-4 relative
// error, with float-float distance sums and accumulation 1.7e-5, and the FP32 rounding
// of k alone left 1e-4 on a float cube with a narrow kernel (exact k: 6e-6); that is why
// these steps carry a second FP32 word.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "../../include/hsad.h"
#include "hsad_internal.h"

using namespace hsad;

namespace {

constexpr int KX_P = 32;        // pixels per CTA
constexpr int KX_T = 256;       // threads per CTA
constexpr int KX_JC = 64;       // background samples per distance chunk
constexpr int KX_BC = 64;       // bands per distance chunk
constexpr int KX_IP = 256;      // outputs per pass of the product with G
constexpr int KX_MAX_M = 512;   // largest background subsample

__host__ __device__ inline int round_up(int v, int q) { return (v + q - 1) / q * q; }

// s + c += p (Knuth's two-sum of s and p, its error added to c)
__device__ __forceinline__ void two_sum_acc(float& s, float& c, float p) {
  const float t = __fadd_rn(s, p);
  const float z = __fsub_rn(t, s);
  c = __fadd_rn(c, __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z)));
  s = t;
}

// Float-float product of a pair and a pair (two-product of the high words with the cross
// terms), renormalised.
__device__ __forceinline__ float2 ffm(float2 a, float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  float e = __fmaf_rn(a.x, b.x, -p);
  e = __fmaf_rn(a.x, b.y, e);
  e = __fmaf_rn(a.y, b.x, e);
  const float h = __fadd_rn(p, e);
  return make_float2(h, __fsub_rn(e, __fsub_rn(h, p)));
}
// a + b in float-float (two-sum of the high words, low words added, renormalised).
__device__ __forceinline__ float2 ffa(float2 a, float2 b) {
  const float s = __fadd_rn(a.x, b.x);
  const float z = __fsub_rn(s, a.x);
  const float e = __fadd_rn(__fadd_rn(__fsub_rn(a.x, __fsub_rn(s, z)), __fsub_rn(b.x, z)), __fadd_rn(a.y, b.y));
  const float h = __fadd_rn(s, e);
  return make_float2(h, __fsub_rn(e, __fsub_rn(h, s)));
}

// Constants of the float-float exponential, formed once per CTA in FP64: 1/i! for
// i = 0 .. 12 and ln 2 in three parts (Cody and Waite's reduction: the first part has
// 11 significant bits, so n ln2_1 is exact for the integers n used here).
struct ExpConsts {
  float2 inv_fact[13];
  float ln2[3];
};
__device__ void exp_consts_init(ExpConsts* ec) {
  if (threadIdx.x == 0) {
    double f = 1.0;
    for (int i = 0; i <= 12; ++i) {
      if (i > 0) f *= i;
      const double v = 1.0 / f;
      const float h = __double2float_rn(v);
      ec->inv_fact[i] = make_float2(h, __double2float_rn(v - (double)h));
    }
    const double ln2 = 0.69314718055994530942;
    const double l1 = rint(ln2 * 2048.0) / 2048.0;
    const float l2 = __double2float_rn(ln2 - l1);
    ec->ln2[0] = (float)l1;
    ec->ln2[1] = l2;
    ec->ln2[2] = __double2float_rn(ln2 - l1 - (double)l2);
  }
}
// exp(-t) for a float-float t >= 0, as a float-float pair (about 45 correct bits): with
// n = rint(t / ln 2) and r = t - n ln 2 (|r| <= ln(2) / 2, formed exactly enough from the
// three parts of ln 2), exp(-t) = 2^-n exp(-r), exp(-r) by its Taylor polynomial of degree
// 12 (truncation below 2^-46) in Horner form. Zero once 2^-n leaves FP32's normal range.
__device__ __forceinline__ float2 ff_exp_neg(float2 t, const ExpConsts& ec) {
  const float n = rintf(__fmul_rn(t.x, 1.4426950408889634f));
  if (n > 120.f) return make_float2(0.f, 0.f);
  const float r1 = __fmaf_rn(-n, ec.ln2[0], t.x);      // exact: n ln2_1 has at most 18 bits
  const float p = __fmul_rn(n, ec.ln2[1]);
  const float pe = __fmaf_rn(n, ec.ln2[1], -p);
  float2 r = ffa(make_float2(r1, 0.f), make_float2(-p, -pe));
  r = ffa(r, make_float2(__fsub_rn(t.y, __fmul_rn(n, ec.ln2[2])), 0.f));
  const float2 mr = make_float2(-r.x, -r.y);
  float2 acc = ec.inv_fact[12];
#pragma unroll
  for (int i = 11; i >= 0; --i) acc = ffa(ffm(acc, mr), ec.inv_fact[i]);
  const float sc = ldexpf(1.f, -(int)n);
  return make_float2(__fmul_rn(acc.x, sc), __fmul_rn(acc.y, sc));
}

__device__ __forceinline__ float2 fk_norm(float s, float c) {
  const float h = __fadd_rn(s, c);
  return make_float2(h, __fsub_rn(c, __fsub_rn(h, s)));
}

template <typename In>
__device__ __forceinline__ float as_float(In v) {
  return (float)v;  // uint16 DN are exact in FP32
}

// ---- background ------------------------------------------------------------------------

template <typename In>
__global__ void krx_gather_kernel(const In* __restrict__ x, const int64_t* __restrict__ idx, int m, int B,
                                  In* __restrict__ S) {
  const int i = blockIdx.x;
  if (i >= m) return;
  const In* src = x + idx[i] * (int64_t)B;
  for (int b = threadIdx.x; b < B; b += blockDim.x) S[(int64_t)i * B + b] = src[b];
}

// D_ij = sum_b (g_b (s_ib - s_jb))^2 in FP64.
template <typename In>
__global__ void krx_gram_kernel(const In* __restrict__ S, int m, int B, const double* __restrict__ g,
                                double* __restrict__ D) {
  const int i = blockIdx.x, j = blockIdx.y * blockDim.x + threadIdx.x;
  if (i >= m || j >= m) return;
  const In* si = S + (int64_t)i * B;
  const In* sj = S + (int64_t)j * B;
  double acc = 0.0;
  for (int b = 0; b < B; ++b) {
    const double t = g[b] * ((double)si[b] - (double)sj[b]);
    acc = fma(t, t, acc);
  }
  D[(int64_t)i * m + j] = acc;
}

// One CTA: the kernel width c (the mean of D over i < j unless c0 > 0), K = exp(-D / c),
// kbar, kall = mean(kbar), lam = eps tr(K~) / m, and A = K~ + lam I (the lower triangle
// of A as the "raw sums" of the factor kernel: with a zero mean and a pixel count of 2
// the factor kernel factors A itself). scal = {c, lam, kall, tr}.
__global__ void krx_center_kernel(const double* __restrict__ D, int m, double c0, double eps,
                                  double* __restrict__ K, double* __restrict__ kbar, double* __restrict__ A,
                                  double* __restrict__ scal) {
  __shared__ double red[32];
  const int tid = threadIdx.x, nt = blockDim.x;
  auto block_sum = [&](double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((tid & 31) == 0) red[tid >> 5] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < nt / 32; ++w) t += red[w];
    __syncthreads();
    return t;
  };
  double c = c0;
  if (!(c > 0.0)) {
    double s = 0.0;
    for (int64_t e = tid; e < (int64_t)m * m; e += nt) {
      const int i = (int)(e / m), j = (int)(e % m);
      if (i < j) s += D[e];
    }
    c = block_sum(s) / (0.5 * (double)m * (m - 1));
  }
  const double rc = 1.0 / c;
  for (int64_t e = tid; e < (int64_t)m * m; e += nt) K[e] = exp(-D[e] * rc);
  __syncthreads();
  for (int i = tid; i < m; i += nt) {
    double s = 0.0;
    for (int j = 0; j < m; ++j) s += K[(int64_t)i * m + j];
    kbar[i] = s / m;
  }
  __syncthreads();
  double ks = 0.0;
  for (int i = tid; i < m; i += nt) ks += kbar[i];
  const double kall = block_sum(ks) / m;
  double ts = 0.0;
  for (int i = tid; i < m; i += nt) ts += K[(int64_t)i * m + i] - 2.0 * kbar[i] + kall;
  const double tr = block_sum(ts);
  const double lam = eps * tr / m;
  for (int64_t e = tid; e < (int64_t)m * m; e += nt) {
    const int i = (int)(e / m), j = (int)(e % m);
    A[e] = (j <= i) ? K[e] - kbar[i] - kbar[j] + kall + (i == j ? lam : 0.0) : 0.0;
  }
  if (tid == 0) {
    scal[0] = c;
    scal[1] = lam;
    scal[2] = kall;
    scal[3] = tr;
  }
}

// G = X^T X H with X = L^{-1} (lower triangular, FP64): M_ij = sum_{k >= max(i, j)} X_ki X_kj,
// G_ij = M_ij - (1/m) sum_k M_ik. One CTA per row i of G.
__global__ void krx_inverse_kernel(const double* __restrict__ X, int m, double* __restrict__ G) {
  __shared__ double red[32];
  const int i = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
  double rs = 0.0;
  for (int j = tid; j < m; j += nt) {
    double acc = 0.0;
    for (int k = max(i, j); k < m; ++k) acc = fma(X[(int64_t)k * m + i], X[(int64_t)k * m + j], acc);
    G[(int64_t)i * m + j] = acc;
    rs += acc;
  }
  for (int o = 16; o > 0; o >>= 1) rs += __shfl_xor_sync(0xffffffffu, rs, o);
  if ((tid & 31) == 0) red[tid >> 5] = rs;
  __syncthreads();
  double tot = 0.0;
  for (int w = 0; w < nt / 32; ++w) tot += red[w];
  const double mean = tot / m;
  __syncthreads();
  for (int j = tid; j < m; j += nt) G[(int64_t)i * m + j] -= mean;
}

// Float-float operands of the per-pixel step: GT[j][i] = G_ij (hi plane, then lo plane;
// zero past m, rows j < mj, columns i < mi), ybar_i = sum_j G_ij kbar_j (FP64, then
// hi / lo), and the per-band gains as FP32.
__global__ void krx_operands_kernel(const double* __restrict__ G, const double* __restrict__ kbar, int m, int mj,
                                    int mi, float* __restrict__ GT, float* __restrict__ ybar) {
  const int j = blockIdx.x;  // row of GT
  for (int i = threadIdx.x; i < mi; i += blockDim.x) {
    const double v = (j < m && i < m) ? G[(int64_t)i * m + j] : 0.0;
    const float hi = __double2float_rn(v);
    GT[(int64_t)j * mi + i] = hi;
    GT[(int64_t)mj * mi + (int64_t)j * mi + i] = __double2float_rn(v - (double)hi);
  }
  if (j == 0) {
    for (int i = threadIdx.x; i < mi; i += blockDim.x) {
      double acc = 0.0;
      if (i < m)
        for (int k = 0; k < m; ++k) acc = fma(G[(int64_t)i * m + k], kbar[k], acc);
      const float hi = __double2float_rn(acc);
      ybar[i] = hi;
      ybar[mi + i] = __double2float_rn(acc - (double)hi);
    }
  }
}

// ---- per pixel ---------------------------------------------------------------------------

// One CTA scores KX_P pixels. Phase A: squared distances to every background sample in
// KX_P x KX_JC tiles (each thread 4 pixels x 2 samples), bands staged KX_BC at a time,
// then k = expf(-d / c) into shared memory kS[j][p]. Phase B: y = G k - ybar for each
// pixel, each thread 4 pixels x 8 outputs per pass of KX_IP outputs, float-float
// accumulation over j; ||y||^2 per pixel summed over the threads in FP64.
template <typename In>
__global__ void __launch_bounds__(KX_T, 2) krx_score_kernel(const In* __restrict__ x, int64_t n_px, int B,
                                                         const In* __restrict__ S, int m, int mj, int mi,
                                                         const float* __restrict__ gw,
                                                         const double* __restrict__ scal,
                                                         const float* __restrict__ GT, const float* __restrict__ ybar,
                                                         float* __restrict__ scores, uint8_t* __restrict__ mask,
                                                         float tau, int write_mask) {
  extern __shared__ __align__(16) float sm[];
  float* kS = sm;                              // [mj][KX_P] high words of the kernel values
  float* kL = kS + (size_t)mj * KX_P;          // [mj][KX_P] low words
  float* Xs = kL + (size_t)mj * KX_P;          // [KX_BC][KX_P]
  float* Ss = Xs + KX_BC * KX_P;               // [KX_BC][KX_JC]
  float* gs = Ss + KX_BC * KX_JC;              // [round_up(B, 4)]
  double* red = (double*)(gs + round_up(B, 4)); // [KX_T / 8][KX_P]
  const int tid = threadIdx.x;
  const int64_t p0 = (int64_t)blockIdx.x * KX_P;
  const int npx = (int)min((int64_t)KX_P, n_px - p0);
  __shared__ ExpConsts ec;
  exp_consts_init(&ec);
  const double rcd = 1.0 / scal[0];
  const float2 rc = make_float2(__double2float_rn(rcd), __double2float_rn(rcd - (double)__double2float_rn(rcd)));
  for (int b = tid; b < B; b += KX_T) gs[b] = gw[b];

  // ---- phase A: kernel values -------------------------------------------------------
  {
    const int tp = tid & 7, tj = tid >> 3;  // pixels 4 tp .. 4 tp + 3, samples 2 tj, 2 tj + 1
    for (int j0 = 0; j0 < mj; j0 += KX_JC) {
      float s[4][2], c[4][2], a[4][2];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 2; ++v) s[u][v] = c[u][v] = a[u][v] = 0.f;
      for (int b0 = 0; b0 < B; b0 += KX_BC) {
        const int nb = min(KX_BC, B - b0);
        __syncthreads();  // previous chunk's readers are done (and gs is written)
        for (int e = tid; e < KX_BC * KX_P; e += KX_T) {
          const int p = e / KX_BC, bb = e % KX_BC;  // consecutive threads: consecutive bands
          Xs[bb * KX_P + p] = (p < npx && bb < nb) ? as_float(x[(p0 + p) * B + b0 + bb]) : 0.f;
        }
        for (int e = tid; e < KX_BC * KX_JC; e += KX_T) {
          const int j = e / KX_BC, bb = e % KX_BC;
          Ss[bb * KX_JC + j] = (j0 + j < m && bb < nb) ? as_float(S[(int64_t)(j0 + j) * B + b0 + bb]) : 0.f;
        }
        __syncthreads();
        for (int bb = 0; bb < nb; ++bb) {
          const float4 xv = *(const float4*)&Xs[bb * KX_P + 4 * tp];
          const float2 sv = *(const float2*)&Ss[bb * KX_JC + 2 * tj];
          const float g = gs[b0 + bb];
          const float xa[4] = {xv.x, xv.y, xv.z, xv.w}, sa[2] = {sv.x, sv.y};
#pragma unroll
          for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 2; ++v) {
              const float t = __fmul_rn(__fsub_rn(xa[u], sa[v]), g);
              a[u][v] = __fmaf_rn(t, t, a[u][v]);
            }
          if ((bb & 7) == 7) {  // 8 bands summed in FP32: gather into the float-float total
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
              for (int v = 0; v < 2; ++v) {
                two_sum_acc(s[u][v], c[u][v], a[u][v]);
                a[u][v] = 0.f;
              }
          }
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 2; ++v) {
          two_sum_acc(s[u][v], c[u][v], a[u][v]);
          const int j = j0 + 2 * tj + v;
          // k = exp(-d / c) with d and 1 / c as float-float pairs
          const float2 kv = (j < m) ? ff_exp_neg(ffm(fk_norm(s[u][v], c[u][v]), rc), ec) : make_float2(0.f, 0.f);
          kS[j * KX_P + 4 * tp + u] = kv.x;
          kL[j * KX_P + 4 * tp + u] = kv.y;
        }
    }
  }
  __syncthreads();

  // ---- phase B: y = G k - ybar, ||y||^2 ------------------------------------------------
  const int tp = tid & 7, ti = tid >> 3;  // pixels 4 tp .. 4 tp + 3, outputs 8 ti .. 8 ti + 7 of a pass
  const float* GTlo = GT + (size_t)mj * mi;
  float nrm[4] = {0.f, 0.f, 0.f, 0.f};
  for (int i0 = 0; i0 < mi; i0 += KX_IP) {
    float s[4][8], c[4][8];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 8; ++v) s[u][v] = c[u][v] = 0.f;
    const float* gh = GT + i0 + 8 * ti;
    const float* gl = GTlo + i0 + 8 * ti;
    float4 h0 = *(const float4*)gh, h1 = *(const float4*)(gh + 4);
    float4 l0 = *(const float4*)gl, l1 = *(const float4*)(gl + 4);
    for (int j = 0; j < m; ++j) {
      const float hv[8] = {h0.x, h0.y, h0.z, h0.w, h1.x, h1.y, h1.z, h1.w};
      const float lv[8] = {l0.x, l0.y, l0.z, l0.w, l1.x, l1.y, l1.z, l1.w};
      if (j + 1 < m) {  // next row of G while this one is used
        const float* nh = gh + (size_t)(j + 1) * mi;
        const float* nl = gl + (size_t)(j + 1) * mi;
        h0 = *(const float4*)nh;
        h1 = *(const float4*)(nh + 4);
        l0 = *(const float4*)nl;
        l1 = *(const float4*)(nl + 4);
      }
      const float4 kv = *(const float4*)&kS[j * KX_P + 4 * tp];
      const float4 kw = *(const float4*)&kL[j * KX_P + 4 * tp];
      const float ka[4] = {kv.x, kv.y, kv.z, kv.w}, kb[4] = {kw.x, kw.y, kw.z, kw.w};
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 8; ++v) {
          // G_ij k_j: product error by FMA (two-product) with the cross terms, sum by two-sum
          const float p = __fmul_rn(hv[v], ka[u]);
          float e = __fmaf_rn(hv[v], ka[u], -p);
          e = __fmaf_rn(lv[v], ka[u], e);
          e = __fmaf_rn(hv[v], kb[u], e);
          two_sum_acc(s[u][v], c[u][v], p);
          c[u][v] = __fadd_rn(c[u][v], e);
        }
    }
    const float* yh = ybar + i0 + 8 * ti;
    const float* yl = ybar + mi + i0 + 8 * ti;
#pragma unroll
    for (int v = 0; v < 8; ++v) {
      const float bh = yh[v], bl = yl[v];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float y = __fadd_rn(__fsub_rn(s[u][v], bh), __fsub_rn(c[u][v], bl));
        nrm[u] = __fmaf_rn(y, y, nrm[u]);
      }
    }
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) red[ti * KX_P + 4 * tp + u] = (double)nrm[u];
  __syncthreads();
  if (tid < KX_P && tid < npx) {
    double tot = 0.0;
    for (int g = 0; g < KX_T / 8; ++g) tot += red[g * KX_P + tid];
    const float dlt = (float)((double)(m - 1) * tot);
    scores[p0 + tid] = dlt;
    if (write_mask) mask[p0 + tid] = dlt > tau ? 1 : 0;
  }
}

size_t score_smem(int B, int mj) {
  return ((size_t)2 * mj * KX_P + KX_BC * KX_P + KX_BC * KX_JC + round_up(B, 4)) * sizeof(float) +
         (size_t)(KX_T / 8) * KX_P * sizeof(double);
}

struct DevBufs {
  std::vector<void*> p;
  cudaStream_t st;
  cudaError_t err = cudaSuccess;
  template <typename T>
  T* get(size_t count) {
    void* q = nullptr;
    if (err == cudaSuccess) err = cudaMallocAsync(&q, std::max<size_t>(count * sizeof(T), 16), st);
    if (err == cudaSuccess) p.push_back(q);
    return (T*)q;
  }
  ~DevBufs() {
    for (void* q : p) cudaFreeAsync(q, st);
  }
};

template <typename In>
cudaError_t launch_krx_score(const In* x, int64_t n_px, int B, const In* S, int m, int mj, int mi, const float* gw,
                             const double* scal, const float* GT, const float* ybar, float* scores, uint8_t* mask,
                             float tau, int write_mask, cudaStream_t st) {
  const size_t smem = score_smem(B, mj);
  cudaError_t e = cudaFuncSetAttribute(krx_score_kernel<In>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t grid = (n_px + KX_P - 1) / KX_P;
  krx_score_kernel<In><<<(unsigned)grid, KX_T, smem, st>>>(x, n_px, B, S, m, mj, mi, gw, scal, GT, ybar, scores,
                                                           mask, tau, write_mask);
  return cudaGetLastError();
}

template <typename In>
cudaError_t krx_run(const In* x, int64_t n_px, int B, const int64_t* idx_host, int m, double c0, double eps,
                    const std::vector<double>& gain, float tau, int rel, int normalize, float* scores,
                    uint8_t* mask, cudaStream_t st, int* status_out) {
  const int mj = round_up(m, KX_JC), mi = round_up(m, KX_IP);
  DevBufs d;
  d.st = st;
  int64_t* idx = d.get<int64_t>(m);
  In* S = d.get<In>((size_t)m * B);
  double* gd = d.get<double>(B);
  float* gw = d.get<float>(B);
  double* D = d.get<double>((size_t)m * m);
  double* K = d.get<double>((size_t)m * m);
  double* kbar = d.get<double>(m);
  double* A = d.get<double>((size_t)m * m);
  double* X = d.get<double>((size_t)m * m);
  double* G = d.get<double>((size_t)m * m);
  double* scal = d.get<double>(4);
  double* mzero = d.get<double>(m);
  double* nline = d.get<double>(1);
  const int mp = pad64(m);
  void* wmat = d.get<char>((size_t)mp * mp * 4);
  float* y0 = d.get<float>(mp);
  float* inv_s2 = d.get<float>(1);
  int32_t* status = d.get<int32_t>(1);
  float* GT = d.get<float>((size_t)2 * mj * mi);
  float* ybar = d.get<float>((size_t)2 * mi);
  unsigned int* dmax = d.get<unsigned int>(1);
  int32_t* h_status = nullptr;
  cudaError_t e = d.err;
  std::vector<float> gf(gain.begin(), gain.end());
  const double two = 2.0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(idx, idx_host, (size_t)m * 8, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(gd, gain.data(), (size_t)B * 8, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(gw, gf.data(), (size_t)B * 4, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(nline, &two, 8, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(mzero, 0, (size_t)m * 8, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, 4, st);
  if (e == cudaSuccess) {
    krx_gather_kernel<In><<<m, 128, 0, st>>>(x, idx, m, B, S);
    krx_gram_kernel<In><<<dim3(m, (m + 127) / 128), 128, 0, st>>>(S, m, B, gd, D);
    krx_center_kernel<<<1, 1024, 0, st>>>(D, m, c0, eps, K, kbar, A, scal);
    e = cudaGetLastError();
  }
  // Cholesky of A and X = L^{-1}: the factor kernel in FP64 arithmetic, explicit-inverse
  // form, raw sums A with a zero mean and a "pixel count" of 2 (so (A - 2 0 0^T) / 1 = A)
  if (e == cudaSuccess)
    e = launch_factor(A, X, mzero, 1, m, P_FP32 | kFactorF64, wmat, y0, inv_s2, status, 0, 0, 0, st, nullptr,
                      nullptr, 1, 0, nline);
  if (e == cudaSuccess) {
    krx_inverse_kernel<<<m, 256, 0, st>>>(X, m, G);
    krx_operands_kernel<<<mj, 256, 0, st>>>(G, kbar, m, mj, mi, GT, ybar);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = launch_krx_score<In>(x, n_px, B, S, m, mj, mi, gw, scal, GT, ybar, scores, mask, tau,
                             (rel || normalize) ? 0 : 1, st);
  if (e == cudaSuccess && (rel || normalize)) {
    ScoreOut o;
    o.scores = scores;
    o.mask = mask;
    o.ring_status = nullptr;
    o.slot0 = 0;
    o.ring = 1;
    o.tau = tau;
    o.write_mask = 1;
    e = launch_cube_normalize(o, 1, (int)n_px, rel, normalize, dmax, st, nullptr);
  }
  if (e == cudaSuccess) e = cudaMallocHost(&h_status, 4);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h_status, status, 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) *status_out = *h_status;
  if (h_status) cudaFreeHost(h_status);
  return e;
}

}  // namespace

extern "C" int hsad_krx(const void* cube, int64_t n_pixels, int32_t bands, int32_t in_dtype, const int64_t* subsample,
                        int32_t m, float kernel_width, float ridge, const float* gain, int32_t threshold_mode,
                        float threshold, int32_t flags, float* scores, uint8_t* mask, void* stream, int32_t device) {
  if (!cube || !subsample || !scores || !mask) return HSAD_E_INVALID;
  if (n_pixels < 2 || n_pixels > 0x7fffffffLL || bands < 1 || bands > 512) return HSAD_E_INVALID;
  if (m < 2 || m > KX_MAX_M || m > n_pixels) return HSAD_E_INVALID;
  if (in_dtype != HSAD_U16 && in_dtype != HSAD_F32) return HSAD_E_INVALID;
  if (!(kernel_width >= 0.f) || kernel_width > 3.0e38f) return HSAD_E_INVALID;
  if (!(ridge > 0.f) || ridge > 1.0e6f) return HSAD_E_INVALID;
  if (threshold_mode != HSAD_ABS && threshold_mode != HSAD_REL) return HSAD_E_INVALID;
  if (!(threshold >= 0.f) || threshold > 3.0e38f) return HSAD_E_INVALID;
  if (flags & ~HSAD_NORMALIZE_SCORES) return HSAD_E_INVALID;
  std::vector<int64_t> idx(subsample, subsample + m), sorted(idx);
  std::sort(sorted.begin(), sorted.end());
  if (sorted.front() < 0 || sorted.back() >= n_pixels) return HSAD_E_INVALID;
  for (int i = 1; i < m; ++i)
    if (sorted[i] == sorted[i - 1]) return HSAD_E_INVALID;
  std::vector<double> g(bands, 1.0);
  if (gain)
    for (int b = 0; b < bands; ++b) {
      g[b] = (double)gain[b];
      if (!(g[b] == g[b]) || g[b] == 0.0 || g[b] > 1e30 || g[b] < -1e30) return HSAD_E_INVALID;
    }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= 0) {
    cudaGetLastError();
    return HSAD_E_CUDA;
  }
  if (device < 0 || device >= ndev) return HSAD_E_INVALID;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != device && cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return HSAD_E_CUDA;
  }
  cudaStream_t st = (cudaStream_t)stream;
  int rc = HSAD_OK;
  // float input: NaN or Inf anywhere makes every distance meaningless
  if (in_dtype == HSAD_F32) {
    int32_t* bad = nullptr;
    int32_t hbad = 0;
    cudaError_t e = cudaMallocAsync(&bad, 4, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(bad, 0, 4, st);
    if (e == cudaSuccess) e = launch_check_finite((const float*)cube, n_pixels * bands, bad, st, nullptr);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hbad, bad, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (bad) cudaFreeAsync(bad, st);
    if (e != cudaSuccess) rc = HSAD_E_CUDA;
    else if (hbad) rc = HSAD_E_INVALID_DATA;
  }
  if (rc == HSAD_OK) {
    const float tau = threshold > 0.f ? threshold
                                      : (threshold_mode == HSAD_ABS ? (float)(bands + 6.0 * sqrt(2.0 * bands)) : 0.f);
    const int rel = threshold_mode == HSAD_REL, norm = (flags & HSAD_NORMALIZE_SCORES) != 0;
    int status = 0;
    const cudaError_t e =
        in_dtype == HSAD_U16
            ? krx_run<uint16_t>((const uint16_t*)cube, n_pixels, bands, idx.data(), m, (double)kernel_width,
                                (double)ridge, g, tau, rel, norm, scores, mask, st, &status)
            : krx_run<float>((const float*)cube, n_pixels, bands, idx.data(), m, (double)kernel_width, (double)ridge,
                             g, tau, rel, norm, scores, mask, st, &status);
    if (e != cudaSuccess) {
      cudaGetLastError();
      rc = HSAD_E_CUDA;
    } else if (status == LS_NOT_PD) {
      rc = HSAD_E_NOT_PD;
    }
  }
  if (prev >= 0 && prev != device) cudaSetDevice(prev);
  return rc;
}
