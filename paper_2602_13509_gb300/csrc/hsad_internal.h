// Internal kernel launchers of the hsad library (not part of the C ABI).
//
// Data layout in HBM (all row-major):
//   input lines     [L][W][B]   uint16 DN or float32 (BIP, bands contiguous)
//   shift c         [B]         int32 (u16 input: integer DN) or float (f32 input)
//   per-line sums   [L][B]      double   s1_t = sum_p (x_p - c)
//   per-line SYRK   [L][B][B]   double   s2_t = sum_p (x_p - c)(x_p - c)^T, then Sigma_t in place
//   factor          [L][Bp][Bp] whitening operand G_t = s_t L_t^{-1} (S_t = L_t L_t^T, the DN-frame
//                               covariance), row n = output coordinate
//                               (FP32: float; FP16/BF16: hi plane then lo plane, 16-bit)
//   y0              [L][Bp]     float   s_t G_t (mu_t - c)
//   inv_s2          [L]         float   1 / s_t^2 (s_t: power-of-two scale of G_t)
//   line status     [L]         int32   LS_*
//   result ring     [R][W]      float scores, uint8 mask, [R] int32 status
// Bp = B rounded up to a multiple of 64 (zero padded).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace hsad {

enum LineStatus : int32_t { LS_OK = 0, LS_NOT_READY = 1, LS_NOT_PD = 2, LS_INVALID_DATA = 3 };
enum InType : int32_t { IN_U16 = 0, IN_F32 = 1 };
enum Prec : int32_t { P_FP32 = 0, P_BF16 = 1, P_FP16 = 2,
                      // factor output for the triangular-solve whitening: L's off-diagonal
                      // 64 x 64 blocks and the inverses of its diagonal blocks, as BF16 hi / lo
                      // planes (tensor cores) or FP32 (SIMT)
                      P_BF16T = 3, P_FP32T = 4,
                      // the same operand as BF16 hi / mid / lo planes: the FP32 value split
                      // into three BF16 terms for an FP32-accurate tensor-core solve
                      P_FP32X = 5 };
__host__ __device__ constexpr bool is_trsm(int prec) {
  return prec == P_BF16T || prec == P_FP32T || prec == P_FP32X;
}
// BF16 planes of the tensor-core triangular-solve operand (0: not that form).
__host__ __device__ constexpr int trsm_planes(int prec) { return prec == P_BF16T ? 2 : prec == P_FP32X ? 3 : 0; }
// Bytes per element of one factor slot's whitening operand (Bp x Bp elements).
__host__ __device__ constexpr int wmat_elem_bytes(int prec) { return prec == P_FP32X ? 6 : 4; }

__host__ __device__ inline int pad64(int b) { return (b + 63) / 64 * 64; }

// Counts every kernel this library launches (per context, host side).
struct LaunchCounter {
  int64_t n = 0;
};

// K1a: integer (u16) or float (f32) centring shift from one line: c_b = rint(mean_b).
cudaError_t launch_shift_init(const void* line, int W, int B, int in_type, int32_t* c_int,
                              float* c_flt, cudaStream_t st, LaunchCounter* lc);

// K1b: per-line column sums s1[t][b] = sum_p (x[t][p][b] - c_b), FP64 (exact for u16).
cudaError_t launch_colsum(const void* x, int64_t n_lines, int W, int B, int in_type,
                          const int32_t* c_int, const float* c_flt, double* s1, cudaStream_t st,
                          LaunchCounter* lc);

// K2 (SIMT): s2 = sum (x - c)(x - c)^T over the pixels of each group of
// lines_per_group lines; out[g] is a full B x B FP64 matrix (row stride B).
// accumulate != 0 adds into out with atomics (split over pixel slices).
cudaError_t launch_syrk_simt(const void* x, int64_t n_groups, int64_t pix_per_group, int B,
                             int in_type, const int32_t* c_int, const float* c_flt, double* out,
                             int64_t out_stride, int accumulate, cudaStream_t st,
                             LaunchCounter* lc);

// K3a: running per-band sums -> per-line mean offset m_t = S1_t / N_t (FP64), line
// readiness, and the updated state S1.
// Per-line gain correction (Sec. 3.2): gain[4 t .. 4 t + 3] = {g_t, 1 / g_t, 1 / g_t^2,
// 1 - g_t} in FP64 (formed on the host, so that no kernel divides). Line t's values are
// u = DN / g_t; with the fixed shift c its sums about c are (s1_t + W e_t) / g_t and
// (s2_t + s1_t e_t^T + e_t s1_t^T + W e_t e_t^T) / g_t^2 with e_t = c (1 - g_t), formed in
// FP64 from the exact integer sums (c_int: the shift, needed with gain).
constexpr int kGainStride = 4;
cudaError_t launch_prefix_mean(const double* s1_line, double* m_out, double* state_s1, int64_t n0,
                               int W, int L, int B, int inclusive, int64_t min_pixels,
                               int32_t* status, cudaStream_t st, LaunchCounter* lc,
                               const int64_t* n0_dev = nullptr, const double* gain = nullptr,
                               const int32_t* c_int = nullptr, double lam = 1.0, const double* n_line = nullptr);
// Exponential forgetting (an extension: lam in (0, 1), every line's sums decay by lam per
// later line): n_line[t] = the forgetting weight of the window after t + incl more lines,
// lam^k n_prev + W (1 - lam^k) / (1 - lam) with k = t + incl; the prefix kernels take lam
// (running sums R_t = lam R_{t-1} + line t) and n_line in place of the pixel count.
cudaError_t launch_forget_n(double n_prev, double lam, int W, int L, int incl, double* n_line, cudaStream_t st,
                            LaunchCounter* lc);
double forget_weight(double n_prev, double lam, int W, int64_t k);
// Writes the per-batch values a replayed CUDA graph reads: desc[0] = pixels in the
// statistics before the batch, desc[1] = ring slot of the batch's second line.
cudaError_t launch_set_batch_desc(int64_t* desc, int64_t n_stats, int64_t slot1, cudaStream_t st,
                                  LaunchCounter* lc);

// K3b: running raw sums S2_t (lower triangle) written in place over the per-line SYRK
// results, and the updated state S2. The factor kernel turns them into Sigma_t.
// gain, s1_line, c_int, W (optional): the per-line gain correction of launch_prefix_mean,
// applied to each line's s2 before it is summed.
cudaError_t launch_prefix_cov(double* buf, double* state_s2, int L, int B, int inclusive, cudaStream_t st,
                              LaunchCounter* lc, const double* gain = nullptr, const double* s1_line = nullptr,
                              const int32_t* c_int = nullptr, int W = 0, double lam = 1.0);

// K2 (tcgen05, uint16 input): exact s2 = sum (x - c)(x - c)^T per group into the lower
// triangle of out[g] (row stride B); groups above 4096 pixels need accumulate != 0
// (atomic adds into a zeroed out). err is set if a bounded wait expires.
// max_pix: pixels one accumulation may sum exactly (4096 for 12-bit DN, fewer for wider
// values); larger groups are cut into slices of max_pix that need accumulate != 0.
cudaError_t launch_syrk_tc(const uint16_t* x, int64_t n_groups, int64_t pix_per_group, int B,
                           const int32_t* c_int, double* out, int64_t out_stride, int accumulate, int32_t* err,
                           cudaStream_t st, LaunchCounter* lc, int64_t max_pix = 4096);
// K2 for streamed statistics in two launches: the integer split of every group's DN into the
// BF16 operand blocks (scratch of syrk_split_bytes), then one tile contraction per block pair
// and group from those blocks (groups of at most 4096 pixels, out as for launch_syrk_tc
// without accumulation).
size_t syrk_split_bytes(int64_t groups, int64_t pix, int B);
// s1 (nullable): also the groups' band sums s1[g][b] = sum_p (x - c) (exact integers in FP64),
// as launch_colsum writes them.
cudaError_t launch_syrk_split(const uint16_t* x, int64_t n_groups, int64_t pix, int B, const int32_t* c_int,
                              uint8_t* hr, double* s1, cudaStream_t st, LaunchCounter* lc);
cudaError_t launch_syrk_pre(const uint8_t* hr, int64_t n_groups, int64_t pix, int B, double* out,
                            int64_t out_stride, int32_t* err, cudaStream_t st, LaunchCounter* lc);
// Front end (Sec. 3.2): out[p][b] = sum_{i < bin} raw[p][first + bin * b + i].
cudaError_t launch_frontend(const uint16_t* raw, int64_t n_px, int raw_bands, int first, int bin, int bands,
                            uint16_t* out, cudaStream_t st, LaunchCounter* lc);

// K3c (cube): raw sums S2 (lower triangle) copied from the state into sigma and
// m = S1 / N; status[0] becomes LS_OK or LS_NOT_READY (fewer than min_pixels pixels).
cudaError_t launch_finalize_cov(const double* state_s1, const double* state_s2, int64_t n, int B, double* sigma,
                                double* m, int64_t min_pixels, int32_t* status, cudaStream_t st, LaunchCounter* lc);

// Arguments of one factor launch (see launch_factor).
struct FactorArgs {
  double* sigma;
  double* scratch;
  const double* m;
  int L, B;
  void* wmat;
  float* y0;
  float* inv_s2;
  int32_t* status;
  int64_t n0;
  int W, incl;
  cudaStream_t st;
  const int64_t* n0_dev;
  int every, q_off;
  const double* n_line;
};
// launch_factor's prec argument: the working precision of the whitening operand (a Prec),
// or'ed with kFactorF64 for FP64 arithmetic in the factor's O(B^3) work (float-float
// otherwise).
constexpr int kFactorF64 = 0x100;
__host__ __device__ constexpr int out_prec(int fprec) { return fprec & 0xff; }

// K4+K5: from each ready line's raw sums (lower triangle of sigma[t]) and mean offset
// m[t]: the DN-frame covariance S_t = (S2_t - n_t m_t m_t^T) / (n_t - 1) with
// n_t = n0 + (t + incl) W (the calibration gains cancel from Eq. 1), Cholesky with FP64
// pivots and 16 x 16 diagonal blocks and float-float (or, with kFactorF64, FP64) panel
// solves and updates, and the triangular inverse, in place (sigma and scratch then hold
// 8-byte float-float pairs or doubles), then the whitening operand in the working
// precision, y0 and 1/s_t^2. scratch: [L][B][B] 8-byte slots.
// The factor kernel with a given launch shape: cl CTAs per line (1, 2, 4, 8, 16) and, for
// cl = 1, ft threads per CTA (128 or 256).
cudaError_t launch_factor_shape(int cl, int ft, double* sigma, double* scratch, const double* m,
                                int L, int B, int prec, void* wmat, float* y0, float* inv_s2, int32_t* status,
                                int64_t n0, int W, int incl, cudaStream_t st, LaunchCounter* lc,
                                const int64_t* n0_dev, int every = 1, int q_off = 0,
                                const double* n_line = nullptr);
// Measure the launch shapes for batch-size buckets 1, 2, 4, ..., max_lines and keep the
// fastest per bucket for launch_factor (current device). report: rows of (bucket, cl, ft,
// ms), up to cap rows. Returns the number of buckets or a negative value on failure.
int factor_autotune(int B, int prec, int max_lines, float* report, int cap);
// Lines one launch of the one-CTA-per-line factor holds resident on the current device
// (SMs x CTAs per SM for its default shape), 0 if unknown.
int factor_wave_lines(int B, int prec);
// Query and cache, once per device, B and precision, how many clusters of each size the
// factor kernel can run at once (host calls that must not land on a line's latency path).
void factor_prepare(int B, int prec);
// n0_dev: if set, n0 is read there at run time (replayed CUDA graphs).
// every > 1: only lines t with (q_off + t) % every == 0 are factored (a cadence); the others
// are left untouched.
cudaError_t launch_factor(double* sigma, double* scratch, const double* m,
                          int L, int B, int prec, void* wmat, float* y0, float* inv_s2,
                          int32_t* status, int64_t n0, int W, int incl, cudaStream_t st, LaunchCounter* lc,
                          const int64_t* n0_dev = nullptr, int every = 1, int q_off = 0,
                          const double* n_line = nullptr);

// K4 + K5 on the tensor cores (k_factor_tc.cu): the same factor output as launch_factor for
// the triangular-solve forms with the float-float factor, the trailing updates as exact
// digit-split BF16 contractions. Needs B >= 192 (the slices live in the inverse scratch);
// err is set if a bounded wait expires.
// Its launches, in order: step 0 forms the covariance; steps 2k + 1 and 2k + 2 are the panel
// and the trailing update of 64-column panel k (the last panel has no update).
bool factor_tc_supported(int B, int prec);
int factor_tc_steps(int B);
int factor_tc_step_kind(int step);  // 0 covariance, 1 diagonal block, 2 rows below, 3 update
// The prefix of a batch's integer covariance sums (as launch_prefix_cov without gains or
// forgetting) with each line's covariance formed in place for the tensor-core factor (its
// step 0, which is then skipped): m, n0, W, incl, n0_dev as for the factor; ffm scratch of
// tcf_form_scratch_bytes(L, B).
size_t tcf_form_scratch_bytes(int L, int B);
cudaError_t launch_tcf_prefix_form(double* buf, double* state_s2, int L, int B, int inclusive, const double* m,
                                   int64_t n0, int W, int incl, const int64_t* n0_dev, float2* ffm,
                                   cudaStream_t st, LaunchCounter* lc);
cudaError_t launch_factor_tc_step(int step, double* sigma, double* scratch, const double* m, int L, int B, int prec,
                                  void* wmat, float* y0, float* inv_s2, int32_t* status, int64_t n0, int W,
                                  int incl, cudaStream_t st, LaunchCounter* lc, const int64_t* n0_dev, int every,
                                  int q_off, const double* n_line, int32_t* err);

// K6 (SIMT): delta_p = inv_s2 * || G (x_p - c) - y0 ||^2 for every pixel of every line,
// threshold, and scatter into the result ring. factor_stride = 0 makes every line
// use factor 0 (cube mode).
struct ScoreOut {
  float* scores;
  uint8_t* mask;
  int32_t* ring_status;
  int64_t slot0;     // ring slot of line 0
  int64_t ring;      // ring capacity in lines
  float tau;
  int write_mask;    // 1: mask = delta > tau here; 0: left to the cube normaliser
  int factor_base = 0;  // factor slot of line 0 (slots advance with factor_stride)
  const int64_t* slot0_dev = nullptr;  // if set, slot0 is read here (replayed CUDA graphs)
  // factorisation cadence: only slots j with (q0 + j) % every == 0 hold a factor; a line
  // whose own slot j does not uses the last such slot at or below j (slot 0 if none)
  int every = 1;
  int q0 = 0;
  // per-line gain correction (triangular-solve forms only): if set, line t of the launch is
  // centred with m_line[t * Bp ..] instead of its factor slot's mean, and its score is
  // multiplied by line_scale[t] = 1 / g_t^2 (see launch_gain_mean)
  const float* m_line = nullptr;
  const float* line_scale = nullptr;
};
#ifdef __CUDACC__
__device__ __forceinline__ int64_t slot0_of(const ScoreOut& o) { return o.slot0_dev ? *o.slot0_dev : o.slot0; }
// Factor slot of line t of a whitening launch.
__device__ __forceinline__ int factor_slot(const ScoreOut& o, int factor_stride, int t) {
  if (!factor_stride) return o.factor_base;
  const int j = o.factor_base + t;
  if (o.every <= 1) return j;
  const int s = j - (o.q0 + j) % o.every;
  return s > 0 ? s : 0;
}
#endif
// Per-line gain correction of a whitening launch of L lines (gain + kGainStride t: line t of
// the launch): the score of a pixel x of line t is ||L^{-1}(x/g - c - m_f)||^2
// = ||L^{-1}(x' - m'_t)||^2 / g^2 with x' = x - c and m'_t = g (m_f + c) - c, m_f the mean
// offset of line t's factor slot f (y0 of the triangular-solve form). Writes m'_t to
// m_out[t * Bp ..] (zero past B) and 1 / g^2 to scale_out[t].
cudaError_t launch_gain_mean(const double* gain, int L, int B, const float* y0, const int32_t* c_int,
                             int factor_stride, ScoreOut out, float* m_out, float* scale_out, cudaStream_t st,
                             LaunchCounter* lc);
cudaError_t launch_whiten_score_simt(const void* x, int L, int W, int B, int in_type,
                                     const int32_t* c_int, const float* c_flt, int prec,
                                     const void* wmat, const float* y0, const float* inv_s2,
                                     const int32_t* status, int factor_stride, ScoreOut out,
                                     cudaStream_t st, LaunchCounter* lc);

// K6 (tcgen05, FP16 / BF16 forms): same contract as the SIMT form; gmap is the
// CUtensorMap over the 16-bit G planes; err is set if a bounded wait expires.
cudaError_t launch_whiten_tc(const void* x, int L, int W, int B, int in_type, const int32_t* c_int,
                             const float* c_flt, int prec, const void* gmap, const float* y0,
                             const float* inv_s2, const int32_t* status, int factor_stride, ScoreOut out,
                             int32_t* err, cudaStream_t st, LaunchCounter* lc);

// K6, triangular-solve form (P_BF16T or P_FP32X factors, uint16 input): delta =
// ||L^{-1} (x' - m)||^2 by blocked forward substitution on the tensor cores; hmap is the
// CUtensorMap over the BF16 planes of H (trsm_planes(prec) of them) with 64 x 64 boxes, m the
// FP32 means (the y0 rows of the factor).
cudaError_t launch_whiten_trsm(const uint16_t* x, int L, int W, int B, int prec, const int32_t* c_int,
                               const void* hmap, const float* m, const float* inv_s2, const int32_t* status,
                               int factor_stride, ScoreOut out, int32_t* err, cudaStream_t st, LaunchCounter* lc);
// K6, triangular-solve form on the SIMT cores (P_FP32T factors): the same blocked forward
// substitution in FP32 with H in FP32 (stored transposed, see h_index), 128 pixels per
// item of a persistent grid; yscratch: whiten_trsm_simt_scratch_bytes(B) of device memory
// (one slot per resident CTA) for the whitened blocks of the items in flight.
cudaError_t launch_whiten_trsm_simt(const void* x, int L, int W, int B, int in_type, const int32_t* c_int,
                                    const float* c_flt, const float* H, const float* m, const float* inv_s2,
                                    const int32_t* status, int factor_stride, ScoreOut out, float* yscratch,
                                    cudaStream_t st, LaunchCounter* lc);
size_t whiten_trsm_simt_scratch_bytes(int B);
// Ring depth the triangular-solve whitening runs with for B bands and an operand of
// `planes` BF16 planes; 0 if it does not fit.
int whiten_trsm_stages(int B, int planes);
// Working form of a context. The triangular solve halves the factor work but its
// whitening is a chain of dependent block steps: it pays where a factorisation per line
// dominates (streamed statistics), not in CUBE mode (one factorisation per cube, the
// whitening dominates), which keeps the explicit inverse.
// BF16: P_BF16T for uint16 input, else P_BF16.
// FP32: P_FP32X (triangular solve on the tensor cores with three-term BF16 operands) for
// uint16 input where the tensor-core factor runs (tc_factor), else P_FP32T (triangular
// solve on the SIMT cores), else P_FP32.
// force_inverse (the HSAD_FORCE_INVERSE configuration flag) keeps the explicit inverse
// everywhere (comparisons).
int bf16_form(int B, int in_type, bool cube, bool force_inverse);
int fp32_form(int B, int in_type, bool cube, bool force_inverse, bool tc_factor);

// K7: cube maximum of delta over n_lines ring lines, then optional normalisation and
// the REL / ABS mask.
cudaError_t launch_cube_normalize(ScoreOut out, int64_t n_lines, int W, int rel, int normalize,
                                  unsigned int* dmax_bits, cudaStream_t st, LaunchCounter* lc);

// Transmit encoding (Sec. 3.4): max_bits (zeroed by the caller) receives the bits of the
// largest finite positive score of s[0, n); then codes = binary16(sqrt(s / max)).
cudaError_t launch_tx_max(const float* s, int64_t n, unsigned int* max_bits, cudaStream_t st, LaunchCounter* lc);
cudaError_t launch_tx_encode(const float* s, int64_t n, uint16_t* codes, const unsigned int* max_bits,
                             cudaStream_t st, LaunchCounter* lc);

// f32 input validation: sets *bad = 1 if any value is NaN or Inf.
cudaError_t launch_check_finite(const float* x, int64_t n, int32_t* bad, cudaStream_t st,
                                LaunchCounter* lc);

}  // namespace hsad
