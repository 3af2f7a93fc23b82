/*
 * hsad.h -- C ABI of the GB300 streaming RX hyperspectral anomaly detector.
 *
 * The detector is the global RX algorithm of Sec. 3.3 ("Detection Algorithm"):
 * per-band mean mu and covariance Sigma of a set of pixel spectra, and for every
 * scored pixel s the squared Mahalanobis distance of Eq. 1,
 *     delta = (s - mu)^T Sigma^{-1} (s - mu),
 * optionally divided by the cube maximum and thresholded into an anomaly mask
 * (Sec. 3.3, last paragraph). Lines of W samples x B bands arrive continuously
 * from a push-broom imager (Sec. 2.1, Sec. 3.2); Sec. 6.1 proposes scoring them
 * line by line, which the EXCLUSIVE and INCLUSIVE statistics modes provide.
 *
 * Conventions shared by every entry point:
 *  - Every call returns an hsad_status (0 = HSAD_OK, negative = error).
 *  - The caller owns every buffer it passes. Nothing is retained after return
 *    except as documented for HSAD_DEVICE input (stream-ordered reads).
 *  - Calls on one context must be serialised by the caller. Different contexts
 *    may be used from different threads.
 *  - A context that hits a CUDA error becomes sticky-failed: every later call
 *    except hsad_destroy / hsad_last_error returns HSAD_E_CUDA.
 *  - Scores are FP32, one per pixel, line-major [n_lines][width]; the mask is one
 *    byte per pixel (1 = anomalous), same layout.
 *  - Input lines are band-interleaved-by-pixel (BIP): [n_lines][width][bands],
 *    bands contiguous, uint16 DN (12-bit sensor values) or float32.
 */
#ifndef HSAD_H
#define HSAD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hsad_ctx hsad_ctx; /* opaque; owned by the library */

typedef enum {
  HSAD_OK = 0,
  HSAD_E_INVALID = -1,      /* bad argument, size or state; nothing was done */
  HSAD_E_NOMEM = -2,        /* device budget or allocation exhausted */
  HSAD_E_NOT_READY = -3,    /* warm-up lines (NaN scores), or not yet computed with timeout 0 */
  HSAD_E_NOT_PD = -4,       /* covariance not positive definite for some requested line (NaN scores) */
  HSAD_E_TIMEOUT = -5,      /* a bounded wait expired */
  HSAD_E_CUDA = -6,         /* CUDA error; the context is now failed */
  HSAD_E_BUSY = -7,         /* no admission slot (serving); retry later */
  HSAD_E_INVALID_DATA = -8  /* non-finite input values in a float32 push */
} hsad_status;

/* input element type */
enum { HSAD_U16 = 0, HSAD_F32 = 1 };
/* working precision of the whitening contraction (the covariance sums are exact for
 * HSAD_U16 input in every mode; the factor's arithmetic follows factor_precision). HSAD_FP32
 * with uint16 input, the float-float factor and B >= 192 on streamed statistics runs the
 * contraction on the tensor cores with every FP32 operand split exactly into three BF16
 * terms (the products kept to FP32 rounding); otherwise FP32 runs on the SIMT cores.
 * HSAD_BF16 and HSAD_FP16 keep two-term operands (about 16 significant bits). */
enum { HSAD_FP32 = 0, HSAD_BF16 = 1, HSAD_FP16 = 2 };
/* arithmetic of the factor (Sec. 3.3 needs Sigma^{-1}): float-float, pairs of FP32 values
 * with about 48 significant bits and FP32's exponent range (default). For streamed
 * statistics at B >= 192 its O(B^3) products run on the tensor cores as exact six-digit
 * BF16 splits (a relative error of about 2^-45 of the row scales per product) and its
 * 64 x 64 diagonal blocks in float-float on the FP32 pipe; elsewhere the CUDA-core factor
 * takes FP64 pivots and 16 x 16 diagonal blocks and float-float for the rest. FP64 (53
 * bits) runs the CUDA-core factor in FP64 throughout, at a fraction of the throughput on
 * this GPU, whose FP64 rate is 1/64 of its FP32 rate. */
enum { HSAD_FACTOR_FF = 0, HSAD_FACTOR_FP64 = 1 };
/* whitening form of a context (Eq. 1, Sec. 3.3), see hsad_whitening_form:
 * HSAD_FORM_INVERSE            y = G x' - y0 with G = s L^{-1}, the full triangular
 *                              inverse: CUBE mode (one factorisation per cube, where the
 *                              whitening dominates), FP16, BF16 with float input;
 * HSAD_FORM_TRIANGULAR_SOLVE   streamed statistics (EXCLUSIVE, INCLUSIVE: a factorisation
 *                              per line): L y = x' - m solved blockwise from L and the
 *                              inverses of its 64 x 64 diagonal blocks only, half the
 *                              factor work; on the tensor cores for uint16 input (BF16:
 *                              two-term operands; FP32 with the float-float factor and
 *                              B >= 192: three-term operands, FP32-accurate products), else
 *                              on the SIMT cores (FP32). */
enum { HSAD_FORM_INVERSE = 0, HSAD_FORM_TRIANGULAR_SOLVE = 1 };
/* statistics window (which pixels form mu and Sigma for a scored line t) */
enum {
  HSAD_EXCLUSIVE = 0, /* lines [r, t): line t scored against earlier lines only */
  HSAD_INCLUSIVE = 1, /* lines [r, t] */
  HSAD_CUBE = 2       /* the whole cube of cube_lines lines containing t (global RX, Sec. 3.3) */
};
/* threshold form */
enum { HSAD_ABS = 0 /* delta > threshold */, HSAD_REL = 1 /* delta / cube max > threshold (CUBE only) */ };
/* memory space of a caller buffer */
enum { HSAD_HOST = 0, HSAD_DEVICE = 1 };
/* flags */
enum {
  HSAD_CREATE_WAIT = 1,      /* hsad_create blocks (bounded) until the device budget admits the context */
  HSAD_NORMALIZE_SCORES = 2, /* CUBE mode: report delta / cube max instead of delta (Sec. 3.3) */
  HSAD_CUDA_GRAPHS = 4,      /* EXCLUSIVE mode, host pushes: the statistics, factor and scoring
                                launches of a batch of up to 8 lines are captured once per batch
                                size and replayed as a CUDA graph (same kernels, same results;
                                fewer host calls); larger batches launch directly. No counterpart
                                in the paper. Ignored while profiling is on. */
  HSAD_FORCE_INVERSE = 8     /* use the explicit-inverse whitening form (HSAD_FORM_INVERSE) also
                                for streamed statistics, where the triangular solve is the
                                default (comparisons of the two forms) */
};

typedef struct {
  int32_t width;               /* W >= 1 samples per line */
  int32_t bands;               /* 1 <= B <= 512 */
  int32_t in_dtype;            /* HSAD_U16 | HSAD_F32 */
  int32_t precision;           /* HSAD_FP32 | HSAD_BF16 | HSAD_FP16 */
  int32_t stats_mode;          /* HSAD_EXCLUSIVE | HSAD_INCLUSIVE | HSAD_CUBE */
  int32_t cube_lines;          /* statistics reset period in lines; 0 = never (stream modes).
                                  Required > 0 in CUBE mode (the paper uses 1000). */
  const float* gain;           /* length B host array or NULL (all 1); copied at create; non-zero */
  const float* offset;         /* length B host array or NULL (all 0); copied at create */
  int32_t threshold_mode;      /* HSAD_ABS | HSAD_REL */
  float threshold;             /* tau; the paper's display value 0.110 is relative (REL) */
  int64_t warmup_pixels;       /* a line is scored only once its statistics hold at least
                                  max(B + 1, warmup_pixels) pixels */
  int64_t device_budget_bytes; /* 0 = no cap for this context */
  int32_t flags;               /* HSAD_CREATE_WAIT | HSAD_NORMALIZE_SCORES | HSAD_CUDA_GRAPHS |
                                  HSAD_FORCE_INVERSE */
  int32_t device;              /* CUDA device ordinal */
  int32_t max_batch_lines;     /* lines processed per internal batch (0 = default 256) */
  int32_t result_lines;        /* lines of scores kept for hsad_scores (0 = default) */
  /* Front end (Sec. 3.2: out-of-specification bands discarded, band_bin consecutive bands
   * summed into one). raw_bands = 0 (default): off, pushed lines have `bands` bands.
   * raw_bands > 0 (HSAD_U16 input of 12-bit DN only): pushed lines have raw_bands bands;
   * band b of the detector is the sum of raw bands band_first + band_bin * b .. + band_bin - 1,
   * band_bin in [1, 4], band_first + band_bin * bands <= raw_bands. The sums stay exact (the
   * covariance sums are accumulated in slices small enough for the wider values). */
  int32_t raw_bands;
  int32_t band_first;
  int32_t band_bin;
  /* Factorisation cadence (an extension; the paper does not define one): 0 or 1 (default)
   * scores every line with the statistics of all lines before it; k in [2, 64] (EXCLUSIVE
   * only) takes the statistics every k lines after a reset and scores line t against the
   * last such snapshot, lines [r, r + k floor((t - r) / k)): k times fewer factorisations,
   * with statistics up to k - 1 lines old. */
  int32_t factor_every;
  /* Exponential forgetting (an extension; the paper does not define one, and names drift and
   * cloud shadow as open problems for the statistics, Sec. 6.1): 0 or 1 (default) keeps every
   * line since the last reset at full weight; forget in (0, 1) (EXCLUSIVE or INCLUSIVE, not
   * with factor_every > 1) weighs the pixels of a line forget^age, age = the number of window
   * lines newer than it (the newest line weighs 1). The mean is the weighted mean and the
   * covariance the weighted centred sum over (N - 1), N = the sum of the weights, which also
   * replaces the pixel count of the warm-up rule: the window saturates at W / (1 - forget)
   * pixels, so a forget with W / (1 - forget) < max(B + 1, warmup_pixels) scores no line.
   * The running sums are then FP64 instead of exact integers; statistics export and import
   * (hsad_get_stats, hsad_set_stats) and CUDA-graph replay are not available. */
  float forget;
  int32_t factor_precision;    /* HSAD_FACTOR_FF (default) | HSAD_FACTOR_FP64 */
} hsad_config;

/* Fill *cfg with defaults: U16, FP32, float-float factor, EXCLUSIVE, cube_lines 0, ABS threshold
 * B + 6 sqrt(2B) once bands is known (threshold 0 here means "use that default"),
 * device 0. Returns HSAD_E_INVALID for NULL. */
int hsad_config_init(hsad_config* cfg);

/* Create a detector context on cfg->device. Validates every field (HSAD_E_INVALID),
 * allocates its device state and checks it against device_budget_bytes and the
 * device-wide budget (HSAD_E_NOMEM, or HSAD_E_BUSY when admission would succeed
 * later; with HSAD_CREATE_WAIT the call waits up to 10 s for admission).
 * On success *out owns the context; release it with hsad_destroy. */
int hsad_create(const hsad_config* cfg, hsad_ctx** out);

/* Append n_lines lines (BIP, in_dtype) to the stream and enqueue their work.
 * mem = HSAD_HOST: the data are copied before return, so the buffer may be reused at
 *   once. Page-locked (pinned) host memory is copied straight to device staging by DMA
 *   (the call returns when those copies have landed, not when the batch is scored);
 *   pageable memory goes through library pinned staging first.
 * mem = HSAD_DEVICE: the lines are read in place, stream-ordered: the buffer must
 *   stay unchanged until hsad_scores has returned for these lines (or
 *   hsad_synchronize). In CUBE mode device lines are copied into the cube buffer
 *   unless the push holds exactly one whole cube starting at its first line.
 * With the front end (raw_bands > 0) the lines have raw_bands bands; they are binned
 * on the device (Sec. 3.2) before anything else reads them.
 * *first_line_id (optional) receives the id of the first pushed line; ids count
 * lines from 0 in push order. n_lines = 0 is a no-op. Returns HSAD_E_INVALID for
 * NULL data, a negative count, a pointer in the wrong memory space, or a push
 * larger than the result ring; HSAD_E_INVALID_DATA when a float32 push holds NaN
 * or Inf (the whole push is rejected and nothing is enqueued). */
int hsad_push_lines(hsad_ctx* ctx, const void* lines, int64_t n_lines, int32_t mem,
                    uint64_t* first_line_id);

/* Push lines recorded at varying gain (Sec. 3.2, "Data Acquisition": the imager adjusts
 * its gain for every line to avoid saturation, and the data is corrected for the varying
 * gain before the radiometric calibration). As hsad_push_lines, plus line_gain: host
 * memory, n_lines floats, line_gain[i] > 0 the gain of line i of this push (of the binned
 * line when the context has a front end: binning commutes with the correction). The
 * detector then works on u = DN / g_t: every line's statistics and scores are those of its
 * values divided by its gain, and the per-band calibration still cancels from Eq. 1.
 * The covariance sums stay exact integers per line; the correction is applied to them in
 * FP64 when the running statistics are formed, and to the mean and the score of each line
 * in the whitening (d = ||L^{-1}(DN - g (mu + c) + c)||^2 / g^2 with the integer shift c).
 * The gains are copied before the call returns. Contexts mix both calls freely (a push
 * without gains has gain 1 on every line). Supported for streamed statistics (EXCLUSIVE,
 * INCLUSIVE) with HSAD_U16 input in the triangular-solve whitening form (HSAD_FP32, or
 * HSAD_BF16); pushes with gains run without CUDA-graph replay. The first call allocates
 * the per-batch gain buffers (Lmax x (4 Bp + 68) bytes of device memory, two pinned slots
 * of Lmax x 32 bytes), outside the context's admission budget.
 * Errors: those of hsad_push_lines; HSAD_E_INVALID for a NULL line_gain with n_lines > 0,
 * a gain outside [2^-16, 2^16] or NaN (checked before anything is enqueued), a CUBE-mode,
 * float-input or explicit-inverse context; HSAD_E_NOMEM if the gain buffers cannot be
 * allocated. */
int hsad_push_lines_gain(hsad_ctx* ctx, const void* lines, const float* line_gain, int64_t n_lines,
                         int32_t mem, uint64_t* first_line_id);

/* CUBE mode: close the current partial cube (fewer than cube_lines lines) and score
 * it as a cube of its own. No-op when no partial cube is open or in stream modes. */
int hsad_flush(hsad_ctx* ctx);

/* Copy scores and/or mask of lines [first_line_id, first_line_id + n_lines) into
 * caller memory (mem = HSAD_HOST or HSAD_DEVICE; scores/mask may be NULL).
 * Waits up to timeout_ms for the lines to be computed (0 = poll: HSAD_E_NOT_READY if
 * not yet done; negative = wait without limit). Lines that were never pushed or have
 * left the result ring give HSAD_E_INVALID. Lines still in warm-up get NaN scores
 * and mask 0 and the call returns HSAD_E_NOT_READY; lines whose covariance was not
 * positive definite likewise return HSAD_E_NOT_PD (which takes precedence). */
int hsad_scores(hsad_ctx* ctx, uint64_t first_line_id, int64_t n_lines, float* scores,
                uint8_t* mask, int32_t mem, int32_t timeout_ms);

/* Per-line status of computed lines: 0 = scored, 1 = warm-up (not ready),
 * 2 = covariance not positive definite, 3 = invalid data. Host array of n_lines.
 * Same waiting rules as hsad_scores. */
int hsad_line_status(hsad_ctx* ctx, uint64_t first_line_id, int64_t n_lines,
                     int32_t* status, int32_t timeout_ms);

/* Transmit encoding (Sec. 3.4, data transmission) of lines [first_line_id, first_line_id +
 * n_lines): code = IEEE binary16 of sqrt(delta / delta_max), delta_max the largest finite
 * score of the block (the cube maximum of the paper when the block is one cube), the
 * division and square root in FP32 (correctly rounded) and the conversion rounded to nearest
 * even. NaN scores (lines in warm-up) give the NaN code 0x7E00; if no score of the block is
 * positive every finite score gives 0. codes: n_lines x width uint16, row-major, in host
 * (mem = HSAD_HOST) or device memory; *max_score (nullable) receives delta_max. Waits and
 * returns like hsad_scores (HSAD_E_NOT_READY after writing the codes if some lines are in
 * warm-up). Runs on the context's copy stream; allocates nothing. */
int hsad_scores_tx(hsad_ctx* ctx, uint64_t first_line_id, int64_t n_lines, uint16_t* codes, float* max_score,
                   int32_t mem, int32_t timeout_ms);

/* The front end alone (Sec. 3.2) on device buffers of `device`: out[p][b] = sum of
 * raw[p][band_first + band_bin * b + i] for i < band_bin, b < bands, p < n_pixels; raw is
 * [n_pixels][raw_bands] uint16, out [n_pixels][bands] uint16 (sums wrap above 65535: use
 * 12-bit DN and band_bin <= 16). stream: a cudaStream_t of that device or NULL; the call
 * synchronises it. Returns HSAD_OK, HSAD_E_INVALID or HSAD_E_CUDA. */
int hsad_frontend(const uint16_t* raw, int64_t n_pixels, int32_t raw_bands, int32_t band_first, int32_t band_bin,
                  int32_t bands, uint16_t* out, int32_t device, void* stream);

/* The same transmit encoding of n scores already in device memory of `device` into n
 * device codes, delta_max over those n scores (returned in *max_score, nullable).
 * stream: a cudaStream_t of that device, or NULL for its default stream; the call
 * synchronises it. Keeps one 4-byte device scratch per device for the process. Returns
 * HSAD_OK, HSAD_E_INVALID (n < 0, NULL pointers, bad device), HSAD_E_NOMEM or HSAD_E_CUDA. */
int hsad_encode_scores(const float* scores, int64_t n, uint16_t* codes, float* max_score, int32_t device,
                       void* stream);

/* Restart the stream: the running statistics, the open cube and the result ring are
 * cleared and line ids start again at 0. Work already enqueued completes first
 * (stream order); no allocation happens. */
int hsad_reset(hsad_ctx* ctx);

/* Export the running statistics (Sec. 3.3: the per-band sums behind mu and Sigma) after
 * all enqueued work: *n_pixels = pixels since the last reset (stream modes) or in the
 * last scored cube (CUBE mode); shift[B] = the per-band centring c (rounded DN for
 * uint16 input, cast to double; float input: the float shift); s1[B] = sum (x - c);
 * s2[B*B] = sum (x - c)(x - c)^T, row-major, lower triangle (row >= column) valid.
 * All arguments are host arrays and may be NULL. For uint16 input every value is an
 * exact integer. Synchronises the context's stream (bounded, 10 s). HSAD_E_INVALID for a
 * context with forgetting (its sums are weighted, not counts of pixels). */
int hsad_get_stats(hsad_ctx* ctx, int64_t* n_pixels, double* shift, double* s1, double* s2);

/* Import running statistics exported by hsad_get_stats (checkpoint / resume of a stream;
 * the paper keeps no detector state). Stream modes only, on a context with no line pushed
 * since creation or hsad_reset. n_pixels >= 0; shift[B] (uint16 input: integers in
 * [0, 65535]), s1[B], s2[B*B] (lower triangle read) are host arrays. Lines pushed next are
 * scored against the imported statistics exactly as if they had followed the exported
 * lines in one stream (for uint16 input the sums are exact, so the scores are bitwise the
 * same); EXCLUSIVE mode also rebuilds the carried factor here (enqueued on the context's
 * stream). Line ids and the reset schedule (cube_lines) count from 0 in the new context.
 * Returns HSAD_E_INVALID for CUBE mode, a context with forgetting, a context already in
 * use, NULL arrays or a bad shift. */
int hsad_set_stats(hsad_ctx* ctx, int64_t n_pixels, const double* shift, const double* s1, const double* s2);

/* Block until all work enqueued on the context has finished (bounded by timeout_ms,
 * negative = no limit). */
int hsad_synchronize(hsad_ctx* ctx, int32_t timeout_ms);

/* The CUDA stream (cudaStream_t) the context launches on, for event timing. */
void* hsad_stream(hsad_ctx* ctx);

/* Number of kernel launches the context has issued so far. */
int64_t hsad_kernel_launches(const hsad_ctx* ctx);

/* Per-kernel timing with CUDA events recorded around every kernel on the context's
 * stream (off by default; costs two event records per launch when on). */
int hsad_profile_enable(hsad_ctx* ctx, int32_t enable);

/* Totals of kernel class `index` (0-based, in first-launch order) since the last
 * reset: its name (copied into name[name_len], NUL-terminated), launches and total
 * milliseconds. Synchronises the context's stream. HSAD_E_INVALID past the last
 * class. */
int hsad_profile_read(hsad_ctx* ctx, int32_t index, char* name, int32_t name_len,
                      int64_t* launches, double* total_ms);

/* Clear the per-kernel totals. */
int hsad_profile_reset(hsad_ctx* ctx);

/* The context's whitening form (HSAD_FORM_*), or HSAD_E_INVALID for a null context. */
int hsad_whitening_form(const hsad_ctx* ctx);
/* 1 if the context's whitening contraction runs on the tensor cores (tcgen05), 0 if on the
 * SIMT cores (FFMA), HSAD_E_INVALID for a null context. An implementation query with no
 * counterpart in the method (Sec. 3.3 fixes what is computed, not on which units). */
int hsad_whitening_tensor_cores(const hsad_ctx* ctx);

/* Bytes of device memory the context holds. */
int64_t hsad_device_bytes(const hsad_ctx* ctx);

/* Device-wide admission budget in bytes shared by every context on `device`
 * (0 = unlimited, the default). Contexts already admitted are not affected. */
int hsad_set_device_budget(int device, int64_t bytes);

/* Bytes currently charged against the device-wide budget of `device`. */
int64_t hsad_device_budget_used(int device);

/* Global RX of one cube already in device memory, with no device allocation.
 * The paper has no counterpart of this call; it exists for callers that cannot
 * allocate device memory (flight or embedded code that forbids the allocator after
 * start-up, or hosts whose external memory manager owns the whole device pool).
 * Same arithmetic and kernels as a CUBE-mode context scoring one cube:
 *   cube    device [n_lines][width][bands], in_dtype (HSAD_U16 | HSAD_F32)
 *   gain    host array of `bands` floats or NULL (all 1), finite and non-zero
 *   threshold_mode / threshold / flags (HSAD_NORMALIZE_SCORES only) as in hsad_config
 *           (threshold 0 with HSAD_ABS means B + 6 sqrt(2B))
 *   scores  device float [n_lines][width], mask device uint8 [n_lines][width]
 *   stream  cudaStream_t to run on (NULL = legacy default stream), device = ordinal
 * Every intermediate lives in one static device array of 16 MiB that each GPU loading
 * the library keeps until exit; the cube must fit it: roughly
 *   16 n_lines B + 24 B^2 + 4 pad64(B)^2 + 8 n_lines bytes <= 16 MiB
 * (e.g. B = 270 up to ~3300 lines, B = 70 up to ~14000 lines), else HSAD_E_INVALID
 * before anything runs. The first call on a device looks up the array's address
 * (cudaGetSymbolAddress, with that device current), which loads the module and commits
 * the array: make it before any stream capture. A call with n_lines = 0 does only that
 * set-up (every other argument is ignored and may be NULL) and returns HSAD_OK:
 * callers that must not allocate after start-up make it once per device at start-up. Calls share the array and keep its last contents (the
 * sums and status words are cleared at the start of each call): calls that overlap
 * on the GPU, from any thread or stream, race and must not be issued. The call
 * returns after the cube is scored: HSAD_OK, HSAD_E_NOT_PD, HSAD_E_NOT_READY (fewer
 * than bands + 1 pixels), HSAD_E_INVALID or HSAD_E_CUDA. No error string is kept. */
int hsad_global_rx_noalloc(const void* cube, int64_t n_lines, int32_t width, int32_t bands,
                           int32_t in_dtype, int32_t precision, const float* gain,
                           int32_t threshold_mode, float threshold, int32_t flags, float* scores,
                           uint8_t* mask, void* stream, int32_t device);

/* Subsampled kernel RX (Sec. 2.2, Table tab:results: the kernel RX variant the paper's prior
 * work compared with global RX, citing Kwon and Nasrabadi's kernel RX and Hidalgo et al.'s
 * subsampled form) of one cube already in device memory of `device`. The background is the m
 * pixels subsample[0 .. m) (distinct flat pixel indices, host array, drawn by the caller);
 * every pixel r of the cube is scored
 *     delta(r) = (m - 1) || (K~ + lam I)^{-1} H (k_r - K 1 / m) ||^2
 * with the Gaussian kernel k(x, y) = exp(-||x - y||^2 / c) on the calibrated bands
 * (x_b = v_b gain_b: offsets cancel), K the m x m kernel matrix of the background,
 * H = I - 1 1^T / m, K~ = H K H, (k_r)_i = k(s_i, r), lam = ridge tr(K~) / m, and
 * c = kernel_width, or the mean squared distance between distinct background pixels when
 * kernel_width is 0.
 *   cube       device [n_pixels][bands], in_dtype (HSAD_U16 | HSAD_F32), bands contiguous
 *   m          2 .. 512, <= n_pixels
 *   ridge      > 0 (relative ridge eps; 1e-2 is a sound default: the scores' sensitivity to
 *              rounding grows with kappa(K~ + lam I), about 1 / eps)
 *   gain       host array of `bands` floats or NULL (all 1), finite and non-zero
 *   threshold_mode / threshold / flags (HSAD_NORMALIZE_SCORES only) as in hsad_config
 *              (threshold 0 with HSAD_ABS means bands + 6 sqrt(2 bands))
 *   scores     device float [n_pixels], mask device uint8 [n_pixels]
 *   stream     cudaStream_t to run on (NULL = legacy default stream)
 * The background statistics are FP64 (Cholesky factor and inverse by the factor kernel);
 * the per-pixel squared distances and the product with (K~ + lam I)^{-1} H carry float-float
 * sums on the FP32 pipe. Allocates its scratch (stream-ordered, about 40 m^2 + 8 m B bytes)
 * and frees it before returning; the call returns after the scores are written: HSAD_OK,
 * HSAD_E_NOT_PD (K~ + lam I not positive definite), HSAD_E_INVALID (bad argument, repeated or
 * out-of-range indices), HSAD_E_INVALID_DATA (non-finite float input) or HSAD_E_CUDA. */
int hsad_krx(const void* cube, int64_t n_pixels, int32_t bands, int32_t in_dtype, const int64_t* subsample,
             int32_t m, float kernel_width, float ridge, const float* gain, int32_t threshold_mode,
             float threshold, int32_t flags, float* scores, uint8_t* mask, void* stream, int32_t device);

/* Factor-kernel autotuner (no counterpart in the paper). Times every launch shape of the
 * factorisation (one 128-thread CTA per line with registers for 4 or 5 CTAs per SM,
 * one 256-thread CTA per line, or a 2/4/8/16-CTA cluster per line) on synthetic
 * positive definite problems of `bands` bands, for batches of 1, 2, 4, ..., max_lines
 * lines (1 .. 4096), and makes contexts on `device` with that band count and precision
 * use the fastest shape per batch size from then on (larger batches keep the built-in
 * rule). Results do not depend on the shape (bitwise). The measurement is kept per
 * process: a second call with no larger max_lines returns at once. report (nullable):
 * rows of 4 floats (largest batch size of the bucket, CTAs per line, threads per CTA
 * (96 = 128 threads sized for 5 CTAs per SM), milliseconds), up to *n_rows rows; *n_rows
 * (nullable only if report is NULL) receives the number of buckets. Allocates (and
 * frees) scratch device memory for max_lines problems. Returns HSAD_OK, HSAD_E_INVALID,
 * or HSAD_E_CUDA. */
int hsad_autotune_factor(int32_t device, int32_t bands, int32_t precision, int32_t max_lines, float* report,
                         int32_t* n_rows);

/* Self-test of the bounded device waits used by the tensor-core kernels (no
 * counterpart in the paper): launches one kernel that waits on an mbarrier nothing
 * arrives at, with a limit of limit_cycles SM clock cycles (1 .. 2e10). The wait gives
 * up, *timed_out becomes 1 and the call returns HSAD_E_TIMEOUT; the device stays usable.
 * HSAD_OK with *timed_out 0 would mean the wait completed, which cannot happen. */
int hsad_selftest_bounded_wait(int32_t device, int64_t limit_cycles, int32_t* timed_out);

/* ---------------------------------------------------------------------------------
 * Serving engine: many concurrent sensor streams on one device (the line-based
 * detector of Sec. 6.1 for several imagers at once). Each admitted stream is a context
 * with its statistics and factor resident on the device and its own CUDA stream; one
 * native worker thread repeatedly pushes every stream's pending lines as one batch, so
 * lines that arrive while a stream's previous batch is on the GPU are batched together
 * and the work of different streams overlaps on the device.
 * ------------------------------------------------------------------------------- */
typedef struct hsad_engine hsad_engine;

/* Start an engine on `device` whose streams share a device budget of budget_bytes
 * (0 = unlimited; this sets the device-wide budget of hsad_set_device_budget). */
int hsad_engine_create(int32_t device, int64_t budget_bytes, hsad_engine** out);

/* Admit a stream with configuration *cfg (its device field is ignored; HSAD_CUDA_GRAPHS
 * is added to its flags). A band count the engine has not served before is first
 * autotuned (hsad_autotune_factor, batches up to min(max_batch_lines, 64)). Returns
 * HSAD_E_BUSY while the budget cannot hold it (retry after a stream closes; with
 * HSAD_CREATE_WAIT in cfg->flags the call waits up to 10 s), HSAD_E_NOMEM if it can
 * never fit, else HSAD_OK and the stream's id. */
int hsad_engine_open(hsad_engine* e, const hsad_config* cfg, int32_t* stream_id);

/* Queue n_lines host lines (BIP, the stream's in_dtype) for scoring; copies them and
 * returns at once. *first_line_id receives the stream-local id of the first line. */
int hsad_engine_submit(hsad_engine* e, int32_t stream_id, const void* lines, int64_t n_lines,
                       uint64_t* first_line_id);

/* Wait (timeout_ms; negative = no limit) until lines [first, first + n) of the stream
 * are scored and copy their scores / mask to host memory (either may be NULL). Status
 * as hsad_scores; HSAD_E_TIMEOUT when the wait expires. */
int hsad_engine_results(hsad_engine* e, int32_t stream_id, uint64_t first_line_id, int64_t n_lines,
                        float* scores, uint8_t* mask, int32_t timeout_ms);

/* Close a stream (waits, bounded, for its work) and return its memory to the budget. */
int hsad_engine_close(hsad_engine* e, int32_t stream_id);

/* Lines pushed, batches pushed and the largest batch so far; returns the last push
 * error (HSAD_OK if none). */
int hsad_engine_counters(hsad_engine* e, int64_t* lines, int64_t* pushes, int64_t* max_batch);

/* Stop the worker and close every stream. NULL-safe. */
int hsad_engine_destroy(hsad_engine* e);

/* Release the context. NULL-safe. Waits (up to 10 s) for in-flight work first. */
int hsad_destroy(hsad_ctx* ctx);

/* Detail string of the last error on this context (or of the last failed
 * hsad_create on this thread when ctx is NULL). Never NULL. */
const char* hsad_last_error(const hsad_ctx* ctx);

/* Static name of a status code. */
const char* hsad_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* HSAD_H */
