// Host engine behind the C ABI declared in include/hsad.h.
//
// One context = one sensor stream: its running statistics (shift c, S1, S2, N) live on
// the device, pushed lines are processed in batches of up to max_batch_lines on the
// context's stream, and per-line scores / mask / status land in a result ring that
// hsad_scores copies out once the batch's completion event has fired.
//
// Per batch in the stream modes (Sec. 6.1's line-based detector; EXCLUSIVE scores line t
// against lines [r, t), INCLUSIVE against [r, t]):
//   K1 shift (first line after a reset) -> K1 column sums -> K2 per-line SYRK
//   -> K3 running mean / covariance per line -> K4+K5 Cholesky + inverse per line (FP64
//   pivots and diagonal blocks, float-float updates)
//   -> K6 whitening + score + threshold.
// In CUBE mode (global RX per cube of cube_lines lines, Sec. 3.3) the cube's lines are
// kept on the device; when the cube is complete: K1, K2 over the whole cube, K3 once,
// K4+K5 once, K6 over every line, K7 maximum / normalisation / threshold.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <chrono>
#include <cmath>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/hsad.h"
#include "hsad_internal.h"

using namespace hsad;

namespace {

thread_local std::string g_thread_error = "";

struct Record {
  uint64_t first, n;
  cudaEvent_t ev;
};

// Device-wide admission budget shared by all contexts of the process.
struct Budget {
  std::mutex mu;
  std::map<int, int64_t> limit, used;
};
Budget& budget() {
  static Budget b;
  return b;
}

using Clock = std::chrono::steady_clock;

}  // namespace

struct hsad_ctx {
  hsad_config cfg{};
  int W = 0, B = 0, Bp = 0, in_type = 0, prec = 0, mode = 0;
  int fprec = 0;  // prec, or'ed with kFactorF64 for the FP64 factor (launch_factor's argument)
  bool tc_factor = false;  // streamed statistics factored by the tensor-core factor (launch_factor_tc)
  int64_t min_pix = 0, elem = 2, line_elems = 0, line_bytes = 0;
  float tau = 0.f;
  int Lmax = 256;
  int64_t ring = 0;
  int device = 0;
  cudaStream_t stream = nullptr, copy_stream = nullptr;
  std::string err;
  bool failed = false;
  LaunchCounter lc;
  std::vector<void*> dev_allocs;
  std::vector<void*> host_allocs;
  int64_t dev_bytes = 0;
  bool budget_charged = false;
  int64_t charged = 0;  // bytes charged to the device budget at admission

  // device state
  int32_t* c_int = nullptr;
  float* c_flt = nullptr;
  double* state_s1 = nullptr;
  double* state_s2 = nullptr;
  // per-batch workspace
  double* s1_line = nullptr;
  double* m_line = nullptr;
  double* sigma = nullptr;
  double* inv = nullptr;
  void* wmat = nullptr;
  float* yscratch = nullptr;  // whitened blocks of the FP32 triangular solve's items in flight
  float* y0 = nullptr;
  float* inv_s2 = nullptr;
  int32_t* status = nullptr;
  unsigned int* dmax_bits = nullptr;
  int32_t* bad_flag = nullptr;
  int32_t* dev_err = nullptr;  // set by a kernel whose bounded wait expired
  int64_t* bdesc = nullptr;    // per-batch values read by replayed CUDA graphs
  alignas(64) CUtensorMap gmap;  // TMA map over the 16-bit G planes (FP16/BF16 forms)
  bool have_gmap = false;
  // result ring
  float* r_scores = nullptr;
  uint8_t* r_mask = nullptr;
  uint16_t* r_codes = nullptr;      // transmit codes of a requested block, for host copies
  unsigned int* tx_max = nullptr;   // bits of the block maximum of the transmit encoding
  int32_t* r_status = nullptr;
  // input staging (host pushes) and cube buffer
  void* h_stage[2] = {nullptr, nullptr};
  void* d_stage[2] = {nullptr, nullptr};
  // front end (raw_bands > 0): raw lines are copied to d_raw (host pushes) and binned into
  // d_bin[i], alternately, before the pipeline reads them
  bool fe = false;
  int64_t raw_line_bytes = 0;
  void* d_raw = nullptr;
  void* d_bin[2] = {nullptr, nullptr};
  int fe_idx = 0;
  int64_t syrk_max_pix = 4096;  // pixels one exact SYRK accumulation may hold
  bool split_syrk = false;      // streamed uint16 lines: split once into hr, then contract per tile
  uint8_t* hr = nullptr;        // the split operand blocks of a batch's lines
  float2* ffm = nullptr;        // per-line float-float means, n m, 1/(n-1) (tensor-core factor)
  int every = 1;                // factorisation cadence in lines (EXCLUSIVE)
  cudaEvent_t stage_ev[2] = {nullptr, nullptr};
  // pinned caller buffers are copied straight to d_stage on h2d_stream: copy_ev marks the
  // copy done, free_ev the end of the last batch that read d_stage[i]
  cudaStream_t h2d_stream = nullptr;
  cudaEvent_t copy_ev[2] = {nullptr, nullptr}, free_ev[2] = {nullptr, nullptr};
  int stage_idx = 0;
  void* cube_buf = nullptr;
  int32_t* h_small = nullptr;  // pinned scratch for small host->device values
  // per-line gain correction (hsad_push_lines_gain), allocated on first use. A batch's
  // per-line factors go through pinned slot h_gain[i] to device slot d_gain + i Lmax
  // kGainStride (slots alternate): gain_ev[i] marks the copy out of h_gain[i] done,
  // gfree_ev[i] the end of the last batch that read device slot i. d_gain_cur is the
  // slot of the batch being enqueued (batch_gain set meanwhile); d_mgain [Lmax][Bp] and
  // d_gscale [Lmax] hold the gain-corrected mean offsets and score scales of a whitening
  // launch.
  double* d_gain = nullptr;  // 2 x [Lmax][kGainStride]: g, 1 / g, 1 / g^2, 1 - g
  double* d_gain_cur = nullptr;
  float* d_mgain = nullptr;
  float* d_gscale = nullptr;
  double* h_gain[2] = {nullptr, nullptr};
  cudaEvent_t gain_ev[2] = {nullptr, nullptr}, gfree_ev[2] = {nullptr, nullptr};
  int gain_idx = 0;
  bool batch_gain = false;

  // host-side stream state
  uint64_t next_line = 0;   // id of the next line to be pushed
  int64_t n_stats = 0;      // pixels in the running statistics (stream modes)
  // exponential forgetting (lam < 1): the window's weight after the last pushed line and the
  // per-line weights of a batch [Lmax] (device)
  double lam = 1.0;
  double n_eff = 0.0;
  double* d_nline = nullptr;
  int64_t cube_fill = 0;    // lines in the open cube (CUBE mode)
  uint64_t cube_first = 0;  // id of the open cube's first line
  int64_t last_cube_lines = 0;  // lines of the most recently scored cube
  std::deque<Record> records;
  std::vector<cudaEvent_t> event_pool;

  // CUDA graphs of the EXCLUSIVE batch tail, one per (lines in the batch, staging buffer)
  bool use_graphs = false;
  struct GraphEntry {
    cudaGraphExec_t exec = nullptr;
    int64_t launches = 0;  // kernels in the graph (added to the launch counter per replay)
  };
  std::map<std::pair<int, int>, GraphEntry> graphs;

  // profiling: pending (name, begin, end) event triples and per-name totals
  bool prof_on = false;
  cudaEvent_t prof_open = nullptr;
  struct Pending {
    std::string name;
    cudaEvent_t a, b;
  };
  std::vector<Pending> prof_pending;
  std::vector<std::string> prof_names;
  std::map<std::string, std::pair<int64_t, double>> prof_tot;
  std::vector<cudaEvent_t> prof_pool;
};

// ------------------------------------------------------------------------------ helpers
namespace {

int fail(hsad_ctx* c, int code, const std::string& msg) {
  if (c) {
    c->err = msg;
    if (code == HSAD_E_CUDA) c->failed = true;
  } else {
    g_thread_error = msg;
  }
  return code;
}

#define CK(expr)                                                                        \
  do {                                                                                  \
    cudaError_t _e = (expr);                                                            \
    if (_e != cudaSuccess)                                                              \
      return fail(ctx, HSAD_E_CUDA, std::string(#expr) + ": " + cudaGetErrorString(_e)); \
  } while (0)

// Per-kernel CUDA-event timing on the launching stream (off unless enabled).
void prof_begin(hsad_ctx* ctx);
void prof_end(hsad_ctx* ctx, const char* name);

#define KL(name, expr)    \
  do {                    \
    prof_begin(ctx);      \
    CK(expr);             \
    prof_end(ctx, name);  \
  } while (0)

cudaEvent_t get_event(hsad_ctx* ctx) {
  if (!ctx->event_pool.empty()) {
    cudaEvent_t e = ctx->event_pool.back();
    ctx->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return nullptr;
  return e;
}

cudaEvent_t prof_event(hsad_ctx* ctx) {
  if (!ctx->prof_pool.empty()) {
    cudaEvent_t e = ctx->prof_pool.back();
    ctx->prof_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

void prof_begin(hsad_ctx* ctx) {
  if (!ctx->prof_on) return;
  ctx->prof_open = prof_event(ctx);
  if (ctx->prof_open) cudaEventRecord(ctx->prof_open, ctx->stream);
}

void prof_end(hsad_ctx* ctx, const char* name) {
  if (!ctx->prof_on || !ctx->prof_open) return;
  cudaEvent_t b = prof_event(ctx);
  if (!b) return;
  cudaEventRecord(b, ctx->stream);
  ctx->prof_pending.push_back({name, ctx->prof_open, b});
  ctx->prof_open = nullptr;
}

// Wait (bounded) for an event. timeout_ms < 0: no limit; 0: single poll.
int wait_event(hsad_ctx* ctx, cudaEvent_t ev, int32_t timeout_ms) {
  const auto t0 = Clock::now();
  for (;;) {
    cudaError_t q = cudaEventQuery(ev);
    if (q == cudaSuccess) return HSAD_OK;
    if (q != cudaErrorNotReady) return fail(ctx, HSAD_E_CUDA, std::string("event: ") + cudaGetErrorString(q));
    if (timeout_ms == 0) return HSAD_E_NOT_READY;
    if (timeout_ms > 0 &&
        std::chrono::duration_cast<std::chrono::milliseconds>(Clock::now() - t0).count() >= timeout_ms)
      return fail(ctx, HSAD_E_TIMEOUT, "timed out waiting for device work");
    std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
}

void* dalloc(hsad_ctx* ctx, int64_t bytes, bool* ok) {
  if (bytes <= 0) return nullptr;
  void* p = nullptr;
  if (cudaMalloc(&p, (size_t)bytes) != cudaSuccess) {
    cudaGetLastError();
    *ok = false;
    return nullptr;
  }
  ctx->dev_allocs.push_back(p);
  ctx->dev_bytes += bytes;
  return p;
}

int64_t plan_bytes(const hsad_ctx* c) {
  const int64_t B = c->B, Bp = c->Bp, L = c->Lmax;
  // factor slots per batch (EXCLUSIVE carries one more)
  const int64_t Lf = (c->mode == HSAD_CUBE) ? 1 : (c->mode == HSAD_EXCLUSIVE ? L + 1 : L);
  const int64_t Ls = (c->mode == HSAD_CUBE) ? c->cfg.cube_lines : L;  // lines per batch
  int64_t b = 0;
  b += B * 4 + B * 4 + B * 8 + B * B * 8;                        // c (int, float), S1, S2
  b += Ls * B * 8 * 2;                                           // s1_line, m_line
  if (c->lam != 1.0) b += Ls * 8;                                // forgetting weights per line
  b += Lf * B * B * 8 * 2;                                       // sigma, inv
  b += Lf * Bp * Bp * wmat_elem_bytes(c->prec) + Lf * Bp * 4 + Lf * 4 + Ls * 4;  // wmat, y0, inv_s2, status
  if (c->prec == P_FP32T) b += (int64_t)whiten_trsm_simt_scratch_bytes(c->B);  // FP32 solve scratch
  if (c->split_syrk) b += (int64_t)syrk_split_bytes(L, c->W, c->B);             // split SYRK operands
  if (c->tc_factor) b += (int64_t)tcf_form_scratch_bytes((int)Lf, c->B);         // formation inputs
  b += c->ring * c->W * 5 + c->ring * 4 + 64;                    // result ring
  b += c->ring * c->W * 2 + 64;                                  // transmit codes scratch
  if (c->mode == HSAD_CUBE) b += (int64_t)c->cfg.cube_lines * c->line_bytes;
  else b += 2 * L * c->line_bytes;                               // device staging
  if (c->fe) b += L * c->raw_line_bytes + 2 * L * c->line_bytes;  // front end: raw copy, binned lines
  return b;
}

int validate(const hsad_config* cfg, std::string* why) {
  auto bad = [&](const char* m) { *why = m; return HSAD_E_INVALID; };
  if (!cfg) return bad("cfg is NULL");
  if (cfg->width < 1) return bad("width must be >= 1");
  if (cfg->bands < 1 || cfg->bands > 512) return bad("bands must be in [1, 512]");
  if (cfg->in_dtype != HSAD_U16 && cfg->in_dtype != HSAD_F32) return bad("in_dtype must be HSAD_U16 or HSAD_F32");
  if (cfg->precision < HSAD_FP32 || cfg->precision > HSAD_FP16) return bad("unknown precision");
  if (cfg->stats_mode < HSAD_EXCLUSIVE || cfg->stats_mode > HSAD_CUBE) return bad("unknown stats_mode");
  if (cfg->cube_lines < 0) return bad("cube_lines must be >= 0");
  if (cfg->stats_mode == HSAD_CUBE && cfg->cube_lines <= 0) return bad("CUBE mode needs cube_lines > 0");
  if (cfg->threshold_mode != HSAD_ABS && cfg->threshold_mode != HSAD_REL) return bad("unknown threshold_mode");
  if (cfg->threshold_mode == HSAD_REL && cfg->stats_mode != HSAD_CUBE) return bad("REL threshold needs CUBE mode");
  if (!std::isfinite(cfg->threshold) || cfg->threshold < 0.f) return bad("threshold must be finite and >= 0");
  if (cfg->warmup_pixels < 0) return bad("warmup_pixels must be >= 0");
  if (cfg->device_budget_bytes < 0) return bad("device_budget_bytes must be >= 0");
  if (cfg->max_batch_lines < 0 || cfg->max_batch_lines > 65535) return bad("max_batch_lines must be in [0, 65535]");
  if (cfg->result_lines < 0) return bad("result_lines must be >= 0");
  if (cfg->flags & ~(HSAD_CREATE_WAIT | HSAD_NORMALIZE_SCORES | HSAD_CUDA_GRAPHS | HSAD_FORCE_INVERSE))
    return bad("unknown flags");
  if (cfg->factor_precision != HSAD_FACTOR_FF && cfg->factor_precision != HSAD_FACTOR_FP64)
    return bad("factor_precision must be HSAD_FACTOR_FF or HSAD_FACTOR_FP64");
  if ((cfg->flags & HSAD_NORMALIZE_SCORES) && cfg->stats_mode != HSAD_CUBE) return bad("HSAD_NORMALIZE_SCORES needs CUBE mode");
  if (cfg->gain)
    for (int b = 0; b < cfg->bands; ++b)
      if (!std::isfinite(cfg->gain[b]) || cfg->gain[b] == 0.f) return bad("gain must be finite and non-zero");
  if (cfg->offset)
    for (int b = 0; b < cfg->bands; ++b)
      if (!std::isfinite(cfg->offset[b])) return bad("offset must be finite");
  if ((int64_t)cfg->width * cfg->bands > (int64_t)1 << 31) return bad("line too large");
  if (cfg->factor_every < 0 || cfg->factor_every > 64) return bad("factor_every must be in [0, 64]");
  if (cfg->factor_every > 1 && cfg->stats_mode != HSAD_EXCLUSIVE) return bad("factor_every > 1 needs EXCLUSIVE mode");
  if (!(cfg->forget >= 0.f && cfg->forget <= 1.f)) return bad("forget must be in [0, 1]");
  if (cfg->forget > 0.f && cfg->forget < 1.f) {
    if (cfg->stats_mode == HSAD_CUBE) return bad("forgetting needs streamed statistics");
    if (cfg->factor_every > 1) return bad("forgetting and factor_every > 1 do not combine");
  }
  if (cfg->raw_bands < 0) return bad("raw_bands must be >= 0");
  if (cfg->raw_bands > 0) {
    if (cfg->in_dtype != HSAD_U16) return bad("the front end (raw_bands > 0) needs HSAD_U16 input");
    if (cfg->band_bin < 1 || cfg->band_bin > 4) return bad("band_bin must be in [1, 4]");
    if (cfg->band_first < 0 || (int64_t)cfg->band_first + (int64_t)cfg->band_bin * cfg->bands > cfg->raw_bands)
      return bad("band_first + band_bin * bands must be <= raw_bands");
    if ((int64_t)cfg->width * cfg->raw_bands > (int64_t)1 << 31) return bad("raw line too large");
  }
  return HSAD_OK;
}

void release(hsad_ctx* ctx) {
  if (!ctx) return;
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  for (auto& r : ctx->records) cudaEventDestroy(r.ev);
  for (auto e : ctx->event_pool) cudaEventDestroy(e);
  for (auto e : ctx->prof_pool) cudaEventDestroy(e);
  for (auto& p : ctx->prof_pending) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  if (ctx->h2d_stream) cudaStreamSynchronize(ctx->h2d_stream);
  for (int i = 0; i < 2; ++i) {
    if (ctx->gain_ev[i]) cudaEventDestroy(ctx->gain_ev[i]);
    if (ctx->gfree_ev[i]) cudaEventDestroy(ctx->gfree_ev[i]);
    if (ctx->stage_ev[i]) cudaEventDestroy(ctx->stage_ev[i]);
    if (ctx->copy_ev[i]) cudaEventDestroy(ctx->copy_ev[i]);
    if (ctx->free_ev[i]) cudaEventDestroy(ctx->free_ev[i]);
  }
  for (auto& g : ctx->graphs)
    if (g.second.exec) cudaGraphExecDestroy(g.second.exec);
  for (void* p : ctx->dev_allocs) cudaFree(p);
  for (void* p : ctx->host_allocs) cudaFreeHost(p);
  if (ctx->stream) cudaStreamDestroy(ctx->stream);
  if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
  if (ctx->h2d_stream) cudaStreamDestroy(ctx->h2d_stream);
  if (ctx->budget_charged) {
    std::lock_guard<std::mutex> g(budget().mu);
    budget().used[ctx->device] -= ctx->charged;
  }
  if (prev >= 0) cudaSetDevice(prev);
  delete ctx;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no libcuda link).
bool encode_gmap(CUtensorMap* map, void* base, int64_t Bp, int64_t rows, int box_rows) {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !p) {
      cudaGetLastError();
      return false;
    }
    fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  const cuuint64_t dims[2] = {(cuuint64_t)Bp, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)Bp * 2};
  // 64 k (128 B, the swizzle span) x one (triangular solve) or two 64-row n blocks
  const cuuint32_t box[2] = {64, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, base, dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

}  // namespace

// Internal (serving engine): 1 when lines [first, first+n) have been scored, 0 while
// pending, negative status on error. Does not wait.
int hsadi_lines_ready(hsad_ctx* ctx, uint64_t first, int64_t n) {
  if (!ctx || n <= 0) return HSAD_E_INVALID;
  if (ctx->failed) return HSAD_E_CUDA;
  const uint64_t last = first + (uint64_t)n - 1;
  if (last >= ctx->next_line) return 0;
  DeviceGuard dg(ctx->device);
  for (auto it = ctx->records.rbegin(); it != ctx->records.rend(); ++it) {
    if (last >= it->first && last < it->first + it->n) {
      const cudaError_t q = cudaEventQuery(it->ev);
      if (q == cudaSuccess) return 1;
      if (q == cudaErrorNotReady) return 0;
      return fail(ctx, HSAD_E_CUDA, std::string("event: ") + cudaGetErrorString(q));
    }
  }
  return 0;
}

// 1 when a host push of up to Lmax lines would not wait for a staging buffer (the
// buffer that push would fill has finished its previous copy), 0 otherwise.
int hsadi_push_ready(hsad_ctx* ctx) {
  if (!ctx || ctx->failed) return 1;  // the push itself reports the error
  if (ctx->mode == HSAD_CUBE) return 1;
  DeviceGuard dg(ctx->device);
  return cudaEventQuery(ctx->stage_ev[ctx->stage_idx]) == cudaErrorNotReady ? 0 : 1;
}

// ------------------------------------------------------------------------------ ABI
extern "C" {

int hsad_autotune_factor(int32_t device, int32_t bands, int32_t precision, int32_t max_lines, float* report,
                         int32_t* n_rows) {
  if (bands < 1 || bands > 512 || max_lines < 1 || max_lines > 4096) return HSAD_E_INVALID;
  if (precision < HSAD_FP32 || precision > HSAD_FP16) return HSAD_E_INVALID;
  if (report && !n_rows) return HSAD_E_INVALID;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return ndev <= 0 ? HSAD_E_CUDA : HSAD_E_INVALID;
  }
  DeviceGuard dg(device);
  // the factor kernel's form for a streamed uint16-input context (the case with a
  // factorisation per line; the tensor-core factor has no tuned shape)
  const int prec = precision == HSAD_FP32 ? fp32_form(bands, IN_U16, false, false, false)
                   : precision == HSAD_BF16 ? bf16_form(bands, IN_U16, false, false)
                                            : P_FP16;
  factor_prepare(bands, prec);
  const int cap = report ? *n_rows : 0;
  const int n = factor_autotune(bands, prec, max_lines, report, cap);
  if (n < 0) return HSAD_E_CUDA;
  if (n_rows) *n_rows = n;
  return HSAD_OK;
}

const char* hsad_status_string(int s) {
  switch (s) {
    case HSAD_OK: return "HSAD_OK";
    case HSAD_E_INVALID: return "HSAD_E_INVALID";
    case HSAD_E_NOMEM: return "HSAD_E_NOMEM";
    case HSAD_E_NOT_READY: return "HSAD_E_NOT_READY";
    case HSAD_E_NOT_PD: return "HSAD_E_NOT_PD";
    case HSAD_E_TIMEOUT: return "HSAD_E_TIMEOUT";
    case HSAD_E_CUDA: return "HSAD_E_CUDA";
    case HSAD_E_BUSY: return "HSAD_E_BUSY";
    case HSAD_E_INVALID_DATA: return "HSAD_E_INVALID_DATA";
    default: return "unknown status";
  }
}

int hsad_config_init(hsad_config* cfg) {
  if (!cfg) return HSAD_E_INVALID;
  memset(cfg, 0, sizeof(*cfg));
  cfg->in_dtype = HSAD_U16;
  cfg->precision = HSAD_FP32;
  cfg->stats_mode = HSAD_EXCLUSIVE;
  cfg->threshold_mode = HSAD_ABS;
  return HSAD_OK;
}

int hsad_set_device_budget(int device, int64_t bytes) {
  if (bytes < 0) return HSAD_E_INVALID;
  std::lock_guard<std::mutex> g(budget().mu);
  budget().limit[device] = bytes;
  return HSAD_OK;
}

int64_t hsad_device_budget_used(int device) {
  std::lock_guard<std::mutex> g(budget().mu);
  return budget().used[device];
}

int hsad_create(const hsad_config* cfg, hsad_ctx** out) {
  hsad_ctx* ctx = nullptr;
  if (!out) return fail(nullptr, HSAD_E_INVALID, "out is NULL");
  *out = nullptr;
  std::string why;
  if (validate(cfg, &why) != HSAD_OK) return fail(nullptr, HSAD_E_INVALID, why);
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= 0) {
    cudaGetLastError();
    return fail(nullptr, HSAD_E_CUDA, "no CUDA device");
  }
  if (cfg->device < 0 || cfg->device >= ndev) return fail(nullptr, HSAD_E_INVALID, "device ordinal out of range");

  ctx = new hsad_ctx();
  ctx->cfg = *cfg;
  ctx->cfg.gain = nullptr;
  ctx->cfg.offset = nullptr;
  ctx->device = cfg->device;
  ctx->W = cfg->width;
  ctx->B = cfg->bands;
  ctx->Bp = pad64(cfg->bands);
  ctx->in_type = cfg->in_dtype == HSAD_U16 ? IN_U16 : IN_F32;
  const bool cube = cfg->stats_mode == HSAD_CUBE;
  const bool force_inverse = (cfg->flags & HSAD_FORCE_INVERSE) != 0;
  ctx->prec = cfg->precision == HSAD_FP32
                  ? fp32_form(ctx->B, ctx->in_type, cube, force_inverse, cfg->factor_precision == HSAD_FACTOR_FF)
              : cfg->precision == HSAD_BF16 ? bf16_form(ctx->B, ctx->in_type, cube, force_inverse)
                                            : P_FP16;
  ctx->fprec = ctx->prec | (cfg->factor_precision == HSAD_FACTOR_FP64 ? kFactorF64 : 0);
  ctx->tc_factor = !cube && cfg->factor_precision == HSAD_FACTOR_FF && factor_tc_supported(ctx->B, ctx->prec);
  ctx->lam = (cfg->forget > 0.f && cfg->forget < 1.f) ? (double)cfg->forget : 1.0;
  ctx->use_graphs = (cfg->flags & HSAD_CUDA_GRAPHS) && cfg->stats_mode == HSAD_EXCLUSIVE && ctx->lam == 1.0;
  ctx->mode = cfg->stats_mode;
  ctx->elem = ctx->in_type == IN_U16 ? 2 : 4;
  ctx->line_elems = (int64_t)ctx->W * ctx->B;
  ctx->line_bytes = ctx->line_elems * ctx->elem;
  ctx->fe = cfg->raw_bands > 0;
  ctx->every = cfg->factor_every > 1 ? cfg->factor_every : 1;
  ctx->raw_line_bytes = ctx->fe ? (int64_t)ctx->W * cfg->raw_bands * 2 : ctx->line_bytes;
  // sums of bin 12-bit DN: |x'| < 2^(12 + ceil(log2 bin)); an exact accumulation holds
  // 2^24 / (|x'| / 64)^2 pixels: 4096 (bin 1), 1024 (bin 2), 256 (bin 3, 4)
  if (ctx->fe) ctx->syrk_max_pix = cfg->band_bin == 1 ? 4096 : (cfg->band_bin == 2 ? 1024 : 256);
  ctx->split_syrk = cfg->stats_mode != HSAD_CUBE && ctx->in_type == IN_U16 && ctx->W <= ctx->syrk_max_pix;
  ctx->min_pix = std::max<int64_t>((int64_t)ctx->B + 1, cfg->warmup_pixels);
  ctx->tau = cfg->threshold > 0.f
                 ? cfg->threshold
                 : (cfg->threshold_mode == HSAD_ABS ? (float)(ctx->B + 6.0 * std::sqrt(2.0 * ctx->B)) : 0.f);
  ctx->cfg.threshold = ctx->tau;
  ctx->Lmax = cfg->max_batch_lines > 0 ? cfg->max_batch_lines : 256;
  {
    int64_t r = cfg->result_lines > 0 ? cfg->result_lines : std::max<int64_t>(4096, 2 * (int64_t)ctx->Lmax);
    if (ctx->mode == HSAD_CUBE) r = std::max<int64_t>(r, 2 * (int64_t)cfg->cube_lines);
    ctx->ring = r;
  }
  DeviceGuard dg(ctx->device);

  // admission
  const int64_t need = plan_bytes(ctx);
  if (cfg->device_budget_bytes > 0 && need > cfg->device_budget_bytes) {
    delete ctx;
    return fail(nullptr, HSAD_E_NOMEM, "context needs " + std::to_string(need) + " bytes, above its budget");
  }
  {
    const auto t0 = Clock::now();
    for (;;) {
      std::unique_lock<std::mutex> g(budget().mu);
      const int64_t lim = budget().limit.count(ctx->device) ? budget().limit[ctx->device] : 0;
      const int64_t used = budget().used[ctx->device];
      if (lim == 0 || used + need <= lim) {
        budget().used[ctx->device] += need;
        ctx->budget_charged = true;
        ctx->charged = need;
        break;
      }
      g.unlock();
      if (need > lim) {
        delete ctx;
        return fail(nullptr, HSAD_E_NOMEM, "context larger than the device budget");
      }
      if (!(cfg->flags & HSAD_CREATE_WAIT) ||
          std::chrono::duration_cast<std::chrono::milliseconds>(Clock::now() - t0).count() > 10000) {
        delete ctx;
        return fail(nullptr, HSAD_E_BUSY, "device budget exhausted; retry when contexts are released");
      }
      std::this_thread::sleep_for(std::chrono::milliseconds(1));
    }
  }
  // the charge is recorded as dev_bytes once allocated; start from the planned amount
  const int64_t charged = need;

  bool ok = true;
  if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&ctx->h2d_stream, cudaStreamNonBlocking) != cudaSuccess) {
    ok = false;
  }
  const int64_t B = ctx->B, Bp = ctx->Bp, L = ctx->Lmax;
  const int64_t Lf = ctx->mode == HSAD_CUBE ? 1 : (ctx->mode == HSAD_EXCLUSIVE ? L + 1 : L);
  const int64_t Ls = ctx->mode == HSAD_CUBE ? cfg->cube_lines : L;
  ctx->c_int = (int32_t*)dalloc(ctx, B * 4, &ok);
  ctx->c_flt = (float*)dalloc(ctx, B * 4, &ok);
  ctx->state_s1 = (double*)dalloc(ctx, B * 8, &ok);
  ctx->state_s2 = (double*)dalloc(ctx, B * B * 8, &ok);
  ctx->s1_line = (double*)dalloc(ctx, Ls * B * 8, &ok);
  if (ctx->lam != 1.0) ctx->d_nline = (double*)dalloc(ctx, Ls * 8, &ok);
  ctx->m_line = (double*)dalloc(ctx, Ls * B * 8, &ok);
  ctx->sigma = (double*)dalloc(ctx, Lf * B * B * 8, &ok);
  ctx->inv = (double*)dalloc(ctx, Lf * B * B * 8, &ok);
  ctx->wmat = dalloc(ctx, Lf * Bp * Bp * wmat_elem_bytes(ctx->prec), &ok);
  if (ctx->prec == P_FP32T) ctx->yscratch = (float*)dalloc(ctx, (int64_t)whiten_trsm_simt_scratch_bytes(B), &ok);
  if (ctx->split_syrk) ctx->hr = (uint8_t*)dalloc(ctx, (int64_t)syrk_split_bytes(L, ctx->W, ctx->B), &ok);
  if (ctx->tc_factor) ctx->ffm = (float2*)dalloc(ctx, (int64_t)tcf_form_scratch_bytes((int)Lf, ctx->B), &ok);
  ctx->y0 = (float*)dalloc(ctx, Lf * Bp * 4, &ok);
  ctx->inv_s2 = (float*)dalloc(ctx, Lf * 4, &ok);
  ctx->status = (int32_t*)dalloc(ctx, std::max(Ls, Lf) * 4, &ok);
  ctx->dmax_bits = (unsigned int*)dalloc(ctx, 64, &ok);
  ctx->bdesc = (int64_t*)dalloc(ctx, 16, &ok);
  ctx->bad_flag = (int32_t*)((char*)ctx->dmax_bits + 32);
  ctx->dev_err = (int32_t*)((char*)ctx->dmax_bits + 48);
  ctx->r_scores = (float*)dalloc(ctx, ctx->ring * ctx->W * 4, &ok);
  ctx->r_mask = (uint8_t*)dalloc(ctx, ctx->ring * ctx->W, &ok);
  ctx->r_codes = (uint16_t*)dalloc(ctx, ctx->ring * ctx->W * 2, &ok);
  ctx->tx_max = (unsigned int*)dalloc(ctx, 64, &ok);
  ctx->r_status = (int32_t*)dalloc(ctx, ctx->ring * 4, &ok);
  if (ctx->mode == HSAD_CUBE) {
    // the cube buffer is allocated on first use: a device push of one whole cube is
    // scored in place and never needs it (its bytes are charged to the budget anyway)
  } else {
    for (int i = 0; i < 2; ++i) ctx->d_stage[i] = dalloc(ctx, L * ctx->line_bytes, &ok);
  }
  if (ctx->fe) {
    ctx->d_raw = dalloc(ctx, L * ctx->raw_line_bytes, &ok);
    for (int i = 0; i < 2; ++i) ctx->d_bin[i] = dalloc(ctx, L * ctx->line_bytes, &ok);
  }
  for (int i = 0; i < 2 && ok; ++i) {
    void* h = nullptr;
    const int64_t hb = (ctx->mode == HSAD_CUBE ? std::min<int64_t>(L, cfg->cube_lines) : L) * ctx->line_bytes;
    if (cudaHostAlloc(&h, (size_t)hb, cudaHostAllocDefault) != cudaSuccess) ok = false;
    else ctx->host_allocs.push_back(h);
    ctx->h_stage[i] = h;
    if (cudaEventCreateWithFlags(&ctx->stage_ev[i], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->copy_ev[i], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->free_ev[i], cudaEventDisableTiming) != cudaSuccess)
      ok = false;
  }
  if (ok) {
    void* h = nullptr;
    if (cudaHostAlloc(&h, 64, cudaHostAllocDefault) != cudaSuccess) ok = false;
    else ctx->host_allocs.push_back(h);
    ctx->h_small = (int32_t*)h;
  }
  ctx->charged = charged;  // released as charged, whatever is allocated later
  if (!ok) {
    cudaGetLastError();
    release(ctx);
    return fail(nullptr, HSAD_E_NOMEM, "device allocation failed");
  }
  // the calibration gain and offset cancel from Eq. 1 (RX is invariant under a per-band
  // affine map): validated above, not needed on the device
  // the tensor-core factor writes only the lower part of the whitening operand and never the
  // zero padding rows of its digit planes: both start (and stay) zero
  if (ctx->tc_factor && (cudaMemsetAsync(ctx->wmat, 0, (size_t)Lf * Bp * Bp * wmat_elem_bytes(ctx->prec),
                                         ctx->stream) != cudaSuccess ||
                         cudaMemsetAsync(ctx->inv, 0, (size_t)Lf * B * B * 8, ctx->stream) != cudaSuccess)) {
    cudaGetLastError();
    release(ctx);
    return fail(nullptr, HSAD_E_CUDA, "device initialisation failed");
  }
  if (cudaMemsetAsync(ctx->state_s1, 0, B * 8, ctx->stream) != cudaSuccess ||
      cudaMemsetAsync(ctx->state_s2, 0, B * B * 8, ctx->stream) != cudaSuccess ||
      cudaMemsetAsync(ctx->r_status, 0xff, ctx->ring * 4, ctx->stream) != cudaSuccess ||
      cudaMemsetAsync(ctx->dmax_bits, 0, 64, ctx->stream) != cudaSuccess ||
      cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
    cudaGetLastError();
    release(ctx);
    return fail(nullptr, HSAD_E_CUDA, "device initialisation failed");
  }
  if (ctx->prec == P_BF16 || ctx->prec == P_FP16 || ctx->prec == P_BF16T || ctx->prec == P_FP32X) {
    // G (H) planes [Lf][2 or 3][Bp][Bp] 16-bit as a 2-D tensor of Lf*planes*Bp rows, 64 x 64
    // boxes (the inverse form: 128-row boxes)
    const int64_t rows = Lf * (ctx->prec == P_FP32X ? 3 : 2) * Bp;
    if (!encode_gmap(&ctx->gmap, ctx->wmat, Bp, rows, trsm_planes(ctx->prec) ? 64 : 128)) {
      release(ctx);
      return fail(nullptr, HSAD_E_CUDA, "cuTensorMapEncodeTiled failed for the whitening operand");
    }
    ctx->have_gmap = true;
  }
  factor_prepare(ctx->B, ctx->fprec);  // cluster capacities: off the first line's latency path
  cudaGetLastError();
  *out = ctx;
  return HSAD_OK;
}

}  // extern "C"

// ------------------------------------------------------------------------------ engine
namespace {

ScoreOut score_out(hsad_ctx* ctx, uint64_t first_line, bool write_mask) {
  ScoreOut o;
  o.scores = ctx->r_scores;
  o.mask = ctx->r_mask;
  o.ring_status = ctx->r_status;
  o.slot0 = (int64_t)(first_line % (uint64_t)ctx->ring);
  o.ring = ctx->ring;
  o.tau = ctx->tau;
  o.write_mask = write_mask ? 1 : 0;
  return o;
}

int add_record(hsad_ctx* ctx, uint64_t first, uint64_t n) {
  cudaEvent_t ev = get_event(ctx);
  if (!ev) return fail(ctx, HSAD_E_CUDA, "event creation failed");
  CK(cudaEventRecord(ev, ctx->stream));
  ctx->records.push_back({first, n, ev});
  // drop records whose lines have left the ring
  while (!ctx->records.empty()) {
    const Record& r = ctx->records.front();
    if (r.first + r.n + (uint64_t)ctx->ring > ctx->next_line) break;
    if (cudaEventQuery(r.ev) != cudaSuccess) break;
    ctx->event_pool.push_back(r.ev);
    ctx->records.pop_front();
  }
  return HSAD_OK;
}

// K6: tensor cores (tcgen05, G by TMA) for the FP16 / BF16 forms, FFMA for FP32.
// gain_off: with a gain-corrected batch, the index of the launch's first line among the
// batch's gains.
int whiten(hsad_ctx* ctx, const void* x, int L, int factor_stride, ScoreOut o, int gain_off = 0) {
  cudaStream_t st = ctx->stream;
  if (ctx->batch_gain) {
    if (!is_trsm(ctx->prec)) return fail(ctx, HSAD_E_INVALID, "gains need the triangular-solve form");
    KL("gain_mean", launch_gain_mean(ctx->d_gain_cur + (size_t)kGainStride * gain_off, L, ctx->B, ctx->y0, ctx->c_int, factor_stride, o,
                                     ctx->d_mgain, ctx->d_gscale, st, &ctx->lc));
    o.m_line = ctx->d_mgain;
    o.line_scale = ctx->d_gscale;
  }
  if (trsm_planes(ctx->prec)) {
    KL("whiten_score", launch_whiten_trsm((const uint16_t*)x, L, ctx->W, ctx->B, ctx->prec, ctx->c_int, &ctx->gmap,
                                          ctx->y0, ctx->inv_s2, ctx->status, factor_stride, o, ctx->dev_err, st,
                                          &ctx->lc));
  } else if (ctx->prec == P_FP32T) {
    KL("whiten_score", launch_whiten_trsm_simt(x, L, ctx->W, ctx->B, ctx->in_type, ctx->c_int, ctx->c_flt,
                                               (const float*)ctx->wmat, ctx->y0, ctx->inv_s2, ctx->status,
                                               factor_stride, o, ctx->yscratch, st, &ctx->lc));
  } else if (ctx->prec != P_FP32) {
    KL("whiten_score", launch_whiten_tc(x, L, ctx->W, ctx->B, ctx->in_type, ctx->c_int, ctx->c_flt, ctx->prec,
                                        &ctx->gmap, ctx->y0, ctx->inv_s2, ctx->status, factor_stride, o,
                                        ctx->dev_err, st, &ctx->lc));
  } else {
    KL("whiten_score", launch_whiten_score_simt(x, L, ctx->W, ctx->B, ctx->in_type, ctx->c_int, ctx->c_flt,
                                                ctx->prec, ctx->wmat, ctx->y0, ctx->inv_s2, ctx->status,
                                                factor_stride, o, st, &ctx->lc));
  }
  return HSAD_OK;
}

// K2: exact covariance sums of n_groups groups of pix pixels into out (lower triangle).
// uint16 input runs on the tensor cores (integer split, exact); float input accumulates
// FP32 x FP32 products in FP64 on the SIMT cores.
// Whether syrk() takes the split path for n_groups lines of pix pixels (which also forms the
// lines' band sums, so that the column-sum launch is skipped).
bool syrk_split_path(const hsad_ctx* ctx, int64_t n_groups, int64_t pix, bool accumulate) {
  return ctx->in_type == IN_U16 && ctx->split_syrk && !accumulate && pix == ctx->W && n_groups <= ctx->Lmax;
}

// K1b + K2 for a batch of streamed lines: the per-line band sums (s1) and the exact covariance
// sums, in one pass over the lines where the split path applies.
int syrk(hsad_ctx* ctx, const void* x, int64_t n_groups, int64_t pix, double* out, int64_t out_stride,
         bool accumulate, double* s1 = nullptr) {
  cudaStream_t st = ctx->stream;
  if (syrk_split_path(ctx, n_groups, pix, accumulate)) {
    // streamed lines: each line's DN split once (band sums on the way), then one contraction
    // per block pair
    KL("syrk_split", launch_syrk_split((const uint16_t*)x, n_groups, pix, ctx->B, ctx->c_int, ctx->hr, s1, st,
                                       &ctx->lc));
    KL("syrk", launch_syrk_pre(ctx->hr, n_groups, pix, ctx->B, out, out_stride, ctx->dev_err, st, &ctx->lc));
  } else if (ctx->in_type == IN_U16) {
    bool acc = accumulate;
    if (!acc && pix > ctx->syrk_max_pix) {  // exactness bound of one accumulation: add slices atomically
      CK(cudaMemsetAsync(out, 0, (size_t)(n_groups * out_stride * 8), st));
      acc = true;
    }
    KL("syrk", launch_syrk_tc((const uint16_t*)x, n_groups, pix, ctx->B, ctx->c_int, out, out_stride, acc ? 1 : 0,
                              ctx->dev_err, st, &ctx->lc, ctx->syrk_max_pix));
  } else {
    KL("syrk", launch_syrk_simt(x, n_groups, pix, ctx->B, ctx->in_type, ctx->c_int, ctx->c_flt, out, out_stride,
                                accumulate ? 1 : 0, st, &ctx->lc));
  }
  return HSAD_OK;
}

// The factor of L lines of streamed statistics: the tensor-core factor where the context
// uses it, else the factor kernel (same output layout; the choice depends only on the
// context, so a line's factor does not depend on how lines are batched).
int factor_lines(hsad_ctx* ctx, double* sigma, double* inv, const double* m, int L, void* wmat, float* y0,
                 float* inv_s2, int32_t* status, int64_t n0, int W, int incl, const int64_t* n0_dev, int every,
                 int q_off, const double* n_line, bool formed = false) {
  if (ctx->tc_factor) {
    static const char* names[4] = {"factor_form", "factor_diag", "factor_panel", "factor_update"};
    for (int s = formed ? 1 : 0; s < factor_tc_steps(ctx->B); ++s)
      KL(names[factor_tc_step_kind(s)],
         launch_factor_tc_step(s, sigma, inv, m, L, ctx->B, ctx->prec, wmat, y0, inv_s2, status, n0, W, incl,
                               ctx->stream, &ctx->lc, n0_dev, every, q_off, n_line, ctx->dev_err));
    return HSAD_OK;
  }
  KL("factor", launch_factor(sigma, inv, m, L, ctx->B, ctx->fprec, wmat, y0, inv_s2, status, n0, W, incl,
                             ctx->stream, &ctx->lc, n0_dev, every, q_off, n_line));
  return HSAD_OK;
}

// Everything of an EXCLUSIVE batch after its first line is scored: the batch's statistics,
// the factors of slots 1..L, the scores of lines 1..L-1 and the carry of slot L to slot 0.
// With dev = true the per-batch values (pixels before the batch, ring slot of line 1) are
// read from ctx->bdesc at run time, so that the launches can be captured once and replayed.
int excl_tail(hsad_ctx* ctx, const void* x, int L, uint64_t first, bool dev) {
  const int W = ctx->W, B = ctx->B, Bp = ctx->Bp;
  // cadence phase of the batch's first line: slot j (statistics through line first + j - 1)
  // is a snapshot iff (q0 + j) % every == 0
  const int q0 = (int)((ctx->n_stats / W) % ctx->every);
  const int64_t BB = (int64_t)B * B;
  cudaStream_t st = ctx->stream;
  const int64_t* n0_dev = dev ? ctx->bdesc : nullptr;
  CK(cudaMemsetAsync(ctx->status + 1, 0, (size_t)L * 4, st));
  {
    const bool fused = syrk_split_path(ctx, L, W, false);
    if (!fused)
      KL("colsum", launch_colsum(x, L, W, B, ctx->in_type, ctx->c_int, ctx->c_flt, ctx->s1_line, st, &ctx->lc));
    int rc = syrk(ctx, x, L, W, ctx->sigma + BB, BB, false, fused ? ctx->s1_line : nullptr);
    if (rc != HSAD_OK) return rc;
  }
  const double* gain = ctx->batch_gain ? ctx->d_gain_cur : nullptr;
  const double* n_line = ctx->lam != 1.0 ? ctx->d_nline : nullptr;
  if (n_line) KL("forget_n", launch_forget_n(ctx->n_eff, ctx->lam, W, L, 1, ctx->d_nline, st, &ctx->lc));
  KL("prefix_mean", launch_prefix_mean(ctx->s1_line, ctx->m_line, ctx->state_s1, ctx->n_stats, W, L, B, 1,
                                       ctx->min_pix, ctx->status + 1, st, &ctx->lc, n0_dev, gain, ctx->c_int,
                                       ctx->lam, n_line));
  // the tensor-core factor takes its covariances formed in the prefix pass (integer sums only)
  const bool fused = ctx->tc_factor && !gain && !n_line;
  if (fused) {
    KL("prefix_cov", launch_tcf_prefix_form(ctx->sigma + BB, ctx->state_s2, L, B, 1, ctx->m_line, ctx->n_stats, W,
                                            1, n0_dev, ctx->ffm, st, &ctx->lc));
  } else {
    KL("prefix_cov", launch_prefix_cov(ctx->sigma + BB, ctx->state_s2, L, B, 1, st, &ctx->lc, gain, ctx->s1_line,
                                       ctx->c_int, W, ctx->lam));
  }
  {
    const int rc_f = factor_lines(ctx, ctx->sigma + BB, ctx->inv + BB, ctx->m_line, L,
                                  (char*)ctx->wmat + (size_t)Bp * Bp * wmat_elem_bytes(ctx->prec), ctx->y0 + Bp,
                                  ctx->inv_s2 + 1, ctx->status + 1, ctx->n_stats, W, 1, n0_dev, ctx->every, q0 + 1,
                                  n_line, fused);
    if (rc_f != HSAD_OK) return rc_f;
  }
  if (L > 1) {
    ScoreOut o1 = score_out(ctx, first + 1, true);
    o1.factor_base = 1;
    o1.every = ctx->every;
    o1.q0 = q0;
    if (dev) o1.slot0_dev = ctx->bdesc + 1;
    int rc = whiten(ctx, (const char*)x + ctx->line_bytes, L - 1, 1, o1, 1);
    if (rc != HSAD_OK) return rc;
  }
  // carry the factor of the last snapshot to slot 0 (every line: slot L, the statistics of all
  // lines so far; with a cadence the last snapshot slot of the batch, or slot 0 unchanged if
  // the batch holds none)
  const int c = L - (q0 + L) % ctx->every;
  if (c > 0) {
    const size_t wb = (size_t)Bp * Bp * wmat_elem_bytes(ctx->prec);
    CK(cudaMemcpyAsync(ctx->wmat, (char*)ctx->wmat + (size_t)c * wb, wb, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(ctx->y0, ctx->y0 + (size_t)c * Bp, (size_t)Bp * 4, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(ctx->inv_s2, ctx->inv_s2 + c, 4, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(ctx->status, ctx->status + c, 4, cudaMemcpyDeviceToDevice, st));
  }
  return HSAD_OK;
}

constexpr int kGraphMaxLines = 8;

// The replayable graph of excl_tail for (L, staging buffer s), captured on first use.
// Returns nullptr if capture or instantiation fails (the caller then launches directly).
hsad_ctx::GraphEntry* excl_graph(hsad_ctx* ctx, const void* x, int L, int s, uint64_t first) {
  // the cadence phase fixes which slots are factored and carried: part of the key
  const int q0 = (int)((ctx->n_stats / ctx->W) % ctx->every);
  auto key = std::make_pair(L, s + 2 * q0);
  auto it = ctx->graphs.find(key);
  if (it != ctx->graphs.end()) return it->second.exec ? &it->second : nullptr;
  hsad_ctx::GraphEntry ge;
  cudaGraph_t graph = nullptr;
  const int64_t lc0 = ctx->lc.n;
  if (cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
    const int rc = excl_tail(ctx, x, L, first, true);
    const cudaError_t e = cudaStreamEndCapture(ctx->stream, &graph);
    if (rc == HSAD_OK && e == cudaSuccess && graph) {
      if (cudaGraphInstantiate(&ge.exec, graph, 0) != cudaSuccess) ge.exec = nullptr;
    }
    if (graph) cudaGraphDestroy(graph);
  }
  ge.launches = ctx->lc.n - lc0;
  ctx->lc.n = lc0;  // captured, not launched
  cudaGetLastError();
  ctx->failed = false;  // a failed capture launched nothing; the batch runs directly
  ctx->err.clear();
  auto& slot = ctx->graphs[key];
  slot = ge;
  return slot.exec ? &slot : nullptr;
}

// One EXCLUSIVE batch (Sec. 6.1 line-based form) of L lines starting at line `first`.
// Line t is scored against the statistics of lines [r, t). Pipelining: slot 0 holds the
// factor of all statistics before the batch, so the batch's first line is scored before
// anything else and its scores become readable at once; the batch's own statistics then
// give the factors of slots 1..L (slot k: lines before line k of the batch), lines 1..L-1
// are scored with slots 1..L-1, and slot L is carried to slot 0 for the next batch.
int stream_batch_excl(hsad_ctx* ctx, const void* x, int L, uint64_t first) {
  const int W = ctx->W, B = ctx->B;
  cudaStream_t st = ctx->stream;
  if (ctx->n_stats == 0) {  // no statistics before this line: not ready
    CK(cudaMemsetAsync(ctx->status, 0, 4, st));
    CK(cudaMemsetAsync(ctx->status, LS_NOT_READY, 1, st));
    KL("shift_init", launch_shift_init(x, W, B, ctx->in_type, ctx->c_int, ctx->c_flt, st, &ctx->lc));
  }
  {
    ScoreOut o0 = score_out(ctx, first, true);
    int rc = whiten(ctx, x, 1, 1, o0);
    if (rc == HSAD_OK) rc = add_record(ctx, first, 1);
    if (rc != HSAD_OK) return rc;
  }
  const int s = x == ctx->d_stage[0] ? 0 : (x == ctx->d_stage[1] ? 1 : -1);
  hsad_ctx::GraphEntry* ge = nullptr;
  // graphs for small batches only: their launch overhead is what a graph saves, and a
  // backlog (large batches of many sizes) must not turn into a capture per new size
  if (ctx->use_graphs && !ctx->prof_on && !ctx->batch_gain && ctx->n_stats > 0 && s >= 0 && L <= kGraphMaxLines)
    ge = excl_graph(ctx, x, L, s, first);
  if (ge) {
    KL("set_batch_desc", launch_set_batch_desc(ctx->bdesc, ctx->n_stats,
                                               (int64_t)((first + 1) % (uint64_t)ctx->ring), st, &ctx->lc));
    CK(cudaGraphLaunch(ge->exec, st));
    ctx->lc.n += ge->launches;
  } else {
    int rc = excl_tail(ctx, x, L, first, false);
    if (rc != HSAD_OK) return rc;
  }
  if (L > 1) {
    int rc = add_record(ctx, first + 1, (uint64_t)(L - 1));
    if (rc != HSAD_OK) return rc;
  }
  ctx->n_stats += (int64_t)L * W;
  if (ctx->lam != 1.0) ctx->n_eff = forget_weight(ctx->n_eff, ctx->lam, W, L);
  return HSAD_OK;
}

// One batch of L lines of a stream-mode context, all inside one statistics segment.
int stream_batch(hsad_ctx* ctx, const void* x, int L, uint64_t first) {
  const int W = ctx->W, B = ctx->B;
  cudaStream_t st = ctx->stream;
  const int incl = ctx->mode == HSAD_INCLUSIVE ? 1 : 0;
  if (!incl) return stream_batch_excl(ctx, x, L, first);
  if (ctx->n_stats == 0) KL("shift_init", launch_shift_init(x, W, B, ctx->in_type, ctx->c_int, ctx->c_flt, st, &ctx->lc));
  CK(cudaMemsetAsync(ctx->status, 0, (size_t)L * 4, st));
  {
    const bool fused = syrk_split_path(ctx, L, W, false);
    if (!fused)
      KL("colsum", launch_colsum(x, L, W, B, ctx->in_type, ctx->c_int, ctx->c_flt, ctx->s1_line, st, &ctx->lc));
    int rc = syrk(ctx, x, L, W, ctx->sigma, (int64_t)B * B, false, fused ? ctx->s1_line : nullptr);
    if (rc != HSAD_OK) return rc;
  }
  const double* gain = ctx->batch_gain ? ctx->d_gain_cur : nullptr;
  const double* n_line = ctx->lam != 1.0 ? ctx->d_nline : nullptr;
  if (n_line) KL("forget_n", launch_forget_n(ctx->n_eff, ctx->lam, W, L, incl, ctx->d_nline, st, &ctx->lc));
  KL("prefix_mean", launch_prefix_mean(ctx->s1_line, ctx->m_line, ctx->state_s1, ctx->n_stats, W, L, B, incl,
                        ctx->min_pix, ctx->status, st, &ctx->lc, nullptr, gain, ctx->c_int, ctx->lam, n_line));
  const bool fused = ctx->tc_factor && !gain && !n_line;
  if (fused) {
    KL("prefix_cov", launch_tcf_prefix_form(ctx->sigma, ctx->state_s2, L, B, incl, ctx->m_line, ctx->n_stats, W,
                                            incl, nullptr, ctx->ffm, st, &ctx->lc));
  } else {
    KL("prefix_cov", launch_prefix_cov(ctx->sigma, ctx->state_s2, L, B, incl, st, &ctx->lc, gain, ctx->s1_line,
                                       ctx->c_int, W, ctx->lam));
  }
  {
    const int rc_f = factor_lines(ctx, ctx->sigma, ctx->inv, ctx->m_line, L, ctx->wmat, ctx->y0, ctx->inv_s2,
                                  ctx->status, ctx->n_stats, W, incl, nullptr, 1, 0, n_line, fused);
    if (rc_f != HSAD_OK) return rc_f;
  }
  {
    int rc = whiten(ctx, x, L, 1, score_out(ctx, first, true));
    if (rc != HSAD_OK) return rc;
  }
  ctx->n_stats += (int64_t)L * W;
  if (ctx->lam != 1.0) ctx->n_eff = forget_weight(ctx->n_eff, ctx->lam, W, L);
  return add_record(ctx, first, (uint64_t)L);
}

// Score the open cube (lines [cube_first, cube_first + n) held in x).
int cube_score(hsad_ctx* ctx, const void* x, int64_t n) {
  const int W = ctx->W, B = ctx->B;
  cudaStream_t st = ctx->stream;
  const int64_t N = n * W;
  KL("shift_init", launch_shift_init(x, W, B, ctx->in_type, ctx->c_int, ctx->c_flt, st, &ctx->lc));
  CK(cudaMemsetAsync(ctx->state_s1, 0, (size_t)B * 8, st));
  CK(cudaMemsetAsync(ctx->state_s2, 0, (size_t)B * B * 8, st));
  KL("colsum", launch_colsum(x, n, W, B, ctx->in_type, ctx->c_int, ctx->c_flt, ctx->s1_line, st, &ctx->lc));
  CK(cudaMemsetAsync(ctx->status, 0, (size_t)n * 4, st));
  KL("prefix_mean", launch_prefix_mean(ctx->s1_line, ctx->m_line, ctx->state_s1, 0, W, (int)n, B, 1, 0, ctx->status, st,
                        &ctx->lc));
  {
    int rc = syrk(ctx, x, 1, N, ctx->state_s2, 0, true);
    if (rc != HSAD_OK) return rc;
  }
  KL("finalize_cov", launch_finalize_cov(ctx->state_s1, ctx->state_s2, N, B, ctx->sigma, ctx->m_line,
                         ctx->min_pix, ctx->status, st, &ctx->lc));
  KL("factor", launch_factor(ctx->sigma, ctx->inv, ctx->m_line, 1, B, ctx->fprec, ctx->wmat, ctx->y0,
                   ctx->inv_s2, ctx->status, N, 0, 0, st, &ctx->lc));
  const bool rel = ctx->cfg.threshold_mode == HSAD_REL;
  const bool norm = (ctx->cfg.flags & HSAD_NORMALIZE_SCORES) != 0;
  ScoreOut o = score_out(ctx, ctx->cube_first, !(rel || norm));
  {
    int rc = whiten(ctx, x, (int)n, 0, o);
    if (rc != HSAD_OK) return rc;
  }
  if (rel || norm)
    KL("cube_normalize", launch_cube_normalize(o, n, W, rel ? 1 : 0, norm ? 1 : 0, ctx->dmax_bits, st, &ctx->lc));
  const uint64_t first = ctx->cube_first;
  ctx->last_cube_lines = n;
  ctx->cube_first += (uint64_t)n;
  ctx->cube_fill = 0;
  return add_record(ctx, first, (uint64_t)n);
}

bool is_pinned_host_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeHost;
}

bool is_device_ptr(const void* p, int device) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (a.type == cudaMemoryTypeDevice && a.device == device) || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" {

static int push_impl(hsad_ctx* ctx, const void* lines, int64_t n_lines, int32_t mem, const float* gain);
static int push_lines(hsad_ctx* ctx, const void* lines, int64_t n_lines, int32_t mem, uint64_t* first_line_id,
                      const float* gain);

int hsad_push_lines(hsad_ctx* ctx, const void* lines, int64_t n_lines, int32_t mem, uint64_t* first_line_id) {
  return push_lines(ctx, lines, n_lines, mem, first_line_id, nullptr);
}

int hsad_push_lines_gain(hsad_ctx* ctx, const void* lines, const float* line_gain, int64_t n_lines, int32_t mem,
                         uint64_t* first_line_id) {
  if (!ctx) return fail(nullptr, HSAD_E_INVALID, "ctx is NULL");
  if (ctx->failed) return HSAD_E_CUDA;
  if (n_lines < 0) return fail(ctx, HSAD_E_INVALID, "n_lines < 0");
  if (n_lines > 0 && !line_gain) return fail(ctx, HSAD_E_INVALID, "line_gain is NULL");
  if (ctx->mode == HSAD_CUBE) return fail(ctx, HSAD_E_INVALID, "per-line gains need streamed statistics");
  if (ctx->in_type != IN_U16) return fail(ctx, HSAD_E_INVALID, "per-line gains need uint16 input");
  if (!is_trsm(ctx->prec))
    return fail(ctx, HSAD_E_INVALID, "per-line gains need the triangular-solve whitening form (FP32 or BF16)");
  for (int64_t i = 0; i < n_lines; ++i) {
    const float g = line_gain[i];
    if (!(g >= 1.0f / 65536.0f && g <= 65536.0f)) return fail(ctx, HSAD_E_INVALID, "gain outside [2^-16, 2^16]");
  }
  if (n_lines > 0 && !ctx->d_gain) {  // first use: per-batch gain buffers
    DeviceGuard dg(ctx->device);
    bool ok = true;
    const int64_t L = ctx->Lmax;
    ctx->d_gain = (double*)dalloc(ctx, 2 * L * kGainStride * 8, &ok);
    ctx->d_mgain = (float*)dalloc(ctx, L * ctx->Bp * 4, &ok);
    ctx->d_gscale = (float*)dalloc(ctx, L * 4, &ok);
    for (int i = 0; i < 2 && ok; ++i) {
      void* h = nullptr;
      if (cudaHostAlloc(&h, (size_t)L * kGainStride * 8, cudaHostAllocDefault) != cudaSuccess) ok = false;
      else ctx->host_allocs.push_back(h);
      ctx->h_gain[i] = (double*)h;
      if (ok && (cudaEventCreateWithFlags(&ctx->gain_ev[i], cudaEventDisableTiming) != cudaSuccess ||
                 cudaEventCreateWithFlags(&ctx->gfree_ev[i], cudaEventDisableTiming) != cudaSuccess))
        ok = false;
    }
    if (!ok) {
      cudaGetLastError();
      ctx->d_gain = nullptr;  // the partial allocations stay with the context until destroy
      return fail(ctx, HSAD_E_NOMEM, "allocation of the gain buffers failed");
    }
  }
  return push_lines(ctx, lines, n_lines, mem, first_line_id, line_gain);
}

static int push_lines(hsad_ctx* ctx, const void* lines, int64_t n_lines, int32_t mem, uint64_t* first_line_id,
                      const float* gain) {
  if (!ctx) return fail(nullptr, HSAD_E_INVALID, "ctx is NULL");
  if (ctx->failed) return HSAD_E_CUDA;
  if (n_lines < 0) return fail(ctx, HSAD_E_INVALID, "n_lines < 0");
  if (mem != HSAD_HOST && mem != HSAD_DEVICE) return fail(ctx, HSAD_E_INVALID, "mem must be HSAD_HOST or HSAD_DEVICE");
  if (first_line_id) *first_line_id = ctx->next_line;
  if (n_lines == 0) return HSAD_OK;
  if (!lines) return fail(ctx, HSAD_E_INVALID, "lines is NULL");
  if (n_lines > ctx->ring) return fail(ctx, HSAD_E_INVALID, "push larger than the result ring");
  DeviceGuard dg(ctx->device);
  if (mem == HSAD_DEVICE && !is_device_ptr(lines, ctx->device))
    return fail(ctx, HSAD_E_INVALID, "lines is not device memory of this context's device");
  if (mem == HSAD_HOST && is_device_ptr(lines, ctx->device))
    return fail(ctx, HSAD_E_INVALID, "lines is device memory but mem = HSAD_HOST");
  if (!ctx->fe) return push_impl(ctx, lines, n_lines, mem, gain);
  // front end: raw lines to the device (host pushes), binned on the context's stream, then
  // pushed as device lines; chunks of at most Lmax lines alternate between two buffers
  const char* raw = (const char*)lines;
  for (int64_t done = 0; done < n_lines;) {
    const int64_t k = std::min<int64_t>(n_lines - done, ctx->Lmax);
    const void* src = raw + done * ctx->raw_line_bytes;
    if (mem == HSAD_HOST) {
      CK(cudaMemcpyAsync(ctx->d_raw, src, (size_t)(k * ctx->raw_line_bytes), cudaMemcpyHostToDevice, ctx->stream));
      src = ctx->d_raw;
    }
    void* bin = ctx->d_bin[ctx->fe_idx];
    ctx->fe_idx ^= 1;
    KL("frontend", launch_frontend((const uint16_t*)src, k * ctx->W, ctx->cfg.raw_bands, ctx->cfg.band_first,
                                   ctx->cfg.band_bin, ctx->B, (uint16_t*)bin, ctx->stream, &ctx->lc));
    const int rc = push_impl(ctx, bin, k, HSAD_DEVICE, gain ? gain + done : nullptr);
    if (rc != HSAD_OK) return rc;
    done += k;
  }
  // the caller may reuse a host buffer once the copies from it have landed
  if (mem == HSAD_HOST) {
    cudaEvent_t ev = get_event(ctx);
    if (!ev) return fail(ctx, HSAD_E_CUDA, "event creation failed");
    CK(cudaEventRecord(ev, ctx->stream));
    const int rc = wait_event(ctx, ev, 60000);
    ctx->event_pool.push_back(ev);
    if (rc != HSAD_OK) return rc;
  }
  return HSAD_OK;
}

static int push_impl(hsad_ctx* ctx, const void* lines, int64_t n_lines, int32_t mem, const float* gain) {

  // float input: reject non-finite values before anything is enqueued
  if (ctx->in_type == IN_F32) {
    const int64_t n = n_lines * ctx->line_elems;
    if (mem == HSAD_HOST) {
      const float* f = (const float*)lines;
      for (int64_t i = 0; i < n; ++i)
        if (!std::isfinite(f[i])) return fail(ctx, HSAD_E_INVALID_DATA, "non-finite value in float32 push");
    } else {
      CK(cudaMemsetAsync(ctx->bad_flag, 0, 4, ctx->stream));
      KL("check_finite", launch_check_finite((const float*)lines, n, ctx->bad_flag, ctx->stream, &ctx->lc));
      CK(cudaMemcpyAsync(ctx->h_small + 1, ctx->bad_flag, 4, cudaMemcpyDeviceToHost, ctx->stream));
      CK(cudaStreamSynchronize(ctx->stream));
      if (ctx->h_small[1]) return fail(ctx, HSAD_E_INVALID_DATA, "non-finite value in float32 push");
    }
  }

  const char* src = (const char*)lines;
  int64_t done = 0;
  if (ctx->mode == HSAD_CUBE) {
    const int64_t CL = ctx->cfg.cube_lines;
    while (done < n_lines) {
      // zero-copy: a device push that holds one whole cube from its first line
      if (mem == HSAD_DEVICE && ctx->cube_fill == 0 && n_lines - done >= CL) {
        ctx->next_line += (uint64_t)CL;
        int rc = cube_score(ctx, src + done * ctx->line_bytes, CL);
        if (rc != HSAD_OK) return rc;
        done += CL;
        continue;
      }
      const int64_t take = std::min<int64_t>(n_lines - done, CL - ctx->cube_fill);
      if (!ctx->cube_buf) {
        bool ok = true;
        ctx->cube_buf = dalloc(ctx, CL * ctx->line_bytes, &ok);
        if (!ok) return fail(ctx, HSAD_E_NOMEM, "cube buffer allocation failed");
      }
      char* dst = (char*)ctx->cube_buf + ctx->cube_fill * ctx->line_bytes;
      if (mem == HSAD_DEVICE) {
        CK(cudaMemcpyAsync(dst, src + done * ctx->line_bytes, (size_t)(take * ctx->line_bytes),
                           cudaMemcpyDeviceToDevice, ctx->stream));
      } else {
        // through pinned staging, in pieces of the staging size
        const int64_t cap = std::min<int64_t>(ctx->Lmax, CL);
        for (int64_t o = 0; o < take; o += cap) {
          const int64_t k = std::min<int64_t>(cap, take - o);
          const int s = ctx->stage_idx;
          int rc = wait_event(ctx, ctx->stage_ev[s], 10000);
          if (rc != HSAD_OK) return rc == HSAD_E_NOT_READY ? fail(ctx, HSAD_E_TIMEOUT, "staging busy") : rc;
          memcpy(ctx->h_stage[s], src + (done + o) * ctx->line_bytes, (size_t)(k * ctx->line_bytes));
          CK(cudaMemcpyAsync(dst + o * ctx->line_bytes, ctx->h_stage[s], (size_t)(k * ctx->line_bytes),
                             cudaMemcpyHostToDevice, ctx->stream));
          CK(cudaEventRecord(ctx->stage_ev[s], ctx->stream));
          ctx->stage_idx ^= 1;
        }
      }
      ctx->cube_fill += take;
      ctx->next_line += (uint64_t)take;
      done += take;
      if (ctx->cube_fill == CL) {
        int rc = cube_score(ctx, ctx->cube_buf, CL);
        if (rc != HSAD_OK) return rc;
      }
    }
    return HSAD_OK;
  }

  // stream modes: batches of <= Lmax lines, never across a statistics reset
  const int64_t CLr = ctx->cfg.cube_lines;
  const bool pinned = mem == HSAD_HOST && is_pinned_host_ptr(lines);
  cudaEvent_t last_copy = nullptr;
  // A large pinned push is cut so that copies overlap kernels: a first batch of one factor
  // wave (the lines one launch of the factor kernel holds resident: its copy is the only
  // one nothing hides), then batches of as many whole waves as fit in a staging buffer,
  // each copied while the previous batch runs. The statistics are exact, so batch
  // boundaries do not change any score.
  int64_t first_batch = ctx->Lmax, pinned_batch = ctx->Lmax;
  if (pinned) {
    const int64_t wave = factor_wave_lines(ctx->B, ctx->fprec);
    if (wave > 0 && n_lines >= 2 * wave && ctx->Lmax >= 2 * wave) {
      first_batch = wave;
      pinned_batch = ctx->Lmax / wave * wave;
    }
  }
  while (done < n_lines) {
    int64_t take = std::min<int64_t>(n_lines - done, !pinned ? ctx->Lmax : done == 0 ? first_batch : pinned_batch);
    // a remainder that fits the staging buffer joins this batch instead of running alone
    if (pinned && done > 0 && n_lines - done - take > 0 && n_lines - done <= ctx->Lmax) take = n_lines - done;
    if (CLr > 0) {
      const int64_t into = (int64_t)(ctx->next_line % (uint64_t)CLr);
      take = std::min<int64_t>(take, CLr - into);
    }
    // the batch's per-line gain factors into a pinned slot whose previous copy has landed
    int gs = -1;
    double* dg = nullptr;
    if (gain) {
      gs = ctx->gain_idx;
      ctx->gain_idx ^= 1;
      int rc = wait_event(ctx, ctx->gain_ev[gs], 10000);
      if (rc != HSAD_OK) return rc == HSAD_E_NOT_READY ? fail(ctx, HSAD_E_TIMEOUT, "gain staging busy") : rc;
      double* hg = ctx->h_gain[gs];
      for (int64_t i = 0; i < take; ++i) {
        const double gi = (double)gain[done + i];
        hg[kGainStride * i] = gi;
        hg[kGainStride * i + 1] = 1.0 / gi;
        hg[kGainStride * i + 2] = 1.0 / (gi * gi);
        hg[kGainStride * i + 3] = 1.0 - gi;
      }
      dg = ctx->d_gain + (size_t)gs * ctx->Lmax * kGainStride;
    }
    const size_t gbytes = (size_t)take * kGainStride * 8;
    const void* x;
    int s = -1;
    if (mem == HSAD_DEVICE) {
      x = src + done * ctx->line_bytes;
    } else if (pinned) {
      // DMA straight from the caller's pinned buffer, on its own stream, once the batch that
      // last read d_stage[s] is done; the kernels wait for the copy. The gains go first on
      // the same stream (the copy engine runs copies in order: queued on the kernels' stream
      // instead, they would wait behind the next batch's lines).
      s = ctx->stage_idx;
      CK(cudaStreamWaitEvent(ctx->h2d_stream, ctx->free_ev[s], 0));
      if (gain) {
        CK(cudaStreamWaitEvent(ctx->h2d_stream, ctx->gfree_ev[gs], 0));
        CK(cudaMemcpyAsync(dg, ctx->h_gain[gs], gbytes, cudaMemcpyHostToDevice, ctx->h2d_stream));
        CK(cudaEventRecord(ctx->gain_ev[gs], ctx->h2d_stream));
      }
      CK(cudaMemcpyAsync(ctx->d_stage[s], src + done * ctx->line_bytes, (size_t)(take * ctx->line_bytes),
                         cudaMemcpyHostToDevice, ctx->h2d_stream));
      CK(cudaEventRecord(ctx->copy_ev[s], ctx->h2d_stream));
      CK(cudaStreamWaitEvent(ctx->stream, ctx->copy_ev[s], 0));
      last_copy = ctx->copy_ev[s];
      ctx->stage_idx ^= 1;
      x = ctx->d_stage[s];
    } else {
      s = ctx->stage_idx;
      int rc = wait_event(ctx, ctx->stage_ev[s], 10000);
      if (rc != HSAD_OK) return rc == HSAD_E_NOT_READY ? fail(ctx, HSAD_E_TIMEOUT, "staging busy") : rc;
      memcpy(ctx->h_stage[s], src + done * ctx->line_bytes, (size_t)(take * ctx->line_bytes));
      CK(cudaMemcpyAsync(ctx->d_stage[s], ctx->h_stage[s], (size_t)(take * ctx->line_bytes),
                         cudaMemcpyHostToDevice, ctx->stream));
      CK(cudaEventRecord(ctx->stage_ev[s], ctx->stream));
      ctx->stage_idx ^= 1;
      x = ctx->d_stage[s];
    }
    if (gain && !pinned) {  // in order on the kernels' stream
      CK(cudaMemcpyAsync(dg, ctx->h_gain[gs], gbytes, cudaMemcpyHostToDevice, ctx->stream));
      CK(cudaEventRecord(ctx->gain_ev[gs], ctx->stream));
    }
    const uint64_t first = ctx->next_line;
    ctx->next_line += (uint64_t)take;
    ctx->batch_gain = gain != nullptr;
    ctx->d_gain_cur = dg;
    int rc = stream_batch(ctx, x, (int)take, first);
    ctx->batch_gain = false;
    if (rc != HSAD_OK) return rc;
    if (gain) CK(cudaEventRecord(ctx->gfree_ev[gs], ctx->stream));
    if (s >= 0) CK(cudaEventRecord(ctx->free_ev[s], ctx->stream));
    done += take;
    if (CLr > 0 && ctx->next_line % (uint64_t)CLr == 0) {  // statistics reset
      CK(cudaMemsetAsync(ctx->state_s1, 0, (size_t)ctx->B * 8, ctx->stream));
      CK(cudaMemsetAsync(ctx->state_s2, 0, (size_t)ctx->B * ctx->B * 8, ctx->stream));
      ctx->n_stats = 0;
      ctx->n_eff = 0.0;
    }
  }
  // the caller may reuse its buffer once the copies from it have landed
  if (last_copy) {
    const int rc = wait_event(ctx, last_copy, 60000);
    if (rc != HSAD_OK) return rc;
  }
  return HSAD_OK;
}

int hsad_flush(hsad_ctx* ctx) {
  if (!ctx) return fail(nullptr, HSAD_E_INVALID, "ctx is NULL");
  if (ctx->failed) return HSAD_E_CUDA;
  if (ctx->mode != HSAD_CUBE || ctx->cube_fill == 0) return HSAD_OK;
  DeviceGuard dg(ctx->device);
  return cube_score(ctx, ctx->cube_buf, ctx->cube_fill);
}

static int find_ready(hsad_ctx* ctx, uint64_t first, int64_t n, int32_t timeout_ms) {
  if (n <= 0) return HSAD_OK;
  const uint64_t last = first + (uint64_t)n - 1;
  if (last >= ctx->next_line) return fail(ctx, HSAD_E_INVALID, "lines not pushed yet");
  if (first + (uint64_t)ctx->ring < ctx->next_line) return fail(ctx, HSAD_E_INVALID, "lines have left the result ring");
  for (auto it = ctx->records.rbegin(); it != ctx->records.rend(); ++it) {
    if (last >= it->first && last < it->first + it->n) return wait_event(ctx, it->ev, timeout_ms);
  }
  // pushed but not yet scored (the open cube in CUBE mode)
  return HSAD_E_NOT_READY;
}

static int copy_ring(hsad_ctx* ctx, void* dst, const void* ring_base, int64_t elem_bytes, uint64_t first,
                     int64_t n, int32_t mem) {
  const int64_t per_line = (int64_t)ctx->W * elem_bytes;
  const cudaMemcpyKind kind = mem == HSAD_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  int64_t done = 0;
  while (done < n) {
    const int64_t slot = (int64_t)((first + (uint64_t)done) % (uint64_t)ctx->ring);
    const int64_t k = std::min<int64_t>(n - done, ctx->ring - slot);
    CK(cudaMemcpyAsync((char*)dst + done * per_line, (const char*)ring_base + slot * per_line,
                       (size_t)(k * per_line), kind, ctx->copy_stream));
    done += k;
  }
  return HSAD_OK;
}

int hsad_line_status(hsad_ctx* ctx, uint64_t first_line_id, int64_t n_lines, int32_t* status,
                     int32_t timeout_ms) {
  if (!ctx) return fail(nullptr, HSAD_E_INVALID, "ctx is NULL");
  if (ctx->failed) return HSAD_E_CUDA;
  if (n_lines < 0 || (n_lines > 0 && !status)) return fail(ctx, HSAD_E_INVALID, "bad status arguments");
  if (n_lines > ctx->ring) return fail(ctx, HSAD_E_INVALID, "request larger than the result ring");
  DeviceGuard dg(ctx->device);
  int rc = find_ready(ctx, first_line_id, n_lines, timeout_ms);
  if (rc != HSAD_OK) return rc;
  int64_t done = 0;
  while (done < n_lines) {
    const int64_t slot = (int64_t)((first_line_id + (uint64_t)done) % (uint64_t)ctx->ring);
    const int64_t k = std::min<int64_t>(n_lines - done, ctx->ring - slot);
    CK(cudaMemcpyAsync(status + done, ctx->r_status + slot, (size_t)k * 4, cudaMemcpyDeviceToHost,
                       ctx->copy_stream));
    done += k;
  }
  CK(cudaStreamSynchronize(ctx->copy_stream));
  return HSAD_OK;
}

int hsad_scores(hsad_ctx* ctx, uint64_t first_line_id, int64_t n_lines, float* scores, uint8_t* mask,
                int32_t mem, int32_t timeout_ms) {
  if (!ctx) return fail(nullptr, HSAD_E_INVALID, "ctx is NULL");
  if (ctx->failed) return HSAD_E_CUDA;
  if (n_lines < 0) return fail(ctx, HSAD_E_INVALID, "n_lines < 0");
  if (mem != HSAD_HOST && mem != HSAD_DEVICE) return fail(ctx, HSAD_E_INVALID, "mem must be HSAD_HOST or HSAD_DEVICE");
  if (n_lines > ctx->ring) return fail(ctx, HSAD_E_INVALID, "request larger than the result ring");
  if (n_lines == 0) return HSAD_OK;
  DeviceGuard dg(ctx->device);
  int rc = find_ready(ctx, first_line_id, n_lines, timeout_ms);
  if (rc != HSAD_OK) return rc;
  if (scores) {
    rc = copy_ring(ctx, scores, ctx->r_scores, 4, first_line_id, n_lines, mem);
    if (rc != HSAD_OK) return rc;
  }
  if (mask) {
    rc = copy_ring(ctx, mask, ctx->r_mask, 1, first_line_id, n_lines, mem);
    if (rc != HSAD_OK) return rc;
  }
  std::vector<int32_t> st((size_t)n_lines);
  int64_t done = 0;
  while (done < n_lines) {
    const int64_t slot = (int64_t)((first_line_id + (uint64_t)done) % (uint64_t)ctx->ring);
    const int64_t k = std::min<int64_t>(n_lines - done, ctx->ring - slot);
    CK(cudaMemcpyAsync(st.data() + done, ctx->r_status + slot, (size_t)k * 4, cudaMemcpyDeviceToHost,
                       ctx->copy_stream));
    done += k;
  }
  int32_t dev_err = 0;
  CK(cudaMemcpyAsync(&dev_err, ctx->dev_err, 4, cudaMemcpyDeviceToHost, ctx->copy_stream));
  CK(cudaStreamSynchronize(ctx->copy_stream));
  if (dev_err) {
    ctx->failed = true;
    return fail(ctx, HSAD_E_TIMEOUT, "a device-side bounded wait expired; the context is failed");
  }
  bool nr = false, npd = false;
  for (int32_t s : st) {
    if (s == LS_NOT_PD) npd = true;
    else if (s != LS_OK) nr = true;
  }
  if (npd) return fail(ctx, HSAD_E_NOT_PD, "covariance not positive definite for some requested lines");
  if (nr) return HSAD_E_NOT_READY;
  return HSAD_OK;
}

int hsad_scores_tx(hsad_ctx* ctx, uint64_t first_line_id, int64_t n_lines, uint16_t* codes, float* max_score,
                   int32_t mem, int32_t timeout_ms) {
  if (!ctx) return fail(nullptr, HSAD_E_INVALID, "ctx is NULL");
  if (ctx->failed) return HSAD_E_CUDA;
  if (n_lines < 0) return fail(ctx, HSAD_E_INVALID, "n_lines < 0");
  if (mem != HSAD_HOST && mem != HSAD_DEVICE) return fail(ctx, HSAD_E_INVALID, "mem must be HSAD_HOST or HSAD_DEVICE");
  if (n_lines > ctx->ring) return fail(ctx, HSAD_E_INVALID, "request larger than the result ring");
  if (n_lines == 0) return HSAD_OK;
  if (!codes) return fail(ctx, HSAD_E_INVALID, "codes is NULL");
  DeviceGuard dg(ctx->device);
  // the block's scores are final once their batches' events have completed
  int rc = find_ready(ctx, first_line_id, n_lines, timeout_ms);
  if (rc != HSAD_OK) return rc;  // not scored yet (e.g. an open cube), timed out, or invalid  // pushed but unscored (an open cube): nothing to encode yet
  cudaStream_t st = ctx->copy_stream;
  uint16_t* out = mem == HSAD_DEVICE ? codes : ctx->r_codes;
  // the ring segments of the block (at most two: the ring wraps)
  int64_t seg_slot[2], seg_n[2], nseg = 0, done = 0;
  while (done < n_lines) {
    const int64_t slot = (int64_t)((first_line_id + (uint64_t)done) % (uint64_t)ctx->ring);
    const int64_t k = std::min<int64_t>(n_lines - done, ctx->ring - slot);
    seg_slot[nseg] = slot;
    seg_n[nseg++] = k;
    done += k;
  }
  const int64_t W = ctx->W;
  CK(cudaMemsetAsync(ctx->tx_max, 0, sizeof(unsigned int), st));
  for (int i = 0; i < nseg; ++i)
    CK(launch_tx_max(ctx->r_scores + seg_slot[i] * W, seg_n[i] * W, ctx->tx_max, st, &ctx->lc));
  for (int i = 0, o = 0; i < nseg; o += (int)seg_n[i], ++i)
    CK(launch_tx_encode(ctx->r_scores + seg_slot[i] * W, seg_n[i] * W, out + (int64_t)o * W, ctx->tx_max, st,
                        &ctx->lc));
  if (mem == HSAD_HOST)
    CK(cudaMemcpyAsync(codes, out, (size_t)(n_lines * W * 2), cudaMemcpyDeviceToHost, st));
  unsigned int bits = 0;
  CK(cudaMemcpyAsync(&bits, ctx->tx_max, sizeof bits, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (max_score) memcpy(max_score, &bits, sizeof bits);
  // the same status report as hsad_scores for the block's lines
  return hsad_scores(ctx, first_line_id, n_lines, nullptr, nullptr, mem, 0);
}

int hsad_reset(hsad_ctx* ctx) {
  if (!ctx) return fail(nullptr, HSAD_E_INVALID, "ctx is NULL");
  if (ctx->failed) return HSAD_E_CUDA;
  DeviceGuard dg(ctx->device);
  CK(cudaMemsetAsync(ctx->state_s1, 0, (size_t)ctx->B * 8, ctx->stream));
  CK(cudaMemsetAsync(ctx->state_s2, 0, (size_t)ctx->B * ctx->B * 8, ctx->stream));
  CK(cudaMemsetAsync(ctx->r_status, 0xff, (size_t)ctx->ring * 4, ctx->stream));
  // completion events may still be pending; re-recording a pooled event later is fine
  for (auto& r : ctx->records) ctx->event_pool.push_back(r.ev);
  ctx->records.clear();
  ctx->next_line = 0;
  ctx->n_stats = 0;
  ctx->n_eff = 0.0;
  ctx->cube_fill = 0;
  ctx->cube_first = 0;
  ctx->last_cube_lines = 0;
  return HSAD_OK;
}

int hsad_get_stats(hsad_ctx* ctx, int64_t* n_pixels, double* shift, double* s1, double* s2) {
  if (!ctx) return fail(nullptr, HSAD_E_INVALID, "ctx is NULL");
  if (ctx->failed) return HSAD_E_CUDA;
  if (ctx->lam != 1.0) return fail(ctx, HSAD_E_INVALID, "no statistics export with forgetting");
  DeviceGuard dg(ctx->device);
  int rc = hsad_synchronize(ctx, 10000);
  if (rc != HSAD_OK) return rc;
  const int B = ctx->B;
  if (n_pixels) {
    if (ctx->mode == HSAD_CUBE) {
      *n_pixels = ctx->last_cube_lines * ctx->W;
    } else {
      *n_pixels = ctx->n_stats;
    }
  }
  if (shift) {
    if (ctx->in_type == IN_U16) {
      std::vector<int32_t> c(B);
      CK(cudaMemcpy(c.data(), ctx->c_int, (size_t)B * 4, cudaMemcpyDeviceToHost));
      for (int b = 0; b < B; ++b) shift[b] = (double)c[b];
    } else {
      std::vector<float> c(B);
      CK(cudaMemcpy(c.data(), ctx->c_flt, (size_t)B * 4, cudaMemcpyDeviceToHost));
      for (int b = 0; b < B; ++b) shift[b] = (double)c[b];
    }
  }
  if (s1) CK(cudaMemcpy(s1, ctx->state_s1, (size_t)B * 8, cudaMemcpyDeviceToHost));
  if (s2) CK(cudaMemcpy(s2, ctx->state_s2, (size_t)B * B * 8, cudaMemcpyDeviceToHost));
  return HSAD_OK;
}

int hsad_set_stats(hsad_ctx* ctx, int64_t n_pixels, const double* shift, const double* s1, const double* s2) {
  if (!ctx) return fail(nullptr, HSAD_E_INVALID, "ctx is NULL");
  if (ctx->failed) return HSAD_E_CUDA;
  if (ctx->mode == HSAD_CUBE) return fail(ctx, HSAD_E_INVALID, "statistics import is for stream modes");
  if (ctx->lam != 1.0) return fail(ctx, HSAD_E_INVALID, "no statistics import with forgetting");
  if (!shift || !s1 || !s2 || n_pixels < 0) return fail(ctx, HSAD_E_INVALID, "NULL array or negative n_pixels");
  if (ctx->every > 1 && (n_pixels % ctx->W != 0 || (n_pixels / ctx->W) % ctx->every != 0))
    return fail(ctx, HSAD_E_INVALID, "with a factorisation cadence the import must be at a snapshot (lines a multiple of it)");
  if (ctx->next_line != 0 || ctx->n_stats != 0)
    return fail(ctx, HSAD_E_INVALID, "import needs a context with no line pushed since creation or reset");
  const int B = ctx->B;
  DeviceGuard dg(ctx->device);
  cudaStream_t st = ctx->stream;
  if (ctx->in_type == IN_U16) {
    std::vector<int32_t> c(B);
    for (int b = 0; b < B; ++b) {
      if (!(shift[b] >= 0.0 && shift[b] <= 65535.0) || shift[b] != std::floor(shift[b]))
        return fail(ctx, HSAD_E_INVALID, "uint16 shift must hold integers in [0, 65535]");
      c[b] = (int32_t)shift[b];
    }
    CK(cudaMemcpyAsync(ctx->c_int, c.data(), (size_t)B * 4, cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
  } else {
    std::vector<float> c(B);
    for (int b = 0; b < B; ++b) {
      if (!std::isfinite(shift[b])) return fail(ctx, HSAD_E_INVALID, "shift must be finite");
      c[b] = (float)shift[b];
    }
    CK(cudaMemcpyAsync(ctx->c_flt, c.data(), (size_t)B * 4, cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
  }
  CK(cudaMemcpyAsync(ctx->state_s1, s1, (size_t)B * 8, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(ctx->state_s2, s2, (size_t)B * B * 8, cudaMemcpyHostToDevice, st));
  if (ctx->mode == HSAD_EXCLUSIVE && n_pixels > 0) {
    // slot 0: the factor of the imported statistics, as the last batch would have left it
    std::vector<double> m(B);
    for (int b = 0; b < B; ++b) m[b] = s1[b] / (double)n_pixels;
    const int32_t st0 = n_pixels >= ctx->min_pix ? LS_OK : LS_NOT_READY;
    CK(cudaMemcpyAsync(ctx->sigma, s2, (size_t)B * B * 8, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(ctx->m_line, m.data(), (size_t)B * 8, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(ctx->status, &st0, 4, cudaMemcpyHostToDevice, st));
    {
    const int rc_f = factor_lines(ctx, ctx->sigma, ctx->inv, ctx->m_line, 1, ctx->wmat, ctx->y0, ctx->inv_s2,
                                      ctx->status, n_pixels, 0, 0, nullptr, 1, 0, nullptr);
    if (rc_f != HSAD_OK) return rc_f;
  }
    CK(cudaStreamSynchronize(st));  // the host vectors above are copied before they go out of scope
  } else {
    CK(cudaStreamSynchronize(st));
  }
  ctx->n_stats = n_pixels;
  return HSAD_OK;
}

int hsad_synchronize(hsad_ctx* ctx, int32_t timeout_ms) {
  if (!ctx) return fail(nullptr, HSAD_E_INVALID, "ctx is NULL");
  if (ctx->failed) return HSAD_E_CUDA;
  DeviceGuard dg(ctx->device);
  cudaEvent_t ev = get_event(ctx);
  if (!ev) return fail(ctx, HSAD_E_CUDA, "event creation failed");
  CK(cudaEventRecord(ev, ctx->stream));
  int rc = wait_event(ctx, ev, timeout_ms < 0 ? -1 : (timeout_ms == 0 ? 1 : timeout_ms));
  ctx->event_pool.push_back(ev);
  return rc;
}

int hsad_profile_enable(hsad_ctx* ctx, int32_t enable) {
  if (!ctx) return fail(nullptr, HSAD_E_INVALID, "ctx is NULL");
  ctx->prof_on = enable != 0;
  return HSAD_OK;
}

int hsad_profile_read(hsad_ctx* ctx, int32_t index, char* name, int32_t name_len, int64_t* launches,
                      double* total_ms) {
  if (!ctx) return fail(nullptr, HSAD_E_INVALID, "ctx is NULL");
  if (ctx->failed) return HSAD_E_CUDA;
  DeviceGuard dg(ctx->device);
  if (!ctx->prof_pending.empty()) {
    CK(cudaStreamSynchronize(ctx->stream));
    for (auto& p : ctx->prof_pending) {
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, p.a, p.b));
      auto& t = ctx->prof_tot[p.name];
      if (t.first == 0 && t.second == 0.0) ctx->prof_names.push_back(p.name);
      t.first += 1;
      t.second += ms;
      ctx->prof_pool.push_back(p.a);
      ctx->prof_pool.push_back(p.b);
    }
    ctx->prof_pending.clear();
  }
  if (index < 0 || index >= (int32_t)ctx->prof_names.size()) return HSAD_E_INVALID;
  const std::string& nm = ctx->prof_names[index];
  const auto& t = ctx->prof_tot[nm];
  if (name && name_len > 0) {
    strncpy(name, nm.c_str(), (size_t)name_len - 1);
    name[name_len - 1] = 0;
  }
  if (launches) *launches = t.first;
  if (total_ms) *total_ms = t.second;
  return HSAD_OK;
}

int hsad_profile_reset(hsad_ctx* ctx) {
  if (!ctx) return fail(nullptr, HSAD_E_INVALID, "ctx is NULL");
  int64_t l;
  double ms;
  hsad_profile_read(ctx, -1, nullptr, 0, &l, &ms);  // drains pending events
  ctx->prof_tot.clear();
  ctx->prof_names.clear();
  return HSAD_OK;
}

void* hsad_stream(hsad_ctx* ctx) { return ctx ? (void*)ctx->stream : nullptr; }

int64_t hsad_kernel_launches(const hsad_ctx* ctx) { return ctx ? ctx->lc.n : 0; }

int64_t hsad_device_bytes(const hsad_ctx* ctx) { return ctx ? ctx->dev_bytes : 0; }

int hsad_whitening_form(const hsad_ctx* ctx) {
  if (!ctx) return HSAD_E_INVALID;
  return is_trsm(ctx->prec) ? HSAD_FORM_TRIANGULAR_SOLVE : HSAD_FORM_INVERSE;
}

int hsad_whitening_tensor_cores(const hsad_ctx* ctx) {
  if (!ctx) return HSAD_E_INVALID;
  return ctx->prec == P_FP32 || ctx->prec == P_FP32T ? 0 : 1;
}

int hsad_destroy(hsad_ctx* ctx) {
  if (!ctx) return HSAD_OK;
  if (ctx->stream) {
    DeviceGuard dg(ctx->device);
    cudaEvent_t ev = nullptr;
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess) {
      cudaEventRecord(ev, ctx->stream);
      const auto t0 = Clock::now();
      while (cudaEventQuery(ev) == cudaErrorNotReady &&
             std::chrono::duration_cast<std::chrono::milliseconds>(Clock::now() - t0).count() < 10000)
        std::this_thread::sleep_for(std::chrono::microseconds(50));
      cudaEventDestroy(ev);
    }
  }
  release(ctx);
  return HSAD_OK;
}

const char* hsad_last_error(const hsad_ctx* ctx) {
  if (!ctx) return g_thread_error.c_str();
  return ctx->err.c_str();
}

}  // extern "C"
