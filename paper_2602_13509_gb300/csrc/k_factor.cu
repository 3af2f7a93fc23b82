// K4 + K5 host side: launch shapes of the factor kernel (one CTA per line for throughput,
// a thread-block cluster per line for latency), the measured-shape table of the factor
// autotuner, and the dispatch to the kernel instances (factor_kernel.cuh, compiled once
// per arithmetic and working precision from k_factor_inst.cu).
#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <mutex>
#include <tuple>
#include <utility>
#include <vector>

#include "hsad_internal.h"

namespace hsad {

// Entry points of the instance translation units: a<arith>_p<working precision>.
#define HSAD_FACTOR_DECL(S)                                              \
  cudaError_t factor_launch_##S(int cl, int ft, const FactorArgs& a);    \
  int factor_capacity_##S(int cl, size_t smem);                          \
  int factor_wave_slots_##S(int ft, size_t smem);
HSAD_FACTOR_DECL(a0_p0)
HSAD_FACTOR_DECL(a0_p1)
HSAD_FACTOR_DECL(a0_p2)
HSAD_FACTOR_DECL(a0_p3)
HSAD_FACTOR_DECL(a0_p4)
HSAD_FACTOR_DECL(a1_p0)
HSAD_FACTOR_DECL(a1_p1)
HSAD_FACTOR_DECL(a1_p2)
HSAD_FACTOR_DECL(a1_p3)
HSAD_FACTOR_DECL(a1_p4)
#undef HSAD_FACTOR_DECL

namespace {

constexpr int NB_PANEL = 16;  // the kernel's panel width (smem: B x (NB + 1) 8-byte slots)
size_t factor_smem(int B) { return (size_t)B * (NB_PANEL + 1) * sizeof(double); }

struct Instance {
  cudaError_t (*launch)(int, int, const FactorArgs&);
  int (*capacity)(int, size_t);
  int (*wave_slots)(int, size_t);
};
#define HSAD_FACTOR_ENTRY(S) {factor_launch_##S, factor_capacity_##S, factor_wave_slots_##S}
const Instance kInstances[2][5] = {
    {HSAD_FACTOR_ENTRY(a0_p0), HSAD_FACTOR_ENTRY(a0_p1), HSAD_FACTOR_ENTRY(a0_p2), HSAD_FACTOR_ENTRY(a0_p3),
     HSAD_FACTOR_ENTRY(a0_p4)},
    {HSAD_FACTOR_ENTRY(a1_p0), HSAD_FACTOR_ENTRY(a1_p1), HSAD_FACTOR_ENTRY(a1_p2), HSAD_FACTOR_ENTRY(a1_p3),
     HSAD_FACTOR_ENTRY(a1_p4)},
};
#undef HSAD_FACTOR_ENTRY

const Instance& instance(int fprec) {
  const int p = out_prec(fprec);
  return kInstances[(fprec & kFactorF64) ? 1 : 0][(p >= 0 && p <= 4) ? p : 0];
}

// Threads of a one-CTA-per-line factorisation without a measured shape: 128 threads with
// registers for 5 CTAs per SM (code 96; so that one CTA's barrier-bound panel step overlaps
// other CTAs' updates). Measured on 4000 lines of B = 270 against 128 threads at 4 per SM
// and 256 threads at 2 per SM: 14.21, 15.77 and 19.81 ms (float-float).
constexpr int kDefaultThreads = 96;

// CTAs per factorisation without a measured shape. A cluster shortens one factorisation
// (the trailing updates and the inverse are shared; each CTA still factors every
// 16-column panel), so few lines (latency) take the largest cluster of which the device can
// run one per line at once, and many lines (throughput) one CTA each.
int factor_cluster_size(int fprec, int L, size_t smem) {
  const Instance& in = instance(fprec);
  if (L <= in.capacity(16, smem)) return 16;
  if (L <= in.capacity(8, smem)) return 8;
  if (L <= in.capacity(4, smem)) return 4;
  if (L <= in.capacity(2, smem)) return 2;
  return 1;
}

}  // namespace

// Measured launch shapes (hsad_autotune_factor): per (device, factor precision, B) a list
// of (largest batch size of the bucket, cluster size, threads of a one-CTA factorisation).
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
bool tuned_shape(int B, int fprec, int L, int* cl, int* ft) {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> g(tune_mu());
  auto it = tune_table().find(std::make_tuple(dev, fprec, B));
  if (it == tune_table().end() || it->second.empty()) return false;
  for (const auto& t : it->second)
    if (L <= t.max_lines) {
      *cl = t.cl;
      *ft = t.ft;
      return true;
    }
  return false;  // larger than every measured batch: the occupancy rule
}

int factor_wave_lines(int B, int fprec) { return instance(fprec).wave_slots(kDefaultThreads, factor_smem(B)); }

void factor_prepare(int B, int fprec) {
  const size_t smem = factor_smem(B);
  const Instance& in = instance(fprec);
  for (int cl : {16, 8, 4, 2}) in.capacity(cl, smem);
  factor_wave_lines(B, fprec);
}

cudaError_t launch_factor(double* sigma, double* scratch, const double* m, int L, int B, int fprec, void* wmat,
                          float* y0, float* inv_s2, int32_t* status, int64_t n0, int W, int incl, cudaStream_t st,
                          LaunchCounter* lc, const int64_t* n0_dev, int every, int q_off, const double* n_line) {
  if (L <= 0) return cudaSuccess;
  int cl = 0, ft = 0;
  if (!tuned_shape(B, fprec, L, &cl, &ft)) {
    cl = factor_cluster_size(fprec, L, factor_smem(B));
    ft = kDefaultThreads;
  }
  return launch_factor_shape(cl, ft, sigma, scratch, m, L, B, fprec, wmat, y0, inv_s2, status, n0, W, incl, st, lc,
                             n0_dev, every, q_off, n_line);
}

cudaError_t launch_factor_shape(int cl, int ft, double* sigma, double* scratch, const double* m, int L, int B,
                                int fprec, void* wmat, float* y0, float* inv_s2, int32_t* status, int64_t n0,
                                int W, int incl, cudaStream_t st, LaunchCounter* lc, const int64_t* n0_dev,
                                int every, int q_off, const double* n_line) {
  if (L <= 0) return cudaSuccess;
  if ((fprec & 0xff) > P_FP32T) return cudaErrorInvalidValue;  // the three-plane form: tensor-core factor only
  const FactorArgs a{sigma, scratch, m, L, B, wmat, y0, inv_s2, status, n0, W, incl, st, n0_dev, every, q_off,
                     n_line};
  const cudaError_t e = instance(fprec).launch(cl, ft, a);
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
int factor_autotune(int B, int fprec, int max_lines, float* report, int cap) {
  int dev = 0;
  cudaGetDevice(&dev);
  {
    std::lock_guard<std::mutex> g(tune_mu());
    auto it = tune_table().find(std::make_tuple(dev, fprec, B));
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
  const size_t smem = factor_smem(B);
  const Instance& in = instance(fprec);
  for (size_t bi = 0; ok && bi < buckets.size(); ++bi) {
    const int L = buckets[bi];
    std::vector<std::pair<int, int>> cands = {{1, 96}, {1, 128}, {1, 256}};
    for (int c : {2, 4, 8, 16}) {
      const int capc = in.capacity(c, smem);
      if (capc > 0 && L <= 2 * capc) cands.push_back({c, 256});  // larger batches only queue
    }
    TunedShape best{L, 1, 128, 1e30f};
    for (const auto& cf : cands) {
      float tot = 0.f;
      for (int rep = 0; ok && rep < 4; ++rep) {  // one untimed run, then three timed
        tune_identity_kernel<<<256, 256, 0, st>>>(sigma, L, B, 1.0e6);
        ok = cudaMemsetAsync(status, 0, (size_t)L * 4, st) == cudaSuccess;
        cudaEventRecord(e0, st);
        if (launch_factor_shape(cf.first, cf.second, sigma, inv, m, L, B, fprec, wmat, y0, inv_s2, status,
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
    tune_table()[std::make_tuple(dev, fprec, B)] = result;
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
