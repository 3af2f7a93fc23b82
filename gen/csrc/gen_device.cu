// Device-side synthetic push-broom DN generator (input infrastructure only; it computes
// no statistic of the data). Used where cubes are too large to draw on the host.
//
// Same scene model as gen/cubes.py PushbroomScene (materials, illumination, drift,
// offsets, gains come from the host scene object), with two simplifications stated in
// the Python wrapper: shot noise is the normal approximation N(s, q s) of q Poisson(s/q)
// (all expected counts here are in the hundreds or more), and anomalies are isolated
// pixels with probability `anomaly_fraction` (no clusters).
//
// Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), counter =
// (pixel index low, pixel index high, draw block, 0), key = seed; normals by Box-Muller.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

namespace {

struct U4 {
  uint32_t x, y, z, w;
};

__device__ __forceinline__ U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
    const uint32_t hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
    c = U4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
    k0 += W0;
    k1 += W1;
  }
  return c;
}

__device__ __forceinline__ float u01(uint32_t v) { return ((float)(v >> 8) + 0.5f) * (1.0f / 16777216.0f); }

__device__ __forceinline__ void box_muller(uint32_t a, uint32_t b, float& z0, float& z1) {
  const float r = sqrtf(-2.0f * logf(u01(a)));
  float s, c;
  sincospif(2.0f * u01(b), &s, &c);
  z0 = r * c;
  z1 = r * s;
}

struct Scene {
  int W, B, K;                 // pixels per line, bands, materials (<= 8)
  const float* materials;      // [K][B]
  const float* illum;          // [B]
  const float* offset;         // [B]
  const float* q;              // [B] DN per photo-electron
  const float* anomaly;        // [4][B]
  float a[8], b[8], period[8], phase[8], c[8], xfreq[8], xphase[8];
  float amplitude, rho, read_noise, anomaly_fraction;
};

}  // namespace

// One thread per pixel: abundances, reflectance, signal, noise, DN for every band.
__global__ void gen_pushbroom_kernel(Scene s, uint16_t* __restrict__ out, int64_t t0, int64_t n_lines,
                                     uint32_t k0, uint32_t k1) {
  const int64_t npx = n_lines * s.W;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < npx; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = t0 + i / s.W;
    const int x = (int)(i % s.W);
    const uint64_t pix = (uint64_t)t * (uint64_t)s.W + (uint64_t)x;
    // abundances: softmax of drifting logits with per-pixel Gaussian noise
    float w[8];
    U4 r = philox4x32_10(U4{(uint32_t)pix, (uint32_t)(pix >> 32), 0u, 0u}, k0, k1);
    float n[8];
    box_muller(r.x, r.y, n[0], n[1]);
    box_muller(r.z, r.w, n[2], n[3]);
    r = philox4x32_10(U4{(uint32_t)pix, (uint32_t)(pix >> 32), 1u, 0u}, k0, k1);
    box_muller(r.x, r.y, n[4], n[5]);
    box_muller(r.z, r.w, n[6], n[7]);
    float mx = -1e30f;
    for (int k = 0; k < s.K; ++k) {
      w[k] = s.a[k] + s.b[k] * sinf(6.283185307f * (float)t / s.period[k] + s.phase[k]) +
             s.c[k] * sinf(6.283185307f * s.xfreq[k] * (float)x / (float)s.W + s.xphase[k]) + 1.2f * n[k];
      mx = fmaxf(mx, w[k]);
    }
    float sum = 0.f;
    for (int k = 0; k < s.K; ++k) {
      w[k] = expf(w[k] - mx);
      sum += w[k];
    }
    for (int k = 0; k < s.K; ++k) w[k] /= sum;
    r = philox4x32_10(U4{(uint32_t)pix, (uint32_t)(pix >> 32), 2u, 0u}, k0, k1);
    const bool anom = u01(r.x) < s.anomaly_fraction;
    const int aspec = (int)(r.y & 3u);
    const float frac = 0.3f + 0.4f * u01(r.z);
    const float drift = 1.0f + 0.05f * sinf(6.283185307f * (float)t / 2500.0f + s.rho);
    uint16_t* o = out + i * (int64_t)s.B;
    for (int b0 = 0; b0 < s.B; b0 += 2) {
      U4 q4 = philox4x32_10(U4{(uint32_t)pix, (uint32_t)(pix >> 32), 3u + (uint32_t)(b0 >> 1), 0u}, k0, k1);
      float z[4];
      box_muller(q4.x, q4.y, z[0], z[1]);
      box_muller(q4.z, q4.w, z[2], z[3]);
      for (int u = 0; u < 2 && b0 + u < s.B; ++u) {
        const int b = b0 + u;
        float refl = 0.f;
        for (int k = 0; k < s.K; ++k) refl += w[k] * s.materials[k * s.B + b];
        if (anom) refl = (1.f - frac) * refl + frac * s.anomaly[aspec * s.B + b];
        const float sig = s.amplitude * s.illum[b] * refl * drift;
        const float qb = s.q[b];
        const float dn = s.offset[b] + sig + sqrtf(fmaxf(qb * sig, 0.f)) * z[u] + s.read_noise * z[2 + u];
        o[b] = (uint16_t)fminf(fmaxf(rintf(dn), 0.f), 4095.f);
      }
    }
  }
}

extern "C" int hsadgen_pushbroom(const void* scene_params, uint16_t* out, int64_t t0, int64_t n_lines,
                                 uint64_t seed, void* stream) {
  const Scene& s = *(const Scene*)scene_params;
  if (!out || n_lines <= 0 || s.W <= 0 || s.B <= 0 || s.K <= 0 || s.K > 8) return -1;
  const int64_t npx = n_lines * s.W;
  int64_t blocks = (npx + 255) / 256;
  if (blocks > 152 * 32) blocks = 152 * 32;
  gen_pushbroom_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(s, out, t0, n_lines, (uint32_t)seed,
                                                                           (uint32_t)(seed >> 32));
  return cudaGetLastError() == cudaSuccess ? 0 : -6;
}

extern "C" int hsadgen_scene_size(void) { return (int)sizeof(Scene); }
