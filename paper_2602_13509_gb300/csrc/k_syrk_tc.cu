// K2 on the tensor cores: exact covariance rank-k update of uint16 DN with tcgen05.mma.
//
// Sec. 3.3 takes each band as a variable and each pixel as a sample; the covariance
// needs S2 = sum_p x'_p x'_p^T with x' = DN - c (an integer, |x'| <= 4095). Splitting
// x' = 64 h + r with h = rint(x'/64) in [-64, 64] and r in [-32, 32] makes both parts
// exact in BF16, their products exact in FP32, and
//     S2 = 4096 H^T H + 64 (H^T R + R^T H) + R^T R,
// three sums that stay exact in FP32 accumulators (TMEM) for up to 4096 pixels
// (|h h| <= 4096, |h r + r h| <= 4096, |r r| <= 1024 per pixel, all below 2^24 in sum).
// Wider values (binned 12-bit DN: |x'| < 2^14, |h| <= 256, h h <= 2^16) keep the same split,
// exact in BF16, with slices of 2^24 / 2^16 = 256 pixels.
// They are combined exactly (int64) in the epilogue and stored as FP64, so S2 is exact.
//
// One CTA: one 128 x N block (bands i in [i0, i0+128), j in [j0, j0+N), j-block >= i-block)
// of one group of pixels (one line, or a slice of a cube). One warp streams each 64-pixel
// chunk (all bands, contiguous in BIP) into shared memory with a bulk copy when aligned;
// eight converter warps write H and R of both band blocks, transposed to K-major (rows =
// bands, K = pixels) with the 128-byte swizzle; one thread issues 4 MMAs per 16 pixels
// (HH, HR, RH, RR) into three accumulators; converter warps 0-3 then read TMEM (one band
// row each) and store the exact sums to the lower triangle (row j >= column i), or add
// them atomically (cube slices). Every wait is bounded; a timeout sets *err.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "hsad_internal.h"
#include "tc_util.cuh"

namespace hsad {

namespace {
constexpr int SK_M = 128, SK_KC = 64, SK_CONV = 256, SK_THREADS = SK_CONV + 64;
constexpr int SK_MMA_WARP = SK_CONV / 32, SK_COPY_WARP = SK_MMA_WARP + 1;
constexpr uint32_t SK_TILE = SK_M * SK_KC * 2;  // 16 KB: 128 rows x 64 pixels, 16-bit
constexpr uint32_t SK_STAGE = 4 * SK_TILE;      // AH, AR, BH, BR
constexpr uint32_t SK_BARS = 256;
constexpr uint32_t SK_SMEM_MAX = 227 * 1024;
constexpr int SK_MAX_PIX = 4096;                // exactness bound of one accumulation

__host__ __device__ inline uint32_t sk_raw_bytes(int B) { return ((uint32_t)SK_KC * B * 2 + 127) / 128 * 128; }

}  // namespace

__global__ void __launch_bounds__(SK_THREADS, 1) syrk_tc_kernel(const uint16_t* __restrict__ x,
                                                                int64_t pix_per_group, int B,
                                                                const int32_t* __restrict__ c_int,
                                                                double* __restrict__ out, int64_t out_stride,
                                                                int64_t pix_per_slice, int accumulate,
                                                                int32_t* __restrict__ err, long long limit,
                                                                int raw_bufs) {
  // decode the block (ib <= jb) of the upper block triangle
  const int nb = (B + SK_M - 1) / SK_M;
  int tile = blockIdx.x, ib = 0;
  while (tile >= nb - ib) {
    tile -= nb - ib;
    ++ib;
  }
  const int jb = ib + tile;
  const int i0 = ib * SK_M, j0 = jb * SK_M;
  const int N = min(SK_M, ((B - j0) + 15) / 16 * 16);
  const bool diag = ib == jb;
  const int64_t g = blockIdx.y;
  const int64_t p_begin = (int64_t)blockIdx.z * pix_per_slice;
  const int64_t p_end = min(p_begin + pix_per_slice, pix_per_group);
  const int nchunks = (int)((p_end - p_begin + SK_KC - 1) / SK_KC);
  if (nchunks <= 0) return;
  const uint16_t* xg = x + g * pix_per_group * (int64_t)B;

  // shared memory: 2 operand stages | raw_bufs DN chunks of 64 pixels x B | barriers
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = tc::align1024(smem_raw);
  const bool bulk = raw_bufs > 0;
  const uint32_t rawb = sk_raw_bytes(B);
  uint8_t* raw = sm + 2 * SK_STAGE;
  uint64_t* bars = (uint64_t*)(raw + (bulk ? raw_bufs * rawb : 0));
  uint32_t* tslot = (uint32_t*)(bars + 16);
  const uint32_t full = tc::smem_u32(bars), empty = full + 16, d_full = empty + 16;
  const uint32_t rfull = d_full + 8, rempty = rfull + 16;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid == 0) {
    for (int s = 0; s < 2; ++s) {
      tc::mbar_init(full + 8 * s, SK_CONV);
      tc::mbar_init(empty + 8 * s, 1);
      tc::mbar_init(rfull + 8 * s, 1);
      tc::mbar_init(rempty + 8 * s, SK_CONV);
    }
    tc::mbar_init(d_full, 1);
    tc::mbar_init_fence();
  }
  if (warp == SK_MMA_WARP) tc::tmem_alloc(tc::smem_u32(tslot), 512);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = *tslot;
  bool ok = true;

  if (warp == SK_MMA_WARP) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      const uint32_t idesc = tc::idesc_f16(1, SK_M, N);
      for (int c = 0; c < nchunks; ++c) {
        const int s = c & 1;
        if (!tc::mbar_wait(full + 8 * s, (uint32_t)((c >> 1) & 1), limit)) { ok = false; break; }
        tc::fence_after_sync();
        const uint32_t aH = tc::smem_u32(sm + s * SK_STAGE), aR = aH + SK_TILE;
        const uint32_t bH = diag ? aH : aH + 2 * SK_TILE, bR = diag ? aR : aH + 3 * SK_TILE;
#pragma unroll
        for (int ks = 0; ks < SK_KC / 16; ++ks) {
          const uint32_t o = ks * 32, acc = (c > 0 || ks > 0) ? 1u : 0u;
          tc::mma_f16(tbase + 0, tc::desc_sw128(aH + o), tc::desc_sw128(bH + o), idesc, acc);
          tc::mma_f16(tbase + 128, tc::desc_sw128(aH + o), tc::desc_sw128(bR + o), idesc, acc);
          tc::mma_f16(tbase + 128, tc::desc_sw128(aR + o), tc::desc_sw128(bH + o), idesc, 1u);
          tc::mma_f16(tbase + 256, tc::desc_sw128(aR + o), tc::desc_sw128(bR + o), idesc, acc);
        }
        tc::mma_commit(empty + 8 * s);
      }
      tc::mma_commit(d_full);
      if (!ok) atomicExch(err, 1);
      if (!tc::mbar_wait(d_full, 0, limit)) atomicExch(err, 1);
    }
  } else if (warp == SK_COPY_WARP) {
    // ---------------- bulk-copy producer: 64 pixels x all bands per chunk ----------------
    if (lane == 0 && bulk) {
      int issued = 0;
      for (int c = 0; c < nchunks && ok; ++c, ++issued) {
        const int r = c % raw_bufs;
        const uint32_t use = (uint32_t)(c / raw_bufs);
        if (!tc::mbar_wait(rempty + 8 * r, (use & 1) ^ 1, limit)) { ok = false; break; }
        const int64_t pc = p_begin + (int64_t)c * SK_KC;
        const uint32_t bytes = (uint32_t)(min((int64_t)SK_KC, p_end - pc) * B * 2);
        tc::mbar_arrive_expect_tx(rfull + 8 * r, bytes);
        tc::bulk_load(tc::smem_u32(raw + r * rawb), xg + pc * B, bytes, rfull + 8 * r);
      }
      for (int r = 0; r < raw_bufs && r < issued; ++r) {  // every copy landed before exit
        const int last = issued - 1 - ((issued - 1 - r) % raw_bufs);
        if (!tc::mbar_wait(rfull + 8 * r, (uint32_t)((last / raw_bufs) & 1), limit)) ok = false;
      }
      if (!ok) atomicExch(err, 1);
    }
  } else {
    // ---------------- converters ----------------
    // Thread = one band row and 8 consecutive pixels at a time: 8 two-byte loads from the
    // raw chunk (a warp reads 32 consecutive bands of one pixel), then one 16-byte store
    // of H and one of R (8 consecutive K elements of one swizzled row; the 8 rows of an
    // atom land in 8 different bank groups). Off the diagonal the first 128 threads
    // convert the i block (A operands), the others the j block (B operands); on the
    // diagonal both halves convert the i block, half of the pixels each.
    const int row = tid & (SK_M - 1), half = tid >> 7;
    const bool jside = !diag && half == 1;
    const int band = (jside ? j0 : i0) + row;
    const bool valid = band < B && (!jside || row < N);
    // x' = DN - c as an exact float: the bits of 1.5 * 2^23 + x' (|x'| < 2^22) minus 1.5 * 2^23
    const int magic_c = 0x4B400000 - (valid ? c_int[band] : 0);
    const int g_begin = diag ? half * (SK_KC / 16) : 0, g_end = diag ? g_begin + SK_KC / 16 : SK_KC / 8;
    for (int c = 0; c < nchunks; ++c) {
      const int s = c & 1;
      if (!tc::mbar_wait(empty + 8 * s, (uint32_t)(((c >> 1) & 1) ^ 1), limit)) {
        ok = false;
        atomicExch(err, 1);
      }
      uint8_t* OH = sm + s * SK_STAGE + (jside ? 2 * SK_TILE : 0);
      uint8_t* OR = OH + SK_TILE;
      const int64_t pc = p_begin + (int64_t)c * SK_KC;
      const int r = bulk ? c % raw_bufs : 0;
      if (bulk && !tc::mbar_wait(rfull + 8 * r, (uint32_t)((c / raw_bufs) & 1), limit)) {
        ok = false;
        atomicExch(err, 1);
      }
      // the chunk's DN: staged in shared memory by the bulk copy, else read from global (two
      // instantiations, so that the shared path uses shared-memory loads)
      const int npx = (int)min((int64_t)SK_KC, p_end - pc);
      auto convert = [&](auto load, auto full) {  // full: a valid row and a whole chunk
        for (int gi = g_begin; gi < g_end; ++gi) {
          uint32_t hw[4], rw[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            float hv[2], rv[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
              const int k = gi * 8 + 2 * q + u;
              const bool in = decltype(full)::value || (valid && k < npx);
              const int dn = in ? load(k * B + band) : 0;
              const float xv = in ? __int_as_float(magic_c + dn) - 12582912.0f : 0.f;
              // h = rint(x'/64) (round to nearest even, exact: |x'/64| <= 64), r = x' - 64 h
              const float hf = __fmaf_rn(xv, 1.f / 64.f, 12582912.0f) - 12582912.0f;
              hv[u] = hf;
              rv[u] = __fmaf_rn(hf, -64.f, xv);
            }
            // both are small integers, exact in BF16: the BF16 bits are the float's top half
            hw[q] = __byte_perm(__float_as_uint(hv[0]), __float_as_uint(hv[1]), 0x7632);
            rw[q] = __byte_perm(__float_as_uint(rv[0]), __float_as_uint(rv[1]), 0x7632);
          }
          const uint32_t off = tc::sw128_offset(row, gi * 8);
          *(uint4*)(OH + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
          *(uint4*)(OR + off) = make_uint4(rw[0], rw[1], rw[2], rw[3]);
        }
      };
      if (ok) {
        const bool whole = valid && npx == SK_KC;
        if (bulk) {
          const uint16_t* rs = (const uint16_t*)(raw + r * rawb);
          auto ld = [&](int idx) { return (int)rs[idx]; };
          if (whole) convert(ld, std::true_type{});
          else convert(ld, std::false_type{});
        } else {
          const uint16_t* gs = xg + pc * B;
          auto ld = [&](int idx) { return (int)__ldg(gs + idx); };
          if (whole) convert(ld, std::true_type{});
          else convert(ld, std::false_type{});
        }
      }
      tc::fence_proxy_async();
      tc::mbar_arrive(full + 8 * s);
      if (bulk) tc::mbar_arrive(rempty + 8 * r);
    }
    // ---------------- epilogue: exact combination, lower-triangle store ----------------
    const bool dok = tc::mbar_wait(d_full, 0, limit);
    __syncwarp();
    tc::fence_after_sync();
    if (!dok) atomicExch(err, 1);
    const uint32_t taddr = tbase + ((uint32_t)(warp * 32) << 16);
    double* o = out + g * out_stride;
    const int bi = i0 + row;  // warps 0-3: row = TMEM lane = band of the i block
    const bool write = dok && ok && bi < B;
    // TMEM has 128 lanes, one quarter per warp of 0..3: only those warps read it
    for (int c0 = 0; warp < 4 && c0 < N; c0 += 32) {
      float hh[32], xr[32], rr[32];
      __syncwarp();
      tc::tmem_ld32(taddr + (uint32_t)c0, hh);
      tc::tmem_ld32(taddr + 128u + (uint32_t)c0, xr);
      tc::tmem_ld32(taddr + 256u + (uint32_t)c0, rr);
      if (write) {
#pragma unroll
        for (int jj = 0; jj < 32; ++jj) {
          const int gj = j0 + c0 + jj;
          if (c0 + jj < N && gj < B && gj >= bi) {
            // the three sums are exact integers below 2^24: combine them in int64 (integer
            // ALU) and convert once; the FP64 pipe is far slower than the integer one
            const long long iv = ((long long)__float2int_rn(hh[jj]) << 12) +
                                 ((long long)__float2int_rn(xr[jj]) << 6) + (long long)__float2int_rn(rr[jj]);
            const double v = (double)iv;
            double* dst = o + (int64_t)gj * B + bi;
            if (accumulate) atomicAdd(dst, v);
            else *dst = v;
          }
        }
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == SK_MMA_WARP) {
    __syncwarp();
    tc::tmem_dealloc(tbase, 512);
  }
}

cudaError_t launch_syrk_tc(const uint16_t* x, int64_t n_groups, int64_t pix_per_group, int B,
                           const int32_t* c_int, double* out, int64_t out_stride, int accumulate, int32_t* err,
                           cudaStream_t st, LaunchCounter* lc, int64_t max_pix) {
  if (n_groups <= 0 || pix_per_group <= 0) return cudaSuccess;
  if (max_pix < SK_KC || max_pix > SK_MAX_PIX || max_pix % SK_KC) return cudaErrorInvalidValue;
  const int nb = (B + SK_M - 1) / SK_M;
  const int tiles = nb * (nb + 1) / 2;
  int64_t slices = (pix_per_group + max_pix - 1) / max_pix;
  if (slices > 1 && !accumulate) return cudaErrorInvalidValue;  // caller zeroes and accumulates
  if (slices > 65535 || n_groups > 65535) return cudaErrorInvalidValue;
  const int64_t per = slices > 1 ? max_pix : pix_per_group;
  // Bulk copies need 16-byte aligned chunk starts and sizes: the input base, every group
  // start (pix_per_group * B * 2 bytes) and the last partial chunk of a group.
  const bool aligned = ((uintptr_t)x % 16 == 0) && ((pix_per_group * B) % 8 == 0) &&
                       (((pix_per_group % SK_KC) * B) % 8 == 0);
  const uint32_t base = 1024 + 2 * SK_STAGE + SK_BARS, rawb = sk_raw_bytes(B);
  int raw_bufs = 0;
  if (aligned) raw_bufs = (base + 2 * rawb <= SK_SMEM_MAX) ? 2 : (base + rawb <= SK_SMEM_MAX ? 1 : 0);
  const uint32_t smem = base + (uint32_t)raw_bufs * rawb;
  cudaError_t e = cudaFuncSetAttribute(syrk_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid(tiles, (unsigned)n_groups, (unsigned)slices), block(SK_THREADS);
  syrk_tc_kernel<<<grid, block, smem, st>>>(x, pix_per_group, B, c_int, out, out_stride, per, accumulate, err,
                                            4000000000LL, raw_bufs);
  if (lc) lc->n += 1;
  return cudaGetLastError();
}

}  // namespace hsad
