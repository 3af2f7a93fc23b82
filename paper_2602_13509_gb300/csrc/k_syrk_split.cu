// K2 for streamed statistics, split once, contracted per tile: the exact integer SYRK of
// k_syrk_tc.cu (S2 = 4096 H^T H + 64 (H^T R + R^T H) + R^T R with x' = 64 h + r, Sec. 3.3's
// covariance sums) with the split taken out of the tile kernel.
//
// In the tile kernel every CTA converts the DN of both of its 128-band blocks for every pixel
// chunk, so each band block is converted once per tile it belongs to (at B = 448: 2048 band
// rows per chunk for 448 distinct ones). Here
//   syrk_split_kernel  converts each (line, 64-pixel chunk) once: H and R of all 128-band
//                      blocks, written to a scratch in exactly the shared-memory operand
//                      layout (per block: H then R, 128 rows x 64 pixels BF16, 128-byte
//                      swizzle; rows past B and pixels past the line zero);
//   syrk_pre_kernel    one CTA per (128-band row block, 64-band column block, line): a
//                      copy warp streams the row block's 32 KB and the column block's 16 KB
//                      of operands per chunk with bulk copies through a 2-stage ring, one thread issues the 4 MMAs per 16 pixels into the three
//                      exact accumulators (TMEM), 4 warps read them out and store the exact
//                      sums (int64 combination, FP64 store) to the lower triangle.
// Every wait is bounded; a timeout sets *err and the CTA drains its copies and exits.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "hsad_internal.h"
#include "tc_util.cuh"

namespace hsad {

namespace {
constexpr int SP_M = 128, SP_KC = 64;
constexpr uint32_t SP_PLANE = SP_M * SP_KC * 2;  // 16 KB: 128 band rows x 64 pixels, 16-bit
constexpr uint32_t SP_BLOCK = 2 * SP_PLANE;      // H then R of one band block
constexpr int SP_STAGES = 2;
constexpr int SP_N = 64;                         // output columns per tile: 3 accumulators in 256 TMEM columns
constexpr uint32_t SP_HALF = SP_PLANE / 2;       // 64 band rows of a plane (the first or second 8 KB)
constexpr uint32_t SP_STAGE = SP_BLOCK + 2 * SP_HALF;
constexpr int SP_THREADS = 192;                  // 4 epilogue warps, copy warp, MMA warp
constexpr int SP_COPY_WARP = 4, SP_MMA_WARP = 5;
constexpr uint32_t SP_SMEM = 1024 + SP_STAGES * SP_STAGE + 256;

__host__ __device__ inline int sp_blocks(int B) { return (B + SP_M - 1) / SP_M; }
__host__ __device__ inline int64_t sp_chunks(int64_t pix) { return (pix + SP_KC - 1) / SP_KC; }
}  // namespace

size_t syrk_split_bytes(int64_t lines, int64_t pix, int B) {
  return (size_t)lines * (size_t)sp_chunks(pix) * (size_t)sp_blocks(B) * SP_BLOCK;
}

// grid (chunks, groups), 256 threads: the chunk's DN (64 pixels x B, contiguous) into shared
// memory with 16-byte loads when aligned; then per 128-band block, thread = one band row and
// 8 pixels at a time (a warp reads 32 consecutive bands of one pixel: conflict free) into a
// staged 32 KB block in the operand layout, written out with coalesced 16-byte stores.
constexpr int SS_T = 256;
__host__ __device__ inline uint32_t ss_raw_bytes(int B) { return ((uint32_t)SP_KC * B * 2 + 15) / 16 * 16; }
__global__ void __launch_bounds__(SS_T) syrk_split_kernel(const uint16_t* __restrict__ x, int64_t pix, int B,
                                                          const int32_t* __restrict__ c_int,
                                                          uint8_t* __restrict__ hr, double* __restrict__ s1,
                                                          int vec) {
  extern __shared__ __align__(16) uint8_t ssm[];
  uint8_t* blk = ssm;                                  // one staged operand block: H then R
  uint16_t* raw = reinterpret_cast<uint16_t*>(ssm + SP_BLOCK);
  const int64_t g = blockIdx.y, chunk = blockIdx.x;
  const int nbb = sp_blocks(B);
  const int64_t pc = chunk * SP_KC;
  const int npx = (int)min((int64_t)SP_KC, pix - pc);
  const uint16_t* src = x + (g * pix + pc) * (int64_t)B;
  const int nval = npx * B;
  if (vec) {  // 16-byte aligned source, whole 8-value groups
    const uint4* s4 = reinterpret_cast<const uint4*>(src);
    uint4* r4 = reinterpret_cast<uint4*>(raw);
    for (int i = threadIdx.x; i < nval / 8; i += SS_T) r4[i] = __ldg(s4 + i);
    for (int i = nval / 8 * 8 + threadIdx.x; i < nval; i += SS_T) raw[i] = __ldg(src + i);
  } else {
    for (int i = threadIdx.x; i < nval; i += SS_T) raw[i] = __ldg(src + i);
  }
  uint8_t* dst = hr + ((size_t)(g * sp_chunks(pix) + chunk) * nbb) * SP_BLOCK;
  if (s1) {  // the chunk's band sums (exact integers; FP64 atomic adds of them are exact in any order)
    __syncthreads();
    for (int b = threadIdx.x; b < B; b += SS_T) {
      int acc = 0;  // |x - c| < 2^16 over 64 pixels
      for (int k = 0; k < npx; ++k) acc += (int)raw[k * B + b];
      atomicAdd(s1 + g * B + b, (double)(acc - npx * c_int[b]));
    }
  }
  for (int bb = 0; bb < nbb; ++bb) {
    __syncthreads();  // the raw chunk is in place; the previous block's stores have read blk
    for (int it = threadIdx.x; it < SP_M * (SP_KC / 8); it += SS_T) {
      const int r = it % SP_M, gi = it / SP_M, row = bb * SP_M + r;
      const bool valid = row < B;
      // x' = DN - c as an exact float: the bits of 1.5 * 2^23 + x' minus 1.5 * 2^23
      const int magic_c = 0x4B400000 - (valid ? c_int[row] : 0);
      uint32_t hw[4], rw[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        float hv[2], rv[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const int k = gi * 8 + 2 * q + u;
          const bool in = valid && k < npx;
          const float xv = in ? __int_as_float(magic_c + (int)raw[k * B + row]) - 12582912.0f : 0.f;
          // h = rint(x'/64) (exact: |x'/64| <= 256), r = x' - 64 h
          const float hf = __fmaf_rn(xv, 1.f / 64.f, 12582912.0f) - 12582912.0f;
          hv[u] = hf;
          rv[u] = __fmaf_rn(hf, -64.f, xv);
        }
        // small integers, exact in BF16: the BF16 bits are the float's top half
        hw[q] = __byte_perm(__float_as_uint(hv[0]), __float_as_uint(hv[1]), 0x7632);
        rw[q] = __byte_perm(__float_as_uint(rv[0]), __float_as_uint(rv[1]), 0x7632);
      }
      const uint32_t off = tc::sw128_offset(r, gi * 8);
      *(uint4*)(blk + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
      *(uint4*)(blk + SP_PLANE + off) = make_uint4(rw[0], rw[1], rw[2], rw[3]);
    }
    __syncthreads();
    uint4* d4 = reinterpret_cast<uint4*>(dst + (size_t)bb * SP_BLOCK);
    const uint4* b4 = reinterpret_cast<const uint4*>(blk);
    for (int i = threadIdx.x; i < (int)(SP_BLOCK / 16); i += SS_T) d4[i] = b4[i];
  }
}

// grid (tiles, groups): the exact sums of one 128 x 64 block of S2 of one group: 128-band row
// block ib, 64-band column block jb >= 2 ib (two CTAs per SM: 96 KB of shared memory and 256
// TMEM columns each, so that one CTA's epilogue overlaps the other's contraction).
__global__ void __launch_bounds__(SP_THREADS, 2) syrk_pre_kernel(const uint8_t* __restrict__ hr, int64_t pix,
                                                                 int B, double* __restrict__ out,
                                                                 int64_t out_stride, int32_t* __restrict__ err,
                                                                 long long limit) {
  const int nb = sp_blocks(B), nc = (B + SP_N - 1) / SP_N;
  int tile = blockIdx.x, ib = 0;
  while (tile >= nc - 2 * ib) {
    tile -= nc - 2 * ib;
    ++ib;
  }
  const int jb = 2 * ib + tile;                  // 64-band column block
  const int i0 = ib * SP_M, j0 = jb * SP_N;
  const int N = min(SP_N, ((B - j0) + 15) / 16 * 16);
  const bool diag = (jb >> 1) == ib;             // the columns lie in the row block's own bands
  const int64_t g = blockIdx.y;
  const int nchunks = (int)sp_chunks(pix);
  const uint8_t* hg = hr + (size_t)g * nchunks * nb * SP_BLOCK;
  const uint32_t stage_bytes = diag ? SP_BLOCK : SP_BLOCK + 2 * SP_HALF;
  const uint32_t half_off = (uint32_t)(jb & 1) * SP_HALF;  // the column block's rows within its 128-band block

  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = tc::align1024(smem_raw);
  uint64_t* bars = (uint64_t*)(sm + SP_STAGES * SP_STAGE);
  uint32_t* tslot = (uint32_t*)(bars + 2 * SP_STAGES + 2);
  const uint32_t full = tc::smem_u32(bars), empty = full + 8 * SP_STAGES, d_full = empty + 8 * SP_STAGES;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid == 0) {
    for (int s = 0; s < SP_STAGES; ++s) {
      tc::mbar_init(full + 8 * s, 1);
      tc::mbar_init(empty + 8 * s, 1);
    }
    tc::mbar_init(d_full, 1);
    tc::mbar_init_fence();
  }
  if (warp == SP_MMA_WARP) tc::tmem_alloc(tc::smem_u32(tslot), 256);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = *tslot;
  bool ok = true;

  if (warp == SP_COPY_WARP) {
    if (lane == 0) {
      int issued = 0;
      for (int c = 0; c < nchunks; ++c, ++issued) {
        const int s = c % SP_STAGES;
        if (!tc::mbar_wait(empty + 8 * s, (uint32_t)(((c / SP_STAGES) & 1) ^ 1), limit)) {
          ok = false;
          break;
        }
        tc::mbar_arrive_expect_tx(full + 8 * s, stage_bytes);
        const uint8_t* cb = hg + (size_t)c * nb * SP_BLOCK;
        uint8_t* st_base = sm + s * SP_STAGE;
        tc::bulk_load(tc::smem_u32(st_base), cb + (size_t)ib * SP_BLOCK, SP_BLOCK, full + 8 * s);
        if (!diag) {  // H and R rows of the 64-band column block
          const uint8_t* jbk = cb + (size_t)(jb >> 1) * SP_BLOCK + half_off;
          tc::bulk_load(tc::smem_u32(st_base + SP_BLOCK), jbk, SP_HALF, full + 8 * s);
          tc::bulk_load(tc::smem_u32(st_base + SP_BLOCK + SP_HALF), jbk + SP_PLANE, SP_HALF, full + 8 * s);
        }
      }
      for (int s = 0; s < SP_STAGES && s < issued; ++s) {  // every copy landed before exit
        const int last = issued - 1 - ((issued - 1 - s) % SP_STAGES);
        if (!tc::mbar_wait(full + 8 * s, (uint32_t)((last / SP_STAGES) & 1), limit)) ok = false;
      }
      if (!ok) atomicExch(err, 1);
    }
  } else if (warp == SP_MMA_WARP) {
    if (lane == 0) {
      const uint32_t idesc = tc::idesc_f16(1, SP_M, N);  // accumulators at columns 0, 64, 128
      bool any = false;
      for (int c = 0; c < nchunks; ++c) {
        const int s = c % SP_STAGES;
        if (!tc::mbar_wait(full + 8 * s, (uint32_t)((c / SP_STAGES) & 1), limit)) {
          ok = false;
          break;
        }
        tc::fence_after_sync();
        const uint32_t aH = tc::smem_u32(sm + s * SP_STAGE), aR = aH + SP_PLANE;
        // B: the column block's 64 rows of H and R (inside A's block on the diagonal)
        const uint32_t bH = diag ? aH + half_off : aH + SP_BLOCK, bR = diag ? aR + half_off : bH + SP_HALF;
        // descriptors by offset: a 32-byte K step adds 2 to the start-address field (address / 16)
        const uint64_t dAH = tc::desc_sw128(aH), dAR = tc::desc_sw128(aR), dBH = tc::desc_sw128(bH),
                       dBR = tc::desc_sw128(bR);
#pragma unroll
        for (int ks = 0; ks < SP_KC / 16; ++ks) {
          const uint64_t o = 2 * ks;
          const uint32_t acc = (c > 0 || ks > 0) ? 1u : 0u;
          tc::mma_f16(tbase + 0, dAH + o, dBH + o, idesc, acc);
          tc::mma_f16(tbase + 64, dAH + o, dBR + o, idesc, acc);
          tc::mma_f16(tbase + 64, dAR + o, dBH + o, idesc, 1u);
          tc::mma_f16(tbase + 128, dAR + o, dBR + o, idesc, acc);
        }
        tc::mma_commit(empty + 8 * s);
        any = true;
      }
      if (any) tc::mma_commit(d_full);
      else tc::mbar_arrive(d_full);
      if (!ok) atomicExch(err, 1);
      if (!tc::mbar_wait(d_full, 0, limit)) atomicExch(err, 1);  // MMAs finished before TMEM is freed
    }
  } else {
    // epilogue: warp w reads TMEM lanes 32 w .. 32 w + 31 (band i0 + row), 32 columns at a time
    const bool dok = tc::mbar_wait(d_full, 0, limit);
    __syncwarp();
    tc::fence_after_sync();
    if (!dok) atomicExch(err, 1);
    const int row = tid;
    const uint32_t taddr = tbase + ((uint32_t)(warp * 32) << 16);
    double* o = out + g * out_stride;
    const int bi = i0 + row;
    const bool write = dok && bi < B;
    for (int c0 = 0; c0 < N; c0 += 32) {
      float hh[32], xr[32], rr[32];
      __syncwarp();
      tc::tmem_ld32(taddr + (uint32_t)c0, hh);
      tc::tmem_ld32(taddr + 64u + (uint32_t)c0, xr);
      tc::tmem_ld32(taddr + 128u + (uint32_t)c0, rr);
      if (write) {
#pragma unroll
        for (int jj = 0; jj < 32; ++jj) {
          const int gj = j0 + c0 + jj;
          if (c0 + jj < N && gj < B && gj >= bi) {
            // exact integer sums below 2^24 each: combined in int64, converted once
            const long long iv = ((long long)__float2int_rn(hh[jj]) << 12) +
                                 ((long long)__float2int_rn(xr[jj]) << 6) + (long long)__float2int_rn(rr[jj]);
            o[(int64_t)gj * B + bi] = (double)iv;
          }
        }
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == SP_MMA_WARP) {
    __syncwarp();
    tc::tmem_dealloc(tbase, 256);
  }
}

cudaError_t launch_syrk_split(const uint16_t* x, int64_t n_groups, int64_t pix, int B, const int32_t* c_int,
                              uint8_t* hr, double* s1, cudaStream_t st, LaunchCounter* lc) {
  if (n_groups <= 0 || pix <= 0) return cudaSuccess;
  if (s1) {
    const cudaError_t e0 = cudaMemsetAsync(s1, 0, (size_t)n_groups * B * sizeof(double), st);
    if (e0 != cudaSuccess) return e0;
  }
  if (n_groups > 65535 || sp_chunks(pix) > 65535) return cudaErrorInvalidValue;
  const uint32_t smem = SP_BLOCK + ss_raw_bytes(B);
  cudaError_t e = cudaFuncSetAttribute(syrk_split_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  // 16-byte loads: the input base and every chunk start (pixel multiples of 64 x B values)
  const int vec = ((uintptr_t)x % 16 == 0) && ((pix * B) % 8 == 0) && ((SP_KC * B) % 8 == 0);
  syrk_split_kernel<<<dim3((unsigned)sp_chunks(pix), (unsigned)n_groups), SS_T, smem, st>>>(x, pix, B, c_int, hr,
                                                                                            s1, vec);
  if (lc) lc->n += 1;
  return cudaGetLastError();
}

cudaError_t launch_syrk_pre(const uint8_t* hr, int64_t n_groups, int64_t pix, int B, double* out,
                            int64_t out_stride, int32_t* err, cudaStream_t st, LaunchCounter* lc) {
  if (n_groups <= 0 || pix <= 0) return cudaSuccess;
  if (n_groups > 65535 || pix > 4096) return cudaErrorInvalidValue;  // one exact accumulation per group
  const int nb = sp_blocks(B), nc = (B + SP_N - 1) / SP_N;
  int tiles = 0;
  for (int ib = 0; ib < nb; ++ib) tiles += nc - 2 * ib;
  cudaError_t e = cudaFuncSetAttribute(syrk_pre_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SP_SMEM);
  if (e != cudaSuccess) return e;
  syrk_pre_kernel<<<dim3(tiles, (unsigned)n_groups), SP_THREADS, SP_SMEM, st>>>(
      hr, pix, B, out, out_stride, err, 4000000000LL);
  if (lc) lc->n += 1;
  return cudaGetLastError();
}

}  // namespace hsad
