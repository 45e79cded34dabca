// SR overlap matrix on the tensor cores (tcgen05, sm_103a):
//   S = (1/N_MC) (O - o)^T (O - o)          (Sec. 3.3.1, S_km = <O_k O_m> - <O_k><O_m>)
// in split-BF16: every centred entry x = x_hi + x_lo with x_hi = bf16(x),
// x_lo = bf16(x - x_hi); each product takes the three terms
// hi*hi + hi*lo + lo*hi (the lo*lo term is below 2^-16 relative), accumulated
// in FP32 in tensor memory.
//
// Pass 1 (k_split_T): O (rows x Np, FP32 or FP64, row-major) -> Hi, Lo
//   (Np_pad x K_pad BF16, parameter-major = K-major for the GEMM, zero padded).
// Pass 2, default (k_syrk_tma): persistent and warp-specialised.  One thread
//   issues TMA tensor copies (128-byte swizzle) of the four operand tiles of
//   a 64-sample chunk (A_hi, A_lo, B_hi, B_lo) into a 3-stage ring; one
//   thread issues tcgen05.mma.kind::f16 (BF16 in, FP32 accumulate into TMEM,
//   M = N = 128, K = 16) into one of two accumulators; four warps read the
//   other accumulator with tcgen05.ld and write the previous tile and its
//   mirror image.  Every wait is bounded.
// Pass 2, fallback (k_syrk_tc): one CTA per 128x128 tile, operands staged
//   by cp.async in the canonical no-swizzle K-major layout (8x8 core
//   matrices of 128 contiguous bytes), three stages.
#include "vmc_common.cuh"

#include <cuda.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <stdlib.h>

namespace {

constexpr int TM = 128;              // tile edge (M = N)
constexpr int TKC = 64;              // samples per chunk (64 BF16 = 128 B per row)
constexpr int STAGES = 3;
constexpr int TILE_BYTES = TM * TKC * 2;          // 16 KB per operand tile
constexpr int STAGE_BYTES = 4 * TILE_BYTES;       // A_hi, A_lo, B_hi, B_lo
constexpr int TC_SMEM = STAGES * STAGE_BYTES + 1024;
constexpr uint32_t TC_WAIT_LIMIT = 1u << 24;
constexpr uint32_t STALL_POLLS = 1u << 14;   // attempts of the test hook's wait

__device__ __forceinline__ uint32_t su32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor (tcgen05): start address, leading (K)
// byte offset, stride (M/N) byte offset, all >> 4; descriptor version 1;
// no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)(lbo >> 4) << 16) |
         ((uint64_t)(sbo >> 4) << 32) | (1ull << 46);
}

// Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major,
// N = 128 (>> 3 at bit 17), M = 128 (>> 4 at bit 24).
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((TM >> 3) << 17) | ((TM >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(IDESC), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   su32(bar))
               : "memory");
}

__device__ __forceinline__ bool bar_wait(uint64_t *bar, uint32_t parity) {
  for (uint32_t it = 0; it < TC_WAIT_LIMIT; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(su32(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// Pass 1: centre, split, transpose.  Block (32, 8) handles a 32x32 tile.
template <typename TO>
__global__ void k_split_T(const TO *O, int ldO, int rows, int Np, const double *obar,
                          __nv_bfloat16 *Hi, __nv_bfloat16 *Lo, int ldK) {
  __shared__ float t[32][33];
  const int r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
  for (int y = threadIdx.y; y < 32; y += 8) {
    const int r = r0 + y, c = c0 + threadIdx.x;
    float v = 0.f;
    if (r < rows && c < Np) v = (float)((double)O[(size_t)r * ldO + c] - obar[c]);
    t[y][threadIdx.x] = v;
  }
  __syncthreads();
  for (int y = threadIdx.y; y < 32; y += 8) {
    const int c = c0 + y, r = r0 + threadIdx.x;   // output row = parameter, column = sample
    const float v = t[threadIdx.x][y];
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    const __nv_bfloat16 l = __float2bfloat16_rn(v - __bfloat162float(h));
    Hi[(size_t)c * ldK + r] = h;
    Lo[(size_t)c * ldK + r] = l;
  }
}

// Offset of the 16-byte chunk (row r, k-group kg) of a 128 x 64 BF16 tile in
// the no-swizzle K-major layout: core matrix (r/8, kg) at (r/8)*1024 + kg*128.
__device__ __forceinline__ uint32_t tile_off(int r, int kg) {
  return (uint32_t)((r >> 3) * 1024 + kg * 128 + (r & 7) * 16);
}

// Issue the cp.async copies of chunk kc (4 operand tiles x 128 rows x 8
// pieces of 16 B) into one stage; 8 consecutive threads fill one core matrix.
__device__ __forceinline__ void load_chunk(unsigned char *stage, const __nv_bfloat16 *const *src,
                                           int ldK, int kc) {
#pragma unroll 4
  for (int q = threadIdx.x; q < 4 * TM * 8; q += 128) {
    const int op = q >> 10, rem = q & 1023;
    const int r = (rem & 7) + ((rem >> 6) << 3);
    const int kg = (rem >> 3) & 7;
    const __nv_bfloat16 *g = src[op] + (size_t)r * ldK + (size_t)kc * TKC + kg * 8;
    const uint32_t d = su32(stage + op * TILE_BYTES + tile_off(r, kg));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(g) : "memory");
  }
}

// One CTA per tile of `tiles` (bi <= bj; the host orders them for L2 reuse).
// Pipeline: STAGES - 1 chunks are in flight while the tensor cores work on
// the current one; a stage is refilled once the MMAs that read it committed.
template <typename TS>
__global__ void __launch_bounds__(128, 1) k_syrk_tc(const __nv_bfloat16 *Hi, const __nv_bfloat16 *Lo,
                                                    int ldK, int K, int Np, double scale, TS *S,
                                                    int ldS, const int2 *tiles, int *status) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t mma_bar[STAGES];
  __shared__ uint32_t tmem_base_sh;
  __shared__ int fail;
  const int2 tile = tiles[blockIdx.x];
  const int bi = tile.x, bj = tile.y;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  unsigned char *base = (unsigned char *)(((uintptr_t)smem + 1023) & ~(uintptr_t)1023);
  if (tid == 0) {
    fail = 0;
    for (int s = 0; s < STAGES; ++s)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&mma_bar[s])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;" ::"r"(
                     su32(&tmem_base_sh))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base_sh;
  const int nchunks = (K + TKC - 1) / TKC;
  const __nv_bfloat16 *src[4] = {Hi + (size_t)bi * TM * ldK, Lo + (size_t)bi * TM * ldK,
                                 Hi + (size_t)bj * TM * ldK, Lo + (size_t)bj * TM * ldK};
  uint32_t phase[STAGES];
#pragma unroll
  for (int s2 = 0; s2 < STAGES; ++s2) phase[s2] = 0;
  // prologue: chunks 0 .. STAGES-2
#pragma unroll
  for (int s2 = 0; s2 < STAGES - 1; ++s2) {
    if (s2 < nchunks) load_chunk(base + s2 * STAGE_BYTES, src, ldK, s2);
    asm volatile("cp.async.commit_group;" ::: "memory");
  }
  for (int kc = 0; kc < nchunks; ++kc) {
    const int st = kc % STAGES;
    unsigned char *stage = base + st * STAGE_BYTES;
    // chunk kc has landed when at most STAGES-2 newer groups are pending
    asm volatile("cp.async.wait_group %0;" ::"n"(STAGES - 2) : "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (__syncthreads_or(fail)) break;
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a_hi = su32(stage), a_lo = su32(stage + TILE_BYTES);
      const uint32_t b_hi = su32(stage + 2 * TILE_BYTES), b_lo = su32(stage + 3 * TILE_BYTES);
#pragma unroll
      for (int ks = 0; ks < TKC / 16; ++ks) {
        const uint32_t off = ks * 256;   // two core matrices along K per MMA
        const uint32_t acc0 = (kc > 0 || ks > 0) ? 1u : 0u;
        mma_bf16(tmem, smem_desc(a_hi + off, 128, 1024), smem_desc(b_hi + off, 128, 1024), acc0);
        mma_bf16(tmem, smem_desc(a_hi + off, 128, 1024), smem_desc(b_lo + off, 128, 1024), 1u);
        mma_bf16(tmem, smem_desc(a_lo + off, 128, 1024), smem_desc(b_hi + off, 128, 1024), 1u);
      }
      mma_commit(&mma_bar[st]);
    }
    // refill the stage of chunk kc-1 with chunk kc+STAGES-1, once its MMAs are done
    const int nxt = kc + STAGES - 1;
    if (nxt < nchunks) {
      const int ps = nxt % STAGES;   // == (kc - 1) mod STAGES
      bool ok = true;
      if (kc >= 1) {
        ok = bar_wait(&mma_bar[ps], phase[ps]);
        phase[ps] ^= 1;
        if (!ok) atomicExch(&fail, 1);
      }
      if (ok) load_chunk(base + ps * STAGE_BYTES, src, ldK, nxt);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  // commits not yet waited for: chunks max(0, nchunks - STAGES) .. nchunks-1
  // (the loop waited for chunks 0 .. nchunks-STAGES-1)
  if (!fail) {
    for (int kc = (nchunks > STAGES ? nchunks - STAGES : 0); kc < nchunks; ++kc) {
      const int st = kc % STAGES;
      if (!bar_wait(&mma_bar[st], phase[st])) atomicExch(&fail, 1);
      phase[st] ^= 1;
    }
  }
  if (fail && tid == 0) {
    // a wait expired: give the tensor cores a bounded chance to finish what
    // was issued before the memory they read or write is released
    for (int s2 = 0; s2 < STAGES; ++s2) bar_wait(&mma_bar[s2], phase[s2]);
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const bool bad = __syncthreads_or(fail);
  if (!bad) {
    // epilogue: TMEM -> shared tile (row-major, padded) -> coalesced rows of S
    // and, off the diagonal, coalesced rows of the mirror image.
    float *Ts = (float *)base;                 // 128 x 129 floats (66 KB), stages are free
    constexpr int LDT = TM + 1;
#pragma unroll 1
    for (int cc = 0; cc < TM; cc += 32) {
      uint32_t v[32];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + cc;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
          "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
            "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
            "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]),
            "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
            "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]),
            "=r"(v[31])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      const int r = warp * 32 + lane;
#pragma unroll
      for (int u = 0; u < 32; ++u) Ts[r * LDT + cc + u] = __uint_as_float(v[u]);
    }
    __syncthreads();
    for (int q = tid; q < TM * TM; q += 128) {
      const int r = q >> 7, c = q & (TM - 1);     // row-major: consecutive threads, consecutive columns
      const int row = bi * TM + r, col = bj * TM + c;
      if (row < Np && col < Np) S[(size_t)row * ldS + col] = (TS)((double)Ts[r * LDT + c] * scale);
      if (bi != bj) {
        const int mrow = bj * TM + r, mcol = bi * TM + c;   // S[mrow][mcol] = tile[c][r]
        if (mrow < Np && mcol < Np) S[(size_t)mrow * ldS + mcol] = (TS)((double)Ts[c * LDT + r] * scale);
      }
    }
  } else if (tid == 0) {
    atomicExch(status, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" ::"r"(tmem) : "memory");
}

// ---------------------------------------------------------------------------
// Persistent, warp-specialised version: the operand tiles arrive by TMA
// tensor copies (128B swizzle) into a STAGES-deep ring; one thread issues the
// MMAs; four warps drain a double-buffered TMEM accumulator, so the epilogue
// of one tile overlaps the MMAs of the next.  CTA = 6 warps:
//   warp 0: TMA producer (one thread), warp 1: TMEM owner and MMA issuer (one
//   thread), warps 2-5: epilogue (TMEM lane quadrant = warp % 4).
// Barriers: full[s] (TMA bytes landed), empty[s] (MMAs that read stage s
// committed), tfull[b] (accumulator b complete), tempty[b] (accumulator b
// drained).  Every wait is bounded; a wait that runs out sets `abort`, the
// other roles see it and leave their loops, and the issued copies and MMAs
// are waited for (bounded) before the TMEM is released.
// ---------------------------------------------------------------------------
constexpr int XW = 6;                 // warps per CTA
constexpr int X_EPI0 = 2;             // first epilogue warp
constexpr uint32_t X_TX = 4 * TILE_BYTES;   // bytes per stage

// K-major, 128-byte swizzle smem descriptor: SBO = 1024 B (8 rows of 128 B),
// LBO unused (1), version 1, layout type 2 (SWIZZLE_128B) in bits 61-63.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFF) >> 4) | (1ull << 16) | ((uint64_t)(1024 >> 4) << 32) |
         (1ull << 46) | (2ull << 61);
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void bar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void bar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// bounded wait that also gives up when another role has aborted
__device__ __forceinline__ bool xwait(uint64_t *bar, uint32_t parity, volatile int *abort) {
  for (uint32_t it = 0; it < TC_WAIT_LIMIT; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(su32(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
    if ((it & 255) == 255 && *abort) return false;
  }
  *abort = 1;
  return false;
}

template <typename TS>
__global__ void __launch_bounds__(XW * 32, 1)
    k_syrk_tma(const __grid_constant__ CUtensorMap map_hi, const __grid_constant__ CUtensorMap map_lo,
               int nchunks, int Np, double scale, TS *S, int ldS, const int2 *tiles, int ntiles,
               int *status, int stall) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t full[STAGES], empty[STAGES], tfull[2], tempty[2];
  __shared__ uint32_t tmem_base_sh;
  __shared__ int abort_sh;
  __shared__ int stalled_sh;
  volatile int *abort = &abort_sh;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  unsigned char *base = (unsigned char *)(((uintptr_t)smem + 1023) & ~(uintptr_t)1023);
  if (tid == 0) {
    abort_sh = 0;
    for (int s = 0; s < STAGES; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&full[s])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&empty[s])) : "memory");
    }
    for (int b = 0; b < 2; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&tfull[b])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 128;" ::"r"(su32(&tempty[b])) : "memory");
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    // test hook (vmc_test_stall): CTA 0 first waits, bounded, on a barrier
    // that no copy or MMA targets; it gives up before allocating TMEM or
    // issuing any copy or MMA, and reports the timeout
    stalled_sh = 0;
    if (stall && blockIdx.x == 0) {
      __shared__ __align__(8) uint64_t never;
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&never)) : "memory");
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
      bool ok = false;
      for (uint32_t it = 0; it < STALL_POLLS && !ok; ++it) {
        uint32_t r;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}"
            : "=r"(r)
            : "r"(su32(&never)), "r"(0u)
            : "memory");
        ok = r != 0;
      }
      if (!ok) stalled_sh = 1;
    }
  }
  __syncthreads();
  if (stalled_sh) {
    if (tid == 0) atomicExch(status, 1);
    return;
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(
                     su32(&tmem_base_sh))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base_sh;

  if (warp == 0 && lane == 0) {
    // ---- producer: stage s of chunk `it`, for this CTA's tiles in order
    uint32_t it = 0;
    for (int t = blockIdx.x; t < ntiles && !*abort; t += gridDim.x) {
      const int2 tl = tiles[t];
      for (int kc = 0; kc < nchunks; ++kc, ++it) {
        const int s = it % STAGES;
        const uint32_t ph = (it / STAGES) & 1;
        if (!xwait(&empty[s], ph ^ 1, abort)) break;
        unsigned char *stage = base + s * STAGE_BYTES;
        const uint32_t fb = su32(&full[s]);
        bar_expect_tx(fb, X_TX);
        const int x = kc * TKC;
        tma_load_2d(su32(stage), &map_hi, x, tl.x * TM, fb);
        tma_load_2d(su32(stage + TILE_BYTES), &map_lo, x, tl.x * TM, fb);
        tma_load_2d(su32(stage + 2 * TILE_BYTES), &map_hi, x, tl.y * TM, fb);
        tma_load_2d(su32(stage + 3 * TILE_BYTES), &map_lo, x, tl.y * TM, fb);
      }
    }
    // every issued stage must land before the shared memory is released
    const uint32_t issued = it;
    for (uint32_t j = (issued > STAGES ? issued - STAGES : 0); j < issued; ++j) {
      // completed phases are skipped immediately; pending ones are waited for
      uint64_t *b = &full[j % STAGES];
      for (uint32_t q = 0; q < TC_WAIT_LIMIT; ++q) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}"
            : "=r"(ok)
            : "r"(su32(b)), "r"((j / STAGES) & 1)
            : "memory");
        if (ok) break;
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer
    uint32_t it = 0, lt = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < ntiles && ok && !*abort; t += gridDim.x, ++lt) {
      const int b = lt & 1;
      const uint32_t tph = (lt >> 1) & 1;
      if (!(ok = xwait(&tempty[b], tph ^ 1, abort))) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t d = tmem + (uint32_t)(b * TM);
      for (int kc = 0; kc < nchunks; ++kc, ++it) {
        const int s = it % STAGES;
        const uint32_t ph = (it / STAGES) & 1;
        if (!(ok = xwait(&full[s], ph, abort))) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        unsigned char *stage = base + s * STAGE_BYTES;
        const uint32_t a_hi = su32(stage), a_lo = su32(stage + TILE_BYTES);
        const uint32_t b_hi = su32(stage + 2 * TILE_BYTES), b_lo = su32(stage + 3 * TILE_BYTES);
#pragma unroll
        for (int ks = 0; ks < TKC / 16; ++ks) {
          const uint32_t off = ks * 32;   // 16 BF16 along K inside the 128-byte swizzle atom
          const uint32_t acc0 = (kc > 0 || ks > 0) ? 1u : 0u;
          mma_bf16(d, smem_desc_sw128(a_hi + off), smem_desc_sw128(b_hi + off), acc0);
          mma_bf16(d, smem_desc_sw128(a_hi + off), smem_desc_sw128(b_lo + off), 1u);
          mma_bf16(d, smem_desc_sw128(a_lo + off), smem_desc_sw128(b_hi + off), 1u);
        }
        mma_commit(&empty[s]);
      }
      if (!ok) break;
      mma_commit(&tfull[b]);
    }
    // wait (bounded) for the MMAs issued so far before the TMEM is released
    __shared__ __align__(8) uint64_t fin;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&fin)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    mma_commit(&fin);
    bar_wait(&fin, 0);
  } else if (warp >= X_EPI0) {
    // ---- epilogue: accumulator b -> S (and its mirror off the diagonal)
    const int q = warp & 3;   // TMEM lane quadrant of this warp
    uint32_t lt = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++lt) {
      const int b = lt & 1;
      if (!xwait(&tfull[b], (lt >> 1) & 1, abort)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int2 tl = tiles[t];
      const int row = tl.x * TM + q * 32 + lane;
#pragma unroll 1
      for (int cc = 0; cc < TM; cc += 32) {
        uint32_t v[32];
        const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * TM + cc);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
            "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
              "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
              "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]),
              "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
              "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]),
              "=r"(v[31])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (cc + 32 >= TM) {
          // the accumulator is in registers: hand it back to the MMA issuer
          asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
          bar_arrive(su32(&tempty[b]));
        }
        const int col0 = tl.y * TM + cc;
        if (row < Np) {
#pragma unroll
          for (int u = 0; u < 32; ++u)
            if (col0 + u < Np) S[(size_t)row * ldS + col0 + u] = (TS)((double)__uint_as_float(v[u]) * scale);
        }
        if (tl.x != tl.y && row < Np) {
          // mirror: S[col][row]; for fixed u the warp writes 32 consecutive rows' entries
#pragma unroll
          for (int u = 0; u < 32; ++u)
            if (col0 + u < Np) S[(size_t)(col0 + u) * ldS + row] = (TS)((double)__uint_as_float(v[u]) * scale);
        }
      }
    }
  }
  __syncthreads();
  if (tid == 0 && *abort) atomicExch(status, 1);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem) : "memory");
}

__global__ void k_shift_diag(double *S, int Np, double shift_rel, double shift_abs) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < Np) S[(size_t)k * Np + k] = S[(size_t)k * Np + k] * (1.0 + shift_rel) + shift_abs;
}

}  // namespace

// 2D tensor map of a split operand (Np_pad rows of ldK BF16, K contiguous):
// box 64 (K) x 128 (rows), 128-byte swizzle.  The encoder is taken from the
// driver through the runtime (no link-time dependency on libcuda).
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
    else
      cudaGetLastError();
  }
  return fn;
}

static bool make_map(CUtensorMap *m, void *base, int ldK, int Np_pad) {
  EncodeTiledFn fn = encode_fn();
  if (!fn || ((uintptr_t)base & 15) || (ldK % TKC)) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)ldK, (cuuint64_t)Np_pad};
  const cuuint64_t strides[1] = {(cuuint64_t)ldK * 2};
  const cuuint32_t box[2] = {(cuuint32_t)TKC, (cuuint32_t)TM};
  const cuuint32_t estr[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Kernel choice for the S GEMM: the persistent TMA kernel unless the
// environment variable VMC_TC_KERNEL is "tiles" (one CTA per tile, cp.async).
static bool vmc_tc_use_tma() {
  const char *v = getenv("VMC_TC_KERNEL");
  return !(v && v[0] == 't' && v[1] == 'i');
}

// Padded sizes of the split operands.
void vmc_tc_dims(int rows, int Np, int *ldK, int *Np_pad) {
  *ldK = (rows + TKC - 1) / TKC * TKC;
  *Np_pad = (Np + TM - 1) / TM * TM;
}

// S (FP64, Np x Np, shifted) from O via split-BF16 tensor-core products.
// hi/lo: device buffers of Np_pad * ldK BF16 each; status: device int.
// Tile order for L2 reuse: groups of 8 block-rows; within a group, for each
// block-column bj the tiles (bi, bj), bi in the group and bi <= bj, are
// consecutive, so a wave of CTAs shares few operand blocks.
int vmc_tc_tile_list(int Np, int2 *out) {
  const int nt = (Np + TM - 1) / TM;
  int k = 0;
  for (int g0 = 0; g0 < nt; g0 += 8)
    for (int bj = g0; bj < nt; ++bj)
      for (int bi = g0; bi < g0 + 8 && bi <= bj; ++bi)
        if (out) out[k++] = make_int2(bi, bj);
        else ++k;
  return k;
}

cudaError_t vmc_sr_build_S_tc(const SrWork &w, void *hi, void *lo, int *status, double shift_rel,
                              double shift_abs, const int2 *tiles, cudaStream_t st, long long *nl,
                              int *which) {
  int ldK, Np_pad;
  vmc_tc_dims(w.rows, w.Np, &ldK, &Np_pad);
  cudaError_t e = cudaMemsetAsync(hi, 0, sizeof(__nv_bfloat16) * (size_t)Np_pad * ldK, st);
  if (e) return e;
  if ((e = cudaMemsetAsync(lo, 0, sizeof(__nv_bfloat16) * (size_t)Np_pad * ldK, st))) return e;
  if ((e = cudaMemsetAsync(status, 0, sizeof(int), st))) return e;
  dim3 g1((w.rows + 31) / 32, (w.Np + 31) / 32), b1(32, 8);
  if (w.precision == 0)
    k_split_T<double><<<g1, b1, 0, st>>>((const double *)w.O, w.ldO, w.rows, w.Np, w.obar,
                                         (__nv_bfloat16 *)hi, (__nv_bfloat16 *)lo, ldK);
  else
    k_split_T<float><<<g1, b1, 0, st>>>((const float *)w.O, w.ldO, w.rows, w.Np, w.obar,
                                        (__nv_bfloat16 *)hi, (__nv_bfloat16 *)lo, ldK);
  ++*nl;
  static bool attr = false;
  if (!attr) {
    if ((e = cudaFuncSetAttribute(k_syrk_tc<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  TC_SMEM)))
      return e;
    if ((e = cudaFuncSetAttribute(k_syrk_tma<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  TC_SMEM)))
      return e;
    attr = true;
  }
  const int nt = Np_pad / TM;
  const int ntiles = nt * (nt + 1) / 2;
  CUtensorMap mh, ml;
  if (vmc_tc_use_tma() && make_map(&mh, hi, ldK, Np_pad) && make_map(&ml, lo, ldK, Np_pad)) {
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int grid = ntiles < nsm ? ntiles : nsm;
    k_syrk_tma<double><<<grid, XW * 32, TC_SMEM, st>>>(mh, ml, ldK / TKC, w.Np, 1.0 / w.rows, w.S,
                                                        w.Np, tiles, ntiles, status, w.stall);
    if (which) *which = VMC_S_KERNEL_TMA;
  } else {
    if (which) *which = VMC_S_KERNEL_TILES;
    k_syrk_tc<double><<<ntiles, 128, TC_SMEM, st>>>(
        (const __nv_bfloat16 *)hi, (const __nv_bfloat16 *)lo, ldK, ldK, w.Np, 1.0 / w.rows, w.S,
        w.Np, tiles, status);
  }
  k_shift_diag<<<(w.Np + 255) / 256, 256, 0, st>>>(w.S, w.Np, shift_rel, shift_abs);
  *nl += 2;
  return cudaGetLastError();
}
