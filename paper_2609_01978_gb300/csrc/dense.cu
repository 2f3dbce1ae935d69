// dense.cu -- form (b): the row transform as a dense tensor-core contraction.
//
// The kernel of Eq. 2 is separable (Sec. 2.6), so the focal-plane field is
//   U = Pre chirp_out .* (K T K^T),   K[m, i] = exp(2 pi i theta(m, i)),
//   theta(m, i) = di^2 kappa/2 - (m - M/2) di delta   (turns),
// and the row pass C1 = K T^T is a real GEMM with
//   A = [Re K; Im K] (2M x N, split as K = K_hi + K_lo, both BF16),
//   B = T (aperture rows x N, binary: exact in BF16),
//   D = FP32 accumulators in tensor memory.
// K_hi T^T + K_lo T^T is accumulated into the same accumulator, so the product
// carries the ~16 significant bits of the split kernel.
//
// GB300 mapping (tcgen05, one CTA per SM, persistent):
//   tile     : 128 kernel rows (64 m values, Re and Im) x 256 aperture rows,
//              K step 64 per stage (one 128-byte swizzle atom of BF16)
//   warp 4   : copies the A stage (hi and lo, pre-swizzled in HBM) with one
//              cp.async.bulk per stage
//   warps 6-13: generate the binary mask of the 256 aperture rows for the
//              stage's 64 columns (exact zone rule, threshold walk), write it
//              in the 128-byte-swizzled K-major layout
//   warp 5   : allocates tensor memory and issues tcgen05.mma (M128 N256 K16)
//   warps 0-3: epilogue; every `promote` K blocks the accumulator (double
//              buffered in TMEM) is read with tcgen05.ld and added in FP32 to
//              the C1 tile in global memory (bounds the growth of the tensor
//              core's FP32 accumulation error).
// Every mbarrier wait is bounded in time; on expiry the kernel records an error
// code, drains what it issued, frees tensor memory and returns.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>

#include "fzp_internal.cuh"

namespace fzp {
namespace {

constexpr int BM = 128, BN = 256, BK = 64, STAGES = 3;
constexpr int A_HALF = BM * BK * 2;  // 16 KiB: one of hi / lo
constexpr int A_BYTES = 2 * A_HALF;  // 32 KiB
constexpr int B_BYTES = BN * BK * 2; // 32 KiB
constexpr int NUM_THREADS = 14 * 32;
constexpr int GEN_WARP0 = 6;
constexpr int TMEM_COLS = 512;
constexpr uint64_t WAIT_NS = 2000000000ull;  // 2 s per wait
constexpr int ERR_TIMEOUT_BASE = 100;

struct DenseArgs {
  MaskGeom mg;
  int64_t N;
  int64_t kblocks;
  int64_t j_begin, j_end;   // aperture rows of this launch [j_begin, j_end)
  int64_t n_stripes;        // ceil((j_end - j_begin) / BN)
  int ntiles;               // 2M / 128
  int promote;              // K blocks per accumulation chunk
  int hi_only;              // 1: BF16 kernel (hi) only
  const uint8_t* A;         // pre-swizzled kernel tiles
  float* C1;                // [2M][c1_stride], column = j - c1_j0
  int64_t c1_stride, c1_j0;
  int* err;
};

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(uint64_t* bar, uint32_t tx) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}" ::"r"(smem_u32(bar)),
               "r"(tx)
               : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: returns false (after recording `code`) when the wait expires
// or another role of this CTA has aborted.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag, int* err,
                                          int code) {
  if (mbar_try(bar, parity)) return true;
  const uint64_t t0 = gtimer();
  while (true) {
    if (mbar_try(bar, parity)) return true;
    if (*abort_flag) return false;
    if (gtimer() - t0 > WAIT_NS) {
      atomicCAS(err, 0, code);
      *abort_flag = 1;
      return false;
    }
  }
}

// Warp-uniform bounded wait: lane 0 polls, the result is broadcast.
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag, int* err, int code) {
  int ok = 0;
  if ((threadIdx.x & 31) == 0) ok = mbar_wait(bar, parity, abort_flag, err, code) ? 1 : 0;
  return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t sdesc(const void* p) {
  const uint64_t a = smem_u32(p);
  return ((a >> 4) & 0x3FFFull) | (1ull << 16) | ((uint64_t)(1024 >> 4) << 32) | (1ull << 46) | (2ull << 61);
}

// Instruction descriptor: kind::f16, D = F32, A = B = BF16, K-major, N = 256, M = 128.
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t ad, uint64_t bd, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(
          dtmem),
      "l"(ad), "l"(bd), "r"(IDESC), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,"
      "%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// ---------------------------------------------------------------- mask rows
__device__ __forceinline__ uint64_t range_bits(int a, int b) {  // bits a..b inclusive, 0 <= a <= b <= 63
  return (~0ull >> (63 - b)) & (~0ull << a);
}

__device__ __forceinline__ int64_t ceil_sqrt(int64_t t) {  // smallest a >= 0 with a^2 >= t
  if (t <= 0) return 0;
  int64_t a = (int64_t)sqrtf((float)t);
  while (a * a < t) ++a;
  while (a > 0 && (a - 1) * (a - 1) >= t) --a;
  return a;
}

__device__ __forceinline__ int64_t isqrt_floor(int64_t t) {  // largest a with a^2 <= t (t >= 0)
  int64_t a = (int64_t)sqrtf((float)t);
  while (a * a > t) --a;
  while ((a + 1) * (a + 1) <= t) ++a;
  return a;
}

// Open bits of row (dj2 = dj^2) for columns [ilo, ihi] inside the disc, relative
// to i0.  The zone index is monotone in |i - c|; its parity flips at the
// columns where dj^2 + (i - c)^2 crosses a threshold S_m.
__device__ uint64_t row_bits(int64_t i0, int64_t ilo, int64_t ihi, int64_t c, int64_t dj2, const MaskGeom& g) {
  uint64_t bits = 0;
  const int64_t r0 = ilo > c ? ilo : c;
  if (r0 <= ihi) {
    const int64_t d0 = r0 - c, d1 = ihi - c;
    const int64_t z0 = zone_of(dj2 + d0 * d0, g), z1 = zone_of(dj2 + d1 * d1, g);
    uint64_t b = (z0 & 1) ? range_bits((int)(r0 - i0), (int)(ihi - i0)) : 0ull;
    for (int64_t m = z0 + 1; m <= z1; ++m) {
      const int64_t p = c + ceil_sqrt(__ldg(g.thr + (m - 1)) - dj2);
      b ^= range_bits((int)(p - i0), (int)(ihi - i0));
    }
    bits |= b;
  }
  const int64_t l1 = ihi < c - 1 ? ihi : c - 1;
  if (ilo <= l1) {
    const int64_t dA = c - ilo, dB = c - l1;
    const int64_t zA = zone_of(dj2 + dA * dA, g), zB = zone_of(dj2 + dB * dB, g);
    uint64_t b = (zA & 1) ? range_bits((int)(ilo - i0), (int)(l1 - i0)) : 0ull;
    for (int64_t m = zA; m > zB; --m) {
      const int64_t p = c - ceil_sqrt(__ldg(g.thr + (m - 1)) - dj2) + 1;
      b ^= range_bits((int)(p - i0), (int)(l1 - i0));
    }
    bits |= b;
  }
  return bits;
}

__device__ __forceinline__ uint32_t pack2(uint32_t two_bits) {  // two samples -> two BF16 (1.0 or 0.0)
  return (two_bits & 1u) * 0x3F80u + ((two_bits >> 1) & 1u) * 0x3F800000u;
}

// ---------------------------------------------------------------- kernel
__global__ void __launch_bounds__(NUM_THREADS, 1) k_dense(DenseArgs a) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  // 1024-byte alignment of the operand tiles (swizzle atoms)
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = base;                       // STAGES x 32 KiB
  uint8_t* sB = base + STAGES * A_BYTES;    // STAGES x 32 KiB
  uint64_t* bars = reinterpret_cast<uint64_t*>(sB + STAGES * B_BYTES);
  uint64_t* fullA = bars;
  uint64_t* fullB = bars + STAGES;
  uint64_t* empty = bars + 2 * STAGES;
  uint64_t* accFull = bars + 3 * STAGES;
  uint64_t* accEmpty = accFull + 2;
  uint64_t* drain = accEmpty + 2;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(drain + 1);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 2);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&fullA[s], 1);
      mbar_init(&fullB[s], 8);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&accFull[b], 1);
      mbar_init(&accEmpty[b], 4);
    }
    mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 5) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  const int64_t n_items = a.n_stripes * a.ntiles;
  const int64_t nkb = a.kblocks;
  const int64_t nchunk = (nkb + a.promote - 1) / a.promote;
  const uint32_t a_bytes = a.hi_only ? A_HALF : A_BYTES;

  if (warp == 4) {
    // ---------------- A loader
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      int last[STAGES];  // parity of the last copy issued into each stage, -1: none
#pragma unroll
      for (int s2 = 0; s2 < STAGES; ++s2) last[s2] = -1;
      for (int64_t it = blockIdx.x; it < n_items && !*abort_flag; it += gridDim.x) {
        const int t = (int)(it / a.n_stripes);
        const uint8_t* At = a.A + (int64_t)t * nkb * A_BYTES;
        for (int64_t kb = 0; kb < nkb; ++kb) {
          if (!mbar_wait(&empty[stage], phase ^ 1, abort_flag, a.err, ERR_TIMEOUT_BASE + 1)) break;
          mbar_arrive_tx(&fullA[stage], a_bytes);
          bulk_g2s(sA + stage * A_BYTES, At + kb * A_BYTES, a_bytes, &fullA[stage]);
          last[stage] = (int)phase;
          if (++stage == STAGES) { stage = 0; phase ^= 1; }
        }
      }
      if (*abort_flag) {
        // the copies already issued must land before shared memory is released
#pragma unroll
        for (int s2 = 0; s2 < STAGES; ++s2) {
          if (last[s2] < 0) continue;
          const uint64_t t0 = gtimer();
          while (!mbar_try(&fullA[s2], (uint32_t)last[s2]) && gtimer() - t0 < WAIT_NS) {
          }
        }
      }
    }
  } else if (warp == 5) {
    // ---------------- MMA issuer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      int buf = 0;
      uint32_t accph = 0;
      bool ok = true;
      for (int64_t it = blockIdx.x; it < n_items && ok; it += gridDim.x) {
        for (int64_t ch = 0; ch < nchunk && ok; ++ch) {
          if (!mbar_wait(&accEmpty[buf], accph ^ 1, abort_flag, a.err, ERR_TIMEOUT_BASE + 2)) { ok = false; break; }
          tc_fence_after();
          const uint32_t dt = tmem + (uint32_t)(buf * BN);
          const int64_t kb0 = ch * a.promote, kb1 = kb0 + a.promote < nkb ? kb0 + a.promote : nkb;
          for (int64_t kb = kb0; kb < kb1; ++kb) {
            if (!mbar_wait(&fullA[stage], phase, abort_flag, a.err, ERR_TIMEOUT_BASE + 3) ||
                !mbar_wait(&fullB[stage], phase, abort_flag, a.err, ERR_TIMEOUT_BASE + 4)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint64_t bdesc = sdesc(sB + stage * B_BYTES);
            const uint64_t adesc = sdesc(sA + stage * A_BYTES);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              if (h == 1 && a.hi_only) break;
#pragma unroll
              for (int kk = 0; kk < BK / 16; ++kk) {
                const uint64_t ad = adesc + (uint64_t)((h * A_HALF + kk * 32) >> 4);
                const uint64_t bd = bdesc + (uint64_t)((kk * 32) >> 4);
                mma_bf16(dt, ad, bd, (kb > kb0 || h > 0 || kk > 0) ? 1u : 0u);
              }
            }
            mma_commit(&empty[stage]);
            if (++stage == STAGES) { stage = 0; phase ^= 1; }
          }
          if (!ok) break;
          mma_commit(&accFull[buf]);
          if (++buf == 2) { buf = 0; accph ^= 1; }
        }
      }
      // all issued MMAs complete before tensor memory is released
      mma_commit(drain);
      const uint64_t t0 = gtimer();
      while (!mbar_try(drain, 0) && gtimer() - t0 < WAIT_NS) {
      }
    }
  } else if (warp >= GEN_WARP0) {
    // ---------------- mask generators: one thread per aperture row of the tile
    const int g = threadIdx.x - GEN_WARP0 * 32;  // 0..255
    int stage = 0;
    uint32_t phase = 0;
    const int64_t c = a.mg.c;
    uint8_t* rowbase0 = sB + (g >> 3) * 1024 + (g & 7) * 128;
    const int sw = g & 7;
    for (int64_t it = blockIdx.x; it < n_items; it += gridDim.x) {
      if (__shfl_sync(0xffffffffu, *abort_flag, 0)) break;
      const int64_t s = it % a.n_stripes;
      const int64_t j = a.j_begin + s * BN + g;
      const int64_t dj = j - c;
      int64_t bmax = -1;
      if (j < a.j_end && dj * dj <= a.mg.sR) bmax = isqrt_floor(a.mg.sR - dj * dj);
      const int64_t dj2 = dj * dj;
      for (int64_t kb = 0; kb < nkb; ++kb) {
        if (!warp_wait(&empty[stage], phase ^ 1, abort_flag, a.err, ERR_TIMEOUT_BASE + 5)) break;
        const int64_t i0 = kb * BK;
        uint64_t bits = 0;
        if (bmax >= 0) {
          int64_t ilo = c - bmax > i0 ? c - bmax : i0;
          int64_t ihi = c + bmax < i0 + BK - 1 ? c + bmax : i0 + BK - 1;
          if (ihi > a.N - 1) ihi = a.N - 1;
          if (ilo <= ihi) bits = row_bits(i0, ilo, ihi, c, dj2, a.mg);
        }
        uint8_t* rowp = rowbase0 + stage * B_BYTES;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const uint32_t byte = (uint32_t)(bits >> (8 * q)) & 0xFFu;
          uint4 v;
          v.x = pack2(byte);
          v.y = pack2(byte >> 2);
          v.z = pack2(byte >> 4);
          v.w = pack2(byte >> 6);
          *reinterpret_cast<uint4*>(rowp + ((q ^ sw) << 4)) = v;
        }
        fence_proxy_async();
        __syncwarp();
        if (lane == 0) mbar_arrive(&fullB[stage]);
        if (++stage == STAGES) { stage = 0; phase ^= 1; }
      }
    }
  } else {
    // ---------------- epilogue: warps 0-3 own TMEM lanes 32w..32w+31
    const int r = warp * 32 + lane;  // kernel row within the tile
    int buf = 0;
    uint32_t accph = 0;
    bool ok = true;
    for (int64_t it = blockIdx.x; it < n_items && ok; it += gridDim.x) {
      const int t = (int)(it / a.n_stripes);
      const int64_t s = it % a.n_stripes;
      float* crow = a.C1 + (int64_t)(t * BM + r) * a.c1_stride + (a.j_begin + s * BN - a.c1_j0);
      for (int64_t ch = 0; ch < nchunk; ++ch) {
        if (!warp_wait(&accFull[buf], accph, abort_flag, a.err, ERR_TIMEOUT_BASE + 6)) { ok = false; break; }
        tc_fence_after();
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(buf * BN);
#pragma unroll 1
        for (int col = 0; col < BN; col += 32) {
          float v[32];
          tmem_ld32(taddr + col, v);
          float4* dst = reinterpret_cast<float4*>(crow + col);
          if (ch == 0) {
#pragma unroll
            for (int q = 0; q < 8; ++q) dst[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
          } else {
#pragma unroll
            for (int q = 0; q < 8; ++q) {
              float4 o = dst[q];
              o.x += v[4 * q]; o.y += v[4 * q + 1]; o.z += v[4 * q + 2]; o.w += v[4 * q + 3];
              dst[q] = o;
            }
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&accEmpty[buf]);
        if (++buf == 2) { buf = 0; accph ^= 1; }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 5) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

// ---------------------------------------------------------------- kernel table
// A image of tile t, K block kb, part h (0 hi, 1 lo): 128 rows x 64 columns,
// K-major, 128-byte swizzle: element (r, k) at byte
//   (r/8)*1024 + (r%8)*128 + ((k/8) ^ (r%8))*16 + (k%8)*2.
__global__ void k_build_A(int M, int64_t N, int64_t kblocks, int64_t c, double kappa, double delta, uint8_t* A) {
  const int64_t total = (int64_t)(2 * M) * kblocks * BK;  // (row, column) pairs
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += stride) {
    const int64_t i = e % (kblocks * BK);
    const int rg = (int)(e / (kblocks * BK));  // global kernel row 0..2M-1
    const int t = rg / BM, r = rg % BM;
    const int m = t * 64 + (r & 63);
    const bool im = r >= 64;
    float v = 0.f;
    if (i < N) {
      const double di = (double)(i - c);
      const double th = di * di * (0.5 * kappa) - (double)(m - M / 2) * di * delta;
      const float2 k = cis_turns_f(th);
      v = im ? k.y : k.x;
    }
    const __nv_bfloat16 hi = __float2bfloat16_rn(v);
    const __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
    const int64_t kb = i / BK;
    const int k = (int)(i % BK);
    const int64_t blk = ((int64_t)t * kblocks + kb) * A_BYTES;
    const int off = (r >> 3) * 1024 + (r & 7) * 128 + (((k >> 3) ^ (r & 7)) << 4) + (k & 7) * 2;
    *reinterpret_cast<__nv_bfloat16*>(A + blk + off) = hi;
    *reinterpret_cast<__nv_bfloat16*>(A + blk + A_HALF + off) = lo;
  }
}

// The generator of k_dense, one (row, 64-column block) per thread, to bytes.
__global__ void k_mask_rows(MaskGeom mg, int64_t N, int64_t j0, int64_t rows, int64_t kblocks, uint8_t* out) {
  const int64_t total = rows * kblocks;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t / kblocks, kb = t % kblocks;
    const int64_t j = j0 + r, c = mg.c, dj = j - c;
    const int64_t i0 = kb * BK;
    uint64_t bits = 0;
    if (dj * dj <= mg.sR) {
      const int64_t bmax = isqrt_floor(mg.sR - dj * dj);
      int64_t ilo = c - bmax > i0 ? c - bmax : i0;
      int64_t ihi = c + bmax < i0 + BK - 1 ? c + bmax : i0 + BK - 1;
      if (ihi > N - 1) ihi = N - 1;
      if (ilo <= ihi) bits = row_bits(i0, ilo, ihi, c, dj * dj, mg);
    }
    for (int k = 0; k < BK && i0 + k < N; ++k) out[r * N + i0 + k] = (uint8_t)((bits >> k) & 1);
  }
}

size_t dense_smem_bytes() { return 1024 + STAGES * (A_BYTES + B_BYTES) + 256; }

}  // namespace

fzp_status dense_build_tables(Plan& P) {
  Dense& d = P.dn;
  d.kblocks = (P.N + BK - 1) / BK;
  d.ntiles = 2 * P.M / BM;
  d.promote_kblocks = 16;
  if (const char* e = getenv("FZP_DENSE_PROMOTE")) d.promote_kblocks = std::max(1, atoi(e));
  int dev = 0;
  FZP_CUDA_TRY(cudaGetDevice(&dev));
  FZP_CUDA_TRY(cudaDeviceGetAttribute(&d.num_sms, cudaDevAttrMultiProcessorCount, dev));
  const size_t bytes = (size_t)d.ntiles * (size_t)d.kblocks * A_BYTES;
  FZP_CUDA_TRY(cudaMalloc(&d.d_A, bytes));
  P.device_bytes += bytes;
  k_build_A<<<4 * d.num_sms, 256>>>(P.M, P.N, d.kblocks, P.c, P.kappa, P.delta, reinterpret_cast<uint8_t*>(d.d_A));
  FZP_CUDA_TRY(cudaGetLastError());
  FZP_CUDA_TRY(cudaFuncSetAttribute(k_dense, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dense_smem_bytes()));
  return FZP_OK;
}

fzp_status dense_mask(Plan& P, int64_t j0, int64_t rows, uint8_t* out, cudaStream_t s) {
  k_mask_rows<<<1024, 256, 0, s>>>(P.mg, P.N, j0, rows, P.dn.kblocks, out);
  P.launches += 1;
  FZP_CUDA_TRY(cudaGetLastError());
  return FZP_OK;
}

fzp_status dense_rows(Plan& P, int64_t j0, int64_t rows, cudaStream_t s) {
  const Dense& d = P.dn;
  DenseArgs a{};
  a.mg = P.mg;
  a.N = P.N;
  a.kblocks = d.kblocks;
  a.j_begin = j0;
  a.j_end = j0 + rows;
  a.n_stripes = (rows + BN - 1) / BN;
  a.ntiles = d.ntiles;
  a.promote = d.promote_kblocks;
  a.hi_only = P.precision == FZP_PREC_BF16 ? 1 : 0;
  a.A = reinterpret_cast<const uint8_t*>(d.d_A);
  a.C1 = P.d_C1;
  a.c1_stride = P.chunk_rows;
  a.c1_j0 = j0;
  a.err = P.d_err;
  const int64_t items = a.n_stripes * a.ntiles;
  const int grid = (int)std::min<int64_t>(items, d.num_sms);
  P.dominant = "dense_tcgen05";
  prof_begin(P, s);
  k_dense<<<grid, NUM_THREADS, dense_smem_bytes(), s>>>(a);
  prof_end(P, s);
  P.launches += 1;
  FZP_CUDA_TRY(cudaGetLastError());
  return FZP_OK;
}

}  // namespace fzp
