// dense.cu -- form (b): the row transform as a dense tensor-core contraction.
//
// The kernel of Eq. 2 is separable (Sec. 2.6), so the focal-plane field is
//   U = Pre chirp_out .* (K T K^T),   K[m, i] = exp(2 pi i theta(m, i)),
//   theta(m, i) = di^2 kappa/2 - (m - msh) di delta   (turns; msh = M/2 for the
//   ROI centred on the focus, -x0/p otherwise),
// and the row pass C1 = K T^T is a real GEMM with
//   A = [Re K; Im K] (2M x N, split as K = K_hi + K_lo, both BF16),
//   B = T (aperture rows x N, binary: exact in BF16),
//   D = FP32 accumulators in tensor memory.
// K_hi T^T + K_lo T^T is accumulated into the same accumulator, so the product
// carries the ~16 significant bits of the split kernel.
//
// GB300 mapping (tcgen05, one CTA per SM, persistent over units, clusters of
// CL = 4 CTAs for M = 512):
//   unit     : one stripe of 256 aperture rows x one pair of kernel tiles
//              (2 x 128 kernel rows = 128 values of m, Re and Im); the CL CTAs
//              of a cluster take CL pairs of the same stripe
//   stage    : K step of 32 columns, 64-byte-swizzled K-major operands
//              (A 32 KiB: [t0 hi][t1 hi][t0 lo][t1 lo]; B 16 KiB), 4 stages
//   warp 8   : copies the A stage, pre-swizzled in HBM, with one cp.async.bulk
//   warps 10-17: mask generators in CL phases; each CTA generates 256 / CL of the
//              stripe's rows for every CL-th stage (two zone evaluations give a
//              block's toggle events; the thresholds of a warp's rows come from
//              one coalesced load) and bulk-copies them to its peers' shared memory
//   warp 9   : allocates 512 TMEM columns and issues tcgen05.mma (M128 N256 K16)
//              into two FP32 accumulators (one per tile), completion multicast
//              to the cluster's empty barriers
//   warps 0-7: epilogue; every `promote` stages both accumulators are read with
//              tcgen05.ld into shared memory and added into C1 by TMA
//              reduce-add (C1 zeroed before the launch).  The tensor core's
//              FP32 accumulation loses precision in proportion to the chunk
//              length (measured: 8e-4 relative error of I over a 0.25 m
//              aperture without promotion, 8e-6 with 4096-sample chunks).
// Phase plates: L = 2 as a +-1 mask (disc and odd-zone bits); L >= 4 as L/2
// passes of -1 / 0 / +1 masks on level sets (level mode of the generator).
// Deformed membranes (complex transmission T e^{i phi}): two passes with the
// real masks T cos(phi) and T sin(phi), whose fields enter the ROI sum with
// weights 1 and i; each mask value is split as BF16 hi + lo (it is not exact
// in BF16), so a K step takes K_hi B_hi + K_lo B_hi + K_hi B_lo (the dropped
// K_lo B_lo is ~2^-17 of the product) in 3 stages of 64 KiB.
// Every mbarrier wait is bounded in time; on expiry the kernel records an error
// code, drains what it issued, frees tensor memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>

#include "fzp_internal.cuh"
#include "tc_ptx.cuh"

namespace fzp {
namespace {

constexpr int BM = 128;               // kernel rows per MMA (tcgen05 M)
constexpr int TILES = 2;               // kernel tiles per item: 256 kernel rows share one mask tile
constexpr int BN = 256;                // aperture rows per item (tcgen05 N)
constexpr int BK = 32;                 // K per stage: one 64-byte swizzle row of BF16
constexpr int STAGES = 4;
constexpr int STAGES_CX = 3;           // membrane passes: A 32 KiB + B hi and lo planes 32 KiB
constexpr int SUB = BM * BK * 2;       // 8 KiB: one (tile, hi|lo) operand image
constexpr int A_BYTES = TILES * 2 * SUB;  // 32 KiB per stage: [t0 hi][t1 hi][t0 lo][t1 lo]
constexpr int B_BYTES = BN * BK * 2;      // 16 KiB per stage (per plane)
constexpr int EPI_WARPS = 8;           // warps 0-7: epilogue (tile = warp / 4)
constexpr int LOAD_WARP = 8, MMA_WARP = 9, GEN_WARP0 = 10;
constexpr int GEN_WARPS = 8;           // warps 10-17: mask generators
constexpr int NUM_THREADS = (GEN_WARP0 + GEN_WARPS) * 32;
constexpr int TMEM_COLS = 512;         // two 128 x 256 FP32 accumulators
constexpr int EPI_BOX = 32;            // epilogue: 32 rows x 32 columns FP32 per bulk reduction
constexpr int EPI_BYTES = EPI_WARPS * EPI_BOX * EPI_BOX * 4;  // 32 KiB of staging, one box per warp
constexpr int ERR_TIMEOUT_BASE = 100;

struct DenseArgs {
  MaskGeom mg;
  int64_t N;
  int64_t kblocks;          // ceil(N / BK)
  int64_t j_begin, j_end;   // aperture rows of this launch [j_begin, j_end)
  int64_t n_stripes;        // ceil((j_end - j_begin) / BN)
  const int* sched;         // work list (k_dense_sched): off[nchunks + 1], slo[nchunks], cnt[nchunks]
  int nchunks;              // ceil(kblocks / group): K chunks of the work list
  int group;                // K blocks per work-list chunk (a multiple of promote)
  int npairs;               // kernel tile pairs (items per stripe; a multiple of the cluster size)
  int M;                    // ROI side: tiles t with 64 t >= M are zero padding, not stored
  int signed_mask;          // 1: binary phase plate, T = +1 / -1 on even / odd zones inside the disc
  int level_mode;           // 1: phase plate pass: +1 on levels in pos, -1 on levels in neg
  int lmod;                 // level count L (level = zone step mod L)
  uint64_t pos, neg;        // level sets of the pass (bit q)
  int promote;              // stages per accumulation chunk
  int hi_only;              // 1: BF16 kernel (hi) only
  int cx_sin;               // membrane pass: 0 -> mask T cos(phi), 1 -> T sin(phi)
  DeformCoef df;            // membrane pass: the deformation phase
  const float* ld_src;      // non-null (membrane-pass kernels): B loaded from this real matrix,
  int64_t ld_stride;        //   row j at ld_src + j * ld_stride, every K block of every stripe
  const uint8_t* A;         // pre-swizzled kernel tiles, [pair][kb][t0hi t1hi t0lo t1lo]
  float* C1;                // [rows][c1_stride], column = j - c1_j0
  int64_t c1_stride, c1_j0;
  int* err;
};

// ---------------------------------------------------------------- form-specific PTX
using namespace tc;

// Shared-memory matrix descriptor: K-major, 64-byte swizzle (rows of 64 B,
// 8-row groups 512 B apart), version 1.
__device__ __forceinline__ uint64_t sdesc(const void* p) {
  const uint64_t a = smem_u32(p);
  return ((a >> 4) & 0x3FFFull) | (1ull << 16) | ((uint64_t)(512 >> 4) << 32) | (1ull << 46) | (4ull << 61);
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
// ---------------------------------------------------------------- mask walker
__device__ __forceinline__ int64_t isqrt_floor(int64_t t) {  // largest a with a^2 <= t (t >= 0)
  int64_t a = (int64_t)sqrtf((float)t);
  while (a * a > t) --a;
  while ((a + 1) * (a + 1) <= t) ++a;
  return a;
}

// Smallest a >= 0 with a^2 >= t, for 0 < t < 2^46.  t converted to float
// (relative error 2^-24) and the approximate square root (relative error
// below 2^-23) give r within 1.3 of sqrt(t) for a < 2^23, so floor(r) lies in
// [a - 3, a + 1]; exact integer corrections follow, without branches.
__device__ __forceinline__ uint32_t ceil_sqrt46(int64_t t) {
  const float tf = __ll2float_rn(t);
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(tf));
  uint32_t a = (uint32_t)r;
  a += ((int64_t)((uint64_t)a * a) < t) ? 1u : 0u;
  a += ((int64_t)((uint64_t)a * a) < t) ? 1u : 0u;
  a += ((int64_t)((uint64_t)a * a) < t) ? 1u : 0u;
  a -= (a > 0 && (int64_t)((uint64_t)(a - 1) * (a - 1)) >= t) ? 1u : 0u;
  return a;
}

// Walks one aperture row from column 0 upwards and yields the columns where
// the binary transmission toggles.  Along the row the zone index is a function
// of d = |i - c|, non-decreasing in d, stepping at d = a_m = ceil(sqrt(S_m - dj^2));
// the open state toggles at every step and at both ends of the disc chord.
// Toggle columns, numbered by the event index e (L = z_e - z_c boundaries per half):
//   c - bmax                       start of the chord (only if the edge zone z_e is odd)
//   c - a_m + 1, m = z_e .. z_c+1  zone drops below m (left half)
//   c + a_m,     m = z_c+1 .. z_e  zone reaches m (right half)
//   c + bmax + 1                   end of the chord (only if z_e is odd)
struct Walker {
  int64_t next;  // column of event e (INT64_MAX: none left)
  int64_t dj2, c, bmax, zc, ze;
  int32_t e, ne, L, odd;
  int32_t in;    // the row meets the aperture disc (chord [c - bmax, c + bmax])
};

__device__ __forceinline__ int64_t walker_event(const Walker& w, int32_t e, const int64_t* __restrict__ thr) {
  if (e >= w.ne) return INT64_MAX;
  const int32_t b = e - w.odd;  // boundary index, -1 = chord start, 2L = chord end
  if (b < 0) return w.c - w.bmax;
  if (b >= 2 * w.L) return w.c + w.bmax + 1;
  const bool left = b < w.L;
  const int64_t m = left ? w.ze - b : w.zc + 1 + (b - w.L);
  const int64_t a = (int64_t)ceil_sqrt46(__ldg(thr + (m - 1)) - w.dj2);
  return left ? w.c - a + 1 : w.c + a;
}

// level_events: the chord's two ends are events of every row (a phase plate
// is nonzero on the whole chord); otherwise only where the edge zone is open.
__device__ __forceinline__ void walker_init(Walker& w, int64_t j, int64_t j_end, const MaskGeom& g,
                                            bool level_events = false) {
  w.c = g.c;
  w.e = 0;
  w.ne = 0;
  w.in = 0;
  w.next = INT64_MAX;
  const int64_t dj = j - g.c;
  if (j >= j_end || dj * dj > g.sR) return;
  w.in = 1;
  w.dj2 = dj * dj;
  w.bmax = isqrt_floor(g.sR - w.dj2);
  w.zc = zone_of(w.dj2, g);
  w.ze = zone_of(w.dj2 + w.bmax * w.bmax, g);
  w.L = (int32_t)(w.ze - w.zc);
  w.odd = level_events ? 1 : (int32_t)(w.ze & 1);
  w.ne = 2 * w.L + 2 * w.odd;
  w.next = walker_event(w, 0, g.thr);
}

// Open bits of columns [i0, i0 + 32) given the open state at i0; updates the state.
__device__ __forceinline__ uint32_t walker_bits(Walker& w, int64_t i0, uint32_t& state, const int64_t* thr) {
  uint32_t bits = 0u - state;
  while (w.next < i0 + 32) {
    bits ^= 0xFFFFFFFFu << (uint32_t)(w.next - i0);
    state ^= 1u;
    w.next = walker_event(w, ++w.e, thr);
  }
  return bits;
}

// Number of toggle events at columns <= X; the open state after column X is
// its parity.  Left of the axis the zone at distance d = c - X says how many
// left boundaries lie at or before X (those with m above it); right of the
// axis the zone at d = X - c counts the right boundaries reached.
__device__ __forceinline__ int32_t walker_count(const Walker& w, int64_t X, const MaskGeom& g) {
  if (w.ne == 0 || X < w.c - w.bmax) return 0;
  if (X < w.c) {
    const int64_t d = w.c - X;
    return w.odd + (int32_t)(w.ze - zone_of(w.dj2 + d * d, g));
  }
  const int64_t d = X - w.c < w.bmax ? X - w.c : w.bmax;
  return w.odd + w.L + (int32_t)(zone_of(w.dj2 + d * d, g) - w.zc) + (X > w.c + w.bmax ? w.odd : 0);
}

// Open bits of columns [i0, i0 + 32) of the walker's row, for a whole warp at
// once (each lane a row of the same stripe; every lane of the warp calls it).
// Two zone evaluations give the block's events [e0, e1) without walking; the
// zone boundaries among them index thresholds S_m that, over the warp's 32
// neighbouring rows, form one short contiguous range of m (at most ~17 at four
// samples per outermost zone), read with one coalesced load and handed to the
// lanes by shuffles.  The events are independent of each other, so the block
// costs one memory round trip instead of one per toggle.  In two halves:
// block_prep finds the events and issues the threshold load, block_finish
// turns them into bits; the generator prepares its next block before it
// finishes the current one, so the load's latency is hidden.
// Per block, a boundary's distance a = ceil(sqrt(S_m - dj^2)) from the axis lies
// in a 32-wide window [d, d + 31] fixed by the block (right of the axis
// d = i0 - c, left of it d = c - i0 - 30).  With a = d + k, k is the smallest
// k >= 0 with k (k + 2d) >= S_m - dj^2 - d^2, a 32-bit quantity; for d >= 1024
// the estimate (S_m - dj^2 - d^2) / (2d) is off by less than 31^2 / (2d) < 1,
// and two steps up and one down in 32-bit arithmetic make k exact.  Blocks
// within 1024 columns of the axis use the 64-bit square root.
struct BlockPrep {
  int32_t e0, e1, wlo, nev;
  int staged;
  long long tv;
  int64_t D2r, D2l;     // dj^2 + d^2, right and left of the axis
  float ir, il;         // 1 / (2 d)
  int32_t tdr, tdl;     // 2 d
  int fr, fl;           // the 32-bit path applies
};

__device__ __forceinline__ int32_t window_k(int32_t D, float inv2d, int32_t two_d) {
  int32_t k = __float2int_ru((float)D * inv2d);
  k = k < 0 ? 0 : k;
  k += (k * (k + two_d) < D) ? 1 : 0;
  k += (k * (k + two_d) < D) ? 1 : 0;
  k -= (k > 0 && (k - 1) * (k - 1 + two_d) >= D) ? 1 : 0;
  return k;
}

// Column of boundary event b (0 <= b < 2L) of the walker's row, relative to i0.
__device__ __forceinline__ uint32_t boundary_col(const Walker& w, int64_t i0, const BlockPrep& p, int32_t b,
                                                 long long S) {
  if (b < w.L) {  // left of the axis: column c - a + 1
    if (p.fl) return 31u - (uint32_t)window_k((int32_t)((int64_t)S - p.D2l), p.il, p.tdl);
    const int64_t aa = (int64_t)ceil_sqrt46((int64_t)S - w.dj2);
    return (uint32_t)(w.c - aa + 1 - i0);
  }
  if (p.fr) return (uint32_t)window_k((int32_t)((int64_t)S - p.D2r), p.ir, p.tdr);
  const int64_t aa = (int64_t)ceil_sqrt46((int64_t)S - w.dj2);
  return (uint32_t)(w.c + aa - i0);
}

__device__ __forceinline__ void block_prep(const Walker& w, int64_t i0, const MaskGeom& g, BlockPrep& p) {
  p.e0 = walker_count(w, i0 - 1, g);
  p.e1 = walker_count(w, i0 + 31, g);
  // thresholds of this lane's boundary events: b = e - odd in [b0, b1) within [0, 2L)
  int32_t mlo = INT32_MAX, mhi = INT32_MIN;
  const int32_t b0 = max(p.e0 - w.odd, 0), b1 = min(p.e1 - w.odd, 2 * w.L);
  if (w.ne > 0 && b1 > b0) {
    if (b0 < w.L) {  // left boundaries: m = ze - b
      mlo = (int32_t)w.ze - (min(b1, w.L) - 1);
      mhi = (int32_t)w.ze - b0;
    }
    if (b1 > w.L) {  // right boundaries: m = zc + 1 + (b - L)
      mlo = min(mlo, (int32_t)w.zc + 1 + (max(b0, w.L) - w.L));
      mhi = max(mhi, (int32_t)w.zc + (b1 - w.L));
    }
  }
  p.wlo = __reduce_min_sync(0xffffffffu, mlo);
  const int32_t whi = __reduce_max_sync(0xffffffffu, mhi);
  p.nev = (int32_t)__reduce_max_sync(0xffffffffu, (uint32_t)(p.e1 - p.e0));
  p.staged = (whi >= p.wlo && whi - p.wlo < 32) ? 1 : 0;
  const int lane = threadIdx.x & 31;
  p.tv = 0;
  if (p.staged && p.wlo + lane <= whi) p.tv = __ldg(g.thr + (p.wlo + lane - 1));
  const int64_t dr = i0 - w.c, dl = w.c - i0 - 30;
  p.fr = dr >= 1024 ? 1 : 0;
  p.fl = dl >= 1024 ? 1 : 0;
  p.D2r = w.dj2 + dr * dr;
  p.D2l = w.dj2 + dl * dl;
  p.tdr = (int32_t)(2 * dr);
  p.tdl = (int32_t)(2 * dl);
  p.ir = p.fr ? 0.5f / (float)dr : 0.0f;
  p.il = p.fl ? 0.5f / (float)dl : 0.0f;
}

__device__ __forceinline__ uint32_t block_finish(const Walker& w, int64_t i0, const MaskGeom& g, const BlockPrep& p) {
  uint32_t bits = 0u - ((uint32_t)p.e0 & 1u);
#pragma unroll 2
  for (int32_t t = 0; t < p.nev; ++t) {
    const int32_t e = p.e0 + t, b = e - w.odd;
    const bool valid = e < p.e1;
    const bool bnd = valid && b >= 0 && b < 2 * w.L;
    const bool left = b < w.L;
    const int32_t m = bnd ? (left ? (int32_t)w.ze - b : (int32_t)w.zc + 1 + (b - w.L)) : p.wlo;
    long long S = __shfl_sync(0xffffffffu, p.tv, (m - p.wlo) & 31);
    if (bnd && !p.staged) S = __ldg(g.thr + (m - 1));
    if (valid) {
      uint32_t cc;
      if (b < 0) cc = (uint32_t)(w.c - w.bmax - i0);            // chord start
      else if (b >= 2 * w.L) cc = (uint32_t)(w.c + w.bmax + 1 - i0);  // chord end
      else cc = boundary_col(w, i0, p, b, S);
      bits ^= 0xFFFFFFFFu << cc;
    }
  }
  return bits;
}


// Zone step of the row after its first e events (walker with level events):
// -1 before the chord start or after its end.
__device__ __forceinline__ int32_t zone_after(const Walker& w, int32_t e) {
  if (e <= 0 || e >= w.ne) return -1;
  const int32_t nb = e - 1;  // zone boundaries passed
  return nb <= w.L ? (int32_t)w.ze - nb : (int32_t)w.zc + (nb - w.L);
}

// Phase-plate pass: bits of columns [i0, i0 + 32) where the level (zone step
// mod lmod) is in `pos` (out_pos) or in `neg` (out_neg), from the block's
// prepared events (block_prep, with level events); whole warp.  Between two
// events the zone step is constant, so each block is a few runs of columns.
__device__ __forceinline__ void block_values(const Walker& w, int64_t i0, const MaskGeom& g, const BlockPrep& p,
                                             int lmod, uint64_t pos, uint64_t neg, uint32_t& out_pos,
                                             uint32_t& out_neg) {
  uint32_t P = 0u, Q = 0u;
  int32_t z = zone_after(w, p.e0);
  uint32_t c0 = 0;  // first column of the current run, relative to i0
  const int lmask = (lmod & (lmod - 1)) == 0 ? lmod - 1 : -1;  // power-of-two L: a mask, no division
  auto fill = [&](int32_t zz, uint32_t a, uint32_t b) {
    if (zz < 0 || b <= a) return;
    const int q = lmask >= 0 ? (zz & lmask) : zz % lmod;
    const uint32_t m = (b >= 32 ? 0xFFFFFFFFu : ((1u << b) - 1u)) & ~((1u << a) - 1u);
    if ((pos >> q) & 1ull) P |= m;
    if ((neg >> q) & 1ull) Q |= m;
  };
  for (int32_t t = 0; t < p.nev; ++t) {
    const int32_t e = p.e0 + t, b = e - w.odd;
    const bool valid = e < p.e1;
    const bool bnd = valid && b >= 0 && b < 2 * w.L;
    const bool left = b < w.L;
    const int32_t m = bnd ? (left ? (int32_t)w.ze - b : (int32_t)w.zc + 1 + (b - w.L)) : p.wlo;
    long long S = __shfl_sync(0xffffffffu, p.tv, (m - p.wlo) & 31);
    if (bnd && !p.staged) S = __ldg(g.thr + (m - 1));
    if (valid) {
      uint32_t cc;
      if (b < 0) cc = (uint32_t)(w.c - w.bmax - i0);
      else if (b >= 2 * w.L) cc = (uint32_t)(w.c + w.bmax + 1 - i0);
      else cc = boundary_col(w, i0, p, b, S);
      fill(z, c0, cc);
      z = zone_after(w, e + 1);
      c0 = cc;
    }
  }
  fill(z, c0, 32u);
  out_pos = P;
  out_neg = Q;
}

// Columns [i0, i0 + 32) of the row that lie on its chord of the aperture disc.
__device__ __forceinline__ uint32_t disc_bits(const Walker& w, int64_t i0) {
  if (!w.in) return 0u;
  const int64_t lo = w.c - w.bmax - i0, hi = w.c + w.bmax - i0;  // inclusive, relative to i0
  if (hi < 0 || lo > 31) return 0u;
  const uint32_t a = lo <= 0 ? 0xFFFFFFFFu : (0xFFFFFFFFu << (uint32_t)lo);
  const uint32_t b = hi >= 31 ? 0xFFFFFFFFu : (0xFFFFFFFFu >> (uint32_t)(31 - hi));
  return a & b;
}

// K blocks [klo, khi) of stripe s that meet the aperture disc: every row's
// chord lies inside the chord of the stripe's row nearest the axis, so blocks
// outside that chord multiply zero mask columns only and are skipped.  At
// least one block (a stripe with no row on the disc still writes its zero
// rows of C1).  Every role of the kernel derives the same range.
__device__ __forceinline__ void stripe_kspan(const DenseArgs& a, int64_t s, int64_t& klo, int64_t& khi) {
  if (a.ld_src) {  // a loaded operand is dense: no chord bound
    klo = 0;
    khi = a.kblocks;
    return;
  }
  const int64_t jb = a.j_begin + s * BN;
  const int64_t je = jb + BN < a.j_end ? jb + BN : a.j_end;
  const int64_t c = a.mg.c;
  const int64_t jn = c < jb ? jb : (c >= je ? je - 1 : c);
  const int64_t t = a.mg.sR - (jn - c) * (jn - c);
  if (t < 0) {
    klo = c / BK < a.kblocks ? c / BK : a.kblocks - 1;
    khi = klo + 1;
    return;
  }
  const int64_t b = isqrt_floor(t);
  klo = c - b > 0 ? (c - b) / BK : 0;
  khi = (c + b) / BK + 1 < a.kblocks ? (c + b) / BK + 1 : a.kblocks;
  if (khi <= klo) khi = klo + 1;
}

// Work units in chunk-major order: unit (g, pair group pu, stripe s) covers the
// K blocks of chunk g, [g Q, (g + 1) Q) with Q = group (a few promotion
// lengths), that meet stripe s's disc chord; units of one chunk are
// consecutive, so the clusters of a wave read the same kernel-matrix blocks
// (one fetch from HBM, the rest from L2).  A unit promotes its accumulators
// into C1 (reduce-add) after every `promote` blocks; its C1 tile stays in L2
// between those promotions.
// Per chunk g the stripes meeting it are a contiguous range [slo_g, slo_g +
// cnt_g) (the chords are nested about the stripe nearest the axis); off_g counts
// the units before chunk g.
struct Unit {
  int64_t s, pu, kb0, kb1;
};

__device__ __forceinline__ Unit unit_at(const DenseArgs& a, int64_t it, int npg) {
  const int* off = a.sched;
  const int* slo = a.sched + a.nchunks + 1;
  const int* cnt = slo + a.nchunks;
  int lo = 0, hi = a.nchunks - 1;  // largest g with off[g] <= it
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if ((int64_t)__ldg(off + mid) <= it) lo = mid;
    else hi = mid - 1;
  }
  const int g = lo;
  const int64_t r = it - __ldg(off + g), c = __ldg(cnt + g);
  Unit u;
  u.pu = r / c;
  u.s = __ldg(slo + g) + r % c;
  int64_t klo, khi;
  stripe_kspan(a, u.s, klo, khi);
  const int64_t c0 = (int64_t)g * a.group, c1 = c0 + a.group;
  u.kb0 = klo > c0 ? klo : c0;
  u.kb1 = khi < c1 ? khi : c1;
  (void)npg;
  return u;
}

// Builds the work list of one k_dense launch (one block).  For each chunk g the
// stripes meeting it are found by bisection on either side of the stripe
// nearest the axis, whose chord holds every other stripe's.
__global__ void k_dense_sched(const DenseArgs a, int npg, int* sched) {
  int* off = sched;
  int* slo = sched + a.nchunks + 1;
  int* cnt = slo + a.nchunks;
  const int64_t ns = a.n_stripes;
  int64_t sc = (a.mg.c - a.j_begin) / BN;
  sc = a.mg.c < a.j_begin ? 0 : (sc >= ns ? ns - 1 : sc);
  for (int g = threadIdx.x; g < a.nchunks; g += blockDim.x) {
    const int64_t c0 = (int64_t)g * a.group, c1 = c0 + a.group;
    auto meets = [&](int64_t st) {
      int64_t klo, khi;
      stripe_kspan(a, st, klo, khi);
      return klo < c1 && khi > c0;
    };
    if (!meets(sc)) {
      slo[g] = (int)sc;
      cnt[g] = 0;
      continue;
    }
    int64_t lo = 0, hi = sc;  // first stripe in [0, sc] that meets the chunk
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (meets(mid)) hi = mid;
      else lo = mid + 1;
    }
    const int64_t first = lo;
    lo = sc;
    hi = ns - 1;  // last stripe in [sc, ns) that meets it
    while (lo < hi) {
      const int64_t mid = (lo + hi + 1) >> 1;
      if (meets(mid)) lo = mid;
      else hi = mid - 1;
    }
    slo[g] = (int)first;
    cnt[g] = (int)(lo - first + 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t acc = 0;
    for (int g = 0; g < a.nchunks; ++g) {
      off[g] = (int)acc;
      acc += (int64_t)cnt[g] * npg;
    }
    off[a.nchunks] = (int)acc;
  }
}

__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel) {
  uint32_t d;
  asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(sel));
  return d;
}

// 32 mask bits -> 32 BF16 values (1.0 = 0x3F80, 0.0) in 16 words.  y_j = bits
// << (7 - j) puts sample 8q + j in the sign bit of byte q; prmt with the
// sign-replicate selector expands two such bytes to 0x00/0xFF per output byte,
// and the AND keeps 0x3F80 in each half-word.
__device__ __forceinline__ void expand_bits(uint32_t bits, uint32_t (&w)[16]) {
  uint32_t y[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) y[j] = bits << (7 - j);
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const int q = k >> 2, j = 2 * (k & 3);  // samples 2k = 8q + j and 8q + j + 1
    const uint32_t sel = (uint32_t)((8 | q) | ((8 | q) << 4) | ((8 | (4 + q)) << 8) | ((8 | (4 + q)) << 12));
    w[k] = prmt(y[j], y[j + 1], sel) & 0x3F803F80u;
  }
}

// Binary phase plate: +1 (0x3F80) on the disc, -1 (0xBF80) where also on an
// odd zone (odd is a subset of disc), 0 off the disc.
__device__ __forceinline__ void expand_signed(uint32_t disc, uint32_t odd, uint32_t (&w)[16]) {
  uint32_t mag[16], sgn[16];
  expand_bits(disc, mag);
  expand_bits(odd, sgn);
#pragma unroll
  for (int k = 0; k < 16; ++k) w[k] = mag[k] | ((sgn[k] << 8) & 0x80008000u);
}

// Membrane pass: one row's T cos(phi) (or T sin(phi)) on 8-column chunks of a
// 32-column block given the block's open bits, as BF16 hi and lo planes (the
// 16-byte chunks of the 64-byte-swizzled row).  phi / 2 pi = 2 w / lambda in
// FP32, walked along the row from the first column: the wrinkle's phasor
// e^{2 pi i t} (t = di kx + dj ky, integer turns dropped exactly) turns by
// e^{2 pi i kx} per column, a ridge's g = exp(-q d^2) by its ratio r, which
// itself scales by rho = exp(-2 q nx^2); the sum is reduced to [-1/2, 1/2]
// turns before one hardware sine or cosine (absolute error below 4e-7; the
// walk adds ~1e-6 relative over 32 columns).  A ridge below 1e-30 at the
// first column stays below 1e-29 in the block (its width is hundreds of
// columns) and is left out.
struct CxRow {
  float fjkh, fjkl, fj2, cr[3];  // row terms: dj kyh, dj kyl, dj^2, ridge offsets
};

__device__ __forceinline__ void cx_row_init(const DeformCoef& d, int64_t dj, CxRow& r) {
  const float fj = (float)dj;
  r.fjkh = fj * d.kyh;
  r.fjkl = fj * d.kyl;
  r.fj2 = fj * fj;
#pragma unroll
  for (int e = 0; e < 3; ++e) r.cr[e] = (fj - d.pj[e]) * d.ny[e] - d.pi_[e] * d.nx[e];
}

// Two FP32 values -> packed BF16 hi (RN) and lo (RN of the remainder), lower
// half from a: one cvt.rn.bf16x2 per plane (a goes to the upper half of the
// instruction's result when given first, so b is given first).
__device__ __forceinline__ void split2(float a, float b, uint32_t& hi, uint32_t& lo) {
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(hi) : "f"(b), "f"(a));
  const float ah = __uint_as_float(hi << 16), bh = __uint_as_float(hi & 0xffff0000u);
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(lo) : "f"(b - bh), "f"(a - ah));
}

// Chunks [q0, q0 + nq) of the row (8 columns each); di0 = column of the block
// start minus c; NR ridges.
template <int NR>
__device__ __forceinline__ void cx_store_n(const DeformCoef& d, const CxRow& r, int64_t di0, uint32_t bits,
                                           int sinpart, uint8_t* hi_row, uint8_t* lo_row, int sw, int q0, int nq) {
  constexpr float TWO_PI = 6.28318530717958648f;
  float fi = (float)(di0 + 8 * q0);
  // wrinkle phasor at the first column
  const float th = fmaf(fi, d.kxh, r.fjkh);
  float tt = (th - rintf(th)) + fmaf(fi, d.kxl, r.fjkl);
  tt -= rintf(tt);
  float ws, wc;
  __sincosf(TWO_PI * tt, &ws, &wc);
  // ridges at the first column, and their ratios to the next column
  float g[NR > 0 ? NR : 1], rr[NR > 0 ? NR : 1];
#pragma unroll
  for (int e = 0; e < NR; ++e) {
    g[e] = 0.0f;
    rr[e] = 1.0f;
    const float d0 = fmaf(fi, d.nx[e], r.cr[e]);
    const float ex = d.q[e] * d0 * d0;
    if (ex < 69.0f) {
      g[e] = __expf(-ex);
      rr[e] = __expf(-d.q[e] * d.nx[e] * fmaf(2.0f, d0, d.nx[e]));
    }
  }
#pragma unroll 1
  for (int q = q0; q < q0 + nq; ++q) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int k = 0; k < 8; k += 2) {
      float v[2];
#pragma unroll
      for (int z = 0; z < 2; ++z) {
        float wz = d.amp2 * ws * fmaf(-d.tq, fmaf(fi, fi, r.fj2), 1.0f);
#pragma unroll
        for (int e = 0; e < NR; ++e) {
          wz = fmaf(d.h2[e], g[e], wz);
          g[e] *= rr[e];
          rr[e] *= d.rho[e];
        }
        const float nws = fmaf(ws, d.zc, wc * d.zs);
        wc = fmaf(wc, d.zc, -ws * d.zs);
        ws = nws;
        fi += 1.0f;
        wz -= rintf(wz);
        const float x = TWO_PI * wz;
        const int col = 8 * q + k + z;
        v[z] = ((bits >> col) & 1u) ? (sinpart ? __sinf(x) : __cosf(x)) : 0.0f;
      }
      split2(v[0], v[1], h[k / 2], l[k / 2]);
    }
    *reinterpret_cast<uint4*>(hi_row + ((q ^ sw) << 4)) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4*>(lo_row + ((q ^ sw) << 4)) = make_uint4(l[0], l[1], l[2], l[3]);
  }
}

// The membrane values of a block's row parts, specialised on the ridge count
// (0 to 3, uniform over the launch).
__device__ __forceinline__ void cx_store(const DeformCoef& d, const CxRow& r, int64_t di0, uint32_t bits, int sinpart,
                                         uint8_t* hi_row, uint8_t* lo_row, int sw, int q0, int nq) {
  switch (d.n) {
    case 0: cx_store_n<0>(d, r, di0, bits, sinpart, hi_row, lo_row, sw, q0, nq); break;
    case 1: cx_store_n<1>(d, r, di0, bits, sinpart, hi_row, lo_row, sw, q0, nq); break;
    case 2: cx_store_n<2>(d, r, di0, bits, sinpart, hi_row, lo_row, sw, q0, nq); break;
    default: cx_store_n<3>(d, r, di0, bits, sinpart, hi_row, lo_row, sw, q0, nq); break;
  }
}

// A loaded B row (the SA-CZT zoom): 8-column parts q0 .. q0 + nq - 1 of one
// K block of an FP32 row (src = its first column, or null for a row past the
// matrix), split into BF16 hi and lo planes like the membrane values.
__device__ __forceinline__ void ld_store(const float* src, uint8_t* hi_row, uint8_t* lo_row, int sw, int q0, int nq) {
#pragma unroll 1
  for (int q = q0; q < q0 + nq; ++q) {
    float4 x = make_float4(0.f, 0.f, 0.f, 0.f), y = x;
    if (src) {
      x = __ldg(reinterpret_cast<const float4*>(src + 8 * q));
      y = __ldg(reinterpret_cast<const float4*>(src + 8 * q + 4));
    }
    uint32_t h[4], l[4];
    split2(x.x, x.y, h[0], l[0]);
    split2(x.z, x.w, h[1], l[1]);
    split2(y.x, y.y, h[2], l[2]);
    split2(y.z, y.w, h[3], l[3]);
    *reinterpret_cast<uint4*>(hi_row + ((q ^ sw) << 4)) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4*>(lo_row + ((q ^ sw) << 4)) = make_uint4(l[0], l[1], l[2], l[3]);
  }
}

// ---------------------------------------------------------------- kernel
// Work units: unit u = (tile-pair group pu = u / n_stripes, stripe s = u % n_stripes);
// CTA rank rk of a cluster of CL takes pair pu * CL + rk, so the CL CTAs of a
// cluster work on the same stripe with different kernel tiles.  Each generates
// RPC = BN / CL of the stripe's mask rows and copies them into its peers' shared
// memory (distributed shared memory, one bulk copy per peer and stage).  Its 8
// generator warps form CL phases of 8 / CL warps; phase p generates the stages of
// the CTA's global K blocks G with G % CL == p, so CL stages are in flight at once
// and each warp has CL stage times for its rows.
template <int CL, bool CX, bool LD = false>
__global__ void __launch_bounds__(NUM_THREADS, 1) k_dense(const DenseArgs a, const __grid_constant__ CUtensorMap tmC1) {
  // CX: membrane pass (B planes hi and lo per stage, 3 stages); else 4 stages of one B plane.
  // LD (with CX): the B planes come from a loaded FP32 matrix (a.ld_src) instead of the generator.
  constexpr int NST = CX ? STAGES_CX : STAGES;
  constexpr int BST = CX ? 2 * B_BYTES : B_BYTES;
  // Generator phases: CL (phase p produces the blocks G = p mod CL; with NST =
  // CL = 4 it is the only producer of stage p).  A membrane pass has 3 stages,
  // so its 8 generator warps form at most two phases: a stage's producer must
  // not get two laps ahead of its consumer, which a parity wait cannot see.
  constexpr int PH = CX ? (CL < 2 ? CL : 2) : CL;
  // A phase's previous wait proves block G - PH - NST consumed; the parity wait
  // for block G is exact only if block G - 2 NST is, i.e. if NST >= PH.
  static_assert(PH <= NST, "a generator phase could run two laps ahead of the issuer");
  static_assert(CX || !LD, "a loaded operand takes the two-plane (membrane) stage layout");
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = base;                  // NST x 32 KiB
  uint8_t* sB = base + NST * A_BYTES;  // NST x BST
  uint8_t* sE = sB + NST * BST;        // EPI_BYTES: epilogue staging (1024-aligned)
  uint64_t* bars = reinterpret_cast<uint64_t*>(sE + EPI_BYTES);
  uint64_t* fullA = bars;
  uint64_t* fullB = bars + NST;
  uint64_t* empty = bars + 2 * NST;
  uint64_t* accFull = bars + 3 * NST;
  uint64_t* accEmpty = accFull + 1;
  uint64_t* drain = accEmpty + 1;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(drain + 1);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 2);
  // common continue/abort decisions, double-buffered by block (or chunk) parity:
  // gen_ok[2 * phase + parity] for each generator phase, epi_ok[parity] for the epilogue
  volatile int* gen_ok = reinterpret_cast<volatile int*>(drain + 3);
  volatile int* epi_ok = gen_ok + 2 * 4;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < NST; ++s) {
      mbar_init(&fullA[s], 1);
      // mask rows: the 8 / CL local warps of the stage's phase, plus (CL > 1) the
      // expect-tx arrival for the rows the peers' bulk copies deliver
      mbar_init(&fullB[s], CL > 1 ? GEN_WARPS / PH + 1 : GEN_WARPS);
      mbar_init(&empty[s], CL);  // MMA completion of every CTA that reads rows this CTA writes
    }
    mbar_init(accFull, 1);
    mbar_init(accEmpty, EPI_WARPS);
    mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == MMA_WARP) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t rk = CL > 1 ? cluster_rank() : 0u;
  if (CL > 1) cluster_sync();  // peers' barriers are initialised before any remote arrive

  const int npg = a.npairs / CL;                           // pair groups per stripe
  const int64_t n_items = __ldg(a.sched + a.nchunks);     // units of the work list
  const int64_t u0 = blockIdx.x / CL, ustep = gridDim.x / CL;
  const int64_t nkb = a.kblocks;
  const uint32_t a_bytes = a.hi_only ? A_BYTES / 2 : A_BYTES;

  if (warp == LOAD_WARP) {
    // ---------------- A loader: one bulk copy of 32 KiB (16 KiB hi only) per stage
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      int last[STAGES];
#pragma unroll
      for (int s2 = 0; s2 < STAGES; ++s2) last[s2] = -1;
      for (int64_t it = u0; it < n_items && !*abort_flag; it += ustep) {
        const Unit un = unit_at(a, it, npg);
        const int64_t pr = un.pu * CL + rk;
        const uint8_t* Ap = a.A + pr * nkb * A_BYTES;
        for (int64_t kb = un.kb0; kb < un.kb1; ++kb) {
          if (!(CL > 1 ? mbar_wait_cl(&empty[stage], phase ^ 1, abort_flag, a.err, ERR_TIMEOUT_BASE + 1)
                       : mbar_wait(&empty[stage], phase ^ 1, abort_flag, a.err, ERR_TIMEOUT_BASE + 1)))
            break;
          mbar_arrive_tx(&fullA[stage], a_bytes);
          bulk_g2s(sA + stage * A_BYTES, Ap + kb * A_BYTES, a_bytes, &fullA[stage]);
          last[stage] = (int)phase;
          if (++stage == NST) { stage = 0; phase ^= 1; }
        }
      }
      if (*abort_flag) {
        // copies already issued must land before shared memory is released
#pragma unroll
        for (int s2 = 0; s2 < NST; ++s2) {
          if (last[s2] < 0) continue;
          const uint64_t t0 = gtimer();
          while (!mbar_try(&fullA[s2], (uint32_t)last[s2]) && gtimer() - t0 < WAIT_NS) {
          }
        }
      }
    }
  } else if (warp == MMA_WARP) {
    // ---------------- MMA issuer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0, accph = 0;
      bool ok = true;
      for (int64_t it = u0; it < n_items && ok; it += ustep) {
        const Unit un = unit_at(a, it, npg);
        const int64_t nch = (un.kb1 - un.kb0 + a.promote - 1) / a.promote;
        for (int64_t ch = 0; ch < nch && ok; ++ch) {
          // the epilogue has drained both accumulators of the previous chunk
          if (!mbar_wait(accEmpty, accph ^ 1, abort_flag, a.err, ERR_TIMEOUT_BASE + 2)) { ok = false; break; }
          tc_fence_after();
          const int64_t kb0 = un.kb0 + ch * a.promote, kb1 = kb0 + a.promote < un.kb1 ? kb0 + a.promote : un.kb1;
          for (int64_t kb = kb0; kb < kb1; ++kb) {
            if (!mbar_wait(&fullA[stage], phase, abort_flag, a.err, ERR_TIMEOUT_BASE + 3) ||
                !(CL > 1 ? mbar_wait_cl(&fullB[stage], phase, abort_flag, a.err, ERR_TIMEOUT_BASE + 4)
                         : mbar_wait(&fullB[stage], phase, abort_flag, a.err, ERR_TIMEOUT_BASE + 4))) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint64_t bdesc = sdesc(sB + stage * BST);
            const uint64_t adesc = sdesc(sA + stage * A_BYTES);
#pragma unroll
            for (int ks = 0; ks < BK / 16; ++ks) {
#pragma unroll
              for (int q = 0; q < TILES; ++q) {
                // products (A part h, B plane b): K_hi B_hi, K_lo B_hi and, for a
                // membrane pass, K_hi B_lo
#pragma unroll
                for (int pi = 0; pi < (CX ? 3 : 2); ++pi) {
                  const int h = pi == 1 ? 1 : 0, b = pi == 2 ? 1 : 0;
                  if (pi > 0 && a.hi_only) continue;
                  const uint64_t ad = adesc + (uint64_t)(((h * TILES + q) * SUB + ks * 32) >> 4);
                  const uint64_t bd = bdesc + (uint64_t)((b * B_BYTES + ks * 32) >> 4);
                  mma_bf16(tmem + (uint32_t)(q * BN), ad, bd, (kb > kb0 || ks > 0 || pi > 0) ? 1u : 0u);
                }
              }
            }
            if (CL > 1) mma_commit_mc(&empty[stage], (uint16_t)((1u << CL) - 1u));
            else mma_commit(&empty[stage]);
            if (++stage == NST) { stage = 0; phase ^= 1; }
          }
          if (!ok) break;
          mma_commit(accFull);
          accph ^= 1;
        }
      }
      // all issued MMAs complete before tensor memory is released
      mma_commit(drain);
      const uint64_t t0 = gtimer();
      while (!mbar_try(drain, 0) && gtimer() - t0 < WAIT_NS) {
      }
    }
  } else if (warp >= GEN_WARP0) {
    // ---------------- mask generators
    // RPC rows of the stripe per CTA in RG groups of 32 (a lane per row); a
    // phase's WPS warps cover them, each group split into WPS / RG column parts
    // (one part except for membrane passes)
    constexpr int RPC = BN / CL, WPS = GEN_WARPS / PH, RG = RPC / 32, NCP = WPS / RG;
    const int gw = warp - GEN_WARP0;
    const int ph = gw / WPS, wr = gw % WPS;
    const int cp = wr / RG;                                 // column part: 16-byte chunks [cp, cp + 1) * 4 / NCP
    const int row = (int)rk * RPC + (wr % RG) * 32 + lane;  // row of the stripe, 0 .. BN - 1
    // 64-byte swizzle, K-major: row at (row/8)*512 + (row%8)*64, 16-byte chunk q at q ^ ((row%8)/2)
    uint8_t* rowbase0 = sB + (row >> 3) * 512 + (row & 7) * 64;
    const int sw = (row & 7) >> 1;
    const bool leader = wr == 0 && lane == 0;
    const int64_t my_units = u0 < n_items ? (n_items - u0 + ustep - 1) / ustep : 0;
    int last[STAGES];  // leader: phase of the last peer copy expected on each stage
#pragma unroll
    for (int s2 = 0; s2 < STAGES; ++s2) last[s2] = -1;
    Walker w;
    CxRow cxr{};
    uint32_t state = 0;  // CL = 1: open state of the sequential walk
    int64_t cur_unit = -1;
    // The CTA's K blocks in MMA order: unit ui (its stripe's span [klo, klo +
    // nlen)), block offset t within it; block G of the sequence (G = ph, ph +
    // PH, ...) sits on stage G % NST like the loader's and the issuer's.
    int64_t ui = 0, t = ph, klo = 0, nlen = 1, ustripe = 0;
    auto unit_span = [&](int64_t u) {
      const Unit un = unit_at(a, u0 + u * ustep, npg);
      klo = un.kb0;
      nlen = un.kb1 - un.kb0;
      ustripe = un.s;
    };
    if (my_units > 0) unit_span(0);
    while (ui < my_units && t >= nlen) {
      t -= nlen;
      if (++ui < my_units) unit_span(ui);
    }
    // block-wise generation (clusters, and every phase-plate pass): the next
    // own block's events and thresholds are prepared (its load issued) before
    // the current block is finished
    const bool prefetch = (CL > 1 || a.level_mode) && !LD;
    BlockPrep pre{}, cur{};
    bool have_pre = false;
    for (int64_t G = ph; ui < my_units; G += PH) {
      const int64_t kb = klo + t;
      const int stage = (int)(G % NST);
      const uint32_t phase = (uint32_t)((G / NST) & 1);
      if (ui != cur_unit) {
        cur_unit = ui;
        const int64_t s = ustripe;
        state = 0;
        if constexpr (!LD) walker_init(w, a.j_begin + s * BN + row, a.j_end, a.mg, a.level_mode != 0);
        if constexpr (CX && !LD) cx_row_init(a.df, a.j_begin + s * BN + row - a.mg.c, cxr);
        if constexpr (CL == 1 && !LD) {
          // the sequential walk starts at the unit's first block: skip the
          // events before it; the open state there is their parity
          if (w.ne > 0) {
            const int32_t e = walker_count(w, klo * BK - 1, a.mg);
            w.e = e;
            w.next = walker_event(w, e, a.mg.thr);
            state = (uint32_t)(e & 1);
          }
        }
        have_pre = false;
      }
      if (prefetch) {
        if (!have_pre) block_prep(w, kb * BK, a.mg, pre);
        cur = pre;
        have_pre = t + PH < nlen;
        if (have_pre) block_prep(w, (kb + PH) * BK, a.mg, pre);
      }
      // One thread per phase waits for the stage; the phase's warps take its
      // decision at a named barrier (waiting there issues no instructions).
      const int slot = 2 * ph + (int)(G / PH & 1);
      if (leader)
        gen_ok[slot] = (CL > 1 ? mbar_wait_cl(&empty[stage], phase ^ 1, abort_flag, a.err, ERR_TIMEOUT_BASE + 5)
                               : mbar_wait(&empty[stage], phase ^ 1, abort_flag, a.err, ERR_TIMEOUT_BASE + 5))
                            ? 1
                            : 0;
      named_bar_sync(1 + ph, WPS * 32);
      if (!gen_ok[slot]) break;
      uint8_t* rowp = rowbase0 + stage * BST;
      uint32_t wd[16];
      if constexpr (LD) {
        // loaded operand: row j of the source, this block's columns
        const int64_t j = a.j_begin + ustripe * BN + row;
        ld_store(j < a.j_end ? a.ld_src + j * a.ld_stride + kb * BK : nullptr, rowp, rowp + B_BYTES, sw,
                 cp * (4 / NCP), 4 / NCP);
      } else if constexpr (CX) {
        // membrane pass: T cos(phi) or T sin(phi), hi and lo planes
        uint32_t bits = CL == 1 ? walker_bits(w, kb * BK, state, a.mg.thr) : block_finish(w, kb * BK, a.mg, cur);
        if (a.mg.centre_open) bits = disc_bits(w, kb * BK) & ~bits;
        cx_store(a.df, cxr, kb * BK - a.mg.c, bits, a.cx_sin, rowp, rowp + B_BYTES, sw, cp * (4 / NCP), 4 / NCP);
      } else if (a.level_mode) {
        // phase-plate pass: +1 / -1 on the pass's level sets
        uint32_t pb, nb;
        block_values(w, kb * BK, a.mg, cur, a.lmod, a.pos, a.neg, pb, nb);
        expand_signed(pb | nb, nb, wd);
      } else {
        // one CTA, consecutive blocks: walk the row; clusters: each phase takes
        // every CL-th block, found directly
        const uint32_t bits = CL == 1 ? walker_bits(w, kb * BK, state, a.mg.thr) : block_finish(w, kb * BK, a.mg, cur);
        if (a.signed_mask) expand_signed(disc_bits(w, kb * BK), bits, wd);
        else expand_bits(bits, wd);
      }
      if constexpr (!CX) {
#pragma unroll
        for (int q = 0; q < 4; ++q)
          *reinterpret_cast<uint4*>(rowp + ((q ^ sw) << 4)) =
              make_uint4(wd[4 * q], wd[4 * q + 1], wd[4 * q + 2], wd[4 * q + 3]);
      }
      fence_proxy_async();
      if constexpr (CL == 1) {
        __syncwarp();
        if (lane == 0) mbar_arrive(&fullB[stage]);
      } else {
        // all of this CTA's rows of the stage are written: one thread sends them
        named_bar_sync(1 + ph, WPS * 32);
        if (leader) {
          constexpr int NPL = CX ? 2 : 1;  // B planes per stage
          const uint32_t off = (uint32_t)(stage * BST + rk * RPC * 64);
          mbar_arrive_tx(&fullB[stage], (uint32_t)((CL - 1) * RPC * 64 * NPL));  // the peers' rows land here
#pragma unroll
          for (int q = 1; q < CL; ++q) {
            const uint32_t peer = (rk + (uint32_t)q) % (uint32_t)CL;
#pragma unroll
            for (int pl = 0; pl < NPL; ++pl)
              bulk_s2peer(mapa(smem_u32(sB + off + pl * B_BYTES), peer), sB + off + pl * B_BYTES,
                          (uint32_t)(RPC * 64), mapa(smem_u32(&fullB[stage]), peer));
          }
          last[stage] = (int)phase;
        }
        if (lane == 0) mbar_arrive(&fullB[stage]);
      }
      t += PH;
      while (ui < my_units && t >= nlen) {
        t -= nlen;
        if (++ui < my_units) unit_span(ui);
      }
    }
    if constexpr (CL > 1) {
      if (leader && *abort_flag) {
        // after an abort the peers' copies already issued must land before this
        // CTA's shared memory is released (bounded: a peer may have stopped first)
#pragma unroll
        for (int s2 = 0; s2 < NST; ++s2) {
          if (last[s2] < 0) continue;
          const uint64_t t0 = gtimer();
          while (!mbar_try_cl(&fullB[s2], (uint32_t)last[s2]) && gtimer() - t0 < WAIT_NS) {
          }
        }
      }
    }
  } else {
    // ---------------- epilogue: warp w drains tile w/4, TMEM lanes 32(w%4)..+31.
    // Each 32 x 32 piece goes registers -> shared memory (128-byte swizzle) ->
    // one TMA reduce-add into C1 (in L2), once per promotion of the unit.
    const int q = warp >> 2;
    uint8_t* eb = sE + warp * (EPI_BOX * EPI_BOX * 4);
    uint32_t accph = 0;
    bool ok = true;
    for (int64_t it = u0; it < n_items && ok; it += ustep) {
      const Unit un = unit_at(a, it, npg);
      const int64_t pr = un.pu * CL + rk;
      const int64_t s = un.s;
      const int64_t nch = (un.kb1 - un.kb0 + a.promote - 1) / a.promote;
      // zero-padding tiles (64 t >= M) have no rows in C1: nothing is stored
      const bool live = (pr * TILES + q) * 64 < (int64_t)a.M;
      const int x0 = (int)(a.j_begin + s * BN - a.c1_j0);       // C1 column of the stripe's first row
      const int y0 = (int)((pr * TILES + q) * BM + (warp & 3) * 32);  // C1 row of lane 0
      for (int64_t ch = 0; ch < nch && ok; ++ch) {
        // thread 0 waits for the accumulators; the 8 warps meet at a named barrier
        if (threadIdx.x == 0) epi_ok[accph] = mbar_wait(accFull, accph, abort_flag, a.err, ERR_TIMEOUT_BASE + 6) ? 1 : 0;
        named_bar_sync(1 + 4, EPI_WARPS * 32);
        if (!epi_ok[accph]) { ok = false; break; }
        tc_fence_after();
        const uint32_t taddr = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(q * BN);
#pragma unroll 1
        for (int col = 0; col < (live ? BN : 0); col += EPI_BOX) {
          float v[32];
          tmem_ld32(taddr + col, v);
          if (lane == 0) bulk_wait_read0();  // the previous piece has been read out of eb
          __syncwarp();
#pragma unroll
          for (int c4 = 0; c4 < 8; ++c4)
            *reinterpret_cast<float4*>(eb + lane * 128 + ((c4 ^ (lane & 7)) << 4)) =
                make_float4(v[4 * c4], v[4 * c4 + 1], v[4 * c4 + 2], v[4 * c4 + 3]);
          fence_proxy_async();
          __syncwarp();
          if (lane == 0) {
            tma_reduce_add_2d(&tmC1, eb, x0 + col, y0);  // C1 was zeroed before the launch
            bulk_commit();
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(accEmpty);
        accph ^= 1;
      }
    }
    if (lane == 0) bulk_wait0();  // C1 complete before the kernel ends
  }
  tc_fence_before();
  __syncthreads();
  if (warp == MMA_WARP) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
  // no CTA leaves while its peer may still write its shared memory or arrive on
  // its barriers (every wait above is bounded, so both CTAs get here)
  if (CL > 1) cluster_sync();
}

// ---------------------------------------------------------------- kernel table
// Block (pair p, K block kb) = 32 KiB: [tile 2p hi][tile 2p+1 hi][tile 2p lo][tile 2p+1 lo],
// each 128 rows x 32 BF16, K-major, 64-byte swizzle: element (r, k) at byte
//   (r/8)*512 + (r%8)*64 + ((k/8) ^ ((r%8)/2))*16 + (k%8)*2.
// Tile t holds Re K for m = 64t + r (r < 64) and Im K for m = 64t + r - 64 (r >= 64);
// tiles with 64t >= M are zero (padding to an even count).
__global__ void k_build_A(int M, double msh, int64_t N, int64_t kblocks, int npairs, int64_t c, double kappa,
                          double delta, uint8_t* A) {
  const int64_t K = kblocks * BK;
  const int64_t total = (int64_t)npairs * TILES * BM * (K / 8);  // one thread per 8 consecutive k
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += stride) {
    const int64_t k8 = e % (K / 8);
    const int64_t rg = e / (K / 8);  // kernel row over all tiles
    const int t = (int)(rg / BM), r = (int)(rg % BM);
    const int m = t * 64 + (r & 63);
    const bool im = r >= 64;
    const int p = t / TILES, q = t % TILES;
    const int64_t i0 = k8 * 8;
    const int64_t kb = i0 / BK;
    const int k = (int)(i0 % BK);
    uint32_t hw[4], lw[4];
#pragma unroll
    for (int u = 0; u < 8; u += 2) {
      float v2[2];
#pragma unroll
      for (int z = 0; z < 2; ++z) {
        const int64_t i = i0 + u + z;
        float v = 0.f;
        if (i < N && m < M) {
          const double di = (double)(i - c);
          const double th = di * di * (0.5 * kappa) - ((double)m - msh) * di * delta;
          const float2 kk = cis_turns_f(th);
          v = im ? kk.y : kk.x;
        }
        v2[z] = v;
      }
      const __nv_bfloat16 h0 = __float2bfloat16_rn(v2[0]), h1 = __float2bfloat16_rn(v2[1]);
      const __nv_bfloat16 l0 = __float2bfloat16_rn(v2[0] - __bfloat162float(h0));
      const __nv_bfloat16 l1 = __float2bfloat16_rn(v2[1] - __bfloat162float(h1));
      hw[u / 2] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
      lw[u / 2] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
    }
    const int64_t blk = ((int64_t)p * kblocks + kb) * A_BYTES;
    const int off = (r >> 3) * 512 + (r & 7) * 64 + (((k >> 3) ^ ((r & 7) >> 1)) << 4);
    *reinterpret_cast<uint4*>(A + blk + (0 * TILES + q) * SUB + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
    *reinterpret_cast<uint4*>(A + blk + (1 * TILES + q) * SUB + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
  }
}

// What a mask export writes per sample (fzp_aperture_mask of a dense plan).
enum MaskExport {
  EXPORT_BITS = 0,    // binary amplitude plate: 1 on open samples
  EXPORT_SIGNED = 1,  // binary phase plate (L = 2): 1 + zone parity inside the disc, 0 outside
  EXPORT_LEVELS = 2,  // level-mode plate (L >= 4): 1 + q inside the disc, q the level
  EXPORT_EVEN = 3     // positive-centred plate (level mode, L = 2): 1 on level 0
};

// The generator of single-CTA k_dense launches (walker), one row per thread,
// to bytes (EXPORT_BITS or EXPORT_SIGNED).
__global__ void k_mask_rows(MaskGeom mg, int64_t N, int64_t j0, int64_t rows, int mode, uint8_t* out) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += (int64_t)gridDim.x * blockDim.x) {
    Walker w;
    walker_init(w, j0 + r, INT64_MAX, mg);
    uint32_t state = 0;
    for (int64_t i0 = 0; i0 < N; i0 += 32) {
      const uint32_t bits = walker_bits(w, i0, state, mg.thr);
      const uint32_t disc = mode == EXPORT_SIGNED ? disc_bits(w, i0) : 0xFFFFFFFFu;
      for (int k = 0; k < 32 && i0 + k < N; ++k) {
        const uint32_t b = (bits >> k) & 1u;
        out[r * N + i0 + k] = (uint8_t)(((disc >> k) & 1u) ? (mode == EXPORT_SIGNED ? 1u + b : b) : 0u);
      }
    }
  }
}

// The block-wise generators of k_dense (cluster launches, and every
// level-mode pass) to bytes: one warp per 32 consecutive rows, a lane per
// row, as the kernel's generator warps run them.  Bits come from block_finish
// (EXPORT_BITS, EXPORT_SIGNED) or from block_values with the one-level set
// {q} for each level q (EXPORT_LEVELS; EXPORT_EVEN takes q = 0 only).  Every
// loop bound is uniform across the warp, as the warp-wide block functions
// require; lanes past the last row walk an empty row and write nothing.
__global__ void k_mask_blocks(MaskGeom mg, int64_t N, int64_t j0, int64_t rows, int mode, int lmod, uint8_t* out) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const bool level = mode >= EXPORT_LEVELS;
  const int nq = mode == EXPORT_LEVELS ? lmod : 1;
  for (int64_t r0 = warp * 32; r0 < rows; r0 += nwarps * 32) {
    const int64_t r = r0 + lane;
    Walker w;
    walker_init(w, j0 + r, j0 + rows, mg, level);
    for (int64_t i0 = 0; i0 < N; i0 += BK) {
      BlockPrep p;
      block_prep(w, i0, mg, p);
      uint8_t v[32];
#pragma unroll
      for (int k = 0; k < 32; ++k) v[k] = 0;
      if (!level) {
        const uint32_t bits = block_finish(w, i0, mg, p);
        const uint32_t disc = mode == EXPORT_SIGNED ? disc_bits(w, i0) : 0xFFFFFFFFu;
#pragma unroll
        for (int k = 0; k < 32; ++k) {
          const uint32_t b = (bits >> k) & 1u;
          v[k] = (uint8_t)(((disc >> k) & 1u) ? (mode == EXPORT_SIGNED ? 1u + b : b) : 0u);
        }
      } else {
        for (int q = 0; q < nq; ++q) {
          uint32_t P, Q;
          block_values(w, i0, mg, p, lmod, 1ull << q, 0ull, P, Q);
#pragma unroll
          for (int k = 0; k < 32; ++k)
            if ((P >> k) & 1u) v[k] = (uint8_t)(mode == EXPORT_LEVELS ? 1 + q : 1);
        }
      }
      if (r < rows)
        for (int k = 0; k < 32 && i0 + k < N; ++k) out[r * N + i0 + k] = v[k];
    }
  }
}

// Both variants take the same shared memory: 4 x (32 + 16) KiB or 3 x (32 + 32) KiB.
static_assert(STAGES * (A_BYTES + B_BYTES) == STAGES_CX * (A_BYTES + 2 * B_BYTES), "stage layouts");
size_t dense_smem_bytes() { return 1024 + STAGES * (A_BYTES + B_BYTES) + EPI_BYTES + 256; }

// 2-D FP32 tensor map of the row intermediate: x = C1 column (aperture row of
// the chunk), y = kernel row; 32 x 32 boxes with the 128-byte swizzle.
fzp_status c1_tensor_map(const Plan& P, CUtensorMap* tm) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    FZP_CUDA_TRY(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q));
    if (q != cudaDriverEntryPointSuccess || !fn) return set_error(FZP_E_CUDA, "cuTensorMapEncodeTiled unavailable");
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  const cuuint64_t dims[2] = {(cuuint64_t)P.chunk_rows, (cuuint64_t)P.c1_rows};
  const cuuint64_t strides[1] = {(cuuint64_t)P.chunk_rows * 4};
  const cuuint32_t box[2] = {EPI_BOX, EPI_BOX};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = encode(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, P.d_C1, dims, strides, box, estr,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return set_error(FZP_E_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return FZP_OK;
}

}  // namespace

namespace {

// Layout of the dense form's tables for a kernel matrix of `ncols` columns.
fzp_status layout_cols(Plan& P, int64_t ncols, FormSizes* out) {
  Dense& d = P.dn;
  d.kblocks = (ncols + BK - 1) / BK;
  d.ntiles = 2 * P.M / BM;
  const int used = (d.ntiles + TILES - 1) / TILES;  // tile pairs holding ROI rows
  // cluster: CTAs sharing each stripe's mask (default: the largest of 4, 2, 1
  // that divides the pairs); pairs padded with zero tiles to a multiple of it
  d.cluster = P.cluster_req > 0 ? P.cluster_req : (used % 4 == 0 ? 4 : used % 2 == 0 ? 2 : 1);
  d.npairs = (used + d.cluster - 1) / d.cluster * d.cluster;
  d.promote_kblocks = P.promote_req > 0 ? P.promote_req : 128;  // 4096 samples per TMEM chunk
  // one promotion per unit: units of several promotions of one stripe
  // (measured with 4) kept C1's DRAM writes the same and, the clusters of a
  // wave drifting apart along K, read the kernel matrix 2.7 times as often
  d.group_kblocks = d.promote_kblocks;
  int dev = 0;
  FZP_CUDA_TRY(cudaGetDevice(&dev));
  FZP_CUDA_TRY(cudaDeviceGetAttribute(&d.num_sms, cudaDevAttrMultiProcessorCount, dev));
  out->A = (size_t)d.npairs * (size_t)d.kblocks * A_BYTES;
  out->sched = sizeof(int) * (size_t)(3 * ((d.kblocks + d.group_kblocks - 1) / d.group_kblocks) + 1);
  static std::atomic<uint64_t> attr1{0}, attr2{0}, attr4{0}, attr1c{0}, attr2c{0}, attr4c{0}, attr1l{0},
      attr2l{0}, attr4l{0};
  FZP_CUDA_TRY(smem_attr_once((const void*)k_dense<1, false>, (int)dense_smem_bytes(), attr1));
  FZP_CUDA_TRY(smem_attr_once((const void*)k_dense<2, false>, (int)dense_smem_bytes(), attr2));
  FZP_CUDA_TRY(smem_attr_once((const void*)k_dense<4, false>, (int)dense_smem_bytes(), attr4));
  FZP_CUDA_TRY(smem_attr_once((const void*)k_dense<1, true>, (int)dense_smem_bytes(), attr1c));
  FZP_CUDA_TRY(smem_attr_once((const void*)k_dense<2, true>, (int)dense_smem_bytes(), attr2c));
  FZP_CUDA_TRY(smem_attr_once((const void*)k_dense<4, true>, (int)dense_smem_bytes(), attr4c));
  FZP_CUDA_TRY(smem_attr_once((const void*)k_dense<1, true, true>, (int)dense_smem_bytes(), attr1l));
  FZP_CUDA_TRY(smem_attr_once((const void*)k_dense<2, true, true>, (int)dense_smem_bytes(), attr2l));
  FZP_CUDA_TRY(smem_attr_once((const void*)k_dense<4, true, true>, (int)dense_smem_bytes(), attr4l));
  // The kernel is persistent: launch only CTAs that are resident at once.  A
  // cluster must fit in one GPC, so with clusters fewer than all SMs may hold one.
  d.max_ctas = d.num_sms;
  if (d.cluster > 1) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(d.num_sms / d.cluster * d.cluster));
    cfg.blockDim = dim3((unsigned)NUM_THREADS);
    cfg.dynamicSmemBytes = dense_smem_bytes();
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)d.cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (d.cluster == 2) FZP_CUDA_TRY(cudaOccupancyMaxActiveClusters(&nclusters, k_dense<2, false>, &cfg));
    else FZP_CUDA_TRY(cudaOccupancyMaxActiveClusters(&nclusters, k_dense<4, false>, &cfg));
    if (nclusters < 1) return set_error(FZP_E_UNSUPPORTED, "no %d-CTA cluster of the dense kernel fits", d.cluster);
    d.max_ctas = std::min(nclusters * d.cluster, d.num_sms / d.cluster * d.cluster);
  }
  d.extra_ctas = d.cluster > 1 ? d.num_sms - d.max_ctas : 0;
  return FZP_OK;
}

// The band of rows for the single-CTA launch on the SMs that hold no whole
// cluster: stripe-aligned, at the end of the row range farther from the axis
// and only where that end reaches the rim (there a row's chord is short and
// crosses few zone boundaries per block, and a single CTA, which generates
// all 256 rows of each of its units alone, keeps `eff` of a cluster CTA's
// rate: 0.64 measured at the rim, 0.51 across the middle of the disc), sized
// to the share of the disc's area the leftover SMs can take.  Sets [b0, b1);
// empty (b0 = b1) when there is no band.
void extra_band(const Plan& P, int64_t j_begin, int64_t j_end, double eff, int64_t& b0, int64_t& b1) {
  const Dense& d = P.dn;
  b0 = b1 = j_end;
  const double R = std::sqrt((double)P.mg.sR);
  auto F = [&](double y) {  // area of the disc below row offset y (continuous)
    y = std::max(-R, std::min(R, y));
    return y * std::sqrt(std::max(0.0, R * R - y * y)) + R * R * std::asin(y / R);
  };
  const double y0 = (double)(j_begin - P.c) - 0.5, y1 = (double)(j_end - P.c) - 0.5;
  const double total = F(y1) - F(y0);
  const bool at_end = std::fabs(y1) >= std::fabs(y0);
  if (!(total > 0) || std::fabs(at_end ? y1 : y0) < 0.95 * R) return;
  const double want = d.extra_ctas * eff / (d.max_ctas + d.extra_ctas * eff) * total;
  double lo = y0, hi = y1;  // the band's inner edge y: its area from the outer end is `want`
  for (int it = 0; it < 60; ++it) {
    const double mid = 0.5 * (lo + hi);
    const double area = at_end ? F(y1) - F(mid) : F(mid) - F(y0);
    if ((area > want) == at_end) lo = mid;
    else hi = mid;
  }
  int64_t jm = (int64_t)std::llround(0.5 * (lo + hi) + 0.5) + P.c;
  jm = j_begin + (jm - j_begin + BN / 2) / BN * BN;  // whole stripes for both launches
  if (jm <= j_begin || jm >= j_end) return;
  if (at_end) b0 = jm;
  else {
    b0 = j_begin;
    b1 = jm;
  }
}

// Memsets C1, builds the work list and launches k_dense over `a` (its rows and
// operand source set): mode 0 generated binary or signed mask, 1 membrane
// pass, 2 loaded operand.  A non-null `name` brackets the launch as the
// plan's dominant kernel.
fzp_status run_dense(Plan& P, DenseArgs& a, int mode, const char* name, cudaStream_t s) {
  const Dense& d = P.dn;
  // binary and phase-plate passes of a single plan also use the SMs left over
  // by the clusters: a single-CTA launch on a second stream takes a band of
  // stripes, both add into C1
  int64_t b0 = a.j_end, b1 = a.j_end;
  if (mode == 0 && d.d_sched2 && d.extra_ctas > 0) extra_band(P, a.j_begin, a.j_end, 0.62, b0, b1);
  const int CL = d.cluster;
  a.npairs = d.npairs;
  a.M = P.M;
  a.kblocks = d.kblocks;
  a.promote = d.promote_kblocks;
  a.group = d.group_kblocks;
  a.A = reinterpret_cast<const uint8_t*>(d.d_A);
  a.C1 = P.d_C1;
  a.c1_stride = P.chunk_rows;
  a.c1_j0 = a.j_begin;
  a.err = P.d_err;
  a.nchunks = (int)((d.kblocks + d.group_kblocks - 1) / d.group_kblocks);
  a.sched = d.d_sched;
  const bool split = b0 < b1;
  DenseArgs b = a;  // the band [b0, b1) of the single-CTA launch (same C1 columns)
  b.j_begin = b0;
  b.j_end = b1;
  b.n_stripes = (b1 - b0 + BN - 1) / BN;
  b.sched = d.d_sched2;
  if (split) {
    if (b0 == a.j_begin) a.j_begin = b1;
    else a.j_end = b0;
    a.n_stripes = (a.j_end - a.j_begin + BN - 1) / BN;
  }
  // every unit adds its promotion into C1 (units of one stripe run in any order)
  FZP_CUDA_TRY(cudaMemsetAsync(P.d_C1, 0, (size_t)P.c1_rows * (size_t)P.chunk_rows * sizeof(float), s));
  k_dense_sched<<<1, 1024, 0, s>>>(a, a.npairs / CL, d.d_sched);
  P.launches += 1;
  FZP_CUDA_TRY(cudaGetLastError());
  // the band's stream starts after the main work list is built (C1 zeroed),
  // so the cluster launch is ready first and its clusters are placed first
  if (split) FZP_CUDA_TRY(cudaEventRecord(d.ev_fork, s));
  // a grid of every resident cluster (the work list's length is known on the device only)
  const int grid = d.max_ctas;
  CUtensorMap tm;
  {
    const fzp_status st = c1_tensor_map(P, &tm);
    if (st != FZP_OK) return st;
  }
  if (name) {
    P.dominant = split ? "k_dense clusters + single-CTA band" : name;
    prof_begin(P, s);
  }
  if (CL > 1) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)NUM_THREADS);
    cfg.dynamicSmemBytes = dense_smem_bytes();
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (mode == 2) {
      if (CL == 2) FZP_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_dense<2, true, true>, a, tm));
      else FZP_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_dense<4, true, true>, a, tm));
    } else if (mode == 1) {
      if (CL == 2) FZP_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_dense<2, true>, a, tm));
      else FZP_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_dense<4, true>, a, tm));
    } else {
      if (CL == 2) FZP_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_dense<2, false>, a, tm));
      else FZP_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_dense<4, false>, a, tm));
    }
  } else if (mode == 2) {
    k_dense<1, true, true><<<grid, NUM_THREADS, dense_smem_bytes(), s>>>(a, tm);
  } else if (mode == 1) {
    k_dense<1, true><<<grid, NUM_THREADS, dense_smem_bytes(), s>>>(a, tm);
  } else {
    k_dense<1, false><<<grid, NUM_THREADS, dense_smem_bytes(), s>>>(a, tm);
  }
  if (split) {
    // the band on the leftover SMs; joined before the launch's end is read
    FZP_CUDA_TRY(cudaStreamWaitEvent(d.s2, d.ev_fork, 0));
    k_dense_sched<<<1, 1024, 0, d.s2>>>(b, b.npairs, d.d_sched2);
    k_dense<1, false><<<d.extra_ctas, NUM_THREADS, dense_smem_bytes(), d.s2>>>(b, tm);
    FZP_CUDA_TRY(cudaEventRecord(d.ev_join, d.s2));
    FZP_CUDA_TRY(cudaStreamWaitEvent(s, d.ev_join, 0));
    P.launches += 2;
  }
  if (name) prof_end(P, s);
  P.launches += 1;
  FZP_CUDA_TRY(cudaGetLastError());
  return FZP_OK;
}

}  // namespace

fzp_status dense_layout(Plan& P, FormSizes* out) { return layout_cols(P, P.N, out); }

fzp_status dense_fill_tables(Plan& P, cudaStream_t s) {
  Dense& d = P.dn;
  k_build_A<<<8 * d.num_sms, 256, 0, s>>>(P.M, P.msh, P.N, d.kblocks, d.npairs, P.c, P.kappa, P.delta,
                                          reinterpret_cast<uint8_t*>(d.d_A));
  P.launches += 1;
  FZP_CUDA_TRY(cudaGetLastError());
  return FZP_OK;
}

fzp_status dense_zoom_build(Plan& P, int64_t ncols, int64_t c, double kappa, double delta) {
  FormSizes z;
  fzp_status st = layout_cols(P, ncols, &z);
  if (st != FZP_OK) return st;
  Dense& d = P.dn;
  FZP_CUDA_TRY(cudaMalloc(&d.d_A, z.A));
  FZP_CUDA_TRY(cudaMalloc(&d.d_sched, z.sched));
  P.device_bytes += z.A + z.sched;
  k_build_A<<<8 * d.num_sms, 256>>>(P.M, P.msh, ncols, d.kblocks, d.npairs, c, kappa, delta,
                                    reinterpret_cast<uint8_t*>(d.d_A));
  P.launches += 1;
  FZP_CUDA_TRY(cudaGetLastError());
  return FZP_OK;
}

fzp_status dense_zoom_rows(Plan& P, const float* src, int64_t rows, int64_t stride, cudaStream_t s) {
  DenseArgs a{};
  a.mg = P.mg;
  a.N = P.dn.kblocks * BK;
  a.j_begin = 0;
  a.j_end = rows;
  a.n_stripes = (rows + BN - 1) / BN;
  a.ld_src = src;
  a.ld_stride = stride;
  return run_dense(P, a, 2, nullptr, s);
}

fzp_status dense_build_tables(Plan& P) {
  FormSizes z;
  fzp_status st = dense_layout(P, &z);
  if (st != FZP_OK) return st;
  FZP_CUDA_TRY(cudaMalloc(&P.dn.d_A, z.A));
  FZP_CUDA_TRY(cudaMalloc(&P.dn.d_sched, z.sched));
  P.device_bytes += z.A + z.sched;
  if (P.dn.extra_ctas > 0) {
    FZP_CUDA_TRY(cudaMalloc(&P.dn.d_sched2, z.sched));
    FZP_CUDA_TRY(cudaStreamCreateWithFlags(&P.dn.s2, cudaStreamNonBlocking));
    FZP_CUDA_TRY(cudaEventCreateWithFlags(&P.dn.ev_fork, cudaEventDisableTiming));
    FZP_CUDA_TRY(cudaEventCreateWithFlags(&P.dn.ev_join, cudaEventDisableTiming));
    P.device_bytes += z.sched;
  }
  return dense_fill_tables(P, 0);
}

// Export through the generator that the plan's row pass runs: the level
// mode for plates with passes (L >= 4, positive-centred), the block-wise
// generator for cluster launches, the walker for single-CTA launches.
fzp_status dense_mask(Plan& P, int64_t j0, int64_t rows, uint8_t* out, cudaStream_t s) {
  const bool level = !P.passes.empty();
  const int mode = level ? (P.mg.centre_open ? EXPORT_EVEN : EXPORT_LEVELS)
                         : (P.levels == 2 ? EXPORT_SIGNED : EXPORT_BITS);
  if (level || P.dn.cluster > 1) {
    const int64_t warps = (rows + 31) / 32;
    const unsigned grid = (unsigned)std::min<int64_t>((warps + 3) / 4, 65535);
    k_mask_blocks<<<grid, 128, 0, s>>>(P.mg, P.N, j0, rows, mode, P.levels > 0 ? P.levels : 2, out);
  } else {
    k_mask_rows<<<(unsigned)((rows + 127) / 128), 128, 0, s>>>(P.mg, P.N, j0, rows, mode, out);
  }
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
  a.signed_mask = P.levels == 2 ? 1 : 0;
  const bool cx = P.pass_index >= 0 && P.passes[P.pass_index].cx >= 0;
  a.level_mode = P.pass_index >= 0 && !cx ? 1 : 0;
  a.lmod = P.levels > 0 ? P.levels : 2;
  if (P.pass_index >= 0 && !cx) {
    a.pos = P.passes[P.pass_index].pos;
    a.neg = P.passes[P.pass_index].neg;
  }
  if (cx) {
    a.cx_sin = P.passes[P.pass_index].cx;
    a.df = deform_coef(P);
  }
  a.hi_only = P.precision == FZP_PREC_BF16 ? 1 : 0;
  return run_dense(P, a, cx ? 1 : 0, "dense_tcgen05", s);
}

}  // namespace fzp
