// colpass_tc.cu -- the column pass of the dense form on the tensor cores.
//
//   Uacc[n, m] += sum_j K[n, j] C[j, m]      (Fig. 2 Stage 3, column CZT as a
//                                            dense product; K is the separable
//                                            kernel of Eq. 2, C the row output)
//
// The real and imaginary parts are concatenated along K so that every output
// lives in one tensor-memory lane:
//   D1[m, c] = sum_j Cr[j, m] B[c, j],   D2[m, c] = sum_j Ci[j, m] B[c, j],
// with B the kernel-matrix images the row pass already holds: a tile pair's 256
// rows are Re K and Im K for 128 values of n (rows 128 q + r: Re K[n], rows
// 128 q + 64 + r: Im K[n], n = 128 p + 64 q + r).  Then
//   Re U[n, m] = D1[m, cRe(n)] - D2[m, cIm(n)],  Im U[n, m] = D2[m, cRe(n)] + D1[m, cIm(n)].
// C (FP32) is split per element into BF16 hi + lo and K is stored split, so
// each accumulator takes Chi Khi + Chi Klo + Clo Khi (the dropped Clo Klo is
// ~2^-18 of the product).  Tensor memory holds FP32 sums of at most 128 K
// blocks (4096 rows); they are promoted into the FP64 ROI accumulator.
//
// Work units: (m tile of 128, n tile of 128 = one tile pair, K slice); one CTA
// per SM, persistent.  Warps 0-3 epilogue, 4-7 split C1 into the A images,
// 8 bulk-copies the kernel block, 9 issues tcgen05.mma (M128 N256 K16).
#include <cuda_bf16.h>

#include <algorithm>

#include "fzp_internal.cuh"
#include "tc_ptx.cuh"

namespace fzp {
namespace {
using namespace tc;

constexpr int TBM = 128;                 // m per unit (MMA M)
constexpr int TBN = 256;                 // B rows: one kernel tile pair
constexpr int TBK = 32;                  // K (aperture rows j) per stage
constexpr int TSTAGES = 3;
constexpr int TSUB = 128 * TBK * 2;      // 8 KiB: one 128 x 32 BF16 image
constexpr int TA_BYTES = 4 * TSUB;       // [Cr hi][Cr lo][Ci hi][Ci lo]
constexpr int TB_BYTES = 4 * TSUB;       // [t0 hi][t1 hi][t0 lo][t1 lo] (as stored)
constexpr int T_EPI_WARPS = 4, T_PROD_WARP0 = 4, T_LOAD_WARP = 8, T_MMA_WARP = 9;
constexpr int T_THREADS = 10 * 32;
// K blocks per tensor-memory chunk: the FP32 accumulator's error grows with
// the chunk's length (a whole 0.25 m aperture: 4.2e-5 relative L2 of I with
// 4096-row chunks), and the column pass is a small part of a step, so its
// chunks are short
constexpr int T_PROMOTE = 32;
constexpr int T_TMEM_COLS = 512;         // D1 at columns 0-255, D2 at 256-511
constexpr int T_ERR_BASE = 200;

// K-major, 64-byte swizzle (rows of 64 B, 8-row groups 512 B apart), version 1.
__device__ __forceinline__ uint64_t sdesc64(const void* p) {
  const uint64_t a = smem_u32(p);
  return ((a >> 4) & 0x3FFFull) | (1ull << 16) | ((uint64_t)(512 >> 4) << 32) | (1ull << 46) | (4ull << 61);
}
// kind::f16, D = F32, A = B = BF16, K-major, N = 256, M = 128.
constexpr uint32_t T_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TBN >> 3) << 17) | ((uint32_t)(TBM >> 4) << 24);

__device__ __forceinline__ void mma(uint32_t dtmem, uint64_t ad, uint64_t bd, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(
          dtmem),
      "l"(ad), "l"(bd), "r"(T_IDESC), "r"(accumulate)
      : "memory");
}

struct ColTcArgs {
  const float* C1;          // [kernel row][c1_stride], column = j - j0
  int64_t c1_stride;
  int64_t j0, rows;         // aperture rows of this chunk
  const uint8_t* A;         // kernel-matrix images [pair][kb] (32 KiB each)
  int64_t kblocks;          // K blocks per pair in the table (ceil(N / 32))
  int M, tiles;             // tiles per side: M / 128
  int64_t kb_lo, nkb;       // table K blocks covering [j0, j0 + rows)
  int slices;               // K slices per output tile
  double2* Uacc;            // [n][m]
  double wr, wi;            // weight of this pass's field (1, 0 for a single-pass plate)
  int* err;
};

// Split x into BF16 hi + lo (round to nearest), two samples per 32-bit word.
__device__ __forceinline__ void split2(float a, float b, uint32_t& hi, uint32_t& lo) {
  const __nv_bfloat16 ah = __float2bfloat16_rn(a), bh = __float2bfloat16_rn(b);
  const __nv_bfloat16 al = __float2bfloat16_rn(a - __bfloat162float(ah));
  const __nv_bfloat16 bl = __float2bfloat16_rn(b - __bfloat162float(bh));
  hi = (uint32_t)__bfloat16_as_ushort(ah) | ((uint32_t)__bfloat16_as_ushort(bh) << 16);
  lo = (uint32_t)__bfloat16_as_ushort(al) | ((uint32_t)__bfloat16_as_ushort(bl) << 16);
}

// 32 consecutive C1 values of kernel row `r`, columns jj0 .. jj0 + 31 (zero
// outside [0, rows)), into the hi and lo images' row t.
__device__ __forceinline__ void load_split_row(const ColTcArgs& a, int r, int64_t jj0, uint8_t* hi_img, uint8_t* lo_img,
                                               int t) {
  float v[32];
  const float* src = a.C1 + (int64_t)r * a.c1_stride + jj0;
  if (jj0 >= 0 && jj0 + 32 <= a.rows && ((reinterpret_cast<uintptr_t>(src) & 15) == 0)) {
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const float4 x = __ldg(reinterpret_cast<const float4*>(src) + q);
      v[4 * q] = x.x; v[4 * q + 1] = x.y; v[4 * q + 2] = x.z; v[4 * q + 3] = x.w;
    }
  } else {
#pragma unroll
    for (int k = 0; k < 32; ++k) {
      const int64_t jj = jj0 + k;
      v[k] = (jj >= 0 && jj < a.rows) ? __ldg(src + k) : 0.0f;
    }
  }
  const int sw = (t & 7) >> 1;
  uint8_t* hrow = hi_img + (t >> 3) * 512 + (t & 7) * 64;
  uint8_t* lrow = lo_img + (t >> 3) * 512 + (t & 7) * 64;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) split2(v[8 * q + 2 * k], v[8 * q + 2 * k + 1], h[k], l[k]);
    *reinterpret_cast<uint4*>(hrow + ((q ^ sw) << 4)) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4*>(lrow + ((q ^ sw) << 4)) = make_uint4(l[0], l[1], l[2], l[3]);
  }
}

__global__ void __launch_bounds__(T_THREADS, 1) k_colpass_tc(const ColTcArgs a) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = base;                       // TSTAGES x 32 KiB
  uint8_t* sB = base + TSTAGES * TA_BYTES;  // TSTAGES x 32 KiB
  uint64_t* bars = reinterpret_cast<uint64_t*>(sB + TSTAGES * TB_BYTES);
  uint64_t* fullA = bars;
  uint64_t* fullB = bars + TSTAGES;
  uint64_t* empty = bars + 2 * TSTAGES;
  uint64_t* accFull = bars + 3 * TSTAGES;
  uint64_t* accEmpty = accFull + 1;
  uint64_t* drain = accEmpty + 1;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(drain + 1);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 2);
  volatile int* epi_ok = reinterpret_cast<volatile int*>(drain + 3);  // [2], by chunk parity

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < TSTAGES; ++s) {
      mbar_init(&fullA[s], 4);  // the four producer warps
      mbar_init(&fullB[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(accFull, 1);
    mbar_init(accEmpty, T_EPI_WARPS);
    mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == T_MMA_WARP) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(T_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  const int64_t n_units = (int64_t)a.tiles * a.tiles * a.slices;
  const int64_t u0 = blockIdx.x, ustep = gridDim.x;
  // K blocks [kbs, kbe) of unit u
  auto unit_range = [&](int64_t u, int64_t& kbs, int64_t& kbe, int& mt, int& nt) {
    const int64_t tile = u / a.slices, sl = u % a.slices;
    mt = (int)(tile / a.tiles);
    nt = (int)(tile % a.tiles);
    kbs = a.kb_lo + a.nkb * sl / a.slices;
    kbe = a.kb_lo + a.nkb * (sl + 1) / a.slices;
  };

  if (warp == T_LOAD_WARP) {
    // ---------------- kernel-matrix block of the unit's tile pair: one bulk copy per stage
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      int last[TSTAGES];
#pragma unroll
      for (int s2 = 0; s2 < TSTAGES; ++s2) last[s2] = -1;
      bool ok = true;
      for (int64_t u = u0; u < n_units && ok; u += ustep) {
        int64_t kbs, kbe;
        int mt, nt;
        unit_range(u, kbs, kbe, mt, nt);
        for (int64_t kb = kbs; kb < kbe; ++kb) {
          if (!mbar_wait(&empty[stage], phase ^ 1, abort_flag, a.err, T_ERR_BASE + 1)) { ok = false; break; }
          mbar_arrive_tx(&fullB[stage], TB_BYTES);
          bulk_g2s(sB + stage * TB_BYTES, a.A + ((int64_t)nt * a.kblocks + kb) * TB_BYTES, TB_BYTES, &fullB[stage]);
          last[stage] = (int)phase;
          if (++stage == TSTAGES) { stage = 0; phase ^= 1; }
        }
      }
      if (*abort_flag) {
#pragma unroll
        for (int s2 = 0; s2 < TSTAGES; ++s2) {
          if (last[s2] < 0) continue;
          const uint64_t t0 = gtimer();
          while (!mbar_try(&fullB[s2], (uint32_t)last[s2]) && gtimer() - t0 < WAIT_NS) {
          }
        }
      }
    }
  } else if (warp >= T_PROD_WARP0 && warp < T_LOAD_WARP) {
    // ---------------- C1 rows -> BF16 hi / lo images of Cr and Ci
    const int t = (warp - T_PROD_WARP0) * 32 + lane;  // row of the A images: m = 128 mt + t
    int stage = 0;
    uint32_t phase = 0;
    bool ok = true;
    for (int64_t u = u0; u < n_units && ok; u += ustep) {
      int64_t kbs, kbe;
      int mt, nt;
      unit_range(u, kbs, kbe, mt, nt);
      const int m = 128 * mt + t;
      for (int64_t kb = kbs; kb < kbe; ++kb) {
        if (!warp_wait(&empty[stage], phase ^ 1, abort_flag, a.err, T_ERR_BASE + 2)) { ok = false; break; }
        uint8_t* img = sA + stage * TA_BYTES;
        const int64_t jj0 = kb * TBK - a.j0;
        load_split_row(a, c1_row_re(m), jj0, img, img + TSUB, t);
        load_split_row(a, c1_row_im(m), jj0, img + 2 * TSUB, img + 3 * TSUB, t);
        fence_proxy_async();
        __syncwarp();
        if (lane == 0) mbar_arrive(&fullA[stage]);
        if (++stage == TSTAGES) { stage = 0; phase ^= 1; }
      }
    }
  } else if (warp == T_MMA_WARP) {
    // ---------------- MMA issuer: D1 += Cr B, D2 += Ci B, three split products each
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0, accph = 0;
      bool ok = true;
      for (int64_t u = u0; u < n_units && ok; u += ustep) {
        int64_t kbs, kbe;
        int mt, nt;
        unit_range(u, kbs, kbe, mt, nt);
        for (int64_t c0 = kbs; c0 < kbe && ok; c0 += T_PROMOTE) {
          const int64_t c1 = c0 + T_PROMOTE < kbe ? c0 + T_PROMOTE : kbe;
          if (!mbar_wait(accEmpty, accph ^ 1, abort_flag, a.err, T_ERR_BASE + 3)) { ok = false; break; }
          tc_fence_after();
          for (int64_t kb = c0; kb < c1; ++kb) {
            if (!mbar_wait(&fullA[stage], phase, abort_flag, a.err, T_ERR_BASE + 4) ||
                !mbar_wait(&fullB[stage], phase, abort_flag, a.err, T_ERR_BASE + 5)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint64_t ad = sdesc64(sA + stage * TA_BYTES), bd = sdesc64(sB + stage * TB_BYTES);
#pragma unroll
            for (int ks = 0; ks < TBK / 16; ++ks) {
              const uint64_t o = (uint64_t)((ks * 32) >> 4);
              const uint64_t b_hi = bd + o, b_lo = bd + (uint64_t)((2 * TSUB) >> 4) + o;
              const uint64_t cr_hi = ad + o, cr_lo = ad + (uint64_t)(TSUB >> 4) + o;
              const uint64_t ci_hi = ad + (uint64_t)((2 * TSUB) >> 4) + o, ci_lo = ad + (uint64_t)((3 * TSUB) >> 4) + o;
              const uint32_t acc = (kb > c0 || ks > 0) ? 1u : 0u;
              mma(tmem, cr_hi, b_hi, acc);
              mma(tmem, cr_hi, b_lo, 1u);
              mma(tmem, cr_lo, b_hi, 1u);
              mma(tmem + 256u, ci_hi, b_hi, acc);
              mma(tmem + 256u, ci_hi, b_lo, 1u);
              mma(tmem + 256u, ci_lo, b_hi, 1u);
            }
            mma_commit(&empty[stage]);
            if (++stage == TSTAGES) { stage = 0; phase ^= 1; }
          }
          if (!ok) break;
          mma_commit(accFull);
          accph ^= 1;
        }
      }
      mma_commit(drain);
      const uint64_t t0 = gtimer();
      while (!mbar_try(drain, 0) && gtimer() - t0 < WAIT_NS) {
      }
    }
  } else {
    // ---------------- epilogue: warp w holds m = 128 mt + 32 w + lane (TMEM lanes 32 w ..)
    uint32_t accph = 0;
    bool ok = true;
    for (int64_t u = u0; u < n_units && ok; u += ustep) {
      int64_t kbs, kbe;
      int mt, nt;
      unit_range(u, kbs, kbe, mt, nt);
      const int m = 128 * mt + 32 * warp + lane;
      for (int64_t c0 = kbs; c0 < kbe; c0 += T_PROMOTE) {
        if (threadIdx.x == 0) epi_ok[accph] = mbar_wait(accFull, accph, abort_flag, a.err, T_ERR_BASE + 6) ? 1 : 0;
        named_bar_sync(1, T_EPI_WARPS * 32);
        if (!epi_ok[accph]) { ok = false; break; }
        tc_fence_after();
        const uint32_t tl = tmem + ((uint32_t)(32 * warp) << 16);
#pragma unroll 1
        for (int q = 0; q < 2; ++q) {
#pragma unroll 1
          for (int r0 = 0; r0 < 64; r0 += 32) {
            const uint32_t cre = (uint32_t)(128 * q + r0), cim = cre + 64u;
            const int n0 = 128 * nt + 64 * q + r0;
            float x[32], y[32];
            // U += (wr + i wi)(Re + i Im): Re feeds x with wr and y with wi,
            // Im feeds x with -wi and y with wr (zero weights are skipped)
            tmem_ld32(tl + cre, x);         // D1 at Re K columns
            tmem_ld32(tl + 256u + cim, y);  // D2 at Im K columns
            if (m < a.M) {
#pragma unroll
              for (int k = 0; k < 32; ++k)
                if (n0 + k < a.M) {
                  const double re = (double)(x[k] - y[k]);
                  double2* u = &a.Uacc[(int64_t)(n0 + k) * a.M + m];
                  if (a.wr != 0.0) atomicAdd(&u->x, a.wr * re);
                  if (a.wi != 0.0) atomicAdd(&u->y, a.wi * re);
                }
            }
            tmem_ld32(tl + 256u + cre, x);  // D2 at Re K columns
            tmem_ld32(tl + cim, y);         // D1 at Im K columns
            if (m < a.M) {
#pragma unroll
              for (int k = 0; k < 32; ++k)
                if (n0 + k < a.M) {
                  const double im = (double)(x[k] + y[k]);
                  double2* u = &a.Uacc[(int64_t)(n0 + k) * a.M + m];
                  if (a.wr != 0.0) atomicAdd(&u->y, a.wr * im);
                  if (a.wi != 0.0) atomicAdd(&u->x, -a.wi * im);
                }
            }
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(accEmpty);
        accph ^= 1;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == T_MMA_WARP) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(T_TMEM_COLS) : "memory");
  }
}

size_t colpass_tc_smem() { return 1024 + TSTAGES * (TA_BYTES + TB_BYTES) + 256; }

}  // namespace

// Usable for dense plans (the kernel-matrix images exist) with M a multiple of 128.
bool column_pass_tc_applies(const Plan& P) {
  return P.form == FZP_FORM_DENSE && P.dn.d_A != nullptr && (P.M % 128) == 0 && P.precision == FZP_PREC_SPLIT_BF16;
}

fzp_status column_pass_tc(Plan& P, int64_t j0, int64_t rows, cudaStream_t s) {
  return column_pass_tc_w(P, j0, rows, P.pass_index >= 0 ? P.passes[P.pass_index].wr : 1.0,
                          P.pass_index >= 0 ? P.passes[P.pass_index].wi : 0.0, s);
}

fzp_status column_pass_tc_w(Plan& P, int64_t j0, int64_t rows, double wr, double wi, cudaStream_t s) {
  static std::atomic<uint64_t> attr{0};
  FZP_CUDA_TRY(smem_attr_once((const void*)k_colpass_tc, (int)colpass_tc_smem(), attr));
  ColTcArgs a{};
  a.C1 = P.d_C1;
  a.c1_stride = P.chunk_rows;
  a.j0 = j0;
  a.rows = rows;
  a.A = reinterpret_cast<const uint8_t*>(P.dn.d_A);
  a.kblocks = P.dn.kblocks;
  a.M = P.M;
  a.tiles = P.M / 128;
  a.kb_lo = j0 / TBK;
  a.nkb = (j0 + rows + TBK - 1) / TBK - a.kb_lo;
  const int64_t tiles2 = (int64_t)a.tiles * a.tiles;
  // about two units per SM, slices of at least 16 K blocks
  int64_t slices = (2 * (int64_t)P.dn.num_sms + tiles2 - 1) / tiles2;
  slices = std::max<int64_t>(1, std::min<int64_t>(slices, a.nkb / 16));
  a.slices = (int)slices;
  a.Uacc = reinterpret_cast<double2*>(P.d_Uacc);
  a.wr = wr;
  a.wi = wi;
  a.err = P.d_err;
  const int64_t units = tiles2 * slices;
  const int grid = (int)std::min<int64_t>(units, P.dn.num_sms);
  k_colpass_tc<<<grid, T_THREADS, colpass_tc_smem(), s>>>(a);
  P.launches += 1;
  FZP_CUDA_TRY(cudaGetLastError());
  return FZP_OK;
}

}  // namespace fzp
