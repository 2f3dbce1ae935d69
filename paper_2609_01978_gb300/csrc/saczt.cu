// saczt.cu -- the semi-analytical chirp-z transform (SA-CZT, Sec. 3.6, Fig. 5):
// angular-spectrum propagation without the paraxial approximation, for the
// binary amplitude plate with the exact zone radii of Eq. 3 (or the paraxial
// ones, to show their aberration under the exact propagator).
//
//   1  A = FFT2 of the mask on a P x P grid (P a power of two >= 1.5 N, mask
//      centre at P/2; no input chirp)
//   2  A *= exp(i h(K) f), h = k_z - c k_max - d K^2 / k_max, k_z = sqrt(k0^2 - K^2),
//      evanescent components zeroed; the quadratic matches k_z at K = 0 and at
//      K = k_max = 2 k0 / 3 (c = k0 / k_max, d = (sqrt(k0^2 - k_max^2) - k0) / k_max)
//   3-4 U1 = IFFT2(A)
//   5  the quadratic part is the Fresnel propagator of z_F = -2 k0 d f / k_max:
//      U(x, y) = e^{i k0 f} / (i lambda z_F) e^{i k0 (x^2 + y^2) / (2 z_F)} dx^2
//                sum_{u,v} U1(u, v) e^{i k0 (u^2 + v^2) / (2 z_F)} e^{-i k0 (x u + y v) / z_F},
//      evaluated only on the ROI samples (the CZT zoom of Fig. 5, step
//      dx_out / (lambda z_F)) as two complex products with the kernel
//      K[m, u] = e^{i k0 u^2 / (2 z_F) - i k0 x_m u / z_F}: rows, then columns.
//
// GB300 mapping: the 2-D transforms are one block per row (the row in shared
// memory, up to 16384 points = 132 KiB with padding), radix-2 stages fused
// four at a time in registers, forward transforms left in bit-reversed order
// for the inverse ones to read back; three row kernels (mask + forward;
// forward + residual phase + inverse; inverse) and two tiled transposes, so
// the padded grid crosses HBM five times each way.  The zoom (M P^2 and M^2 P complex
// multiply-adds) is a dense contraction with the structure of the dense
// form's: K U1 K^T with the kernel K[m][u] above.  For M a multiple of 128 it
// runs on the tensor cores through the dense form's kernels: the last inverse
// transform writes U1 as two real planes, each plane is the loaded B operand
// of one k_dense row pass (split BF16 hi + lo, three products, FP32 tensor
// memory, C1 by reduce-add) against split-BF16 images of K, and the tensor
// column pass adds K C1^T into the FP64 ROI field with weight 1 (real plane)
// or i (imaginary plane).  Other M take two FP32 complex products on the CUDA
// cores.  The zoom kernel's phases are reduced in FP64 before the FP32
// (co)sines; the residual phase of step 2, once per grid sample, without FP64.
#include <cmath>
#include <vector>

#include "fzp_internal.cuh"

namespace fzp {
namespace {

constexpr int64_t SA_PMAX = 16384;  // rows of the transforms live in shared memory

struct SaMaskArgs {
  MaskGeom mg;  // disc limit, centre, paraxial zone rule, centre configuration
  int64_t N, P, j0, j1;
  int exact;
  const int64_t* xthr;  // exact radii: xthr[m - 1] = smallest s in zone >= m, m = 1 .. nx
  int64_t nx;
  float dx2f, ff, lamf;  // FP32 estimate of the exact zone index
};

// Zone of sample s = dj^2 + di^2 for the exact radii (Eq. 3): the zone index
// is floor(n(r)), n(r) = 2 (sqrt(f^2 + r^2) - f) / lambda, r^2 = s dx^2.  The
// host tabulates, by bisection on the same expression in FP64 written without
// the cancellation (2 r^2 / (lambda (sqrt(f^2 + r^2) + f))), the first s of
// every zone; here an FP32 estimate of n picks the entry and the table
// decides.
__device__ __forceinline__ int64_t zone_exact(const SaMaskArgs& a, int64_t s) {
  const float r2 = (float)s * a.dx2f;
  int64_t m = (int64_t)(2.0f * r2 / (a.lamf * (sqrtf(fmaf(a.ff, a.ff, r2)) + a.ff)));
  m = m < 0 ? 0 : (m > a.nx ? a.nx : m);
  while (m > 0 && __ldg(a.xthr + m - 1) > s) --m;
  while (m < a.nx && __ldg(a.xthr + m) <= s) ++m;
  return m;
}

// Open state of sample (j, i) (dj = j - c, di = i - c) inside the disc: the
// exact radii's zone rule above, or the paraxial radii's exact integer rule.
__device__ __forceinline__ bool sa_open(const SaMaskArgs& a, int64_t dj, int64_t di) {
  const int64_t s = dj * dj + di * di;
  if (s > a.mg.sR) return false;
  const int64_t z = a.exact ? zone_exact(a, s) : zone_of(s, a.mg);
  return ((z ^ a.mg.centre_open) & 1) != 0;
}

// Export of rows [j0, j0 + rows) of the mask (1 open, 0 closed), N per row.
__global__ void k_sa_mask_export(SaMaskArgs a, int64_t rows, uint8_t* __restrict__ out) {
  const int64_t total = rows * a.N;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t / a.N, i = t % a.N;
    out[t] = sa_open(a, a.j0 + r - a.mg.c, i - a.mg.c) ? 1 : 0;
  }
}

// tw[t] = e^{-2 pi i t / P}, t < P / 2, from an FP64 argument.
__global__ void k_sa_twiddles(int64_t P, float2* __restrict__ tw) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < P / 2; t += (int64_t)gridDim.x * blockDim.x) {
    double s, c;
    sincospi(-2.0 * (double)t / (double)P, &s, &c);
    tw[t] = make_float2((float)c, (float)s);
  }
}

__device__ __forceinline__ int sa_brev(int v, int bits) { return (int)(__brev((unsigned)v) >> (32 - bits)); }

// Shared-memory slot of element i of a row: one padding slot per 32 keeps
// the strided group accesses of the late passes within two-way bank
// conflicts.
__device__ __forceinline__ int spad(int i) { return i + (i >> 5); }

// One pass of R radix-2 stages of the decimation-in-frequency transform
// (natural order in, bit-reversed out; twiddles e^{-2 pi i t / P}):
// halves H, H/2, ..., H / 2^(R-1); each thread takes groups of 2^R elements
// at stride sig = H / 2^(R-1) and runs the R stages in registers.
template <int R>
__device__ __forceinline__ void dif_pass(float2* x, int P, int logP, int H, int lgH, const float2* __restrict__ tw) {
  constexpr int NE = 1 << R;
  const int lsig = lgH - (R - 1), sig = 1 << lsig;
  for (int g = threadIdx.x; g < (P >> R); g += blockDim.x) {
    const int k0 = g & (sig - 1);
    const int base = ((g >> lsig) << (lgH + 1)) + k0;
    float2 v[NE];
#pragma unroll
    for (int j = 0; j < NE; ++j) v[j] = x[spad(base + j * sig)];
#pragma unroll
    for (int t = 0; t < R; ++t) {
      const int span = 1 << (R - 1 - t);             // pair distance in j; half = sig * span
      const int tsh = logP - 1 - (lsig + R - 1 - t);  // twiddle step P / (2 half) = 2^tsh
#pragma unroll
      for (int j = 0; j < NE; ++j) {
        if (j & span) continue;
        const float2 u = v[j], w = v[j + span];
        const float2 w2 = tw[(k0 + (j & (span - 1)) * sig) << tsh];
        v[j] = cadd(u, w);
        v[j + span] = cmul(csub(u, w), w2);
      }
    }
#pragma unroll
    for (int j = 0; j < NE; ++j) x[spad(base + j * sig)] = v[j];
  }
}

// One pass of R radix-2 stages of the inverse decimation-in-time transform
// (bit-reversed order in, natural out; twiddles e^{+2 pi i t / P}, no 1/P):
// halves sig, 2 sig, ..., sig 2^(R-1).
template <int R>
__device__ __forceinline__ void dit_inv_pass(float2* x, int P, int logP, int lsig, const float2* __restrict__ tw) {
  constexpr int NE = 1 << R;
  const int sig = 1 << lsig;
  for (int g = threadIdx.x; g < (P >> R); g += blockDim.x) {
    const int k0 = g & (sig - 1);
    const int base = ((g >> lsig) << (lsig + R)) + k0;
    float2 v[NE];
#pragma unroll
    for (int j = 0; j < NE; ++j) v[j] = x[spad(base + j * sig)];
#pragma unroll
    for (int t = 0; t < R; ++t) {
      const int span = 1 << t;               // half = sig * span
      const int tsh = logP - 1 - (lsig + t);  // twiddle step P / (2 half)
#pragma unroll
      for (int j = 0; j < NE; ++j) {
        if (j & span) continue;
        float2 w2 = tw[(k0 + (j & (span - 1)) * sig) << tsh];
        w2.y = -w2.y;
        const float2 u = v[j], b = cmul(v[j + span], w2);
        v[j] = cadd(u, b);
        v[j + span] = csub(u, b);
      }
    }
#pragma unroll
    for (int j = 0; j < NE; ++j) x[spad(base + j * sig)] = v[j];
  }
}

// The row in shared memory, forward (bit-reversed result) or inverse (from
// bit-reversed order), in passes of four stages and one shorter pass.
__device__ __forceinline__ void row_fft_fwd(float2* x, int P, int logP, const float2* __restrict__ tw) {
  for (int done = 0; done < logP;) {
    const int r = logP - done < 4 ? logP - done : 4;
    const int lgH = logP - 1 - done;
    switch (r) {
      case 4: dif_pass<4>(x, P, logP, 1 << lgH, lgH, tw); break;
      case 3: dif_pass<3>(x, P, logP, 1 << lgH, lgH, tw); break;
      case 2: dif_pass<2>(x, P, logP, 1 << lgH, lgH, tw); break;
      default: dif_pass<1>(x, P, logP, 1 << lgH, lgH, tw); break;
    }
    __syncthreads();
    done += r;
  }
}

__device__ __forceinline__ void row_fft_inv(float2* x, int P, int logP, const float2* __restrict__ tw) {
  for (int done = 0; done < logP;) {
    const int r = logP - done < 4 ? logP - done : 4;
    switch (r) {
      case 4: dit_inv_pass<4>(x, P, logP, done, tw); break;
      case 3: dit_inv_pass<3>(x, P, logP, done, tw); break;
      case 2: dit_inv_pass<2>(x, P, logP, done, tw); break;
      default: dit_inv_pass<1>(x, P, logP, done, tw); break;
    }
    __syncthreads();
    done += r;
  }
}

// out[x][y] = in[y][x] for a P x P complex64 matrix (32 x 32 tiles, block 32 x 8).
__global__ void k_sa_transpose(const float2* __restrict__ in, float2* __restrict__ out, int64_t P) {
  __shared__ float2 tile[32][33];
  const int64_t x0 = (int64_t)blockIdx.x * 32, y0 = (int64_t)blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += 8) tile[r][threadIdx.x] = in[(y0 + r) * P + x0 + threadIdx.x];
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += 8) out[(x0 + r) * P + y0 + threadIdx.x] = tile[threadIdx.x][r];
}

// Step 2's phase in turns, h f / (2 pi), for spectrum sample (a, b) with
// signed frequency indices (fa, fb) and s = fa^2 + fb^2 (an exact integer):
// q = K^2 / k0^2 = eps s, eps = (lambda / (P dx))^2, and with z = 1 - sqrt(1 - q)
// (= K^2 / (k0 (k0 + k_z)), no cancellation) and A = f / lambda,
//   h f / (2 pi) = -A z - C s,   C = A (d k0 / k_max) eps.
// It is evaluated without FP64 (FP64 runs at a small fraction of the FP32
// rate here): z as a float-float pair (Dekker's two-sum and two-product with
// a fused multiply-add, one correction of the FP32 square root), A z reduced
// mod 1 in the same pairs, C s mod 1 in 64-bit fixed point.  Absolute error
// about 1e-7 turns where A z is 1e4 turns (checked against FP64 on the host
// in the same single-precision steps).
struct SaPhase {
  float eh, el;    // eps as a float-float pair
  float ah, al;    // A as a float-float pair
  uint64_t cfix;   // |C| 2^64 (|C| < 1)
  int cneg;        // C < 0
  int64_t s_ev;    // smallest s with eps s >= 1: evanescent from there
  float scale;     // 1 / P^2 of the inverse transform
};

// The error-free transforms use the _rn intrinsics, which the compiler never
// contracts into fused multiply-adds.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ float sa_turns(const SaPhase& c, int64_t s) {
  // x = eps s; s < 2^28 splits exactly into two floats, each product exact
  // as a pair (two-product)
  const float sh = (float)(s & ~(int64_t)0xFFF), sl = (float)(s & 0xFFF);
  const float p1 = __fmul_rn(c.eh, sh), p2 = __fmul_rn(c.eh, sl);
  const float e1 = fmaf(c.eh, sh, -p1), e2 = fmaf(c.eh, sl, -p2);
  float xh, xl;
  two_sum(p1, p2, xh, xl);
  xl = fmaf(c.el, __fadd_rn(sh, sl), __fadd_rn(xl, __fadd_rn(e1, e2)));
  fast_two_sum(xh, xl, xh, xl);
  // w = 1 - x, y = sqrt(w) (correctly rounded root, one correction)
  float wh, wl;
  two_sum(1.0f, -xh, wh, wl);
  wl = __fsub_rn(wl, xl);
  fast_two_sum(wh, wl, wh, wl);  // near the evanescent edge xl is not small against wh
  const float y0 = __fsqrt_rn(wh);
  const float y1 = (fmaf(-y0, y0, wh) + wl) * __frcp_rn(y0 + y0);
  // z = 1 - y
  float zh, ze;
  two_sum(1.0f, -y0, zh, ze);
  float zl = __fsub_rn(ze, y1);
  fast_two_sum(zh, zl, zh, zl);
  // A z mod 1
  const float ph = __fmul_rn(c.ah, zh);
  const float pl = fmaf(c.ah, zh, -ph) + fmaf(c.ah, zl, c.al * zh);
  const float t1 = __fsub_rn(ph, rintf(ph)) + pl;
  // |C| s mod 1
  const uint64_t prod = c.cfix * (uint64_t)s;
  const float t2 = (float)(uint32_t)(prod >> 40) * 0x1p-24f;
  const float t = c.cneg ? t2 - t1 : -t2 - t1;
  return t - rintf(t);
}

// The three row kernels of the 2-D transforms, one block per row of the P x P
// grid, the row in shared memory:
//   MODE 0: the mask row (step 1's input, generated here: aperture row
//           j = p - P/2 + c, zero outside [j0, j1)), forward transform;
//   MODE 1: a row of the transposed spectrum: forward transform along it,
//           the residual phase of step 2 with the 1 / P^2 of the inverse
//           transform (evanescent components zeroed), inverse transform;
//   MODE 2: inverse transform, the result as two real planes (real parts at
//           planar, imaginary parts at planar + P^2) for the zoom's loaded
//           operand, or complex rows in place when planar is null.
// Forward results stay in bit-reversed order along the row, which the
// phase step and the inverse transforms read as such: no reordering pass.
struct SaRowArgs {
  int64_t P;
  int logP;
  const float2* tw;  // P / 2 twiddles e^{-2 pi i t / P}
  SaMaskArgs m;      // MODE 0
  SaPhase ph;        // MODE 1
  const float2* in;  // MODES 1, 2 (may equal out)
  float2* out;       // MODES 0, 1, 2 (complex rows)
  float* planar;     // MODE 2
};

// Row <-> shared memory with 16-byte accesses, eight in flight per thread
// (one block per SM holds a row, so the loads' latency is covered by their
// number, not by other blocks).
__device__ __forceinline__ void row_load(float2* x, const float2* __restrict__ src, int P) {
  const float4* s4 = reinterpret_cast<const float4*>(src);
  const int n4 = P / 2;
  for (int b = threadIdx.x; b < n4; b += 8 * blockDim.x) {
    float4 v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int i = b + u * blockDim.x;
      v[u] = i < n4 ? __ldg(s4 + i) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int i = b + u * blockDim.x;
      if (i < n4) {
        x[spad(2 * i)] = make_float2(v[u].x, v[u].y);
        x[spad(2 * i + 1)] = make_float2(v[u].z, v[u].w);
      }
    }
  }
}

__device__ __forceinline__ void row_store(float2* __restrict__ dst, const float2* x, int P) {
  float4* d4 = reinterpret_cast<float4*>(dst);
  for (int i = threadIdx.x; i < P / 2; i += blockDim.x) {
    const float2 a = x[spad(2 * i)], b = x[spad(2 * i + 1)];
    d4[i] = make_float4(a.x, a.y, b.x, b.y);
  }
}

// The twiddle table (P/2 entries) is copied into shared memory behind the
// row at the start, so the transform passes read it from there.
__device__ __forceinline__ void tw_load(float2* tws, const float2* __restrict__ tw, int P) {
  const float4* t4 = reinterpret_cast<const float4*>(tw);
  for (int i = threadIdx.x; i < P / 4; i += blockDim.x) {
    const float4 w = __ldg(t4 + i);
    tws[2 * i] = make_float2(w.x, w.y);
    tws[2 * i + 1] = make_float2(w.z, w.w);
  }
}

template <int MODE>
__global__ void __launch_bounds__(512, 1) k_sa_rows(const SaRowArgs a) {
  extern __shared__ float2 x[];
  const int P = (int)a.P, logP = a.logP;
  float2* tws = x + (P + P / 32);  // behind the padded row
  const int64_t row = blockIdx.x;
  if (MODE == 0) {
    const int64_t o = a.P / 2 - a.m.mg.c;
    const int64_t j = row - o, dj = j - a.m.mg.c;
    float2* dst = a.out + row * a.P;
    if (j < a.m.j0 || j >= a.m.j1 || j < 0 || j >= a.m.N || dj * dj > a.m.mg.sR) {
      float4* d4 = reinterpret_cast<float4*>(dst);
      for (int i = threadIdx.x; i < P / 2; i += blockDim.x) d4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
      return;
    }
    tw_load(tws, a.tw, P);
    for (int q = threadIdx.x; q < P; q += blockDim.x) {
      const int64_t i = q - o;
      const bool open = i >= 0 && i < a.m.N && sa_open(a.m, dj, i - a.m.mg.c);
      x[spad(q)] = make_float2(open ? 1.0f : 0.0f, 0.0f);
    }
    __syncthreads();
    row_fft_fwd(x, P, logP, tws);
    row_store(dst, x, P);
    return;
  }
  tw_load(tws, a.tw, P);
  row_load(x, a.in + row * a.P, P);
  __syncthreads();
  if (MODE == 1) {
    row_fft_fwd(x, P, logP, tws);
    // this row is the bit-reversed position of fb; element q of fa
    const int rb = sa_brev((int)row, logP), fb = rb < P / 2 ? rb : rb - P;
    for (int q = threadIdx.x; q < P; q += blockDim.x) {
      const int ra = sa_brev(q, logP), fa = ra < P / 2 ? ra : ra - P;
      const int64_t s2 = (int64_t)fa * fa + (int64_t)fb * fb;
      float2 v = make_float2(0.0f, 0.0f);
      if (s2 < a.ph.s_ev) {
        float sn, cs;
        sincospif(2.0f * sa_turns(a.ph, s2), &sn, &cs);
        const float2 u = x[spad(q)];
        v = make_float2(a.ph.scale * (u.x * cs - u.y * sn), a.ph.scale * (u.x * sn + u.y * cs));
      }
      x[spad(q)] = v;
    }
    __syncthreads();
  }
  row_fft_inv(x, P, logP, tws);
  if (MODE == 2 && a.planar) {
    float4* re = reinterpret_cast<float4*>(a.planar + row * a.P);
    float4* im = reinterpret_cast<float4*>(a.planar + row * a.P + a.P * a.P);
    for (int i = threadIdx.x; i < P / 4; i += blockDim.x) {
      const float2 v0 = x[spad(4 * i)], v1 = x[spad(4 * i + 1)], v2 = x[spad(4 * i + 2)], v3 = x[spad(4 * i + 3)];
      re[i] = make_float4(v0.x, v1.x, v2.x, v3.x);
      im[i] = make_float4(v0.y, v1.y, v2.y, v3.y);
    }
  } else {
    row_store(a.out + row * a.P, x, P);
  }
}

// K[m][q] = e^{i k0 u_q^2 / (2 z_F) - i k0 x_m u_q / z_F}, u_q = (q - P/2) dx,
// x_m = (m - msh) p; the phase in turns reduced in FP64.
__global__ void k_sa_kernel(int M, int64_t P, double msh, double p, double dx, double lzF, float2* __restrict__ K) {
  const int64_t total = (int64_t)M * P;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t m = t / P, q = t % P;
    const double u = (double)(q - P / 2) * dx, x = ((double)m - msh) * p;
    K[t] = cis_turns_f((0.5 * u * u - x * u) / lzF);
  }
}

// C[a][b] = sum_k X[a][k] Y[b][k] (complex, FP32 accumulation), a < na, b < nb,
// k < nk; rows of X and Y contiguous in k.  64 x 64 tile per block, 256
// threads with 4 x 4 outputs each, k in steps of 16 through shared memory.
// Out = float2 (stored) or double2 (stored as FP64).
template <typename Out>
__global__ void __launch_bounds__(256) k_sa_gemm_nt(const float2* __restrict__ X, const float2* __restrict__ Y,
                                                    int64_t na, int64_t nb, int64_t nk, Out* __restrict__ C) {
  __shared__ float2 sX[16][65];
  __shared__ float2 sY[16][65];
  const int64_t a0 = (int64_t)blockIdx.y * 64, b0 = (int64_t)blockIdx.x * 64;
  const int tid = threadIdx.x, ta = tid >> 4, tb = tid & 15;
  float2 acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.0f, 0.0f);
  for (int64_t k0 = 0; k0 < nk; k0 += 16) {
    for (int t = tid; t < 64 * 16; t += 256) {
      const int r = t >> 4, kk = t & 15;
      const int64_t a = a0 + r, b = b0 + r, k = k0 + kk;
      sX[kk][r] = (a < na && k < nk) ? X[a * nk + k] : make_float2(0.0f, 0.0f);
      sY[kk][r] = (b < nb && k < nk) ? Y[b * nk + k] : make_float2(0.0f, 0.0f);
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < 16; ++kk) {
      float2 xv[4], yv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) xv[i] = sX[kk][ta + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) yv[j] = sY[kk][tb + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          acc[i][j].x = fmaf(xv[i].x, yv[j].x, fmaf(-xv[i].y, yv[j].y, acc[i][j].x));
          acc[i][j].y = fmaf(xv[i].x, yv[j].y, fmaf(xv[i].y, yv[j].x, acc[i][j].y));
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t a = a0 + ta + 16 * i, b = b0 + tb + 16 * j;
      if (a < na && b < nb) {
        Out o;
        o.x = acc[i][j].x;
        o.y = acc[i][j].y;
        C[a * nb + b] = o;
      }
    }
}

SaMaskArgs mask_args(const Plan& P, int64_t j0, int64_t j1) {
  SaMaskArgs a{};
  a.mg = P.mg;
  a.N = P.N;
  a.P = P.sa.P;
  a.j0 = j0;
  a.j1 = j1;
  a.exact = P.sa.exact;
  a.xthr = P.sa.d_xthr;
  a.nx = P.sa.nx;
  a.dx2f = (float)P.dx2;
  a.ff = (float)P.f;
  a.lamf = (float)P.lambda;
  return a;
}

// Zone index of the exact radii (Eq. 3) at s = (r / dx)^2, in FP64.
int64_t zone_exact_host(const Plan& P, int64_t s) {
  const double r2 = (double)s * P.dx2;
  return (int64_t)std::floor(2.0 * r2 / (P.lambda * (std::sqrt(P.f * P.f + r2) + P.f)));
}

// First s of every zone m = 1 .. (the zone of s_R) of the exact radii, by
// bisection (the zone index is non-decreasing in s).
std::vector<int64_t> exact_thresholds(const Plan& P) {
  std::vector<int64_t> t;
  const int64_t zmax = zone_exact_host(P, P.mg.sR);
  for (int64_t m = 1; m <= zmax; ++m) {
    int64_t lo = t.empty() ? 0 : t.back(), hi = P.mg.sR;  // zone(hi) >= m
    while (lo < hi) {
      const int64_t mid = lo + (hi - lo) / 2;
      if (zone_exact_host(P, mid) >= m) hi = mid;
      else lo = mid + 1;
    }
    t.push_back(lo);
  }
  return t;
}

size_t rows_smem(int64_t P) { return (size_t)(P + P / 32 + P / 2) * sizeof(float2); }  // row + twiddles

// 512 threads (a group of 16 elements each per pass, two at P = 16384): the
// 16 values of a group stay in registers without spilling.
unsigned rows_threads(int64_t P) { return (unsigned)std::max<int64_t>(32, std::min<int64_t>(512, P / 16)); }

// Host constants of k_sa_phase (FP64 here, split into float-float pairs and
// 64-bit fixed point).
SaPhase sa_phase_consts(const Plan& P) {
  const SaCzt& s = P.sa;
  SaPhase c{};
  const double lr = P.lambda / ((double)s.P * P.dx);
  const double eps = lr * lr;
  const double A = P.f / P.lambda;
  const double k0 = 2.0 * M_PI / P.lambda;
  const double C = A * (s.d * k0 / s.kmax) * eps;
  c.eh = (float)eps;
  c.el = (float)(eps - (double)c.eh);
  c.ah = (float)A;
  c.al = (float)(A - (double)c.ah);
  c.cneg = C < 0 ? 1 : 0;
  c.cfix = (uint64_t)std::ldexp(std::fabs(C), 64);
  int64_t sev = (int64_t)std::ceil(1.0 / eps);
  while (sev > 0 && eps * (double)(sev - 1) >= 1.0) --sev;
  while (eps * (double)sev < 1.0) ++sev;
  c.s_ev = sev;
  c.scale = (float)(1.0 / ((double)s.P * (double)s.P));
  return c;
}

unsigned grid_for(int64_t items) { return (unsigned)std::min<int64_t>((items + 255) / 256, 152 * 32); }

}  // namespace

fzp_status saczt_layout(Plan& P) {
  SaCzt& s = P.sa;
  int64_t n = 64;  // at least two 32 x 32 transpose tiles
  int lg = 6;
  while ((double)n < 1.5 * (double)P.N) { n <<= 1; ++lg; }
  if (n > SA_PMAX)
    return set_error(FZP_E_UNSUPPORTED, "SA-CZT: padded grid %lld above %lld (N = %lld)", (long long)n,
                     (long long)SA_PMAX, (long long)P.N);
  s.P = n;
  s.logP = lg;
  const double k0 = 2.0 * M_PI / P.lambda;
  s.kmax = 2.0 * k0 / 3.0;
  s.d = (std::sqrt(k0 * k0 - s.kmax * s.kmax) - k0) / s.kmax;
  s.zF = -2.0 * k0 * s.d * P.f / s.kmax;
  return FZP_OK;
}

// The zoom runs on the tensor cores when the column pass's 128-row tiles fit M.
static bool saczt_zoom_tc(const Plan& P) { return P.M % 128 == 0; }

fzp_status saczt_build(Plan& P) {
  SaCzt& s = P.sa;
  fzp_status st = saczt_layout(P);
  if (st != FZP_OK) return st;
  const size_t grid = (size_t)s.P * (size_t)s.P * sizeof(float2);
  const size_t kern = (size_t)P.M * (size_t)s.P * sizeof(float2);
  FZP_CUDA_TRY(cudaMalloc(&s.d_G, grid));
  FZP_CUDA_TRY(cudaMalloc(&s.d_T, grid));
  FZP_CUDA_TRY(cudaMalloc(&s.d_tw, (size_t)s.P / 2 * sizeof(float2)));
  P.device_bytes += 2 * grid + (size_t)s.P / 2 * sizeof(float2);
  static std::atomic<uint64_t> attr0{0}, attr1{0}, attr2{0};
  FZP_CUDA_TRY(smem_attr_once((const void*)k_sa_rows<0>, (int)rows_smem(SA_PMAX), attr0));
  FZP_CUDA_TRY(smem_attr_once((const void*)k_sa_rows<1>, (int)rows_smem(SA_PMAX), attr1));
  FZP_CUDA_TRY(smem_attr_once((const void*)k_sa_rows<2>, (int)rows_smem(SA_PMAX), attr2));
  if (s.exact) {
    const std::vector<int64_t> t = exact_thresholds(P);
    s.nx = (int64_t)t.size();
    FZP_CUDA_TRY(cudaMalloc(&s.d_xthr, std::max<size_t>(1, t.size()) * sizeof(int64_t)));
    if (!t.empty())
      FZP_CUDA_TRY(cudaMemcpy(s.d_xthr, t.data(), t.size() * sizeof(int64_t), cudaMemcpyHostToDevice));
    P.device_bytes += t.size() * sizeof(int64_t);
  }
  k_sa_twiddles<<<grid_for(s.P / 2), 256>>>(s.P, reinterpret_cast<float2*>(s.d_tw));
  P.launches += 1;
  FZP_CUDA_TRY(cudaGetLastError());
  if (saczt_zoom_tc(P)) {
    // kernel images of K over the P padded columns: u = (q - P/2) dx, so the
    // phase is di^2 kappa / 2 - (m - msh) di delta turns with z_F for f
    const double lz = P.lambda * s.zF;
    return dense_zoom_build(P, s.P, s.P / 2, P.dx2 / lz, P.p * P.dx / lz);
  }
  FZP_CUDA_TRY(cudaMalloc(&s.d_K, kern));
  FZP_CUDA_TRY(cudaMalloc(&s.d_RT, kern));
  P.device_bytes += 2 * kern;
  k_sa_kernel<<<grid_for((int64_t)P.M * s.P), 256>>>(P.M, s.P, P.msh, P.p, P.dx, P.lambda * s.zF,
                                                      reinterpret_cast<float2*>(s.d_K));
  P.launches += 1;
  FZP_CUDA_TRY(cudaGetLastError());
  return FZP_OK;
}

fzp_status saczt_propagate(Plan& P, int64_t j0, int64_t j1, cudaStream_t st) {
  const SaCzt& s = P.sa;
  float2* G = reinterpret_cast<float2*>(s.d_G);
  float2* T = reinterpret_cast<float2*>(s.d_T);
  const float2* tw = reinterpret_cast<const float2*>(s.d_tw);
  const dim3 tgrid((unsigned)(s.P / 32), (unsigned)(s.P / 32)), tblock(32, 8);
  const bool tc = saczt_zoom_tc(P);
  SaRowArgs ra{};
  ra.P = s.P;
  ra.logP = s.logP;
  ra.tw = tw;
  ra.m = mask_args(P, j0, j1);
  ra.ph = sa_phase_consts(P);
  const unsigned nb = (unsigned)s.P, nt = rows_threads(s.P);
  const size_t smem = rows_smem(s.P);
  // step 1: mask rows and their forward transforms (G), transposed (T)
  ra.out = G;
  k_sa_rows<0><<<nb, nt, smem, st>>>(ra);
  k_sa_transpose<<<tgrid, tblock, 0, st>>>(G, T, s.P);
  // steps 2-3 along the other axis: forward, residual phase, inverse (T in place)
  ra.in = T;
  ra.out = T;
  P.dominant = "k_sa_rows<1> (forward transforms, residual phase, inverse transforms)";
  prof_begin(P, st);
  k_sa_rows<1><<<nb, nt, smem, st>>>(ra);
  prof_end(P, st);
  k_sa_transpose<<<tgrid, tblock, 0, st>>>(T, G, s.P);
  // the last inverse rows: U1 in place, or as two real planes in T for the tensor cores
  ra.in = G;
  ra.out = G;
  ra.planar = tc ? reinterpret_cast<float*>(T) : nullptr;
  k_sa_rows<2><<<nb, nt, smem, st>>>(ra);
  P.launches += 5;
  FZP_CUDA_TRY(cudaGetLastError());
  // the Fresnel part on the ROI: C1[m][v] = sum_u K[m][u] U1[v][u], then
  // U[n][m] += sum_v K[n][v] C1[m][v] into the FP64 accumulator
  if (tc) {
    const float* re = reinterpret_cast<const float*>(T);
    for (int part = 0; part < 2; ++part) {
      fzp_status e = dense_zoom_rows(P, re + (size_t)part * s.P * s.P, s.P, s.P, st);
      if (e == FZP_OK) e = column_pass_tc_w(P, 0, s.P, part ? 0.0 : 1.0, part ? 1.0 : 0.0, st);
      if (e != FZP_OK) return e;
    }
    return FZP_OK;
  }
  const float2* K = reinterpret_cast<const float2*>(s.d_K);
  float2* RT = reinterpret_cast<float2*>(s.d_RT);
  k_sa_gemm_nt<float2><<<dim3((unsigned)((s.P + 63) / 64), (unsigned)((P.M + 63) / 64)), 256, 0, st>>>(
      K, G, P.M, s.P, s.P, RT);
  k_sa_gemm_nt<double2><<<dim3((unsigned)((P.M + 63) / 64), (unsigned)((P.M + 63) / 64)), 256, 0, st>>>(
      K, RT, P.M, P.M, s.P, P.d_Uacc);
  P.launches += 2;
  FZP_CUDA_TRY(cudaGetLastError());
  return FZP_OK;
}

fzp_status saczt_mask(Plan& P, int64_t j0, int64_t rows, uint8_t* out, cudaStream_t st) {
  k_sa_mask_export<<<grid_for(rows * P.N), 256, 0, st>>>(mask_args(P, j0, j0 + rows), rows, out);
  P.launches += 1;
  FZP_CUDA_TRY(cudaGetLastError());
  return FZP_OK;
}

}  // namespace fzp
