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
// memory, up to 16384 points = 128 KiB, radix-2 passes) with tiled transposes
// between the two directions; the phase step and the transposes are HBM
// passes over the padded grid; the zoom is two FP32 complex products on the
// CUDA cores (M P^2 and M^2 P complex multiply-adds), accumulated into the
// FP64 ROI field.  Phases are reduced in FP64 before the FP32 (co)sines.
#include <cmath>

#include "fzp_internal.cuh"

namespace fzp {
namespace {

constexpr int FFT_THREADS = 1024;
constexpr int64_t SA_PMAX = 16384;  // rows of the transforms live in shared memory

struct SaMaskArgs {
  MaskGeom mg;  // disc limit, centre, paraxial zone rule, centre configuration
  int64_t N, P, j0, j1;
  int exact;
  double dx2, f, lambda;
};

// Open state of sample (j, i) (dj = j - c, di = i - c) inside the disc: exact
// radii (Eq. 3) take the zone index n(r) = 2 (sqrt(f^2 + r^2) - f) / lambda,
// written as 2 r^2 / (lambda (sqrt(f^2 + r^2) + f)) to avoid the cancellation;
// paraxial radii the library's exact integer rule.
__device__ __forceinline__ bool sa_open(const SaMaskArgs& a, int64_t dj, int64_t di) {
  const int64_t s = dj * dj + di * di;
  if (s > a.mg.sR) return false;
  if (!a.exact) return ((zone_of(s, a.mg) ^ a.mg.centre_open) & 1) != 0;
  const double r2 = (double)s * a.dx2;
  const double n = 2.0 * r2 / (a.lambda * (sqrt(a.f * a.f + r2) + a.f));
  return ((((int64_t)floor(n)) ^ (int64_t)a.mg.centre_open) & 1) != 0;
}

// The mask on the padded grid (rows outside [j0, j1) zero): G[p][q] for
// aperture sample (j, i) = (p, q) - P/2 + c.
__global__ void k_sa_mask(SaMaskArgs a, float2* __restrict__ G) {
  const int64_t total = a.P * a.P, o = a.P / 2 - a.mg.c;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = t / a.P, q = t % a.P;
    const int64_t j = p - o, i = q - o;
    float v = 0.0f;
    if (j >= a.j0 && j < a.j1 && i >= 0 && i < a.N && sa_open(a, j - a.mg.c, i - a.mg.c)) v = 1.0f;
    G[t] = make_float2(v, 0.0f);
  }
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

__device__ __forceinline__ int sa_brev(int64_t v, int bits) { return (int)(__brev((unsigned)v) >> (32 - bits)); }

// In-place P-point FFT of every row (one block per row): bit-reversed load
// into shared memory, log2 P radix-2 passes, store.  Forward e^{-2 pi i k n / P};
// inverse the conjugate (no 1/P).
__global__ void __launch_bounds__(FFT_THREADS) k_sa_fft_rows(float2* __restrict__ data, int64_t P, int logP,
                                                             const float2* __restrict__ tw, int inverse) {
  extern __shared__ float2 srow[];
  float2* row = data + (int64_t)blockIdx.x * P;
  for (int64_t t = threadIdx.x; t < P; t += blockDim.x) srow[sa_brev(t, logP)] = row[t];
  __syncthreads();
  for (int st = 1; st <= logP; ++st) {
    const int64_t half = 1ll << (st - 1);
    const int64_t step = P >> st;
    for (int64_t b = threadIdx.x; b < P / 2; b += blockDim.x) {
      const int64_t k = b & (half - 1);
      const int64_t i0 = ((b >> (st - 1)) << st) + k, i1 = i0 + half;
      float2 w = __ldg(tw + k * step);
      if (inverse) w.y = -w.y;
      const float2 u = srow[i0], v = cmul(srow[i1], w);
      srow[i0] = cadd(u, v);
      srow[i1] = csub(u, v);
    }
    __syncthreads();
  }
  for (int64_t t = threadIdx.x; t < P; t += blockDim.x) row[t] = srow[t];
}

// out[x][y] = in[y][x] for a P x P complex64 matrix (32 x 32 tiles, block 32 x 8).
__global__ void k_sa_transpose(const float2* __restrict__ in, float2* __restrict__ out, int64_t P) {
  __shared__ float2 tile[32][33];
  const int64_t x0 = (int64_t)blockIdx.x * 32, y0 = (int64_t)blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += 8) tile[r][threadIdx.x] = in[(y0 + r) * P + x0 + threadIdx.x];
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += 8) out[(x0 + r) * P + y0 + threadIdx.x] = tile[threadIdx.x][r];
}

// Step 2 with the 1 / P^2 of the inverse transform: element (a, b) of the
// spectrum has K = 2 pi (fa, fb) / (P dx), fa the signed frequency index of a.
// h = k_z - k0 - d K^2 / k_max with k_z - k0 = -K^2 / (k0 + k_z) (c k_max = k0).
__global__ void k_sa_phase(float2* __restrict__ A, int64_t P, double dx, double k0, double f, double kmax, double d,
                           float scale) {
  const int64_t total = P * P;
  const double dk = 2.0 * 3.14159265358979323846 / ((double)P * dx);
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = t / P, b = t % P;
    const double ka = (double)(a < P / 2 ? a : a - P) * dk, kb = (double)(b < P / 2 ? b : b - P) * dk;
    const double K2 = ka * ka + kb * kb;
    float2 v = make_float2(0.0f, 0.0f);
    if (K2 < k0 * k0) {
      const double kz = sqrt(k0 * k0 - K2);
      const double h = -K2 / (k0 + kz) - d * K2 / kmax;
      const float2 w = cis_turns_f(h * f / (2.0 * 3.14159265358979323846));
      const float2 x = A[t];
      v = make_float2(scale * (x.x * w.x - x.y * w.y), scale * (x.x * w.y + x.y * w.x));
    }
    A[t] = v;
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
  a.dx2 = P.dx2;
  a.f = P.f;
  a.lambda = P.lambda;
  return a;
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

fzp_status saczt_build(Plan& P) {
  SaCzt& s = P.sa;
  fzp_status st = saczt_layout(P);
  if (st != FZP_OK) return st;
  const size_t grid = (size_t)s.P * (size_t)s.P * sizeof(float2);
  const size_t kern = (size_t)P.M * (size_t)s.P * sizeof(float2);
  FZP_CUDA_TRY(cudaMalloc(&s.d_G, grid));
  FZP_CUDA_TRY(cudaMalloc(&s.d_T, grid));
  FZP_CUDA_TRY(cudaMalloc(&s.d_tw, (size_t)s.P / 2 * sizeof(float2)));
  FZP_CUDA_TRY(cudaMalloc(&s.d_K, kern));
  FZP_CUDA_TRY(cudaMalloc(&s.d_RT, kern));
  P.device_bytes += 2 * grid + 2 * kern + (size_t)s.P / 2 * sizeof(float2);
  static std::atomic<uint64_t> attr{0};
  FZP_CUDA_TRY(smem_attr_once((const void*)k_sa_fft_rows, (int)(SA_PMAX * sizeof(float2)), attr));
  k_sa_twiddles<<<grid_for(s.P / 2), 256>>>(s.P, reinterpret_cast<float2*>(s.d_tw));
  k_sa_kernel<<<grid_for((int64_t)P.M * s.P), 256>>>(P.M, s.P, P.msh, P.p, P.dx, P.lambda * s.zF,
                                                      reinterpret_cast<float2*>(s.d_K));
  P.launches += 2;
  FZP_CUDA_TRY(cudaGetLastError());
  return FZP_OK;
}

fzp_status saczt_propagate(Plan& P, int64_t j0, int64_t j1, cudaStream_t st) {
  const SaCzt& s = P.sa;
  float2* G = reinterpret_cast<float2*>(s.d_G);
  float2* T = reinterpret_cast<float2*>(s.d_T);
  const float2* tw = reinterpret_cast<const float2*>(s.d_tw);
  const size_t smem = (size_t)s.P * sizeof(float2);
  const dim3 tgrid((unsigned)(s.P / 32), (unsigned)(s.P / 32)), tblock(32, 8);
  P.dominant = "saczt_pipeline";
  prof_begin(P, st);
  k_sa_mask<<<grid_for(s.P * s.P), 256, 0, st>>>(mask_args(P, j0, j1), G);
  // FFT2: rows, transpose, rows (the spectrum in transposed layout)
  k_sa_fft_rows<<<(unsigned)s.P, FFT_THREADS, smem, st>>>(G, s.P, s.logP, tw, 0);
  k_sa_transpose<<<tgrid, tblock, 0, st>>>(G, T, s.P);
  k_sa_fft_rows<<<(unsigned)s.P, FFT_THREADS, smem, st>>>(T, s.P, s.logP, tw, 0);
  const double k0 = 2.0 * M_PI / P.lambda;
  k_sa_phase<<<grid_for(s.P * s.P), 256, 0, st>>>(T, s.P, P.dx, k0, P.f, s.kmax, s.d,
                                                  (float)(1.0 / ((double)s.P * (double)s.P)));
  // inverse FFT2: rows, transpose back, rows
  k_sa_fft_rows<<<(unsigned)s.P, FFT_THREADS, smem, st>>>(T, s.P, s.logP, tw, 1);
  k_sa_transpose<<<tgrid, tblock, 0, st>>>(T, G, s.P);
  k_sa_fft_rows<<<(unsigned)s.P, FFT_THREADS, smem, st>>>(G, s.P, s.logP, tw, 1);
  // the Fresnel part on the ROI: RT[m][v] = sum_u K[m][u] U1[v][u], then
  // U[n][m] = sum_v K[n][v] RT[m][v] into the FP64 accumulator
  const float2* K = reinterpret_cast<const float2*>(s.d_K);
  float2* RT = reinterpret_cast<float2*>(s.d_RT);
  k_sa_gemm_nt<float2><<<dim3((unsigned)((s.P + 63) / 64), (unsigned)((P.M + 63) / 64)), 256, 0, st>>>(
      K, G, P.M, s.P, s.P, RT);
  k_sa_gemm_nt<double2><<<dim3((unsigned)((P.M + 63) / 64), (unsigned)((P.M + 63) / 64)), 256, 0, st>>>(
      K, RT, P.M, P.M, s.P, P.d_Uacc);
  prof_end(P, st);
  P.launches += 11;
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
