// metrics.cu -- metric extractor on the device (Fig. 2 Stage 4; Fig. 18 Stage 5).
//
//   FWHM  : centre row (and column) through the on-axis sample M/2; peak from
//           the 3-point parabola there; half-maximum crossings are roots of the
//           not-a-knot cubic spline through the row, solved by bisection.
//   DE    : sum of I p^2 over ROI samples with r <= r_null, divided by
//           P_in = (# aperture samples with r <= R_eff) dx^2; also over the ROI.
//   MTF   : |fft2(I)| / |fft2(I)|(0,0), averaged in 200 equal radial bins over
//           [0, nu_Nyq], nu_Nyq = 1/(2p); sample (ku, kv) lies in bin
//           floor(200 |k| / (M/2)) evaluated exactly in integers; read by linear
//           interpolation between bin centres at nu_cut/2 and at 16 frequencies.
//   Strehl: I(M/2, M/2) / (pi R^2 / (lambda f))^2.
#include <cmath>
#include <cstring>
#include <mutex>

#include "fzp_internal.cuh"

namespace fzp {
namespace {

constexpr int NBINS = 200;
// scratch layout in P.d_metrics (doubles)
constexpr int S_SUM = 0, S_LOBE = 1, S_COUNT = 2 /* int64 bits */, S_OUT = 8, S_BINS = 64;
constexpr int S_BINCNT = S_BINS + NBINS;  // int64 bits
constexpr int S_FFT = 1024;               // complex work area starts here (doubles)
// S_OUT..: fwhm_x, fwhm_y, peak
constexpr double AIRY_NULL = 3.8317059702075125 / 3.14159265358979323846;

__device__ __forceinline__ int64_t isqrt64(int64_t v) {
  if (v <= 0) return 0;
  int64_t r = (int64_t)sqrt((double)v);
  while (r * r > v) --r;
  while ((r + 1) * (r + 1) <= v) ++r;
  return r;
}

__global__ void k_sums(int M, double p, double rnull2, const double2* __restrict__ U, double* scratch) {
  __shared__ double sh[2][256];
  double s = 0, l = 0;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < M * M; t += gridDim.x * blockDim.x) {
    const int n = t / M, m = t % M;
    const double I = U[t].x * U[t].x + U[t].y * U[t].y;
    s += I;
    const double xm = (double)(m - M / 2) * p, yn = (double)(n - M / 2) * p;
    if (xm * xm + yn * yn <= rnull2) l += I;
  }
  sh[0][threadIdx.x] = s;
  sh[1][threadIdx.x] = l;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      sh[0][threadIdx.x] += sh[0][threadIdx.x + w];
      sh[1][threadIdx.x] += sh[1][threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    atomicAdd(&scratch[S_SUM], sh[0][0]);
    atomicAdd(&scratch[S_LOBE], sh[1][0]);
  }
}

__global__ void k_count(int64_t N, int64_t c, int64_t sR, double* scratch) {
  unsigned long long acc = 0;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < N; j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t dj = j - c;
    if (dj * dj <= sR) acc += (unsigned long long)(2 * isqrt64(sR - dj * dj) + 1);
  }
  atomicAdd(reinterpret_cast<unsigned long long*>(&scratch[S_COUNT]), acc);
}

// In-place radix-2 DIT on SMEM (bit-reversed input), FP64, twiddles computed here.
__device__ void dit64(double2* x, int logn) {
  const int n = 1 << logn;
  for (int s = 1; s <= logn; ++s) {
    const int half = 1 << (s - 1);
    for (int b = threadIdx.x; b < n / 2; b += blockDim.x) {
      const int k = b & (half - 1);
      const int i0 = ((b >> (s - 1)) << s) + k, i1 = i0 + half;
      double sn, cs;
      sincospi(-(double)k / (double)half, &sn, &cs);
      const double2 a = x[i0], v = x[i1];
      const double2 t = make_double2(v.x * cs - v.y * sn, v.x * sn + v.y * cs);
      x[i0] = make_double2(a.x + t.x, a.y + t.y);
      x[i1] = make_double2(a.x - t.x, a.y - t.y);
    }
    __syncthreads();
  }
}

// Row FFTs of I: F[n][k] = sum_m I[n][m] e^{-2 pi i m k / M}.
__global__ void k_fft_rows(int M, int logM, const double2* __restrict__ U, double2* F) {
  extern __shared__ double2 sm[];
  const int n = blockIdx.x;
  for (int m = threadIdx.x; m < M; m += blockDim.x) {
    const double2 u = U[(int64_t)n * M + m];
    sm[__brev(m) >> (32 - logM)] = make_double2(u.x * u.x + u.y * u.y, 0.0);
  }
  __syncthreads();
  dit64(sm, logM);
  for (int k = threadIdx.x; k < M; k += blockDim.x) F[(int64_t)n * M + k] = sm[k];
}

// Column FFTs and radial binning of |OTF|.
__global__ void k_fft_cols(int M, int logM, const double2* __restrict__ F, double* scratch) {
  extern __shared__ double2 sm[];
  const int k = blockIdx.x;
  for (int n = threadIdx.x; n < M; n += blockDim.x) sm[__brev(n) >> (32 - logM)] = F[(int64_t)n * M + k];
  __syncthreads();
  dit64(sm, logM);
  const int ku = k < M / 2 ? k : k - M;
  unsigned long long* cnt = reinterpret_cast<unsigned long long*>(scratch + S_BINCNT);
  for (int q = threadIdx.x; q < M; q += blockDim.x) {
    const int kv = q < M / 2 ? q : q - M;
    const int64_t r2 = (int64_t)ku * ku + (int64_t)kv * kv;
    // bin = floor(2 NBINS sqrt(r2) / M), exact
    const int64_t b = isqrt64((int64_t)(4 * NBINS * NBINS) * r2 / ((int64_t)M * M));
    if (b < NBINS) {
      const double a = sqrt(sm[q].x * sm[q].x + sm[q].y * sm[q].y);
      atomicAdd(&scratch[S_BINS + b], a);
      atomicAdd(&cnt[b], 1ull);
    }
  }
}

// Not-a-knot cubic spline slopes on a unit grid; y has n points.
__device__ void spline_slopes(const double* y, int n, double* s, double* cp) {
  // unknowns s_1..s_{n-2}: tridiagonal (Thomas); diag/rhs built on the fly
  // row 1: 2 s1 + s2 = (d0 + 5 d1)/2 ; rows i: s_{i-1} + 4 s_i + s_{i+1} = 3 (d_{i-1} + d_i)
  // row n-2: s_{n-3} + 2 s_{n-2} = (5 d_{n-3} + d_{n-2})/2, d_i = y_{i+1} - y_i
  const int K = n - 2;
  auto d = [&](int i) { return y[i + 1] - y[i]; };
  // forward sweep: cp = modified super-diagonal, s = modified rhs
  for (int r = 0; r < K; ++r) {
    const int i = r + 1;
    double a = 1.0, b = 4.0, c = 1.0, rhs = 3.0 * (d(i - 1) + d(i));
    if (r == 0) { a = 0.0; b = 2.0; c = 1.0; rhs = 0.5 * (d(0) + 5.0 * d(1)); }
    if (r == K - 1) { a = 1.0; b = 2.0; c = 0.0; rhs = 0.5 * (5.0 * d(n - 3) + d(n - 2)); }
    if (r == 0) {
      cp[r] = c / b;
      s[i] = rhs / b;
    } else {
      const double den = b - a * cp[r - 1];
      cp[r] = c / den;
      s[i] = (rhs - a * s[i - 1]) / den;
    }
  }
  for (int r = K - 2; r >= 0; --r) s[r + 1] -= cp[r] * s[r + 2];
  s[0] = s[2] + 2.0 * d(0) - 2.0 * d(1);
  s[n - 1] = s[n - 3] - 2.0 * d(n - 3) + 2.0 * d(n - 2);
}

__device__ double hermite(const double* y, const double* s, int i, double t) {
  const double dl = y[i + 1] - y[i];
  const double c2 = 3.0 * dl - 2.0 * s[i] - s[i + 1];
  const double c3 = s[i] + s[i + 1] - 2.0 * dl;
  return y[i] + t * (s[i] + t * (c2 + t * c3));
}

__device__ double crossing(const double* y, const double* s, int i, double half) {
  // root of hermite(i, t) = half in t in [0, 1] (sign change guaranteed by the scan)
  double lo = 0.0, hi = 1.0;
  const double flo = hermite(y, s, i, 0.0) - half;
  for (int it = 0; it < 64; ++it) {
    const double mid = 0.5 * (lo + hi);
    const double fm = hermite(y, s, i, mid) - half;
    if ((fm < 0) == (flo < 0)) lo = mid; else hi = mid;
  }
  return (double)i + 0.5 * (lo + hi);
}

// One thread: FWHM along the centre row (axis 0) or column (axis 1).
__global__ void k_fwhm(int M, double p, const double2* __restrict__ U, double* work, double* scratch) {
  if (threadIdx.x != 0) return;
  const int axis = blockIdx.x;
  double* y = work + (size_t)axis * 3 * M;
  double* s = y + M;
  double* cp = s + M;
  const int k = M / 2;
  for (int i = 0; i < M; ++i) {
    const double2 u = axis == 0 ? U[(int64_t)k * M + i] : U[(int64_t)i * M + k];
    y[i] = u.x * u.x + u.y * u.y;
  }
  const double ym = y[k - 1], y0 = y[k], yp = y[k + 1];
  const double den = ym - 2.0 * y0 + yp;
  const double peak = den != 0.0 ? y0 - 0.125 * (yp - ym) * (yp - ym) / den : y0;
  const double half = 0.5 * peak;
  spline_slopes(y, M, s, cp);
  int m = k;
  while (m > 0 && y[m] >= half) --m;
  const double xl = crossing(y, s, m, half);
  m = k;
  while (m < M - 1 && y[m] >= half) ++m;
  const double xr = crossing(y, s, m - 1, half);
  scratch[S_OUT + axis] = (xr - xl) * p;
  if (axis == 0) scratch[S_OUT + 2] = y0;
}

}  // namespace

// The extractor's kernels on `scr` (sums, counts and bins cleared first),
// then the scratch header copied to h[] (host); the caller synchronises.
static fzp_status extract_enqueue(int M, double p, double rnull, int64_t N, int64_t c, int64_t sR,
                                  const double2* U, double* scr, double* h, cudaStream_t s) {
  int logM = 0;
  while ((1 << logM) < M) ++logM;
  double2* F = reinterpret_cast<double2*>(scr + S_FFT + 6 * 1024);
  FZP_CUDA_TRY(cudaMemsetAsync(scr, 0, S_FFT * sizeof(double), s));
  k_sums<<<256, 256, 0, s>>>(M, p, rnull * rnull, U, scr);
  k_count<<<256, 256, 0, s>>>(N, c, sR, scr);
  k_fft_rows<<<M, 256, M * sizeof(double2), s>>>(M, logM, U, F);
  k_fft_cols<<<M, 256, M * sizeof(double2), s>>>(M, logM, F, scr);
  k_fwhm<<<2, 32, 0, s>>>(M, p, U, scr + S_FFT, scr);
  FZP_CUDA_TRY(cudaGetLastError());
  FZP_CUDA_TRY(cudaMemcpyAsync(h, scr, S_FFT * sizeof(double), cudaMemcpyDeviceToHost, s));
  return FZP_OK;
}

// Host post-processing of the scratch header h[] into the metrics: DE over
// P_in = count dx^2, Strehl, and the radial MTF read at nu_cut/2 and at the
// 16 sample frequencies (linear interpolation between bin centres).
static void extract_finish(const double* h, double p, double R2, double lf, double dx2, fzp_metrics_t* out) {
  const double sum = h[S_SUM], lobe = h[S_LOBE];
  int64_t count;
  memcpy(&count, &h[S_COUNT], sizeof(count));
  const double pin = (double)count * dx2;
  out->aperture_count = count;
  out->p_in = pin;
  out->p_in_disc = 3.14159265358979323846 * R2;
  out->de_lobe = lobe * p * p / pin;
  out->de_roi = sum * p * p / pin;
  out->fwhm_x = h[S_OUT];
  out->fwhm_y = h[S_OUT + 1];
  out->peak = h[S_OUT + 2];
  const double ip = 3.14159265358979323846 * R2 / lf;
  out->strehl = out->peak / (ip * ip);
  // radial MTF: bin means normalised by |OTF(0,0)| = sum I
  double centre[NBINS], mean[NBINS];
  int nb = 0;
  const double nyq = 1.0 / (2.0 * p);
  for (int b = 0; b < NBINS; ++b) {
    int64_t c;
    memcpy(&c, &h[S_BINCNT + b], sizeof(c));
    if (c > 0) {
      centre[nb] = (b + 0.5) * nyq / NBINS;
      mean[nb] = h[S_BINS + b] / (double)c / sum;
      ++nb;
    }
  }
  auto interp = [&](double nu) -> double {
    if (nb == 0) return (double)NAN;
    if (nu <= centre[0]) return mean[0];
    if (nu >= centre[nb - 1]) return mean[nb - 1];
    int i = 0;
    while (centre[i + 1] < nu) ++i;
    const double t = (nu - centre[i]) / (centre[i + 1] - centre[i]);
    return mean[i] + t * (mean[i + 1] - mean[i]);
  };
  const double nucut = 2.0 * std::sqrt(R2) / lf;
  out->mtf_half_cut = interp(0.5 * nucut);
  for (int q = 0; q < 16; ++q) out->mtf16[q] = interp((q + 0.5) * nucut / 16.0);
}

fzp_status metrics(Plan& P, const void* d_field, cudaStream_t s, fzp_metrics_t* out) {
  const int M = P.M;
  if ((M & (M - 1)) != 0) return set_error(FZP_E_UNSUPPORTED, "metrics need a power-of-two M (got %d)", M);
  if (P.msh != (double)(M / 2))
    return set_error(FZP_E_UNSUPPORTED, "metrics read the focus at the ROI centre: the plan's ROI is off axis");
  const double lf = P.lambda * P.f;
  double h[S_FFT];
  fzp_status st = extract_enqueue(M, P.p, AIRY_NULL * lf / (2.0 * P.R), P.N, P.c, P.mg.sR,
                                  reinterpret_cast<const double2*>(d_field), P.d_metrics, h, s);
  if (st != FZP_OK) return st;
  P.launches += 5;
  int err = 0;
  FZP_CUDA_TRY(cudaMemcpyAsync(&err, P.d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  FZP_CUDA_TRY(cudaStreamSynchronize(s));
  if (err) return set_error(FZP_E_TIMEOUT, "a device-side wait timed out (code %d); results are invalid", err);
  extract_finish(h, P.p, P.R2, lf, P.dx2, out);
  return FZP_OK;
}

// ---------------------------------------------------------------- no-allocation variant
// Scratch of fzp_metrics_noalloc: same layout as the plan's metric scratch for
// M <= 512 (sums, bins, spline work, then the M x M complex FFT buffer).
constexpr int kNoAllocMaxM = 512;
constexpr size_t kNoAllocDoubles = (size_t)S_FFT + 6 * 1024 + 2 * (size_t)kNoAllocMaxM * kNoAllocMaxM;
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device; looked up once
// per device with that device current.
fzp_status noalloc_scratch(double** out) {
  int dev = 0;
  FZP_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return set_error(FZP_E_UNSUPPORTED, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return set_error(FZP_E_CUDA, "cudaGetSymbolAddress(scratch) failed on device %d: %s", dev,
                       cudaGetErrorString(e));
    g_noalloc_ptr[dev] = p;
  }
  *out = reinterpret_cast<double*>(g_noalloc_ptr[dev]);
  return FZP_OK;
}

}  // namespace

}  // namespace fzp

extern "C" fzp_status fzp_metrics_noalloc(const fzp_params* in, const void* d_field, void* stream,
                                          fzp_metrics_t* out) {
  using namespace fzp;
  if (!in || !d_field || !out) return set_error(FZP_E_INVALID, "NULL argument");
  // the plan's own host path: validation (Eq. 6, N, levels, centre
  // configuration, ROI origin) and grids (Fig. 2 / Fig. 18 Stage 1-2), no
  // CUDA call and no allocation
  Plan P;
  int64_t sR = 0, zmax = 0;
  fzp_status st = plan_host(in, P, &sR, &zmax);
  if (st != FZP_OK) return st;
  if (P.M > kNoAllocMaxM)
    return set_error(FZP_E_INVALID, "M = %d outside the static scratch of fzp_metrics_noalloc "
                     "(a power of two in [64, %d])", P.M, kNoAllocMaxM);
  if (P.msh != (double)(P.M / 2))
    return set_error(FZP_E_UNSUPPORTED, "metrics read the focus at the ROI centre: the ROI is off axis");
  double* scr = nullptr;
  st = noalloc_scratch(&scr);
  if (st != FZP_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const double lf = P.lambda * P.f;
  double h[S_FFT];
  st = extract_enqueue(P.M, P.p, AIRY_NULL * lf / (2.0 * P.R), P.N, P.c, sR,
                       reinterpret_cast<const double2*>(d_field), scr, h, s);
  if (st != FZP_OK) return st;
  FZP_CUDA_TRY(cudaStreamSynchronize(s));
  extract_finish(h, P.p, P.R2, lf, P.dx2, out);
  return FZP_OK;
}
