// fzp_internal.cuh -- shared declarations of libfzp (CUDA C++, sm_103a).
//
// Notation (Eq. 2 and Fig. 2):
//   aperture sample (j, i), i, j in [0, N), centred index di = i - c, c = (N-1)/2,
//   u_i = di * dx;  ROI sample (n, m), x_m = (m - msh) p, msh = -x0 / p
//   (msh = M/2 for the ROI centred on the focus).
//   Row kernel K[m, i] = exp(2 pi i theta(m, i)) with the phase in turns
//     theta(m, i) = di^2 kappa / 2 - (m - msh) di delta,
//     kappa = dx^2 / (lambda f),  delta = p dx / (lambda f)   (Eq. 2, Eq. 10).
//   The same matrix serves the column pass (the grids of both axes coincide):
//     U = Pre * chirp_out .* (K T K^T).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <utility>
#include <vector>

#include "../../include/fzp.h"

namespace fzp {

// --------------------------------------------------------------------------
// Host-side error handling (thread-local message, no exceptions across ABI)
// --------------------------------------------------------------------------
fzp_status set_error(fzp_status st, const char* fmt, ...);

#define FZP_CUDA_TRY(call)                                                              \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return ::fzp::set_error(e_ == cudaErrorMemoryAllocation ? FZP_E_OOM : FZP_E_CUDA, \
                              "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),   \
                              __FILE__, __LINE__);                                      \
  } while (0)

// Dynamic shared memory above 48 KiB is an attribute of a kernel on one
// device: set it on each device that launches the kernel, once.  `done` holds
// a bit per device ordinal (ordinals from 64 up set it at every call).
inline cudaError_t smem_attr_once(const void* kernel, int bytes, std::atomic<uint64_t>& done) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const uint64_t bit = dev < 64 ? (1ull << dev) : 0ull;
  if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_acq_rel);
  return e;
}

// --------------------------------------------------------------------------
// Mask geometry: exact binary FZP rule (paraxial radii, centre opaque)
//   open(s) = s <= s_R  and  zone(s) odd,   zone(s) = floor(fl(s * kappa)),
//   s = di^2 + dj^2 an exact integer.  zone(s) = #{m >= 1 : S_m <= s} with the
//   threshold table S_m = min{s : floor(fl(s kappa)) >= m} built on the host.
// --------------------------------------------------------------------------
struct MaskGeom {
  int64_t c;          // on-axis index
  int64_t sR;         // largest s inside the aperture disc
  uint64_t K64;       // floor(kappa * 2^64): fixed-point zone rate
  const int64_t* thr; // device: thr[m-1] = S_m, m = 1..nthr
  int64_t nthr;
  int levels;         // 0: binary amplitude (open on odd zones); L >= 2: phase level = zone mod L
  int centre_open;    // binary amplitude: 1 = open on even zones (positive-centred)
};

// zone(s) for 0 <= s <= sR (the zone rate kappa is kappa_L for phase plates).
// The 64x64->128 fixed-point product s K64 / 2^64 lies below s kappa by less
// than s / 2^64 < 2^-18 (s < 2^46), and fl(s kappa) differs from s kappa by
// less than 2^-29 (s kappa < 2^24); so outside a window of 2^-17 below and
// 2^-28 above an integer the product's integer part is floor(fl(s kappa)), and
// inside it the threshold table decides, bit for bit.
__device__ __forceinline__ int64_t zone_of(int64_t s, const MaskGeom& g) {
  const uint64_t hi = __umul64hi((uint64_t)s, g.K64);
  const uint64_t lo = (uint64_t)s * g.K64;
  int64_t z = (int64_t)hi;
  if (lo < (1ull << 36) || lo >= 0xFFFF800000000000ull) {
    if (z >= 1 && __ldg(g.thr + (z - 1)) > s) z -= 1;
    else if (z < g.nthr && __ldg(g.thr + z) <= s) z += 1;
  }
  return z;
}

__device__ __forceinline__ bool mask_open(int64_t dj, int64_t di, const MaskGeom& g) {
  const int64_t s = dj * dj + di * di;
  if (s > g.sR) return false;
  return ((zone_of(s, g) ^ g.centre_open) & 1) != 0;
}

// --------------------------------------------------------------------------
// Membrane deformation phase in turns, 2 w / lambda (phi / 2 pi, phi = (4 pi /
// lambda) w), as FP32 coefficients in sample units (di = i - c, dj = j - c):
//   amp2 sin(2 pi (di kx + dj ky)) (1 - tq (di^2 + dj^2)) + sum_k h2_k exp(-q_k d_k^2),
//   d_k = (di - pi_k) nx_k + (dj - pj_k) ny_k  ((pi_k, pj_k) on the k-th crease).
// kx, ky are split hi + lo with hi a multiple of 2^-14: for |di| < 2^20 and the
// configured wrinkle periods (>= 1 mm at sub-micron pitch) di * kxh is exact in
// FP32, so the integer turns drop exactly before the sine.
// --------------------------------------------------------------------------
struct DeformCoef {
  float kxh, kxl, kyh, kyl, amp2, tq;
  int n;
  float nx[3], ny[3], pi_[3], pj[3], q[3], h2[3];
  // steps along a row (di -> di + 1) for generators that walk columns:
  // the wrinkle phasor turns by e^{2 pi i kx}; a ridge's ratio g(di+1)/g(di)
  // is multiplied by rho_k = exp(-2 q_k nx_k^2)
  float zc, zs, rho[3];
};

// --------------------------------------------------------------------------
// Phase helpers.  Phases are carried in turns; the integer part is removed in
// FP64 before the (co)sine is evaluated.
// --------------------------------------------------------------------------
__device__ __forceinline__ double frac_turns(double t) { return t - rint(t); }

__device__ __forceinline__ float2 cis_turns_f(double t) {
  float s, c;
  sincospif((float)(2.0 * frac_turns(t)), &s, &c);
  return make_float2(c, s);
}

__device__ __forceinline__ double2 cis_turns_d(double t) {
  double s, c;
  sincospi(2.0 * frac_turns(t), &s, &c);
  return make_double2(c, s);
}

template <typename R> struct Cplx;
template <> struct Cplx<float> { using T = float2; };
template <> struct Cplx<double> { using T = double2; };

template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  C r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { C r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { C r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }

template <typename R> __device__ __forceinline__ typename Cplx<R>::T cis_turns(double t);
template <> __device__ __forceinline__ float2 cis_turns<float>(double t) { return cis_turns_f(t); }
template <> __device__ __forceinline__ double2 cis_turns<double>(double t) { return cis_turns_d(t); }

// e^{sign 2 pi i r / L} for an exact integer r (0 <= r < L, L a power of two).
template <typename R> __device__ __forceinline__ typename Cplx<R>::T twiddle(int64_t r, int64_t L, float sign);
template <> __device__ __forceinline__ float2 twiddle<float>(int64_t r, int64_t L, float sign) {
  float s, c;
  sincospif(sign * 2.0f * (float)r / (float)L, &s, &c);
  return make_float2(c, s);
}
template <> __device__ __forceinline__ double2 twiddle<double>(int64_t r, int64_t L, float sign) {
  double s, c;
  sincospi((double)sign * 2.0 * (double)r / (double)L, &s, &c);
  return make_double2(c, s);
}

// --------------------------------------------------------------------------
// Plan
// --------------------------------------------------------------------------
struct Bluestein {
  int64_t L = 0;     // convolution length, power of two >= N + M - 1
  int64_t L1 = 1;    // four-step split L = L1 * L2 (L1 = 1: single pass)
  int64_t L2 = 0;
  void* d_pre = nullptr;  // N entries: e^{2 pi i pre(i)} (complex64 or complex128)
  void* d_H = nullptr;    // L entries: FFT_L of the convolution chirp, stored [k1][k2]
  void* d_Z = nullptr;    // workspace [rows][L1][L2]
  void* d_G = nullptr;    // workspace [rows][L1][M]
  void* d_tab = nullptr;  // table block: chirp v (L) | twiddles (L2/2) | post (M)
  void* d_tw = nullptr;   // into d_tab
  void* d_post = nullptr; // into d_tab
  void* d_twL = nullptr;  // into d_tab: e^{-2 pi i t / L}, t < 4096
  int64_t rows = 0;       // rows per batch of the workspace
  // partitioned convolution (FP32): blocks of S columns, 4096-point spectra of
  // the chirp pieces in d_H as [nseg][4096]; d_Z, d_G unused
  int seg = 0;
  int S = 0;
  int64_t nseg = 0;
};

// One signed-mask pass of a phase plate in the dense form: the mask is +1 on
// the levels in `pos`, -1 on those in `neg` (bit q for level q), 0 elsewhere,
// and the pass's field enters the ROI accumulator times (wr + i wi).
struct MaskPass {
  uint64_t pos = 0, neg = 0;
  double wr = 1.0, wi = 0.0;
  int cx = -1;  // membrane deformation (complex T e^{i phi}): 0 -> mask T cos(phi), 1 -> T sin(phi)
};

struct Dense {
  void* d_A = nullptr;     // kernel matrix, split-BF16, pre-swizzled tiles
  int64_t kblocks = 0;     // ceil(N / 32)
  int ntiles = 0;          // 2M / 128 row tiles of the kernel matrix
  int promote_kblocks = 0; // K blocks per TMEM accumulation chunk
  int group_kblocks = 0;   // K blocks per work-list chunk (promotions of one unit)
  int npairs = 0;          // kernel tile pairs, padded to a multiple of the cluster size
  int cluster = 1;         // CTAs per cluster sharing each mask tile
  int num_sms = 0;
  int max_ctas = 0;        // CTAs that can be resident at once (whole clusters)
  int* d_sched = nullptr;  // work list of a row-pass launch (3 nchunks + 1 ints)
  // SMs that hold no whole cluster: a concurrent single-CTA launch takes a
  // band of stripes there (single plans of cluster launches only)
  int extra_ctas = 0;
  int* d_sched2 = nullptr;
  cudaStream_t s2 = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
};

// SA-CZT (Sec. 3.6, Fig. 5): padded grid and its buffers.
struct SaCzt {
  int64_t P = 0;           // padded grid side, a power of two >= 1.5 N
  int logP = 0;
  int exact = 0;           // 1: exact zone radii of Eq. 3; 0: paraxial radii
  double zF = 0;           // distance of the Fresnel part
  double kmax = 0, d = 0;  // quadratic fit of k_z: c k_max + d K^2 / k_max, c = k0 / k_max
  void* d_G = nullptr;     // P x P complex64
  void* d_T = nullptr;     // P x P complex64 (transposed layout)
  void* d_tw = nullptr;    // P / 2 twiddles e^{-2 pi i t / P}, complex64
  void* d_K = nullptr;     // M x P complex64: Fresnel chirp and zoom kernel
  void* d_RT = nullptr;    // M x P complex64: row pass, transposed
  int64_t* d_xthr = nullptr;  // exact radii: first s of every zone m = 1 .. nx
  int64_t nx = 0;
};

struct Plan {
  // problem
  double D, f, lambda, dx, R, p, x0;
  double msh = 0;  // ROI shift in pitches: x_m = (m - msh) p (M/2 when centred)
  int64_t N, c;
  int M;
  int form, precision, stripe_rows;
  int promote_req = 0, row_batch_req = 0, cluster_req = 0;  // tuning knobs as requested (0: default)
  int conv_req = 0;  // Bluestein row convolution as requested (fzp_params.conv)
  bool owns_buffers = true;  // false: tables and workspace belong to a batch
  // derived
  double kappa, delta, dx2, R2;
  int64_t total_zones;
  int levels = 0;               // 0: binary amplitude FZP; L >= 2: L-level phase FZP
  std::vector<MaskPass> passes; // dense form, L >= 4: the signed-mask passes summing to T
  int pass_index = -1;          // pass being run (-1: the plate's single pass)
  double kappa_mask = 0;        // zone rate of the mask rule: kappa, or kappa_L = fl(kappa L/2)
  MaskGeom mg;
  int64_t* d_thr = nullptr;
  bool has_deform = false;
  fzp_deform deform{};
  // workspace shared by both forms
  float* d_C1 = nullptr;       // row intermediate [2M][chunk_rows] (FP32 forms)
  double* d_C1d = nullptr;     // row intermediate [2M][chunk_rows] (FP64 form)
  int64_t chunk_rows = 0;
  int64_t c1_rows = 0;          // rows of C1: 2M rounded up to 512
  double2* d_Uacc = nullptr;   // FP64 ROI accumulator M*M
  int* d_err = nullptr;        // device error word (bounded waits)
  double* d_metrics = nullptr; // device scratch for the metric extractor
  size_t device_bytes = 0;
  Bluestein bs;
  SaCzt sa;
  Dense dn;
  // tracing: kernel launches issued, and CUDA events around the dominant
  // kernel (recorded on the launching stream when profiling is enabled)
  int64_t launches = 0;
  bool profiling = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_events;
  size_t prof_used = 0;
  const char* dominant = "";
};

// FP32 deformation coefficients of a plan with a deformation (host).
DeformCoef deform_coef(const Plan& P);

// Bracket one launch of the dominant kernel with events (no-op unless profiling).
void prof_begin(Plan& P, cudaStream_t s);
void prof_end(Plan& P, cudaStream_t s);

// Launchers implemented in the .cu files.  All enqueue on `stream`.
// Form layouts: sizes in bytes of the form's tables and transform workspace.
struct FormSizes {
  size_t pre = 0, H = 0, tab = 0, Z = 0, G = 0;  // Bluestein
  size_t A = 0, sched = 0;                       // dense
};
fzp_status bluestein_layout(Plan& P, FormSizes* out);
fzp_status bluestein_fill_tables(Plan& P, cudaStream_t s);  // buffers already assigned
fzp_status bluestein_build_tables(Plan& P);                 // layout + allocate + fill
fzp_status bluestein_rows(Plan& P, int64_t j0, int64_t rows, cudaStream_t stream);
fzp_status dense_layout(Plan& P, FormSizes* out);
fzp_status dense_fill_tables(Plan& P, cudaStream_t s);
fzp_status dense_build_tables(Plan& P);
fzp_status dense_rows(Plan& P, int64_t j0, int64_t rows, cudaStream_t stream);
// The SA-CZT zoom on the tensor cores: kernel images of `ncols` columns with
// the chirp-kernel phase di^2 kappa / 2 - (m - msh) di delta turns (di = i - c),
// then row passes over a real FP32 matrix [rows][stride] loaded as the B operand.
fzp_status dense_zoom_build(Plan& P, int64_t ncols, int64_t c, double kappa, double delta);
fzp_status dense_zoom_rows(Plan& P, const float* src, int64_t rows, int64_t stride, cudaStream_t stream);
fzp_status column_pass(Plan& P, int64_t j0, int64_t rows, cudaStream_t stream);
bool column_pass_tc_applies(const Plan& P);
// Row pass and column pass of rows [j0, j0 + rows) (every mask pass of a dense
// phase plate), accumulated into the ROI accumulator.
fzp_status chunk_passes(Plan& P, int64_t j0, int64_t rows, cudaStream_t stream);
fzp_status column_pass_tc(Plan& P, int64_t j0, int64_t rows, cudaStream_t stream);
// The same with the pass's field weighted by (wr + i wi).
fzp_status column_pass_tc_w(Plan& P, int64_t j0, int64_t rows, double wr, double wi, cudaStream_t stream);
fzp_status epilogue(Plan& P, void* d_field, int accumulate, cudaStream_t stream);
// The epilogue with the Fresnel part's distance z in the output chirp and the
// amplitude dx^2 / (lambda z) (the phase e^{ikf} keeps the focal length).
fzp_status epilogue_z(Plan& P, void* d_field, int accumulate, double z, cudaStream_t stream);
fzp_status saczt_layout(Plan& P);                      // P, fit, z_F (host)
fzp_status saczt_build(Plan& P);                       // allocate and fill its tables
fzp_status saczt_propagate(Plan& P, int64_t j0, int64_t j1, cudaStream_t stream);  // into d_Uacc
fzp_status saczt_mask(Plan& P, int64_t j0, int64_t rows, uint8_t* out, cudaStream_t stream);
fzp_status intensity(Plan& P, const void* d_field, void* d_I, cudaStream_t stream);
fzp_status metrics(Plan& P, const void* d_field, cudaStream_t stream, fzp_metrics_t* out);
fzp_status bluestein_mask(Plan& P, int64_t j0, int64_t rows, uint8_t* out, cudaStream_t stream);
fzp_status dense_mask(Plan& P, int64_t j0, int64_t rows, uint8_t* out, cudaStream_t stream);

// Row index into the C1 layout: kernel row tile t = m / 64 holds the real parts
// of m = 64t..64t+63 in rows [0,64) and the imaginary parts in rows [64,128).
__host__ __device__ __forceinline__ int c1_row_re(int m) { return (m >> 6) * 128 + (m & 63); }
__host__ __device__ __forceinline__ int c1_row_im(int m) { return (m >> 6) * 128 + 64 + (m & 63); }

}  // namespace fzp

// The opaque handle of the C ABI is the plan itself.
struct fzp_plan_s : public fzp::Plan {};

namespace fzp {
// Host part of fzp_plan (validation, grids, zone-rule limits; no CUDA call):
// fills P and returns the disc limit s_R and the last zone step.
fzp_status plan_host(const fzp_params* params, Plan& P, int64_t* sR, int64_t* zmax);
fzp_status autotune(const fzp_params* in, fzp_params* chosen, fzp_plan_t* keep);
}
