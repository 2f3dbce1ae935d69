// plan.cu -- C ABI entry points, parameter validation, grids and the exact
// zone-threshold table (Fig. 2 Stage 1-2; Fig. 18 Stage 1-2).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "fzp_internal.cuh"

namespace fzp {

static thread_local char g_errmsg[512] = "";

fzp_status set_error(fzp_status st, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_errmsg, sizeof(g_errmsg), fmt, ap);
  va_end(ap);
  return st;
}

// fl(s * a) with s an exact integer below 2^53 (one IEEE multiply).
static inline double mul_exact_int(int64_t s, double a) {
  volatile double prod = (double)s * a;  // volatile: no contraction, no reassociation
  return prod;
}

// Largest s >= 0 with fl(s * dx2) <= R2 (aperture disc, Fig. 2 Stage 2).
static int64_t disc_limit(double dx2, double R2) {
  int64_t s = (int64_t)std::floor(R2 / dx2);
  if (s < 0) s = 0;
  while (mul_exact_int(s + 1, dx2) <= R2) ++s;
  while (s > 0 && mul_exact_int(s, dx2) > R2) --s;
  return s;
}

static inline int64_t zone_host(int64_t s, double kappa) {
  return (int64_t)std::floor(mul_exact_int(s, kappa));
}

// S_m = min{s : floor(fl(s kappa)) >= m}, m = 1..count.
static void thresholds(double kappa, int64_t count, std::vector<int64_t>& S) {
  S.resize((size_t)count);
  for (int64_t m = 1; m <= count; ++m) {
    int64_t s = (int64_t)std::ceil((double)m / kappa);
    if (s < 0) s = 0;
    while (s > 0 && zone_host(s - 1, kappa) >= m) --s;
    while (zone_host(s, kappa) < m) ++s;
    S[(size_t)(m - 1)] = s;
  }
}

void prof_begin(Plan& P, cudaStream_t s) {
  if (!P.profiling) return;
  if (P.prof_used == P.prof_events.size()) {
    cudaEvent_t a = nullptr, b = nullptr;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
      if (a) cudaEventDestroy(a);
      cudaGetLastError();
      return;
    }
    P.prof_events.emplace_back(a, b);
  }
  cudaEventRecord(P.prof_events[P.prof_used].first, s);
}

void prof_end(Plan& P, cudaStream_t s) {
  if (!P.profiling || P.prof_used >= P.prof_events.size()) return;
  cudaEventRecord(P.prof_events[P.prof_used].second, s);
  ++P.prof_used;
}

void release_plan(Plan* P) {
  if (!P) return;
  for (auto& e : P->prof_events) {
    cudaEventDestroy(e.first);
    cudaEventDestroy(e.second);
  }
  if (P->d_thr) cudaFree(P->d_thr);
  if (P->dn.d_sched2) cudaFree(P->dn.d_sched2);
  if (P->dn.ev_fork) cudaEventDestroy(P->dn.ev_fork);
  if (P->dn.ev_join) cudaEventDestroy(P->dn.ev_join);
  if (P->dn.s2) cudaStreamDestroy(P->dn.s2);
  if (P->owns_buffers) {
    void* ptrs[] = {P->d_C1, P->d_C1d, P->d_Uacc, P->d_err, P->d_metrics,
                    P->bs.d_pre, P->bs.d_H, P->bs.d_Z, P->bs.d_G, P->bs.d_tab, P->dn.d_A, P->dn.d_sched,
                    P->sa.d_G, P->sa.d_T, P->sa.d_tw, P->sa.d_K, P->sa.d_RT, P->sa.d_xthr};
    for (void* q : ptrs)
      if (q) cudaFree(q);
  }
}

static void release(fzp_plan_s* P) {
  if (!P) return;
  release_plan(P);
  delete P;
}

fzp_status validate_and_derive(const fzp_params* in, Plan& P) {
  if (!(in->D > 0) || !(in->f > 0) || !(in->lambda > 0) || !(in->pitch > 0) || !std::isfinite(in->D) ||
      !std::isfinite(in->f) || !std::isfinite(in->lambda) || !std::isfinite(in->pitch))
    return set_error(FZP_E_INVALID, "D, f, lambda and pitch must be finite and positive");
  if (in->dx < 0 || !std::isfinite(in->dx)) return set_error(FZP_E_INVALID, "dx must be >= 0");
  if (in->M < 64 || in->M > 1024 || (in->M & (in->M - 1)) != 0)
    return set_error(FZP_E_INVALID, "M must be a power of two in [64, 1024] (got %d)", in->M);
  if (in->N < 0 || (in->N > 0 && (in->N % 2) == 0))
    return set_error(FZP_E_INVALID, "N must be 0 (derive) or odd (got %lld)", (long long)in->N);
  if (in->stripe_rows < 0 || (in->stripe_rows % 256) != 0)
    return set_error(FZP_E_INVALID, "stripe_rows must be 0 or a positive multiple of 256");
  if (in->promote < 0 || in->row_batch < 0) return set_error(FZP_E_INVALID, "promote and row_batch must be >= 0");
  if (in->form < FZP_FORM_AUTO || in->form > FZP_FORM_SACZT) return set_error(FZP_E_INVALID, "unknown form");
  if (in->exact_radii != 0 && in->exact_radii != 1) return set_error(FZP_E_INVALID, "exact_radii must be 0 or 1");
  if (in->conv < 0 || in->conv > 2) return set_error(FZP_E_INVALID, "conv must be 0, 1 or 2");
  if (in->conv == 2 && in->precision == FZP_PREC_FP64)
    return set_error(FZP_E_UNSUPPORTED, "the partitioned Bluestein convolution runs in FP32 only");
  if (in->precision < FZP_PREC_FP64 || in->precision > FZP_PREC_AUTO_1E4)
    return set_error(FZP_E_INVALID, "unknown precision");
  if (in->deform && (in->deform->n_ridges < 0 || in->deform->n_ridges > 3))
    return set_error(FZP_E_INVALID, "deform.n_ridges must be in [0, 3]");
  if (in->levels < 0 || in->levels > 64) return set_error(FZP_E_INVALID, "levels must be in [0, 64]");
  if (in->centre_open != 0 && in->centre_open != 1) return set_error(FZP_E_INVALID, "centre_open must be 0 or 1");
  if (in->centre_open && in->levels >= 2)
    return set_error(FZP_E_INVALID, "centre_open applies to the binary amplitude plate (levels 0 or 1)");
  if (in->roi_origin != 0 && in->roi_origin != 1) return set_error(FZP_E_INVALID, "roi_origin must be 0 or 1");
  if (in->reserved != 0) return set_error(FZP_E_INVALID, "reserved must be 0");
  if (in->roi_origin == 1) {
    if (!std::isfinite(in->x0) || !std::isfinite(in->y0))
      return set_error(FZP_E_INVALID, "x0 and y0 must be finite");
    if (in->x0 != in->y0)
      return set_error(FZP_E_UNSUPPORTED, "off-axis ROI with x0 != y0 (one kernel matrix serves both axes)");
  }
  P.levels = in->levels >= 2 ? in->levels : 0;
  P.mg.centre_open = in->centre_open;
  const double lf = in->lambda * in->f;
  P.D = in->D; P.f = in->f; P.lambda = in->lambda; P.p = in->pitch; P.M = in->M;
  // Fig. 2 / Fig. 18 Stage 1: dx_in = Lambda_edge / (S_samp max(L, 2)), Lambda_edge =
  // lambda f / R, S_samp = 4: lambda f / (4 D) for the amplitude plate and L = 2
  P.dx = in->dx > 0 ? in->dx : lf / (2.0 * (P.levels > 2 ? P.levels : 2) * in->D);
  // Eq. 6: dx <= lambda f / (2 D)  (two samples across the outermost zone)
  if (P.dx > lf / (2.0 * in->D) * (1.0 + 1e-12))
    return set_error(FZP_E_INVALID, "dx = %g violates Eq. 6 (dx <= lambda f / (2D) = %g)", P.dx, lf / (2.0 * in->D));
  if (in->N > 0) {
    P.N = in->N;
  } else {
    const double n = std::ceil(in->D / P.dx);
    if (!(n < 1e9)) return set_error(FZP_E_INVALID, "grid too large (N = %g)", n);
    P.N = (int64_t)n;
    if ((P.N % 2) == 0) P.N += 1;  // forced odd: sample c on the axis (Fig. 2 Stage 1)
  }
  if (P.N < 3) return set_error(FZP_E_INVALID, "N must be >= 3");
  P.c = (P.N - 1) / 2;
  P.R = std::min(in->D / 2.0, lf / (2.0 * P.dx));  // R_eff (Fig. 2 Stage 2)
  // ROI grid x_m = x0 + m p = (m - msh) p on both axes (Eq. 10's A from x0):
  // centred on the focus, msh = M/2 exactly
  if (in->roi_origin == 1) {
    P.x0 = in->x0;
    P.msh = -in->x0 / P.p;
  } else {
    P.x0 = -(double)(P.M / 2) * P.p;
    P.msh = (double)(P.M / 2);
  }
  P.dx2 = P.dx * P.dx;
  P.R2 = P.R * P.R;
  P.kappa = P.dx2 / lf;
  P.kappa_mask = P.levels >= 2 ? P.kappa * (0.5 * (double)P.levels) : P.kappa;
  P.delta = P.p * P.dx / lf;  // Eq. 10: W = exp(-2 pi i dx_out dx_in / (lambda z))
  // Eq. 3 zone count: (lambda^2/4) n^2 + lambda f n - R^2 = 0
  {
    const double a = in->lambda * in->lambda / 4.0, b = lf, cc = -P.R2;
    P.total_zones = (int64_t)std::floor((-b + std::sqrt(b * b - 4 * a * cc)) / (2 * a));
  }
  // form / precision
  P.precision = in->precision;
  P.form = in->form;
  const bool dense_prec = (P.precision == FZP_PREC_SPLIT_BF16 || P.precision == FZP_PREC_BF16);
  if (P.form == FZP_FORM_AUTO) P.form = dense_prec ? FZP_FORM_DENSE : FZP_FORM_BLUESTEIN;
  if (P.form == FZP_FORM_DENSE && !dense_prec)
    return set_error(FZP_E_UNSUPPORTED, "dense form runs in split-BF16 or BF16 precision only");
  if (P.form == FZP_FORM_BLUESTEIN && dense_prec)
    return set_error(FZP_E_UNSUPPORTED, "Bluestein form runs in FP32 or FP64 precision only");
  if (P.form == FZP_FORM_SACZT) {
    if (P.precision != FZP_PREC_FP32) return set_error(FZP_E_UNSUPPORTED, "SA-CZT form runs in FP32 precision only");
    if (P.levels >= 2) return set_error(FZP_E_UNSUPPORTED, "SA-CZT form: binary amplitude plates only");
    if (in->deform) return set_error(FZP_E_UNSUPPORTED, "SA-CZT form: flat membranes only");
    if (in->stripe_rows || in->promote || in->row_batch || in->cluster)
      return set_error(FZP_E_INVALID, "SA-CZT form takes no stripe, promotion, row-batch or cluster knobs");
  }
  if (in->exact_radii && P.form != FZP_FORM_SACZT)
    return set_error(FZP_E_UNSUPPORTED, "exact zone radii (Eq. 3) are taken by the SA-CZT form only");
  P.sa.exact = in->exact_radii;
  if (P.form == FZP_FORM_DENSE && P.levels > 2) {
    // T = e^{-2 pi i q/L} = sum over passes of w (pos - neg): Re T by magnitude
    // classes cos(2 pi k/L) > 0, Im T by sin(2 pi k/L) > 0; each pass's mask
    // is -1 / 0 / +1, exact in BF16 (L/2 passes)
    if (P.levels % 2) return set_error(FZP_E_UNSUPPORTED, "dense form: phase plates need an even level count");
    const int L = P.levels;
    for (int k = 0; 4 * k < L; ++k) {
      MaskPass mp;
      mp.pos = (1ull << (k % L)) | (1ull << ((L - k) % L));
      mp.neg = (1ull << ((L / 2 - k) % L)) | (1ull << ((L / 2 + k) % L));
      mp.wr = std::cos(2.0 * M_PI * k / L);
      mp.wi = 0.0;
      P.passes.push_back(mp);
    }
    for (int k = 1; 4 * k <= L; ++k) {
      MaskPass mp;
      mp.neg = (1ull << (k % L)) | (1ull << ((L / 2 - k) % L));
      mp.pos = (1ull << ((L / 2 + k) % L)) | (1ull << ((L - k) % L));
      mp.wr = 0.0;
      mp.wi = std::sin(2.0 * M_PI * k / L);
      P.passes.push_back(mp);
    }
  }
  if (P.form == FZP_FORM_DENSE && P.mg.centre_open) {
    // positive-centred binary plate: one pass of the generator's level mode,
    // +1 where the zone index is even (level 0 of 2) inside the disc
    MaskPass mp;
    mp.pos = 1ull;
    P.passes.push_back(mp);
  }
  if (in->deform) {
    const fzp_deform& d = *in->deform;
    bool ok = d.period > 0 && std::isfinite(d.period) && std::isfinite(d.amp) && std::isfinite(d.theta) &&
              std::isfinite(d.taper);
    for (int k = 0; k < d.n_ridges; ++k)
      ok = ok && d.ridge_width[k] > 0 && std::isfinite(d.ridge_width[k]) && std::isfinite(d.ridge_h[k]) &&
           std::isfinite(d.ridge_px[k]) && std::isfinite(d.ridge_py[k]) && std::isfinite(d.ridge_alpha[k]);
    if (!ok) return set_error(FZP_E_INVALID, "deformation: period and ridge widths must be positive, all finite");
    if (P.form == FZP_FORM_DENSE && P.levels >= 2)
      return set_error(FZP_E_UNSUPPORTED, "dense form: a deformed membrane must be a binary amplitude plate");
    P.has_deform = true;
    P.deform = d;
    if (P.form == FZP_FORM_DENSE) {
      // complex transmission T e^{i phi}: the real masks T cos(phi) and T sin(phi)
      // in two passes, their fields weighted 1 and i (the centre configuration
      // is applied by the membrane generator itself)
      P.passes.clear();
      MaskPass re, im;
      re.cx = 0;
      im.cx = 1;
      im.wr = 0.0;
      im.wi = 1.0;
      P.passes.push_back(re);
      P.passes.push_back(im);
    }
  }
  P.stripe_rows = in->stripe_rows;
  P.promote_req = in->promote;
  P.row_batch_req = in->row_batch;
  P.conv_req = in->conv;
  if (in->cluster != 0 && in->cluster != 1 && in->cluster != 2 && in->cluster != 4)
    return set_error(FZP_E_INVALID, "cluster must be 0, 1, 2 or 4");
  P.cluster_req = in->cluster;
  return FZP_OK;
}

fzp_status build_mask_tables(Plan& P) {
  P.mg.c = P.c;
  P.mg.sR = disc_limit(P.dx2, P.R2);
  P.mg.levels = P.levels;
  const int64_t zmax = zone_host(P.mg.sR, P.kappa_mask);
  // zone_of() error analysis needs s_R < 2^46 and zone < 2^24.
  if (P.mg.sR >= (1ll << 46) || zmax + 1 >= (1ll << 24))
    return set_error(FZP_E_UNSUPPORTED, "aperture too large for the exact zone rule (s_R=%lld, zones=%lld)",
                     (long long)P.mg.sR, (long long)zmax);
  const double k64 = std::ldexp(P.kappa_mask, 64);
  if (!(k64 < 18446744073709551616.0)) return set_error(FZP_E_INVALID, "kappa >= 1: grid far too coarse");
  P.mg.K64 = (uint64_t)std::floor(k64);
  std::vector<int64_t> S;
  thresholds(P.kappa_mask, zmax + 2, S);
  P.mg.nthr = (int64_t)S.size();
  FZP_CUDA_TRY(cudaMalloc(&P.d_thr, S.size() * sizeof(int64_t)));
  P.device_bytes += S.size() * sizeof(int64_t);
  FZP_CUDA_TRY(cudaMemcpy(P.d_thr, S.data(), S.size() * sizeof(int64_t), cudaMemcpyHostToDevice));
  P.mg.thr = P.d_thr;
  return FZP_OK;
}

fzp_status chunk_passes(Plan& P, int64_t j0, int64_t rows, cudaStream_t s) {
  const int np = (P.form == FZP_FORM_DENSE && !P.passes.empty()) ? (int)P.passes.size() : 1;
  fzp_status st = FZP_OK;
  for (int k = 0; k < np && st == FZP_OK; ++k) {
    P.pass_index = np > 1 || !P.passes.empty() ? k : -1;
    st = (P.form == FZP_FORM_DENSE) ? dense_rows(P, j0, rows, s) : bluestein_rows(P, j0, rows, s);
    if (st == FZP_OK)
      st = column_pass_tc_applies(P) ? column_pass_tc(P, j0, rows, s) : column_pass(P, j0, rows, s);
  }
  P.pass_index = -1;
  return st;
}

// cudaMalloc of a plan's row intermediate.  Host-side fault injection for
// tests: with the environment variable FZP_FAULT_ALLOC_LIMIT set to a byte
// count, larger requests fail as out of memory without reaching the device.
cudaError_t workspace_malloc(void** p, size_t bytes) {
  const char* lim = std::getenv("FZP_FAULT_ALLOC_LIMIT");
  if (lim && *lim && bytes > (size_t)std::strtoull(lim, nullptr, 10)) return cudaErrorMemoryAllocation;
  return cudaMalloc(p, bytes);
}

// Rows per row-pass chunk: requested (multiple of 256), else as many as an
// 8 GiB row intermediate holds; never more than the grid (rounded to 256).
// SA-CZT plans: the padded grid's side (rounded to 256).
int64_t chunk_rows_for(const Plan& P) {
  if (P.form == FZP_FORM_SACZT) {
    // the zoom's row pass covers the padded grid's P rows in one chunk
    int64_t n = 64;
    while ((double)n < 1.5 * (double)P.N) n <<= 1;
    return (n + 255) / 256 * 256;
  }
  const int64_t M2 = (2 * (int64_t)P.M + 511) / 512 * 512;
  const int64_t budget_rows = (int64_t)((8ull << 30) / (uint64_t)(M2 * (P.precision == FZP_PREC_FP64 ? 8 : 4)));
  int64_t rows = P.stripe_rows > 0 ? (int64_t)P.stripe_rows : budget_rows;
  rows = std::min<int64_t>(rows, P.N);
  return (rows + 255) / 256 * 256;
}

// Rows of [0, N) that intersect the aperture disc: dj^2 <= s_R.
void disc_rows(const Plan& P, int64_t& jlo, int64_t& jhi) {
  int64_t b = (int64_t)std::floor(std::sqrt((double)P.mg.sR));
  while ((b + 1) * (b + 1) <= P.mg.sR) ++b;
  while (b * b > P.mg.sR) --b;
  jlo = P.c - b;
  jhi = P.c + b + 1;
  if (jlo < 0) jlo = 0;
  if (jhi > P.N) jhi = P.N;
}

}  // namespace fzp

using namespace fzp;

extern "C" {

const char* fzp_last_error(void) { return g_errmsg; }

const char* fzp_version(void) { return "libfzp 0.1 (sm_103a)"; }

fzp_status fzp_plan(const fzp_params* params, fzp_plan_t* out) {
  if (!out) return set_error(FZP_E_INVALID, "out is NULL");
  *out = nullptr;
  if (!params) return set_error(FZP_E_INVALID, "params is NULL");
  if (params->precision == FZP_PREC_AUTO_1E4) {
    fzp_params chosen;
    return autotune(params, &chosen, out);
  }
  fzp_plan_s* P = new (std::nothrow) fzp_plan_s();
  if (!P) return set_error(FZP_E_OOM, "host allocation failed");
  fzp_status st = validate_and_derive(params, *P);
  if (st != FZP_OK) { release(P); return st; }
  g_errmsg[0] = 0;
  st = build_mask_tables(*P);
  if (st == FZP_OK) {
    // rows of C1: 2M kernel rows, rounded up to whole couples of 2 x 128-row tile pairs (dense form)
    const int64_t M2 = (2 * (int64_t)P->M + 511) / 512 * 512;
    P->chunk_rows = chunk_rows_for(*P);
    P->c1_rows = M2;
    // The row intermediate of one chunk.  When it cannot be allocated the
    // chunk is halved (down to 256 rows) and the allocation retried, as the
    // paper's engine halves its row batch on a GPU out-of-memory error
    // (Fig. 18 Stage 2); only then is FZP_E_OOM returned.
    const size_t esz = P->precision == FZP_PREC_FP64 ? sizeof(double) : sizeof(float);
    cudaError_t e = cudaSuccess;
    while (true) {
      const size_t bytes = (size_t)(M2 * P->chunk_rows) * esz;
      void* c1 = nullptr;
      e = workspace_malloc(&c1, bytes);
      if (e == cudaSuccess) {
        if (P->precision == FZP_PREC_FP64) P->d_C1d = static_cast<double*>(c1);
        else P->d_C1 = static_cast<float*>(c1);
        P->device_bytes += bytes;
        break;
      }
      if (e != cudaErrorMemoryAllocation || P->chunk_rows <= 256) break;
      cudaGetLastError();
      P->chunk_rows = std::max<int64_t>(256, (P->chunk_rows / 2 + 255) / 256 * 256);
    }
    if (e == cudaSuccess) e = cudaMalloc(&P->d_Uacc, (size_t)P->M * P->M * sizeof(double2));
    if (e == cudaSuccess) e = cudaMalloc(&P->d_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&P->d_metrics, 8192 * sizeof(double) + (size_t)P->M * P->M * sizeof(double2));
    if (e == cudaSuccess) e = cudaMemset(P->d_err, 0, sizeof(int));
    P->device_bytes += (size_t)P->M * P->M * sizeof(double2) * 2 + 8192 * sizeof(double) + sizeof(int);
    if (e != cudaSuccess) {
      st = set_error(e == cudaErrorMemoryAllocation ? FZP_E_OOM : FZP_E_CUDA, "workspace allocation: %s",
                     cudaGetErrorString(e));
      cudaGetLastError();
    }
  }
  if (st == FZP_OK)
    st = P->form == FZP_FORM_DENSE ? dense_build_tables(*P)
         : P->form == FZP_FORM_SACZT ? saczt_build(*P)
                                     : bluestein_build_tables(*P);
  if (st == FZP_OK) {
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) st = set_error(FZP_E_CUDA, "plan build: %s", cudaGetErrorString(e));
  }
  if (st != FZP_OK) {
    cudaGetLastError();
    release(P);
    return st;
  }
  *out = P;
  return FZP_OK;
}

}  // extern "C"

// Host part of a plan: validation, grids and the zone-rule limits, without
// any CUDA call.  Returns the disc limit and the last zone step through *sR
// and *zmax.
fzp_status fzp::plan_host(const fzp_params* params, Plan& P, int64_t* sR, int64_t* zmax) {
  fzp_status st = validate_and_derive(params, P);
  if (st != FZP_OK) return st;
  *sR = disc_limit(P.dx2, P.R2);
  *zmax = zone_host(*sR, P.kappa_mask);
  if (*sR >= (1ll << 46) || *zmax + 1 >= (1ll << 24))
    return set_error(FZP_E_UNSUPPORTED, "aperture too large for the exact zone rule (s_R=%lld, zones=%lld)",
                     (long long)*sR, (long long)*zmax);
  if (!(std::ldexp(P.kappa_mask, 64) < 18446744073709551616.0))
    return set_error(FZP_E_INVALID, "kappa >= 1: grid far too coarse");
  return FZP_OK;
}

extern "C" {

fzp_status fzp_plan_query(const fzp_params* params, fzp_plan_info* out) {
  if (!params || !out) return set_error(FZP_E_INVALID, "NULL argument");
  Plan P;
  int64_t sR = 0, zmax = 0;
  const fzp_status st = plan_host(params, P, &sR, &zmax);
  if (st != FZP_OK) return st;
  *out = fzp_plan_info{};
  out->N = P.N; out->c = P.c; out->total_zones = P.total_zones; out->n_thresholds = zmax + 2;
  out->dx = P.dx; out->R = P.R; out->kappa = P.kappa; out->x0 = P.x0;
  out->M = P.M;
  const bool tuned = params->precision == FZP_PREC_AUTO_1E4;  // form chosen by measurement
  out->form = tuned ? FZP_FORM_AUTO : P.form;
  out->precision = P.precision;
  out->stripe_rows = P.stripe_rows;
  out->chunk_rows = chunk_rows_for(P);
  if (!tuned && P.form == FZP_FORM_BLUESTEIN) {
    int64_t L = 1;
    while (L < P.N + P.M - 1) L <<= 1;
    // the four-step split L = L1 L2 with L1 <= L2 <= 4096 (bluestein.cu)
    if (L > (1ll << 24)) return set_error(FZP_E_UNSUPPORTED, "FFT length %lld above %lld", (long long)L, 1ll << 24);
    out->fft_length = L;
    out->conv = (P.precision == FZP_PREC_FP32 && P.conv_req != 1) ? 2 : 1;
    out->fft_inner = out->conv == 2 ? 4096 : (int32_t)std::min<int64_t>(L, 4096);
  }
  if (!tuned && P.form == FZP_FORM_SACZT) {
    const fzp_status sst = saczt_layout(P);  // host only
    if (sst != FZP_OK) return sst;
    out->fft_length = P.sa.P;
  }
  out->promote = !tuned && P.form == FZP_FORM_DENSE ? (P.promote_req > 0 ? P.promote_req : 128) : 0;
  out->cluster = !tuned && P.form == FZP_FORM_DENSE ? P.cluster_req : 0;
  out->levels = P.levels;
  out->passes = P.passes.empty() ? 1 : (int32_t)P.passes.size();
  out->centre_open = P.mg.centre_open;
  out->s_R = sR;
  return FZP_OK;
}

fzp_status fzp_zone_thresholds(const fzp_params* params, int64_t* out, int64_t capacity, int64_t* count) {
  if (!params || !count) return set_error(FZP_E_INVALID, "NULL argument");
  if (capacity < 0 || (capacity > 0 && !out)) return set_error(FZP_E_INVALID, "bad output buffer");
  Plan P;
  int64_t sR = 0, zmax = 0;
  const fzp_status st = plan_host(params, P, &sR, &zmax);
  if (st != FZP_OK) return st;
  std::vector<int64_t> S;
  thresholds(P.kappa_mask, zmax + 2, S);
  *count = (int64_t)S.size();
  const int64_t n = std::min<int64_t>(capacity, *count);
  for (int64_t k = 0; k < n; ++k) out[k] = S[(size_t)k];
  return FZP_OK;
}

fzp_status fzp_plan_info_get(fzp_plan_t plan, fzp_plan_info* out) {
  if (!plan || !out) return set_error(FZP_E_INVALID, "NULL argument");
  const Plan& P = *plan;
  out->N = P.N; out->c = P.c; out->total_zones = P.total_zones; out->n_thresholds = P.mg.nthr;
  out->dx = P.dx; out->R = P.R; out->kappa = P.kappa; out->x0 = P.x0;
  out->M = P.M; out->form = P.form; out->precision = P.precision;
  out->stripe_rows = P.stripe_rows;
  out->fft_length = P.form == FZP_FORM_SACZT ? P.sa.P : P.bs.L;
  out->promote = P.form == FZP_FORM_DENSE ? P.dn.promote_kblocks : 0;
  out->row_batch = P.form == FZP_FORM_BLUESTEIN ? (int32_t)P.bs.rows : 0;
  out->chunk_rows = P.chunk_rows;
  out->cluster = P.form == FZP_FORM_DENSE ? P.dn.cluster : 0;
  out->fft_inner = P.form == FZP_FORM_BLUESTEIN ? (P.bs.seg ? 4096 : (int32_t)P.bs.L2) : 0;
  out->conv = P.form == FZP_FORM_BLUESTEIN ? (P.bs.seg ? 2 : 1) : 0;
  out->ctas = P.form == FZP_FORM_DENSE ? P.dn.max_ctas : 0;
  out->levels = P.levels;
  out->passes = P.passes.empty() ? 1 : (int32_t)P.passes.size();
  out->centre_open = P.mg.centre_open;
  out->s_R = P.mg.sR;
  out->device_bytes = P.device_bytes;
  return FZP_OK;
}

fzp_status fzp_plan_destroy(fzp_plan_t plan) {
  if (!plan) return FZP_OK;
  cudaDeviceSynchronize();
  release(plan);
  return FZP_OK;
}

fzp_status fzp_propagate_roi(fzp_plan_t plan, int64_t row_begin, int64_t row_end, void* d_field, int accumulate,
                             void* stream) {
  if (!plan || !d_field) return set_error(FZP_E_INVALID, "NULL plan or field");
  Plan& P = *plan;
  if (row_begin < 0 || row_end > P.N || row_begin > row_end)
    return set_error(FZP_E_INVALID, "row range [%lld, %lld) outside [0, %lld]", (long long)row_begin,
                     (long long)row_end, (long long)P.N);
  cudaStream_t s = (cudaStream_t)stream;
  FZP_CUDA_TRY(cudaMemsetAsync(P.d_Uacc, 0, (size_t)P.M * P.M * sizeof(double2), s));
  int64_t jlo, jhi;
  disc_rows(P, jlo, jhi);
  const int64_t a = std::max(row_begin, jlo), b = std::min(row_end, jhi);
  if (P.form == FZP_FORM_SACZT) {
    // the whole padded plane at once (rows outside the range masked to zero)
    if (a < b) {
      const fzp_status st = saczt_propagate(P, a, b, s);
      if (st != FZP_OK) return st;
    }
    return epilogue_z(P, d_field, accumulate, P.sa.zF, s);
  }
  for (int64_t j0 = a; j0 < b; j0 += P.chunk_rows) {
    const fzp_status st = chunk_passes(P, j0, std::min(P.chunk_rows, b - j0), s);
    if (st != FZP_OK) return st;
  }
  return epilogue(P, d_field, accumulate, s);
}

fzp_status fzp_aperture_mask(fzp_plan_t plan, int64_t row_begin, int64_t row_end, void* d_mask, void* stream) {
  if (!plan || !d_mask) return set_error(FZP_E_INVALID, "NULL plan or mask");
  Plan& P = *plan;
  if (row_begin < 0 || row_end > P.N || row_begin > row_end)
    return set_error(FZP_E_INVALID, "row range [%lld, %lld) outside [0, %lld]", (long long)row_begin,
                     (long long)row_end, (long long)P.N);
  if (row_end == row_begin) return FZP_OK;
  uint8_t* out = reinterpret_cast<uint8_t*>(d_mask);
  // each form exports through the generator its row pass runs (the dense
  // form: walker, block-wise generator or level mode, as the plan launches it)
  return P.form == FZP_FORM_DENSE   ? dense_mask(P, row_begin, row_end - row_begin, out, (cudaStream_t)stream)
         : P.form == FZP_FORM_SACZT ? saczt_mask(P, row_begin, row_end - row_begin, out, (cudaStream_t)stream)
                                    : bluestein_mask(P, row_begin, row_end - row_begin, out, (cudaStream_t)stream);
}

fzp_status fzp_profile_enable(fzp_plan_t plan, int enable) {
  if (!plan) return set_error(FZP_E_INVALID, "NULL plan");
  plan->profiling = enable != 0;
  return FZP_OK;
}

fzp_status fzp_profile_read(fzp_plan_t plan, fzp_profile_t* out) {
  if (!plan || !out) return set_error(FZP_E_INVALID, "NULL argument");
  double total = 0;
  for (size_t i = 0; i < plan->prof_used; ++i) {
    FZP_CUDA_TRY(cudaEventSynchronize(plan->prof_events[i].second));
    float ms = 0;
    FZP_CUDA_TRY(cudaEventElapsedTime(&ms, plan->prof_events[i].first, plan->prof_events[i].second));
    total += ms;
  }
  out->dominant_ms = total;
  out->dominant_launches = (int64_t)plan->prof_used;
  out->kernel_launches = plan->launches;
  snprintf(out->dominant_name, sizeof(out->dominant_name), "%s", plan->dominant);
  plan->prof_used = 0;
  plan->launches = 0;
  return FZP_OK;
}

fzp_status fzp_intensity(fzp_plan_t plan, const void* d_field, void* d_intensity, void* stream) {
  if (!plan || !d_field || !d_intensity) return set_error(FZP_E_INVALID, "NULL argument");
  return intensity(*plan, d_field, d_intensity, (cudaStream_t)stream);
}

fzp_status fzp_metrics(fzp_plan_t plan, const void* d_field, void* stream, fzp_metrics_t* out) {
  if (!plan || !d_field || !out) return set_error(FZP_E_INVALID, "NULL argument");
  return metrics(*plan, d_field, (cudaStream_t)stream, out);
}

}  // extern "C"
