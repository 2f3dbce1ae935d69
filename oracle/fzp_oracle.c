/*
 * fzp_oracle.c -- CPU FP64 oracle for the Fresnel zone plate (FZP) propagator.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark do.  It shares no code with the CUDA path.
 *
 * Everything here is a plain, slow, obviously-correct statement of what the
 * paper computes, in IEEE double precision:
 *
 *   Eq. 1  U(x,y) = e^{ikz}/(i lambda z) * sum U0(u,v) e^{ik[(x-u)^2+(y-v)^2]/2z} du dv
 *   Eq. 2  the same integral with the quadratic phase expanded into an input
 *          chirp, a Fourier kernel and an output chirp (the target of every
 *          propagator in the paper); z = f (focal plane).
 *   Eq. 9  X[m] = sum_n x[n] A^{-n} W^{mn}              (chirp-z transform)
 *   Eq. 10 W = exp(-2 pi i dx_out dx_in / (lambda z)), A = exp(2 pi i x0 dx_in / (lambda z))
 *   Sec. 2.6  Bluestein's identity mn = [n^2 + m^2 - (m-n)^2]/2 turns Eq. 9
 *          into chirp * linear convolution (by FFT) * chirp; the 2-D kernel is
 *          separable, so a row pass is followed by a column pass (Fig. 2,
 *          "Separable batched execution").
 *   Fig. 2 Stage 2: binary amplitude mask, paraxial radii r_m^2 = m lambda f
 *          (Eq. 4), a pixel is open where its zone index is odd, the centre
 *          zone (index 0) is opaque ("negative-centred", Sec. 4.1); the
 *          aperture is limited to R_eff = min(D/2, lambda f / (2 dx_in)).
 *          The positive-centred plate (centre zone open) is the second
 *          centre configuration the Fig. 18 engine offers.
 *
 * Three independent evaluations of the focal-plane field are provided:
 *   O1  orc_field_direct    : Eq. 1 summed literally over every aperture
 *                             sample and every ROI sample (tiny inputs).
 *   O2  orc_field_separable : Eq. 2 as two dense matrix products,
 *                             U = Pre * chirp_out * (K T K^T).
 *   O3  orc_field_czt       : the paper's method -- row CZT by Bluestein with
 *                             an FFT written here, then column CZT (Fig. 2).
 * They must agree to rounding; the test-suite checks that.
 *
 * Readings of the paper taken here (each is listed in the design notes):
 *   - mask rule: s = (i-c)^2 + (j-c)^2 is an exact integer; a pixel is open iff
 *     fl(s*dx^2) <= fl(R^2) and floor(fl(s*kappa)) is odd, with
 *     kappa = fl(fl(dx*dx) / fl(lambda*f)), i.e. floor(r^2/(lambda f)) odd.
 *   - grid: pixel c = (N-1)/2 lies on the optical axis (N odd), u_i = (i-c) dx.
 *   - ROI: x_m = x0 + m p, same grid on both axes.
 *   - field layout: out[n*M + m] is the sample at (x_m, y_n).
 *
 * Build: gcc -O2 -fopenmp -fPIC -shared -o liboracle.so fzp_oracle.c -lm
 * (no -ffast-math: the mask rule depends on IEEE rounding of one multiply).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

typedef double complex cplx;

/* Aperture kinds. */
enum {
  ORC_FZP_PARAXIAL = 0, /* binary amplitude FZP, paraxial radii (Eq. 4, Fig. 2) */
  ORC_LENS = 1,         /* ideal thin lens: circ(r<=R) * exp(-i pi r^2/(lambda f)) */
  ORC_FZP_EXACT = 2,    /* binary amplitude FZP, exact radii (Eq. 3)             */
  ORC_CIRC = 3,         /* clear circular pupil (no focusing phase)              */
  ORC_FZP_PHASE = 4,    /* L-level phase FZP (Fig. 18 Stage 3), levels = L >= 2  */
  ORC_FZP_POSITIVE = 5  /* binary amplitude FZP, paraxial radii, centre zone open */
};

/* Deformation of the membrane, w(u,v) in metres; phase phi = (4 pi/lambda) w.
 *   w = amp * sin(2 pi (u cos th + v sin th)/period) * (1 - taper (r/R)^2)
 *     + sum_k h_k exp(-d_k^2 / (2 sigma_k^2)),
 *   d_k = distance of (u,v) to the straight crease line through (px_k,py_k)
 *         at angle alpha_k, sigma_k = width_k / (2 sqrt(2 ln 2)).          */
typedef struct {
  double amp, period, theta, taper;
  int32_t n_ridges;
  int32_t pad_;
  double ridge_px[3], ridge_py[3], ridge_alpha[3], ridge_h[3], ridge_width[3];
} orc_deform;

typedef struct {
  int64_t N;        /* samples per side of the aperture grid (odd)          */
  double dx;        /* aperture pitch dx_in [m]                              */
  double lambda;    /* wavelength [m]                                        */
  double f;         /* focal length = propagation distance z [m]             */
  double R;         /* aperture radius R_eff [m]                             */
  int32_t M;        /* ROI samples per side                                  */
  int32_t kind;     /* ORC_* aperture kind                                   */
  double p;         /* ROI pitch dx_out [m]                                  */
  double x0;        /* first ROI coordinate (both axes) [m]                  */
  const orc_deform* deform; /* NULL: flat membrane                           */
  int32_t levels;   /* ORC_FZP_PHASE: phase levels L per 2 pi (>= 2)         */
  int32_t pad2_;
} orc_params;

/* ------------------------------------------------------------------ */
/* Aperture                                                            */
/* ------------------------------------------------------------------ */

static double orc_kappa(const orc_params* P) {
  double dx2 = P->dx * P->dx;
  double lf = P->lambda * P->f;
  return dx2 / lf;
}

/* Binary transmission of pixel (j,i) for the two FZP kinds, the clear pupil
 * and the lens support. */
static int orc_open(const orc_params* P, int64_t j, int64_t i) {
  const int64_t c = (P->N - 1) / 2;
  const int64_t di = i - c, dj = j - c;
  const int64_t s = di * di + dj * dj; /* exact */
  const double dx2 = P->dx * P->dx;
  const double R2 = P->R * P->R;
  if ((double)s * dx2 > R2) return 0;
  if (P->kind == ORC_FZP_PARAXIAL) {
    const double zone = floor((double)s * orc_kappa(P));
    return ((int64_t)zone & 1) ? 1 : 0;
  }
  if (P->kind == ORC_FZP_POSITIVE) {
    /* the other centre configuration of the v8 engine (Fig. 18): the even
     * zones, the centre zone among them, are the open ones */
    const double zone = floor((double)s * orc_kappa(P));
    return ((int64_t)zone & 1) ? 0 : 1;
  }
  if (P->kind == ORC_FZP_EXACT) {
    /* Eq. 3: r^2 = n lambda f + n^2 lambda^2/4  =>  n(r) = 2 (sqrt(f^2 + r^2) - f) / lambda */
    const double r2 = (double)s * dx2;
    const double n = 2.0 * (sqrt(P->f * P->f + r2) - P->f) / P->lambda;
    return ((int64_t)floor(n) & 1) ? 1 : 0;
  }
  return 1; /* lens / clear pupil / phase FZP: full disc */
}

/* Level index of an L-level phase FZP (Fig. 18 Stage 3: z = r^2/(lambda f),
 * L-level phase).  The lens phase -pi z wrapped to [0, 2 pi) and quantised to
 * L steps: q = floor(L frac(z / 2)) = floor(s kappa_L) mod L with
 * kappa_L = fl(kappa * (L/2)), so that for L = 2 the steps are the zones of the
 * amplitude rule.  Transmission e^{-2 pi i q / L}. */
static int64_t orc_level(const orc_params* P, int64_t j, int64_t i) {
  const int64_t c = (P->N - 1) / 2;
  const int64_t di = i - c, dj = j - c;
  const int64_t s = di * di + dj * dj;
  const double kL = orc_kappa(P) * (0.5 * (double)P->levels);
  const int64_t step = (int64_t)floor((double)s * kL);
  return step % P->levels;
}

static double orc_deform_w(const orc_deform* d, double u, double v, double R) {
  double r2 = (u * u + v * v) / (R * R);
  double w = d->amp * sin(2.0 * M_PI * (u * cos(d->theta) + v * sin(d->theta)) / d->period) *
             (1.0 - d->taper * r2);
  for (int k = 0; k < d->n_ridges && k < 3; ++k) {
    double nx = -sin(d->ridge_alpha[k]), ny = cos(d->ridge_alpha[k]);
    double dist = (u - d->ridge_px[k]) * nx + (v - d->ridge_py[k]) * ny;
    double sigma = d->ridge_width[k] / (2.0 * sqrt(2.0 * log(2.0)));
    w += d->ridge_h[k] * exp(-dist * dist / (2.0 * sigma * sigma));
  }
  return w;
}

/* Complex aperture field U0[j,i] (unit incident amplitude). */
static cplx orc_u0(const orc_params* P, int64_t j, int64_t i) {
  if (!orc_open(P, j, i)) return 0.0;
  const int64_t c = (P->N - 1) / 2;
  const double u = (double)(i - c) * P->dx, v = (double)(j - c) * P->dx;
  cplx a = 1.0;
  if (P->kind == ORC_LENS) a = cexp(-I * M_PI * (u * u + v * v) / (P->lambda * P->f));
  if (P->kind == ORC_FZP_PHASE) a = cexp(-I * 2.0 * M_PI * (double)orc_level(P, j, i) / (double)P->levels);
  if (P->deform) a *= cexp(I * (4.0 * M_PI / P->lambda) * orc_deform_w(P->deform, u, v, P->R));
  return a;
}

int orc_mask_rows(const orc_params* P, int64_t j0, int64_t j1, uint8_t* out) {
  if (!P || !out || j0 < 0 || j1 > P->N || j0 > j1) return 1;
  for (int64_t j = j0; j < j1; ++j)
    for (int64_t i = 0; i < P->N; ++i) {
      const int open = orc_open(P, j, i);
      /* phase FZP: 1 + level inside the aperture, 0 outside */
      out[(j - j0) * P->N + i] =
          (uint8_t)(P->kind == ORC_FZP_PHASE ? (open ? 1 + orc_level(P, j, i) : 0) : open);
    }
  return 0;
}

int orc_aperture_rows(const orc_params* P, int64_t j0, int64_t j1, double* re, double* im) {
  if (!P || !re || !im || j0 < 0 || j1 > P->N || j0 > j1) return 1;
  for (int64_t j = j0; j < j1; ++j)
    for (int64_t i = 0; i < P->N; ++i) {
      cplx a = orc_u0(P, j, i);
      re[(j - j0) * P->N + i] = creal(a);
      im[(j - j0) * P->N + i] = cimag(a);
    }
  return 0;
}

/* Number of pixels inside the aperture disc, fl(s dx^2) <= fl(R^2), counted by
 * bisection on each row (the predicate is monotone in |i - c|). */
int64_t orc_count_aperture(const orc_params* P) {
  const int64_t N = P->N, c = (N - 1) / 2;
  const double dx2 = P->dx * P->dx, R2 = P->R * P->R;
  int64_t total = 0;
  for (int64_t j = 0; j < N; ++j) {
    const int64_t dj = j - c;
    if ((double)(dj * dj) * dx2 > R2) continue;
    int64_t lo = 0, hi = c; /* largest d in [0,c] with (dj^2 + d^2) dx2 <= R2 */
    while (lo < hi) {
      int64_t mid = lo + (hi - lo + 1) / 2;
      if ((double)(dj * dj + mid * mid) * dx2 <= R2) lo = mid; else hi = mid - 1;
    }
    total += 2 * lo + 1;
  }
  return total;
}

/* ------------------------------------------------------------------ */
/* FFT: iterative radix-2 Cooley-Tukey, in place, power-of-two length.   */
/* Forward: X[k] = sum x[n] e^{-2 pi i nk/L}; inverse without 1/L.        */
/* ------------------------------------------------------------------ */

static int orc_fft_inplace(int64_t L, cplx* x, int inverse) {
  if (L < 1 || (L & (L - 1))) return 1;
  for (int64_t i = 1, j = 0; i < L; ++i) { /* bit reversal */
    int64_t bit = L >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) { cplx t = x[i]; x[i] = x[j]; x[j] = t; }
  }
  const double sgn = inverse ? 1.0 : -1.0;
  for (int64_t len = 2; len <= L; len <<= 1) {
    const int64_t half = len >> 1;
    for (int64_t k = 0; k < half; ++k) {
      const double ang = sgn * 2.0 * M_PI * (double)k / (double)len;
      const cplx w = cos(ang) + I * sin(ang);
      for (int64_t s = 0; s < L; s += len) {
        cplx a = x[s + k], b = x[s + k + half] * w;
        x[s + k] = a + b;
        x[s + k + half] = a - b;
      }
    }
  }
  return 0;
}

int orc_fft(int64_t L, double* re, double* im, int inverse) {
  cplx* x = (cplx*)malloc(sizeof(cplx) * (size_t)L);
  if (!x) return 2;
  for (int64_t i = 0; i < L; ++i) x[i] = re[i] + I * im[i];
  int rc = orc_fft_inplace(L, x, inverse);
  for (int64_t i = 0; i < L; ++i) { re[i] = creal(x[i]); im[i] = cimag(x[i]); }
  free(x);
  return rc;
}

/* ------------------------------------------------------------------ */
/* Chirp-z transform (Eq. 9) with A = e^{2 pi i alpha}, W = e^{-2 pi i omega}:
 *   X[m] = sum_n x[n] e^{-2 pi i (alpha n + omega m n)},  m = 0..M-1.       */
/* ------------------------------------------------------------------ */

int orc_czt_direct(int64_t N, const double* xr, const double* xi, int64_t M, double alpha,
                   double omega, double* Xr, double* Xi) {
  for (int64_t m = 0; m < M; ++m) {
    cplx acc = 0.0;
    for (int64_t n = 0; n < N; ++n)
      acc += (xr[n] + I * xi[n]) * cexp(-2.0 * M_PI * I * (alpha * (double)n + omega * (double)m * (double)n));
    Xr[m] = creal(acc);
    Xi[m] = cimag(acc);
  }
  return 0;
}

/* Bluestein workspace for one transform size. */
typedef struct {
  int64_t N, M, L;
  double alpha, omega;
  cplx* Vf;   /* FFT of the convolution chirp v[k] = W^{-k^2/2}, k in (-N, M) */
  cplx* pre;  /* A^{-n} W^{n^2/2}, n < N */
  cplx* post; /* W^{m^2/2} / L, m < M   */
} orc_bluestein;

static int64_t orc_next_pow2(int64_t v) { int64_t L = 1; while (L < v) L <<= 1; return L; }

static void orc_bluestein_free(orc_bluestein* b) { free(b->Vf); free(b->pre); free(b->post); }

static int orc_bluestein_init(orc_bluestein* b, int64_t N, int64_t M, double alpha, double omega) {
  b->N = N; b->M = M; b->alpha = alpha; b->omega = omega;
  b->L = orc_next_pow2(N + M - 1);
  b->Vf = (cplx*)calloc((size_t)b->L, sizeof(cplx));
  b->pre = (cplx*)malloc(sizeof(cplx) * (size_t)N);
  b->post = (cplx*)malloc(sizeof(cplx) * (size_t)M);
  if (!b->Vf || !b->pre || !b->post) { orc_bluestein_free(b); return 2; }
  /* W^{t^2/2} = e^{-i pi omega t^2}; t^2 is exact in double for t < 2^26. */
  for (int64_t k = 0; k < M; ++k) b->Vf[k] = cexp(I * M_PI * omega * (double)k * (double)k);
  for (int64_t k = 1; k < N; ++k) b->Vf[b->L - k] = cexp(I * M_PI * omega * (double)k * (double)k);
  orc_fft_inplace(b->L, b->Vf, 0);
  for (int64_t n = 0; n < N; ++n)
    b->pre[n] = cexp(-2.0 * M_PI * I * alpha * (double)n) * cexp(-I * M_PI * omega * (double)n * (double)n);
  for (int64_t m = 0; m < M; ++m)
    b->post[m] = cexp(-I * M_PI * omega * (double)m * (double)m) / (double)b->L;
  return 0;
}

/* X = CZT(x) through Bluestein; work has room for L values. */
static void orc_bluestein_apply(const orc_bluestein* b, const cplx* x, cplx* X, cplx* work) {
  for (int64_t n = 0; n < b->N; ++n) work[n] = x[n] * b->pre[n];
  for (int64_t n = b->N; n < b->L; ++n) work[n] = 0.0;
  orc_fft_inplace(b->L, work, 0);
  for (int64_t k = 0; k < b->L; ++k) work[k] *= b->Vf[k];
  orc_fft_inplace(b->L, work, 1);
  for (int64_t m = 0; m < b->M; ++m) X[m] = work[m] * b->post[m];
}

int orc_czt(int64_t N, const double* xr, const double* xi, int64_t M, double alpha, double omega,
            double* Xr, double* Xi) {
  orc_bluestein b;
  if (orc_bluestein_init(&b, N, M, alpha, omega)) return 2;
  cplx* x = (cplx*)malloc(sizeof(cplx) * (size_t)N);
  cplx* X = (cplx*)malloc(sizeof(cplx) * (size_t)M);
  cplx* w = (cplx*)malloc(sizeof(cplx) * (size_t)b.L);
  if (!x || !X || !w) { free(x); free(X); free(w); orc_bluestein_free(&b); return 2; }
  for (int64_t n = 0; n < N; ++n) x[n] = xr[n] + I * xi[n];
  orc_bluestein_apply(&b, x, X, w);
  for (int64_t m = 0; m < M; ++m) { Xr[m] = creal(X[m]); Xi[m] = cimag(X[m]); }
  free(x); free(X); free(w); orc_bluestein_free(&b);
  return 0;
}

/* ------------------------------------------------------------------ */
/* Focal-plane field                                                    */
/* ------------------------------------------------------------------ */

/* Pre = e^{ikz} dx^2 / (i lambda z), z = f; the dx^2 is the area element. */
static cplx orc_prefactor(const orc_params* P) {
  return cexp(I * 2.0 * M_PI * (P->f / P->lambda)) * (P->dx * P->dx) / (I * P->lambda * P->f);
}

static double orc_coord_in(const orc_params* P, int64_t i) { return (double)(i - (P->N - 1) / 2) * P->dx; }
static double orc_coord_out(const orc_params* P, int64_t m) { return P->x0 + (double)m * P->p; }

/* O1: Eq. 1 summed literally.  Rows [j0, j1) of the aperture contribute. */
int orc_field_direct(const orc_params* P, int64_t j0, int64_t j1, double* re, double* im) {
  const int M = P->M;
  const double lf = P->lambda * P->f;
  const cplx pre = cexp(I * 2.0 * M_PI * (P->f / P->lambda)) / (I * lf) * (P->dx * P->dx);
#pragma omp parallel for schedule(dynamic)
  for (int64_t t = 0; t < (int64_t)M * M; ++t) {
    const int64_t n = t / M, m = t % M;
    const double x = orc_coord_out(P, m), y = orc_coord_out(P, n);
    cplx acc = 0.0;
    for (int64_t j = j0; j < j1; ++j) {
      const double v = orc_coord_in(P, j);
      for (int64_t i = 0; i < P->N; ++i) {
        const cplx a = orc_u0(P, j, i);
        if (a == 0.0) continue;
        const double u = orc_coord_in(P, i);
        acc += a * cexp(I * M_PI * ((x - u) * (x - u) + (y - v) * (y - v)) / lf);
      }
    }
    acc *= pre;
    re[t] = creal(acc);
    im[t] = cimag(acc);
  }
  return 0;
}

/* O2: Eq. 2 as U = Pre * chirp_out * (K T K^T), K[m,i] = e^{i pi u_i^2/lf} e^{-2 pi i x_m u_i/lf}. */
int orc_field_separable(const orc_params* P, int64_t j0, int64_t j1, double* re, double* im) {
  const int64_t N = P->N, M = P->M, rows = j1 - j0;
  const double lf = P->lambda * P->f;
  if (rows < 0 || j0 < 0 || j1 > N) return 1;
  cplx* C1 = (cplx*)calloc((size_t)(rows * M), sizeof(cplx));
  if (!C1) return 2;
#pragma omp parallel for schedule(dynamic)
  for (int64_t r = 0; r < rows; ++r) {
    const int64_t j = j0 + r;
    for (int64_t i = 0; i < N; ++i) {
      const cplx a = orc_u0(P, j, i);
      if (a == 0.0) continue;
      const double u = orc_coord_in(P, i);
      const cplx aq = a * cexp(I * M_PI * u * u / lf);
      for (int64_t m = 0; m < M; ++m)
        C1[r * M + m] += aq * cexp(-2.0 * M_PI * I * orc_coord_out(P, m) * u / lf);
    }
  }
  const cplx pre = orc_prefactor(P);
#pragma omp parallel for schedule(static)
  for (int64_t n = 0; n < M; ++n) {
    const double y = orc_coord_out(P, n);
    for (int64_t m = 0; m < M; ++m) {
      cplx acc = 0.0;
      for (int64_t r = 0; r < rows; ++r) {
        const double v = orc_coord_in(P, j0 + r);
        acc += cexp(I * M_PI * v * v / lf) * cexp(-2.0 * M_PI * I * y * v / lf) * C1[r * M + m];
      }
      const double x = orc_coord_out(P, m);
      acc *= pre * cexp(I * M_PI * (x * x + y * y) / lf);
      re[n * M + m] = creal(acc);
      im[n * M + m] = cimag(acc);
    }
  }
  free(C1);
  return 0;
}

/* O3: the paper's CZT method (Fig. 2).  Rows [j0, j1) contribute.
 * Row pass : a_i = U0[j,i] e^{i pi u_i^2/lf};  R[j,m] = e^{-2 pi i (x0 u_0 + m p u_0)/lf} CZT(a)[m]
 *            with Eq. 10: alpha = x0 dx/lf (A), omega = p dx/lf (W), u_0 = first input coordinate.
 * Column   : b_j = e^{i pi v_j^2/lf} R[j,m]; the same CZT over j starting at v_{j0}.
 * Output   : U = Pre e^{i pi (x^2+y^2)/lf} * column result.
 * nthreads <= 0 uses the OpenMP default. */
int orc_field_czt(const orc_params* P, int64_t j0, int64_t j1, int nthreads, double* re, double* im) {
  const int64_t N = P->N, M = P->M, rows = j1 - j0;
  const double lf = P->lambda * P->f;
  if (rows <= 0 || j0 < 0 || j1 > N) return 1;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
  const double alpha = P->x0 * P->dx / lf, omega = P->p * P->dx / lf;
  orc_bluestein brow, bcol;
  if (orc_bluestein_init(&brow, N, M, alpha, omega)) return 2;
  if (orc_bluestein_init(&bcol, rows, M, alpha, omega)) { orc_bluestein_free(&brow); return 2; }
  cplx* R = (cplx*)malloc(sizeof(cplx) * (size_t)(rows * M));
  if (!R) { orc_bluestein_free(&brow); orc_bluestein_free(&bcol); return 2; }
  const double u0 = orc_coord_in(P, 0);
  int fail = 0;
#pragma omp parallel
  {
    cplx* a = (cplx*)malloc(sizeof(cplx) * (size_t)N);
    cplx* w = (cplx*)malloc(sizeof(cplx) * (size_t)brow.L);
    if (!a || !w) {
#pragma omp atomic write
      fail = 1;
    } else {
#pragma omp for schedule(dynamic, 4)
      for (int64_t r = 0; r < rows; ++r) {
        const int64_t j = j0 + r;
        for (int64_t i = 0; i < N; ++i) {
          const cplx t = orc_u0(P, j, i);
          if (t == 0.0) { a[i] = 0.0; continue; }
          const double u = orc_coord_in(P, i);
          a[i] = t * cexp(I * M_PI * u * u / lf); /* chirp written at open pixels only */
        }
        orc_bluestein_apply(&brow, a, R + r * M, w);
        for (int64_t m = 0; m < M; ++m)
          R[r * M + m] *= cexp(-2.0 * M_PI * I * (P->x0 * u0 + (double)m * P->p * u0) / lf);
      }
    }
    free(a); free(w);
  }
  if (fail) { free(R); orc_bluestein_free(&brow); orc_bluestein_free(&bcol); return 2; }
  const double v0 = orc_coord_in(P, j0);
  const cplx pre = orc_prefactor(P);
#pragma omp parallel
  {
    cplx* b = (cplx*)malloc(sizeof(cplx) * (size_t)rows);
    cplx* X = (cplx*)malloc(sizeof(cplx) * (size_t)M);
    cplx* w = (cplx*)malloc(sizeof(cplx) * (size_t)bcol.L);
    if (!b || !X || !w) {
#pragma omp atomic write
      fail = 1;
    } else {
#pragma omp for schedule(dynamic, 4)
      for (int64_t m = 0; m < M; ++m) {
        for (int64_t r = 0; r < rows; ++r) {
          const double v = orc_coord_in(P, j0 + r);
          b[r] = cexp(I * M_PI * v * v / lf) * R[r * M + m];
        }
        orc_bluestein_apply(&bcol, b, X, w);
        const double x = orc_coord_out(P, m);
        for (int64_t n = 0; n < M; ++n) {
          const double y = orc_coord_out(P, n);
          const cplx U = X[n] * cexp(-2.0 * M_PI * I * (P->x0 * v0 + (double)n * P->p * v0) / lf) * pre *
                         cexp(I * M_PI * (x * x + y * y) / lf);
          re[n * M + m] = creal(U);
          im[n * M + m] = cimag(U);
        }
      }
    }
    free(b); free(X); free(w);
  }
  free(R);
  orc_bluestein_free(&brow);
  orc_bluestein_free(&bcol);
  return fail ? 2 : 0;
}

int orc_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
