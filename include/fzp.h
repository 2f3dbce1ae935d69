/*
 * fzp.h -- C ABI of libfzp.so, a GB300 (sm_103a) library that evaluates the
 * Fresnel diffraction integral of a full-aperture Fresnel zone plate (FZP) on a
 * fixed focal-plane region of interest (ROI) by stripe-processed chirp-z
 * transforms.
 *
 * The operation (Eq. 1-2, Sec. 2.1; Fig. 2 and Fig. 18):
 *
 *   U(x_m, y_n) = e^{ikf} e^{i pi (x_m^2 + y_n^2)/(lambda f)} dx^2 / (i lambda f)
 *                 * sum_{j,i} T[j,i] e^{i phi[j,i]} e^{i pi (u_i^2 + v_j^2)/(lambda f)}
 *                   * e^{-2 pi i (x_m u_i + y_n v_j)/(lambda f)},           I = |U|^2
 *
 * with the aperture grid u_i = (i - c) dx, c = (N-1)/2 (N odd, Fig. 2 Stage 1),
 * the ROI grid x_m = (m - M/2) p (sample M/2 on the axis; or x_m = x0 + m p,
 * y_n = y0 + n p for an off-axis ROI, see fzp_params.roi_origin), T the binary FZP
 * mask (open where floor(r^2/(lambda f)) is odd and r <= R_eff, Fig. 2 Stage 2,
 * paraxial radii of Eq. 4, centre zone opaque) and phi an optional membrane
 * deformation phase (4 pi / lambda) w(u, v).  With fzp_params.levels = L >= 2
 * T is instead the L-level phase transmission e^{-2 pi i q / L} inside R_eff,
 * q = floor(L r^2 / (2 lambda f)) mod L (Fig. 18 Stage 3; Tables 3-5).  The mask is
 * generated inside the kernels stripe by stripe and never stored.
 *
 * Conventions shared by every call:
 *   - Units are SI (metres).  Complex data are interleaved (re, im) pairs of
 *     IEEE doubles ("complex128"); 2-D arrays are row-major with the y index n
 *     slowest: element (n, m) at offset n*M + m.
 *   - "device" pointers are CUDA global-memory addresses on the current device;
 *     the caller allocates and owns them.  `stream` is a cudaStream_t passed as
 *     void* (NULL = legacy default stream).  Calls that take a stream enqueue
 *     work and return without synchronising unless stated otherwise.
 *   - Every call returns an fzp_status; nothing throws or aborts across the
 *     ABI.  fzp_last_error() gives a human-readable message for the calling
 *     thread's last failure.
 *   - Invalid arguments are rejected with FZP_E_INVALID before any device
 *     memory is allocated or any work is enqueued.
 */
#ifndef FZP_H_
#define FZP_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define FZP_API __attribute__((visibility("default")))
#else
#define FZP_API
#endif

typedef enum {
  FZP_OK = 0,
  FZP_E_INVALID = 1,     /* bad argument; nothing was allocated or enqueued          */
  FZP_E_OOM = 2,         /* device or host allocation failed; nothing leaked          */
  FZP_E_CUDA = 3,        /* a CUDA runtime call failed (message names it)             */
  FZP_E_TIMEOUT = 4,     /* a bounded device-side wait ran out; results are invalid   */
  FZP_E_UNSUPPORTED = 5  /* valid request the library does not implement              */
} fzp_status;

/* Kernel form of the row transform. */
typedef enum {
  FZP_FORM_AUTO = 0,      /* dense for split-BF16/BF16 precision, Bluestein otherwise  */
  FZP_FORM_BLUESTEIN = 1, /* (a) separable Bluestein CZT with hand-written FFTs (Sec. 2.6) */
  FZP_FORM_DENSE = 2,     /* (b) tensor-core contraction U = K diag T K^T (separability of Eq. 2) */
  FZP_FORM_SACZT = 3      /* semi-analytical CZT (Sec. 3.6, Fig. 5): angular-spectrum propagation
                             without the paraxial approximation on a padded grid, then a Fresnel
                             chirp and a CZT zoom onto the ROI; FP32; with exact_radii = 1 the
                             zone radii of Eq. 3 */
} fzp_form;

/* Arithmetic of the row transform.  Phase arguments are always reduced in
 * FP64 and the cross-stripe ROI sum is always FP64. */
typedef enum {
  FZP_PREC_FP64 = 0,       /* Bluestein in FP64 throughout                          */
  FZP_PREC_FP32 = 1,       /* Bluestein in FP32 (complex64)                          */
  FZP_PREC_SPLIT_BF16 = 2, /* dense: K = K_hi + K_lo in BF16, T exact, FP32 accumulate */
  FZP_PREC_BF16 = 3,       /* dense: K_hi only (reduced accuracy, for error studies)   */
  FZP_PREC_AUTO_1E4 = 4    /* any arithmetic whose ROI-intensity error is <= 1e-4: the
                              autotuner measures split-BF16 dense and FP32 Bluestein
                              (and their knobs) on a probe stripe and keeps the faster */
} fzp_precision;

/* Membrane deformation w(u,v) [m]; phase phi = (4 pi / lambda) w:
 *   w = amp sin(2 pi (u cos theta + v sin theta) / period) (1 - taper (r/R)^2)
 *     + sum_{k < n_ridges} h_k exp(-d_k^2 / (2 sigma_k^2)),
 *   d_k = distance of (u,v) to the line through (px_k, py_k) at angle alpha_k,
 *   sigma_k = width_k / (2 sqrt(2 ln 2)).   n_ridges <= 3.                    */
typedef struct fzp_deform {
  double amp, period, theta, taper;
  int32_t n_ridges;
  int32_t reserved;
  double ridge_px[3], ridge_py[3], ridge_alpha[3], ridge_h[3], ridge_width[3];
} fzp_deform;

/* Problem statement (Fig. 2 ENTRY: N_in, N_out, D, f, lambda0). */
typedef struct fzp_params {
  double D;            /* aperture diameter [m], > 0                                   */
  double f;            /* focal length = propagation distance [m], > 0                 */
  double lambda;       /* wavelength [m], > 0                                          */
  double dx;           /* aperture pitch [m]; 0 -> lambda f / (4 D): four samples per
                          outermost zone width (Eq. 5); must satisfy Eq. 6,
                          dx <= lambda f / (2 D)                                       */
  int64_t N;           /* samples per aperture side; 0 -> ceil(D / dx) forced odd;
                          a given N must be odd                                        */
  int32_t M;           /* ROI samples per side: a power of two in [64, 1024]          */
  int32_t form;        /* fzp_form                                                     */
  double pitch;        /* ROI pitch p [m], > 0                                         */
  int32_t precision;   /* fzp_precision                                                */
  int32_t stripe_rows; /* aperture rows per row-pass chunk (multiple of 256); 0 ->
                          as many as an 8 GiB row intermediate holds               */
  const fzp_deform* deform; /* NULL: flat membrane.  Copied by fzp_plan.               */
  int32_t promote;     /* dense: 32-column K blocks accumulated in tensor memory before
                          promotion to FP32 global sums; 0 -> 128 (error ~8e-6 at
                          D = 0.25 m; it grows in proportion to this length)       */
  int32_t row_batch;   /* Bluestein: aperture rows per FFT pass launch; 0 -> rows of a
                          1 GiB transform workspace                               */
  int32_t cluster;     /* dense: CTAs of a thread-block cluster that share each
                          generated mask tile through distributed shared memory,
                          each generating its share of the rows (1, 2 or 4;
                          0 -> the largest of 4, 2, 1 dividing the M/64 tile
                          pairs; other values pad the pairs with zero tiles)      */
  int32_t levels;      /* 0 or 1: binary amplitude FZP (Fig. 2: open where the
                          paraxial zone index is odd).  L >= 2: L-level phase FZP
                          (Fig. 18 Stage 3): transmission e^{-2 pi i q/L} inside
                          the aperture, q = floor(fl(s kappa_L)) mod L with
                          kappa_L = fl(kappa L/2), so L = 2 steps on the zones.
                          The default dx becomes lambda f/(2 D max(L, 2))
                          (Fig. 18 Stage 1, S_samp = 4).  The dense form takes
                          even L: L = 2 as one +-1 mask, L >= 4 as L/2 passes of
                          masks with values -1, 0, +1 (exact in BF16) whose
                          fields are summed with the weights of Re T and Im T */
  int32_t centre_open; /* centre configuration of the binary amplitude plate
                          (Fig. 18 engine): 0 = negative-centred, odd zones open,
                          the centre zone opaque (Sec. 4.1's plate); 1 =
                          positive-centred, even zones open.  Must be 0 for a
                          phase plate (levels >= 2), where it would only shift
                          every level by one phase; other values are invalid */
  int32_t roi_origin;  /* 0: ROI centred on the focus, x_m = (m - M/2) p and
                          y_n = (n - M/2) p.  1: the first ROI sample is at
                          (x0, y0): x_m = x0 + m p, y_n = y0 + n p (Eq. 10's A
                          from the first ROI coordinate, Sec. 2.6).  Both forms
                          use one kernel matrix for the two axes, so x0 must
                          equal y0 (FZP_E_UNSUPPORTED otherwise); fzp_metrics
                          reads the focus at the ROI centre and rejects an
                          off-axis plan with FZP_E_UNSUPPORTED.  Other values
                          are invalid                                          */
  int32_t reserved;    /* must be 0                                            */
  double x0, y0;       /* first ROI coordinates [m] when roi_origin = 1 (finite) */
  int32_t exact_radii; /* 0: paraxial zone radii r_m^2 = m lambda f (Eq. 4), every
                          form; 1: exact radii of Eq. 3, r_m^2 = m lambda f +
                          (m lambda / 2)^2, the binary amplitude plate under
                          FZP_FORM_SACZT only (the paraxial forms' kernel would
                          aberrate it; FZP_E_UNSUPPORTED elsewhere)          */
  int32_t conv;        /* Bluestein row convolution (Sec. 2.6: the row CZT as a
                          convolution with the chirp h_k = e^{i pi delta k^2}):
                          0 -> partitioned with FP32, single with FP64;
                          1 = single: one L-point FFT convolution per row
                          (four-step FFTs through a global-memory workspace,
                          the paper's structure);
                          2 = partitioned: the row cut into blocks of S
                          columns, S = 256 min(15, floor((4097 - M) / 256)),
                          each block's 4096-point spectrum times the
                          precomputed spectrum of its chirp piece, summed over
                          the blocks that meet the row's disc chord, then one
                          inverse 4096-point FFT per row, all on chip; FP32
                          only (FZP_E_UNSUPPORTED with FP64).  Other values
                          are invalid; the other forms ignore it            */
} fzp_params;

/* Opaque plan: geometry, zone-threshold table, chirp / kernel tables and the
 * workspace of one problem.  Owned by the caller between fzp_plan and
 * fzp_plan_destroy.  A plan must not be used by two streams at once. */
typedef struct fzp_plan_s* fzp_plan_t;

/* Read-only description of a plan. */
typedef struct fzp_plan_info {
  int64_t N;             /* aperture samples per side                              */
  int64_t c;             /* index of the on-axis sample, (N-1)/2                   */
  int64_t total_zones;   /* floor(n_exact) of Eq. 3 (Fig. 2 Stage 2)               */
  int64_t n_thresholds;  /* entries of the zone-threshold table                    */
  double dx;             /* aperture pitch [m]                                     */
  double R;              /* aperture radius R_eff = min(D/2, lambda f/(2 dx)) [m]  */
  double kappa;          /* dx^2 / (lambda f): zone index = floor(s kappa)         */
  double x0;             /* first ROI coordinate [m] (both axes)                   */
  int32_t M;             /* ROI samples per side                                   */
  int32_t form;          /* resolved fzp_form                                      */
  int32_t precision;     /* fzp_precision                                          */
  int32_t stripe_rows;   /* resolved stripe height                                 */
  int64_t fft_length;    /* Bluestein length L = 2^ceil(log2(N + M - 1)) (Sec. 2.6) */
  size_t device_bytes;   /* device memory owned by the plan (batch: by the batch)  */
  int32_t promote;       /* dense: K blocks per tensor-memory accumulation chunk   */
  int32_t row_batch;     /* Bluestein: aperture rows per FFT pass launch           */
  int64_t chunk_rows;    /* aperture rows per row-pass chunk                       */
  int32_t cluster;       /* dense: CTAs per cluster sharing each mask tile         */
  int32_t fft_inner;     /* Bluestein: inner FFT length L2 of the four-step split
                            L = L1 L2 (L itself when L <= the inner limit)        */
  int32_t ctas;          /* dense: CTAs of the persistent row-pass launch (whole
                            clusters that are resident at once)                   */
  int32_t levels;        /* phase levels L (0: binary amplitude FZP)               */
  int32_t passes;        /* dense form: signed-mask passes per row chunk (1, or L/2
                            for a phase plate with L >= 4)                         */
  int32_t centre_open;   /* 1: positive-centred binary plate (even zones open)     */
  int32_t conv;          /* Bluestein: 1 single L-point convolution per row, 2
                            partitioned into 4096-point blocks; 0 other forms      */
  int64_t s_R;           /* largest squared distance from the axis, in samples, of a
                            sample inside the aperture disc (fl(s_R dx^2) <= fl(R^2)) */
} fzp_plan_info;

/* Metrics of Fig. 2 Stage 4 / Fig. 18 Stage 5. */
typedef struct fzp_metrics_t {
  double fwhm_x, fwhm_y; /* FWHM of the centre row / column [m]: parabolic peak,
                            half-maximum crossings of the not-a-knot cubic spline */
  double de_lobe;        /* sum_{r <= r_null} I p^2 / P_in, r_null = 1.21967 lambda f / (2R) */
  double de_roi;         /* sum_ROI I p^2 / P_in                                  */
  double p_in;           /* incident power: (# samples with r <= R_eff) dx^2       */
  double p_in_disc;      /* pi R^2 (the v8 normalisation, Fig. 18)                 */
  double peak;           /* I at the on-axis sample (M/2, M/2)                     */
  double strehl;         /* peak / (pi R^2 / (lambda f))^2 (Fig. 18 Stage 5)       */
  double mtf_half_cut;   /* radial MTF at nu_cut/2, nu_cut = 2R/(lambda f)         */
  double mtf16[16];      /* radial MTF at (q + 1/2) nu_cut / 16, q = 0..15         */
  int64_t aperture_count;/* samples with r <= R_eff                                */
} fzp_metrics_t;

/* Build a plan (Fig. 2 Stage 1-2; Fig. 18 Stage 1-2): validate `params`,
 * derive the grids, build the zone-threshold table and the form's tables,
 * and allocate the workspace.  Synchronises the device.  On failure *out is
 * NULL and nothing is leaked.  If the row intermediate of one chunk cannot be
 * allocated, the chunk is halved (down to 256 rows) and the allocation
 * retried; fzp_plan_info_get reports the chunk that was allocated.  For
 * tests, the environment variable FZP_FAULT_ALLOC_LIMIT (bytes) makes larger
 * row-intermediate requests fail as out of memory on the host.
 * Size limits (FZP_E_UNSUPPORTED beyond them): the exact zone rule needs the
 * squared disc radius in samples s_R < 2^46 (N up to about 1.67e7 for a
 * full-aperture plate) and fewer than 2^24 zone steps; the Bluestein form
 * needs N + M - 1 <= 2^24 (its FFT length, a power of two); the SA-CZT form
 * a padded grid P <= 16384 (P the power of two >= 1.5 N, N <= 10922; the
 * plan holds two P x P complex64 grids, 4 GiB at the limit).  Errors:
 * FZP_E_INVALID (bad parameters, Eq. 6 violated, M out of range), FZP_E_OOM,
 * FZP_E_CUDA, FZP_E_UNSUPPORTED (e.g. dense form with FP64 precision). */
FZP_API fzp_status fzp_plan(const fzp_params* params, fzp_plan_t* out);

/* The host part of fzp_plan alone: validate `params`, derive the grids (Fig. 2
 * and Fig. 18 Stage 1) and check the zone-rule limits, without any CUDA call
 * or allocation (it runs on a machine without a GPU), and describe the plan
 * that fzp_plan would build: N, c, the Eq. 3 zone count, the threshold count,
 * dx, R_eff, kappa, x0, M, form, precision, chunk rows, FFT length (Bluestein),
 * promotion length (dense), levels, passes, centre configuration.  Fields
 * that depend on the device (fft_inner, ctas, device_bytes, an automatic
 * cluster size, row_batch) are 0, and so are the form-specific fields when the
 * precision is FZP_PREC_AUTO_1E4 (form reported as FZP_FORM_AUTO).  The chunk
 * is the one fzp_plan tries first.  Errors: as fzp_plan's validation. */
FZP_API fzp_status fzp_plan_query(const fzp_params* params, fzp_plan_info* out);

/* The zone-threshold table that fzp_plan builds on the host and uploads
 * (Sec. 2.2, Eq. 4; the exact mask rule): S_m = min{s : floor(fl(s kappa_L))
 * >= m} for m = 1 .. count, s the integer squared distance from the axis in
 * samples, kappa_L the zone-step rate (kappa, or kappa L / 2 for an L-level
 * plate).  Writes *count and the first min(capacity, count) entries to `out`
 * (host memory; NULL with capacity 0 asks for the count).  No CUDA call.
 * Errors: as fzp_plan's validation; FZP_E_INVALID for a NULL count or a NULL
 * out with capacity > 0. */
FZP_API fzp_status fzp_zone_thresholds(const fzp_params* params, int64_t* out, int64_t capacity, int64_t* count);

/* Copy the plan description into *out (host memory). */
FZP_API fzp_status fzp_plan_info_get(fzp_plan_t plan, fzp_plan_info* out);

/* Release everything the plan owns.  NULL is accepted.  Synchronises the device. */
FZP_API fzp_status fzp_plan_destroy(fzp_plan_t plan);

/* Contribution of aperture rows [row_begin, row_end) to the ROI field
 * (Fig. 2 Stage 3 / Fig. 18 Stage 3-4: row pass per stripe, column pass, output
 * chirp and Fresnel prefactor).  The field is linear in the rows, so calls over
 * disjoint row ranges with accumulate = 1 sum to the full-aperture field
 * (resumable and shardable, Sec. 7.2).
 *   d_field    device, complex128, M*M, caller-owned; written (accumulate = 0)
 *              or added to (accumulate != 0).
 *   stream     cudaStream_t; work is enqueued, no host synchronisation.
 * Errors: FZP_E_INVALID (range outside [0, N], NULL field), FZP_E_CUDA. */
FZP_API fzp_status fzp_propagate_roi(fzp_plan_t plan, int64_t row_begin, int64_t row_end, void* d_field,
                             int accumulate, void* stream);

/* I = |U|^2 (Fig. 2: I(x', y') = |U_out|^2).
 *   d_field device complex128 M*M (input), d_intensity device double M*M (output). */
FZP_API fzp_status fzp_intensity(fzp_plan_t plan, const void* d_field, void* d_intensity, void* stream);

/* Metric extractor on a full ROI field (Fig. 2 Stage 4; Fig. 18 Stage 5).
 * Runs on the device, then synchronises `stream` and writes *out (host).
 * Also reports any device-side timeout recorded by earlier calls on this plan
 * (FZP_E_TIMEOUT). */
FZP_API fzp_status fzp_metrics(fzp_plan_t plan, const void* d_field, void* stream, fzp_metrics_t* out);

/* Run outputs of the simulation engine (Fig. 18, RETURN: result, text report
 * and JSON sidecar in a run folder, read against the analytic references).
 * Runs fzp_metrics on d_field (a full ROI field of this plan), then writes
 *   <run_dir>/result_<tag>.npy   I = |U|^2, M x M float64, NumPy .npy 1.0
 *   <run_dir>/report_<tag>.txt   problem, grids, metrics, references, timing
 *   <run_dir>/result_<tag>.json  the same as one JSON object
 * References: FWHM against the Airy value 1.0289939 lambda f / (2 R_eff) and
 * the outermost zone width lambda f / (2 R_eff); main-lobe DE against
 * EE(r_null) eta with EE(r_null) = 0.8377850 and eta = 1/pi^2 (binary
 * amplitude) or sinc^2(1/L) (L-level phase, the level ladder); MTF at
 * nu_cut/2 against the clear pupil's 0.3910022.
 *   d_field       device complex128 M*M (input).
 *   t_propagate_s the caller's propagation time [s], reported with the
 *                 throughput N^2 / t (0: not timed).
 *   run_dir       existing directory (host string); tag: letters, digits,
 *                 '-', '_', '.' only.  Existing files of the same tag are
 *                 overwritten.
 *   stream        cudaStream_t; the call synchronises it.
 *   out           optional (NULL): receives the metrics.
 * Errors: FZP_E_INVALID (NULL, bad tag, a file that cannot be written),
 * FZP_E_UNSUPPORTED (off-axis ROI, as fzp_metrics), FZP_E_CUDA, FZP_E_TIMEOUT. */
FZP_API fzp_status fzp_report_write(fzp_plan_t plan, const void* d_field, double t_propagate_s, const char* run_dir,
                                    const char* tag, void* stream, fzp_metrics_t* out);

/* ---- Batches: many apertures in one CUDA graph ----------------------------
 *
 * A batch holds n problems (different D, lambda, deformation, ROI) that share
 * one set of device buffers sized for the largest.  Each instance's form
 * tables are regenerated inside the batch, and its work -- tables, row passes
 * (the dense form as one persistent launch), column pass and epilogue -- is
 * captured with all other instances into one CUDA graph that
 * fzp_batch_propagate replays with a single launch.  Instances with
 * precision FZP_PREC_AUTO_1E4 are autotuned first (see fzp_precision).
 * The per-instance stages follow Fig. 18 (tables, row stage, column stage,
 * output chirp); the batching itself has no counterpart in the paper. */
typedef struct fzp_batch_s* fzp_batch_t;

/* Plan a batch of n >= 1 problems.  params[i] as for fzp_plan.  Errors as
 * fzp_plan; the message names the failing instance. */
FZP_API fzp_status fzp_batch_plan(const fzp_params* params, int n, fzp_batch_t* out);

/* Full-aperture field of every instance: d_fields[i] is a device complex128
 * M_i*M_i buffer (caller-owned), overwritten.  The first call (and any call
 * with different field pointers) captures the graph; later calls replay it.
 * Asynchronous on `stream`. */
FZP_API fzp_status fzp_batch_propagate(fzp_batch_t batch, void* const* d_fields, void* stream);

/* Plan description of instance `index` (the form and knobs chosen for it). */
FZP_API fzp_status fzp_batch_info(fzp_batch_t batch, int index, fzp_plan_info* out);

/* Metric extractor for instance `index` (as fzp_metrics). */
FZP_API fzp_status fzp_batch_metrics(fzp_batch_t batch, int index, const void* d_field, void* stream,
                                     fzp_metrics_t* out);

/* I = |U|^2 of instance `index` (as fzp_intensity): d_field device complex128
 * M_i*M_i (input), d_intensity device double M_i*M_i (output).  Asynchronous. */
FZP_API fzp_status fzp_batch_intensity(fzp_batch_t batch, int index, const void* d_field, void* d_intensity,
                                       void* stream);

/* Kernel launches of one replay: the kernel nodes of the captured graph
 * (0 before the first fzp_batch_propagate).  Host only. */
FZP_API fzp_status fzp_batch_kernels(fzp_batch_t batch, int64_t* kernels);

/* Release the batch.  NULL is accepted.  Synchronises the device. */
FZP_API fzp_status fzp_batch_destroy(fzp_batch_t batch);

/* ---- Learned surrogate (no counterpart in the paper) ------------------------
 *
 * A multilayer perceptron n_in -> hidden (x n_hidden_layers, SiLU) -> n_out
 * (linear), trained with mean squared error and AdamW (decoupled weight decay
 * on weights), by kernels in this library: every matrix product takes BF16
 * operands and accumulates in FP32 on the tensor cores (tcgen05); master
 * weights, optimiser state and gradients are FP32.  It learns the map from
 * membrane-deformation parameters to the PSF and metrics that this library's
 * propagation computes; the propagation stays the reference its error is measured against.
 * Parameters are one flat FP32 vector: for each layer W (n_out x n_in,
 * row-major) then b (n_out). */
typedef struct fzp_surrogate_s* fzp_surrogate_t;

/* Create with weights ~ U(-1/sqrt(fan_in), 1/sqrt(fan_in)) from `seed`, biases 0.
 * All sizes in [1, 65536]; max_batch bounds every later batch. */
FZP_API fzp_status fzp_surrogate_create(int n_in, int hidden, int n_hidden_layers, int n_out, int max_batch,
                                        uint64_t seed, fzp_surrogate_t* out);

/* Number of FP32 parameters (0 for NULL). */
FZP_API size_t fzp_surrogate_param_count(fzp_surrogate_t s);

/* Copy the master parameters to (set = 0) or from (set = 1) host memory;
 * count must equal fzp_surrogate_param_count.  Synchronous. */
FZP_API fzp_status fzp_surrogate_params(fzp_surrogate_t s, float* h_params, size_t count, int set);

/* y = network(x): d_x device FP32 [batch][n_in], d_y device FP32 [batch][n_out],
 * 1 <= batch <= max_batch.  Asynchronous on `stream`. */
FZP_API fzp_status fzp_surrogate_infer(fzp_surrogate_t s, const float* d_x, int batch, float* d_y, void* stream);

/* Loss (mean squared error, written to d_loss, device FP32 scalar, optional)
 * and its gradient (d_grad, device FP32 [param_count], optional) for a batch
 * (multiple of 8, <= max_batch) of inputs d_x and targets d_y [batch][n_out]. */
FZP_API fzp_status fzp_surrogate_grad(fzp_surrogate_t s, const float* d_x, const float* d_y, int batch,
                                      float* d_grad, float* d_loss, void* stream);

/* One AdamW step (beta1 0.9, beta2 0.999, eps 1e-8) on a batch (multiple of 8). */
FZP_API fzp_status fzp_surrogate_train_step(fzp_surrogate_t s, const float* d_x, const float* d_y, int batch,
                                            float lr, float weight_decay, float* d_loss, void* stream);

/* Release.  NULL is accepted. */
FZP_API fzp_status fzp_surrogate_destroy(fzp_surrogate_t s);

/* Metric extractor that allocates nothing (no counterpart in the paper).
 *
 * Some callers cannot allocate device memory: a process whose device memory is
 * owned by another allocator (for example a framework's caching pool that must
 * stay the only owner), a real-time loop that forbids allocation once it has
 * started, or a process running at its memory limit where a fresh allocation
 * can fail mid-run.  fzp_plan allocates its tables and workspace, so such a
 * caller cannot obtain fzp_metrics; this call computes the same metrics (same
 * kernels) from the problem parameters alone.
 *
 * Its scratch is one file-scope device array of 4.25 MiB, which every GPU that
 * loads libfzp holds until the process exits.  Limit: M <= 512 (power of two,
 * >= 64); larger M is rejected with FZP_E_INVALID.  The first call on a device
 * looks up the array's device address with that device current (once per
 * device) and keeps it for the life of the process; make that first call
 * before any stream capture.  cudaDeviceReset discards the array's address
 * with the context, so a process that resets a device must not call this
 * entry point on that device afterwards.  The parameters are validated as
 * fzp_plan validates them (no CUDA call for that).  All calls share
 * the array and it keeps the last call's contents (the call clears what must
 * start at zero); calls that overlap on the GPU, on any streams, race and give
 * wrong results, so serialise them.
 *   params  problem statement as for fzp_plan (M <= 512).
 *   d_field device complex128 M*M, the focal-plane field (input).
 *   stream  cudaStream_t; the call synchronises it and writes *out (host).
 * Calls no cudaMalloc, cudaFree or allocating library routine. */
FZP_API fzp_status fzp_metrics_noalloc(const fzp_params* params, const void* d_field, void* stream,
                                       fzp_metrics_t* out);

/* Self-test of the failure path shared by the library's kernels (no
 * counterpart in the paper).  Every device-side wait is bounded: when it
 * expires, the kernel records a code in an error word, stops, and the host
 * reports FZP_E_TIMEOUT (fzp_metrics does for a propagation).  This call runs
 * one such wait on a barrier that nothing completes, with a limit of limit_us
 * microseconds (1 .. 2,000,000; the production kernels use 2 s), so that the
 * path can be tested without a fault: nothing else is in flight and the
 * context stays usable.
 *   stream  cudaStream_t; the call synchronises it.
 * Returns FZP_E_TIMEOUT when the wait ran out and was reported (the expected
 * outcome), FZP_E_CUDA if it was not, FZP_E_INVALID for a limit out of range.
 * Allocates nothing (the error word is a file-scope device variable). */
FZP_API fzp_status fzp_selftest_wait_timeout(uint32_t limit_us, void* stream);

/* Binary aperture transmission T[j, i] of rows [row_begin, row_end), produced
 * by the same device code that feeds the plan's row transform (Fig. 2 Stage 2:
 * open where the paraxial zone index floor(r^2/(lambda f)) is odd and
 * r <= R_eff; even instead of odd for a positive-centred plate), for
 * inspection and testing.  The Bluestein form evaluates each sample; the
 * dense form exports through the generator its row pass launches: the row
 * walker (single-CTA launches), the block-wise generator (2- and 4-CTA
 * clusters) or the level mode (phase plates with L >= 4, positive-centred
 * plates).  For an L-level phase plate (levels >= 2) the level map: 1 + q
 * inside the aperture (q = the phase level, Fig. 18 Stage 3), 0 outside.
 *   d_mask  device uint8, (row_end - row_begin) * N, row-major.
 * Errors: FZP_E_INVALID (range outside [0, N], NULL). */
FZP_API fzp_status fzp_aperture_mask(fzp_plan_t plan, int64_t row_begin, int64_t row_end, void* d_mask,
                                     void* stream);

/* Tracing of one plan (Sec. 5 of the paper times t_row / t_col with tic/toc;
 * here CUDA events are recorded on the launching stream around every launch of
 * the form's dominant kernel while profiling is enabled). */
typedef struct fzp_profile_t {
  double dominant_ms;        /* summed device time of the dominant kernel [ms]      */
  int64_t dominant_launches; /* its launches since the last read                    */
  int64_t kernel_launches;   /* all kernels this plan launched since the last read  */
  char dominant_name[48];    /* kernel name                                         */
} fzp_profile_t;

/* Enable (1) or disable (0) event recording for `plan`. */
FZP_API fzp_status fzp_profile_enable(fzp_plan_t plan, int enable);

/* Synchronise on the recorded events, write the totals to *out (host) and
 * reset them. */
FZP_API fzp_status fzp_profile_read(fzp_plan_t plan, fzp_profile_t* out);

/* Message of the calling thread's last failed call ("" if none). */
FZP_API const char* fzp_last_error(void);

/* Library version string. */
FZP_API const char* fzp_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FZP_H_ */
