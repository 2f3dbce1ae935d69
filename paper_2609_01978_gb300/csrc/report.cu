// report.cu -- the run outputs of the simulation engine (Fig. 18, RETURN:
// result, text report and JSON sidecar written to a run folder, with FWHM read
// against the Airy value and the zone width, DE against the level ladder,
// Strehl and MTF).
//
//   result_<tag>.npy   I = |U|^2 on the M x M ROI (float64, row-major, n slowest;
//                      NumPy .npy format 1.0 so that any NumPy reads it)
//   report_<tag>.txt   the problem, the grids, the metrics and their analytic
//                      references, the timings
//   result_<tag>.json  the same as one JSON object (the sidecar)
//
// Analytic references (Sec. 2.3, Fig. 18 "verification against the analytical
// references"):
//   FWHM_Airy = 1.0289939 lambda f / (2 R): the full width at half maximum of
//     (2 J1(x)/x)^2, x = pi r 2R / (lambda f) (half maximum at x = 1.6163);
//   outermost zone width dr_N = lambda f / (2 R) (Eq. 5 with D = 2R);
//   main-lobe DE = EE(r_null) eta, EE(r_null) = 1 - J0(j1,1)^2 = 0.8377850 the
//     Airy energy inside the first null j1,1 = 3.8317, eta the first-order
//     efficiency: 1/pi^2 for the binary amplitude plate, sinc^2(1/L) =
//     (sin(pi/L)/(pi/L))^2 for an L-level phase plate (the level ladder);
//   MTF of the clear circular pupil at nu_cut / 2: (2/pi)(acos(1/2) -
//     (1/2) sqrt(3/4)) = 0.3910022.
#include <cctype>
#include <cerrno>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "fzp_internal.cuh"

namespace fzp {
namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr double kAiryFwhm = 1.0289939;   // FWHM of the Airy pattern in lambda f / D
constexpr double kEeNull = 0.8377850;     // encircled energy inside the first Airy null
constexpr double kMtfHalf = 0.3910022;    // circular-pupil MTF at half the cut-off

double level_efficiency(int levels) {
  if (levels < 2) return 1.0 / (kPi * kPi);
  const double x = kPi / levels;
  return (std::sin(x) / x) * (std::sin(x) / x);
}

// NumPy .npy (format 1.0) header for a C-ordered float64 array of shape (M, M).
std::string npy_header(int M) {
  char dict[128];
  snprintf(dict, sizeof(dict), "{'descr': '<f8', 'fortran_order': False, 'shape': (%d, %d), }", M, M);
  std::string h(dict);
  const size_t base = 10;  // magic (6) + version (2) + header length (2)
  size_t total = base + h.size() + 1;
  const size_t pad = (64 - total % 64) % 64;
  h.append(pad, ' ');
  h.push_back('\n');
  std::string out("\x93NUMPY\x01\x00", 8);
  const uint16_t len = (uint16_t)h.size();
  out.push_back((char)(len & 0xFF));
  out.push_back((char)(len >> 8));
  return out + h;
}

bool little_endian() {
  const uint16_t v = 1;
  uint8_t b;
  memcpy(&b, &v, 1);
  return b == 1;
}

}  // namespace
}  // namespace fzp

using namespace fzp;

extern "C" fzp_status fzp_report_write(fzp_plan_t plan, const void* d_field, double t_propagate_s,
                                       const char* run_dir, const char* tag, void* stream, fzp_metrics_t* out) {
  if (!plan || !d_field || !run_dir || !tag) return set_error(FZP_E_INVALID, "NULL argument");
  for (const char* c = tag; *c; ++c)
    if (!(std::isalnum((unsigned char)*c) || *c == '-' || *c == '_' || *c == '.'))
      return set_error(FZP_E_INVALID, "tag may hold letters, digits, '-', '_' and '.' only");
  if (!*tag) return set_error(FZP_E_INVALID, "empty tag");
  if (!little_endian()) return set_error(FZP_E_UNSUPPORTED, "the .npy writer assumes a little-endian host");
  Plan& P = *plan;
  cudaStream_t s = (cudaStream_t)stream;
  fzp_metrics_t m{};
  fzp_status st = metrics(P, d_field, s, &m);
  if (st != FZP_OK) return st;
  // I = |U|^2 into the metric scratch's transform area (free once the
  // extractor has finished on this stream), then to the host
  const int M = P.M;
  double* dI = P.d_metrics + 8192;
  st = intensity(P, d_field, dI, s);
  if (st != FZP_OK) return st;
  std::vector<double> I((size_t)M * M);
  FZP_CUDA_TRY(cudaMemcpyAsync(I.data(), dI, I.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
  FZP_CUDA_TRY(cudaStreamSynchronize(s));

  const std::string dir(run_dir), t(tag);
  const std::string f_npy = dir + "/result_" + t + ".npy", f_txt = dir + "/report_" + t + ".txt",
                    f_json = dir + "/result_" + t + ".json";
  {
    FILE* fh = std::fopen(f_npy.c_str(), "wb");
    if (!fh) return set_error(FZP_E_INVALID, "cannot write %s: %s", f_npy.c_str(), std::strerror(errno));
    const std::string h = npy_header(M);
    const bool ok = std::fwrite(h.data(), 1, h.size(), fh) == h.size() &&
                    std::fwrite(I.data(), sizeof(double), I.size(), fh) == I.size();
    if (std::fclose(fh) != 0 || !ok) return set_error(FZP_E_INVALID, "short write to %s", f_npy.c_str());
  }
  // analytic references
  const double lf = P.lambda * P.f;
  const double zone_width = lf / (2.0 * P.R);
  const double fwhm_airy = kAiryFwhm * zone_width;
  const double eta = level_efficiency(P.levels);
  const double de_ref = kEeNull * eta;
  const char* plate = P.levels >= 2 ? "L-level phase" : (P.mg.centre_open ? "binary amplitude, positive-centred"
                                                                          : "binary amplitude, negative-centred");
  const char* form = P.form == FZP_FORM_DENSE ? "dense tcgen05 contraction" : "separable Bluestein CZT";
  const char* prec = P.precision == FZP_PREC_FP64 ? "fp64" : P.precision == FZP_PREC_FP32 ? "fp32"
                     : P.precision == FZP_PREC_SPLIT_BF16 ? "split-bf16" : "bf16";
  const double samples = (double)P.N * (double)P.N;
  {
    FILE* fh = std::fopen(f_txt.c_str(), "w");
    if (!fh) return set_error(FZP_E_INVALID, "cannot write %s: %s", f_txt.c_str(), std::strerror(errno));
    std::fprintf(fh, "%s -- Fresnel zone plate, full-aperture CZT propagation\n\n", fzp_version());
    std::fprintf(fh, "plate      %s, L = %d\n", plate, P.levels >= 2 ? P.levels : 2);
    std::fprintf(fh, "aperture   D = %.9g m, R_eff = %.9g m, f = %.9g m, lambda = %.9g m\n", P.D, P.R, P.f, P.lambda);
    std::fprintf(fh, "grid       dx_in = %.9g m, N = %lld (%.4g samples), zones (Eq. 3) = %lld\n", P.dx,
                 (long long)P.N, samples, (long long)P.total_zones);
    std::fprintf(fh, "ROI        M = %d, pitch = %.9g m, x0 = %.9g m\n", M, P.p, P.x0);
    std::fprintf(fh, "form       %s, %s\n\n", form, prec);
    std::fprintf(fh, "FWHM x     %.9g m   Airy %.9g m (%+.3e)   / zone width %.6f\n", m.fwhm_x, fwhm_airy,
                 m.fwhm_x / fwhm_airy - 1.0, m.fwhm_x / zone_width);
    std::fprintf(fh, "FWHM y     %.9g m   Airy %.9g m (%+.3e)\n", m.fwhm_y, fwhm_airy, m.fwhm_y / fwhm_airy - 1.0);
    std::fprintf(fh, "DE lobe    %.9f   ladder EE(r_null) eta = %.9f (%+.3e)\n", m.de_lobe, de_ref,
                 m.de_lobe / de_ref - 1.0);
    std::fprintf(fh, "DE ROI     %.9f\n", m.de_roi);
    std::fprintf(fh, "P_in       %.9g m^2 (%lld samples); pi R^2 = %.9g m^2\n", m.p_in, (long long)m.aperture_count,
                 m.p_in_disc);
    std::fprintf(fh, "Strehl     %.9f\n", m.strehl);
    std::fprintf(fh, "MTF        %.9f at nu_cut/2 (clear pupil %.7f)\n", m.mtf_half_cut, kMtfHalf);
    std::fprintf(fh, "time       propagation %.6f s (%.4g Gsamples/s)\n", t_propagate_s,
                 t_propagate_s > 0 ? samples / t_propagate_s / 1e9 : 0.0);
    if (std::fclose(fh) != 0) return set_error(FZP_E_INVALID, "short write to %s", f_txt.c_str());
  }
  {
    FILE* fh = std::fopen(f_json.c_str(), "w");
    if (!fh) return set_error(FZP_E_INVALID, "cannot write %s: %s", f_json.c_str(), std::strerror(errno));
    std::fprintf(fh, "{\"library\": \"%s\", \"tag\": \"%s\", \"result\": \"result_%s.npy\",\n", fzp_version(),
                 t.c_str(), t.c_str());
    std::fprintf(fh, " \"config\": {\"plate\": \"%s\", \"levels\": %d, \"D\": %.17g, \"R_eff\": %.17g, \"f\": %.17g, "
                 "\"lambda\": %.17g, \"dx\": %.17g, \"N\": %lld, \"total_zones\": %lld, \"M\": %d, \"pitch\": %.17g, "
                 "\"x0\": %.17g, \"form\": \"%s\", \"precision\": \"%s\"},\n",
                 plate, P.levels, P.D, P.R, P.f, P.lambda, P.dx, (long long)P.N, (long long)P.total_zones, M, P.p,
                 P.x0, form, prec);
    std::fprintf(fh, " \"metrics\": {\"fwhm_x\": %.17g, \"fwhm_y\": %.17g, \"de_lobe\": %.17g, \"de_roi\": %.17g, "
                 "\"p_in\": %.17g, \"p_in_disc\": %.17g, \"aperture_count\": %lld, \"peak\": %.17g, \"strehl\": %.17g, "
                 "\"mtf_half_cut\": %.17g, \"mtf16\": [",
                 m.fwhm_x, m.fwhm_y, m.de_lobe, m.de_roi, m.p_in, m.p_in_disc, (long long)m.aperture_count, m.peak,
                 m.strehl, m.mtf_half_cut);
    for (int q = 0; q < 16; ++q) std::fprintf(fh, "%s%.17g", q ? ", " : "", m.mtf16[q]);
    std::fprintf(fh, "]},\n");
    std::fprintf(fh, " \"references\": {\"fwhm_airy\": %.17g, \"zone_width\": %.17g, \"fwhm_over_airy_minus_1\": %.17g, "
                 "\"fwhm_over_zone_width\": %.17g, \"de_lobe_ladder\": %.17g, \"first_order_efficiency\": %.17g, "
                 "\"de_lobe_over_ladder_minus_1\": %.17g, \"mtf_half_cut_clear_pupil\": %.17g},\n",
                 fwhm_airy, zone_width, m.fwhm_x / fwhm_airy - 1.0, m.fwhm_x / zone_width, de_ref, eta,
                 m.de_lobe / de_ref - 1.0, kMtfHalf);
    std::fprintf(fh, " \"timing\": {\"propagate_s\": %.9g, \"samples\": %.17g, \"gsamples_per_s\": %.9g}}\n",
                 t_propagate_s, samples, t_propagate_s > 0 ? samples / t_propagate_s / 1e9 : 0.0);
    if (std::fclose(fh) != 0) return set_error(FZP_E_INVALID, "short write to %s", f_json.c_str());
  }
  if (out) *out = m;
  return FZP_OK;
}
