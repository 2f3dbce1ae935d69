// batch.cu -- autotuner and batched execution of many apertures.
//
// Autotuner: for FZP_PREC_AUTO_1E4 (any arithmetic whose ROI-intensity error is
// <= 1e-4) it builds the candidate plans -- the split-BF16 dense form with two
// accumulation-chunk lengths, and the FP32 Bluestein form (its partitioned
// convolution unless the request asks for conv = 1) -- times each on a
// probe stripe of central aperture rows sized to fill the GPU twice with dense
// work items, and keeps the fastest.  Deformed membranes (complex
// transmission) are dense candidates as binary amplitude plates (two membrane
// passes); odd-level phase plates and deformed phase plates have the
// Bluestein form only.  Results are cached
// per (N, M, deformed, levels, centre configuration, requested convolution)
// for the process and, when FZP_TUNE_CACHE names a file, in that file (one
// "key value..." line per problem).
//
// Batch: many apertures of different diameter, wavelength and deformation share
// one set of device buffers sized for the largest; every instance regenerates
// its form tables (chirps, FFT of the convolution chirp, or split-BF16 kernel
// tiles) inside the batch, so tables are never held for all instances at once.
// The whole batch -- per instance: tables, row passes, column pass, epilogue
// into the caller's field -- is captured once into a CUDA graph and replayed
// with a single cudaGraphLaunch.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "fzp_internal.cuh"

namespace fzp {

fzp_status validate_and_derive(const fzp_params* in, Plan& P);
fzp_status build_mask_tables(Plan& P);
int64_t chunk_rows_for(const Plan& P);
void disc_rows(const Plan& P, int64_t& jlo, int64_t& jhi);
void release_plan(Plan* P);

namespace {

struct Choice {
  int form, precision, promote, row_batch, cluster;
  double ms_probe;
};

std::mutex g_tune_mu;
std::map<std::string, Choice> g_tune;
bool g_tune_loaded = false;

// The request's Bluestein convolution is part of the key: a choice measured
// with the partitioned convolution does not hold for the single one.
std::string tune_key(int64_t N, int M, bool deformed, int levels, int centre_open, int conv) {
  char buf[112];
  snprintf(buf, sizeof(buf), "N=%lld,M=%d,deformed=%d,levels=%d,centre_open=%d,conv=%d", (long long)N, M,
           deformed ? 1 : 0, levels, centre_open, conv);
  return buf;
}

void tune_load() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  const char* path = getenv("FZP_TUNE_CACHE");
  if (!path) return;
  FILE* fh = fopen(path, "r");
  if (!fh) return;
  char key[96];
  Choice c;
  while (fscanf(fh, "%95s %d %d %d %d %d %lf", key, &c.form, &c.precision, &c.promote, &c.row_batch, &c.cluster,
                &c.ms_probe) == 7)
    g_tune[key] = c;
  fclose(fh);
}

void tune_store(const std::string& key, const Choice& c) {
  g_tune[key] = c;
  const char* path = getenv("FZP_TUNE_CACHE");
  if (!path) return;
  FILE* fh = fopen(path, "a");
  if (!fh) return;
  fprintf(fh, "%s %d %d %d %d %d %.6f\n", key.c_str(), c.form, c.precision, c.promote, c.row_batch, c.cluster,
          c.ms_probe);
  fclose(fh);
}

}  // namespace

// Times one candidate on the probe stripe; returns the plan (caller owns) or null.
static fzp_plan_t probe_candidate(const fzp_params& base, const Choice& c, double* ms) {
  fzp_params p = base;
  p.form = c.form;
  p.precision = c.precision;
  p.promote = c.promote;
  p.row_batch = c.row_batch;
  p.cluster = c.cluster;
  fzp_plan_t plan = nullptr;
  if (fzp_plan(&p, &plan) != FZP_OK) return nullptr;
  void* field = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  bool ok = cudaMalloc(&field, (size_t)p.M * p.M * 16) == cudaSuccess && cudaEventCreate(&e0) == cudaSuccess &&
            cudaEventCreate(&e1) == cudaSuccess;
  fzp_plan_info info;
  fzp_plan_info_get(plan, &info);
  // probe stripe: enough rows for two full waves of dense work items (one item =
  // 256 rows x one pair of 128-row kernel tiles) so that neither form is timed
  // on an under-filled GPU; centred rows carry the most zone boundaries
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t pairs = std::max<int64_t>(1, (2 * (int64_t)p.M / 128 + 1) / 2);
  const int64_t half = 128 * ((2 * sms + pairs - 1) / pairs);
  const int64_t j0 = std::max<int64_t>(0, info.c - half), j1 = std::min<int64_t>(info.N, info.c + half);
  float t = 0;
  if (ok) ok = fzp_propagate_roi(plan, j0, j1, field, 0, nullptr) == FZP_OK;  // warm
  if (ok) {
    cudaEventRecord(e0, 0);
    ok = fzp_propagate_roi(plan, j0, j1, field, 0, nullptr) == FZP_OK;
    cudaEventRecord(e1, 0);
    ok = ok && cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&t, e0, e1) == cudaSuccess;
  }
  if (field) cudaFree(field);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaGetLastError();
  if (!ok) {
    fzp_plan_destroy(plan);
    return nullptr;
  }
  *ms = t;
  return plan;
}

// Chooses form, precision and knobs for an FZP_PREC_AUTO_1E4 request.  If
// `keep` is non-null the winning candidate plan is returned through it.
fzp_status autotune(const fzp_params* in, fzp_params* chosen, fzp_plan_t* keep) {
  Plan geo;
  fzp_params probe = *in;
  probe.precision = FZP_PREC_FP32;
  probe.form = FZP_FORM_BLUESTEIN;
  fzp_status st = validate_and_derive(&probe, geo);
  if (st != FZP_OK) return st;
  const bool deformed = in->deform != nullptr;
  const std::string key = tune_key(geo.N, geo.M, deformed, geo.levels, geo.mg.centre_open, in->conv);
  *chosen = *in;
  std::lock_guard<std::mutex> lock(g_tune_mu);
  tune_load();
  auto hit = g_tune.find(key);
  if (hit != g_tune.end()) {
    chosen->form = hit->second.form;
    chosen->precision = hit->second.precision;
    chosen->promote = hit->second.promote;
    chosen->row_batch = hit->second.row_batch;
    chosen->cluster = hit->second.cluster;
    if (keep) return fzp_plan(chosen, keep);
    return FZP_OK;
  }
  std::vector<Choice> cands;
  // the dense form takes binary and even-level plates, and deformed binary
  // amplitude plates (membrane passes with split mask values)
  if (!deformed && geo.levels % 2 == 0) {
    // cluster 0: the plan's own choice (4 CTAs for M = 512); 1: single-CTA kernel
    cands.push_back({FZP_FORM_DENSE, FZP_PREC_SPLIT_BF16, 128, 0, 0, 0});
    cands.push_back({FZP_FORM_DENSE, FZP_PREC_SPLIT_BF16, 256, 0, 0, 0});
    cands.push_back({FZP_FORM_DENSE, FZP_PREC_SPLIT_BF16, 128, 0, 1, 0});
  } else if (deformed && geo.levels == 0) {
    // membrane passes are limited by their generators: single CTAs and 2- and
    // 4-CTA clusters (small ROIs padded) trade generator share per CTA against
    // peer copies and padded tiles; measured, the single CTA wins at M = 128
    cands.push_back({FZP_FORM_DENSE, FZP_PREC_SPLIT_BF16, 128, 0, 1, 0});
    cands.push_back({FZP_FORM_DENSE, FZP_PREC_SPLIT_BF16, 128, 0, 2, 0});
    cands.push_back({FZP_FORM_DENSE, FZP_PREC_SPLIT_BF16, 128, 0, 4, 0});
  }
  cands.push_back({FZP_FORM_BLUESTEIN, FZP_PREC_FP32, 0, 0, 0, 0});
  fzp_plan_t best = nullptr;
  Choice bc{};
  double bms = 1e300;
  for (Choice& c : cands) {
    double ms = 0;
    fzp_plan_t p = probe_candidate(*in, c, &ms);
    if (!p) continue;
    c.ms_probe = ms;
    if (ms < bms) {
      if (best) fzp_plan_destroy(best);
      best = p;
      bms = ms;
      bc = c;
    } else {
      fzp_plan_destroy(p);
    }
  }
  if (!best) return set_error(FZP_E_CUDA, "autotune: no candidate ran (%s)", key.c_str());
  tune_store(key, bc);
  chosen->form = bc.form;
  chosen->precision = bc.precision;
  chosen->promote = bc.promote;
  chosen->row_batch = bc.row_batch;
  chosen->cluster = bc.cluster;
  if (keep) *keep = best;
  else fzp_plan_destroy(best);
  return FZP_OK;
}

}  // namespace fzp

using namespace fzp;

struct fzp_batch_s {
  std::vector<fzp_plan_s*> inst;
  std::vector<void*> buffers;  // shared device buffers (owned)
  cudaStream_t cap = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<void*> fields;   // fields the graph was captured with
  size_t device_bytes = 0;
};

static void batch_release(fzp_batch_s* b) {
  if (!b) return;
  cudaDeviceSynchronize();
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->cap) cudaStreamDestroy(b->cap);
  for (fzp_plan_s* p : b->inst) {
    release_plan(p);
    delete p;
  }
  for (void* q : b->buffers)
    if (q) cudaFree(q);
  delete b;
}

extern "C" {

fzp_status fzp_batch_plan(const fzp_params* params, int n, fzp_batch_t* out) {
  if (!out) return set_error(FZP_E_INVALID, "out is NULL");
  *out = nullptr;
  if (!params || n <= 0) return set_error(FZP_E_INVALID, "need n >= 1 parameter sets");
  fzp_batch_s* b = new (std::nothrow) fzp_batch_s();
  if (!b) return set_error(FZP_E_OOM, "host allocation failed");
  FormSizes mx;
  size_t c1 = 0, c1d = 0, uacc = 0, metr = 0;
  for (int i = 0; i < n; ++i) {
    fzp_params p = params[i];
    if (p.precision == FZP_PREC_AUTO_1E4) {
      fzp_params chosen;
      fzp_status st = autotune(&p, &chosen, nullptr);
      if (st != FZP_OK) { batch_release(b); return st; }
      p = chosen;
    }
    if (p.form == FZP_FORM_SACZT) {
      batch_release(b);
      return set_error(FZP_E_UNSUPPORTED, "instance %d: the SA-CZT form does not run in batches", i);
    }
    fzp_plan_s* P = new (std::nothrow) fzp_plan_s();
    if (!P) { batch_release(b); return set_error(FZP_E_OOM, "host allocation failed"); }
    P->owns_buffers = false;
    b->inst.push_back(P);
    fzp_status st = validate_and_derive(&p, *P);
    if (st == FZP_OK) st = build_mask_tables(*P);
    if (st != FZP_OK) {
      batch_release(b);
      return set_error(st, "instance %d: %s", i, fzp_last_error());
    }
    P->chunk_rows = chunk_rows_for(*P);
    P->c1_rows = (2 * (int64_t)P->M + 511) / 512 * 512;
    FormSizes z;
    st = P->form == FZP_FORM_DENSE ? dense_layout(*P, &z) : bluestein_layout(*P, &z);
    if (st != FZP_OK) { batch_release(b); return st; }
    mx.pre = std::max(mx.pre, z.pre); mx.H = std::max(mx.H, z.H); mx.tab = std::max(mx.tab, z.tab);
    mx.Z = std::max(mx.Z, z.Z); mx.G = std::max(mx.G, z.G); mx.A = std::max(mx.A, z.A);
    mx.sched = std::max(mx.sched, z.sched);
    const size_t rowsC1 = (size_t)((2 * (int64_t)P->M + 511) / 512 * 512) * (size_t)P->chunk_rows;
    if (P->precision == FZP_PREC_FP64) c1d = std::max(c1d, rowsC1 * 8);
    else c1 = std::max(c1, rowsC1 * 4);
    uacc = std::max(uacc, (size_t)P->M * P->M * sizeof(double2));
    metr = std::max(metr, 8192 * sizeof(double) + (size_t)P->M * P->M * sizeof(double2));
  }
  auto alloc = [&](size_t bytes) -> void* {
    if (!bytes) return nullptr;
    void* q = nullptr;
    if (cudaMalloc(&q, bytes) != cudaSuccess) return nullptr;
    b->buffers.push_back(q);
    b->device_bytes += bytes;
    return q;
  };
  void *pre = alloc(mx.pre), *H = alloc(mx.H), *tab = alloc(mx.tab), *Z = alloc(mx.Z), *G = alloc(mx.G),
       *A = alloc(mx.A), *sched = alloc(mx.sched), *C1 = alloc(c1), *C1d = alloc(c1d), *U = alloc(uacc), *M = alloc(metr),
       *err = alloc(sizeof(int));
  if ((mx.pre && !pre) || (mx.H && !H) || (mx.tab && !tab) || (mx.Z && !Z) || (mx.G && !G) || (mx.A && !A) ||
      (mx.sched && !sched) ||
      (c1 && !C1) || (c1d && !C1d) || !U || !M || !err) {
    cudaGetLastError();
    batch_release(b);
    return set_error(FZP_E_OOM, "batch workspace allocation failed");
  }
  if (cudaMemset(err, 0, sizeof(int)) != cudaSuccess) { batch_release(b); return set_error(FZP_E_CUDA, "memset"); }
  for (fzp_plan_s* P : b->inst) {
    P->bs.d_pre = pre; P->bs.d_H = H; P->bs.d_tab = tab; P->bs.d_Z = Z; P->bs.d_G = G;
    P->dn.d_A = A;
    P->dn.d_sched = reinterpret_cast<int*>(sched);
    P->d_C1 = reinterpret_cast<float*>(C1);
    P->d_C1d = reinterpret_cast<double*>(C1d);
    P->d_Uacc = reinterpret_cast<double2*>(U);
    P->d_metrics = reinterpret_cast<double*>(M);
    P->d_err = reinterpret_cast<int*>(err);
    P->device_bytes = 0;
  }
  if (cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess) {
    batch_release(b);
    return set_error(FZP_E_CUDA, "stream creation failed");
  }
  *out = b;
  return FZP_OK;
}

// Enqueue instance i on stream s: tables, rows, column pass, epilogue.
static fzp_status batch_enqueue(Plan& P, void* field, cudaStream_t s) {
  fzp_status st = P.form == FZP_FORM_DENSE ? dense_fill_tables(P, s) : bluestein_fill_tables(P, s);
  if (st != FZP_OK) return st;
  FZP_CUDA_TRY(cudaMemsetAsync(P.d_Uacc, 0, (size_t)P.M * P.M * sizeof(double2), s));
  int64_t jlo, jhi;
  disc_rows(P, jlo, jhi);
  for (int64_t j0 = jlo; j0 < jhi; j0 += P.chunk_rows) {
    const int64_t rows = std::min(P.chunk_rows, jhi - j0);
    st = chunk_passes(P, j0, rows, s);
    if (st != FZP_OK) return st;
  }
  return epilogue(P, field, 0, s);
}

fzp_status fzp_batch_propagate(fzp_batch_t b, void* const* d_fields, void* stream) {
  if (!b || !d_fields) return set_error(FZP_E_INVALID, "NULL batch or fields");
  for (size_t i = 0; i < b->inst.size(); ++i)
    if (!d_fields[i]) return set_error(FZP_E_INVALID, "field %zu is NULL", i);
  const bool same = b->exec && std::equal(b->fields.begin(), b->fields.end(), d_fields);
  if (!same) {
    if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
    if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
    FZP_CUDA_TRY(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
    fzp_status st = FZP_OK;
    for (size_t i = 0; i < b->inst.size() && st == FZP_OK; ++i) st = batch_enqueue(*b->inst[i], d_fields[i], b->cap);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(b->cap, &g);
    if (st != FZP_OK) {
      if (g) cudaGraphDestroy(g);
      return st;
    }
    if (e != cudaSuccess) return set_error(FZP_E_CUDA, "graph capture: %s", cudaGetErrorString(e));
    b->graph = g;
    FZP_CUDA_TRY(cudaGraphInstantiate(&b->exec, b->graph, 0));
    b->fields.assign(d_fields, d_fields + b->inst.size());
  }
  FZP_CUDA_TRY(cudaGraphLaunch(b->exec, (cudaStream_t)stream));
  return FZP_OK;
}

fzp_status fzp_batch_info(fzp_batch_t b, int i, fzp_plan_info* out) {
  if (!b || !out || i < 0 || i >= (int)b->inst.size()) return set_error(FZP_E_INVALID, "bad batch index");
  fzp_status st = fzp_plan_info_get(b->inst[i], out);
  out->device_bytes = b->device_bytes;
  return st;
}

fzp_status fzp_batch_metrics(fzp_batch_t b, int i, const void* d_field, void* stream, fzp_metrics_t* out) {
  if (!b || !d_field || !out || i < 0 || i >= (int)b->inst.size())
    return set_error(FZP_E_INVALID, "bad batch index or NULL argument");
  return metrics(*b->inst[i], d_field, (cudaStream_t)stream, out);
}

fzp_status fzp_batch_intensity(fzp_batch_t b, int i, const void* d_field, void* d_intensity, void* stream) {
  if (!b || !d_field || !d_intensity || i < 0 || i >= (int)b->inst.size())
    return set_error(FZP_E_INVALID, "bad batch index or NULL argument");
  return intensity(*b->inst[i], d_field, d_intensity, (cudaStream_t)stream);
}

fzp_status fzp_batch_kernels(fzp_batch_t b, int64_t* kernels) {
  if (!b || !kernels) return set_error(FZP_E_INVALID, "NULL argument");
  *kernels = 0;
  if (!b->graph) return FZP_OK;
  size_t n = 0;
  FZP_CUDA_TRY(cudaGraphGetNodes(b->graph, nullptr, &n));
  std::vector<cudaGraphNode_t> nodes(n);
  FZP_CUDA_TRY(cudaGraphGetNodes(b->graph, nodes.data(), &n));
  for (cudaGraphNode_t nd : nodes) {
    cudaGraphNodeType t;
    FZP_CUDA_TRY(cudaGraphNodeGetType(nd, &t));
    if (t == cudaGraphNodeTypeKernel) ++*kernels;
  }
  return FZP_OK;
}

fzp_status fzp_batch_destroy(fzp_batch_t b) {
  batch_release(b);
  return FZP_OK;
}

}  // extern "C"
