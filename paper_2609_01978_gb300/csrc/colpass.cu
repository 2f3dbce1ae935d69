// colpass.cu -- column pass, cross-stripe FP64 accumulation and output
// epilogue (Fig. 2 Stage 3 "column czt * dx_in^2/(lambda0 f)"; Fig. 18 Stage 4
// "output chirp and Fresnel prefactor").
//
//   Uacc[n, m] += sum_{j in rows} K[n, j] C[j, m]            (column pass)
//   U[n, m]     = Pre e^{i pi (x_m^2 + y_n^2)/(lambda f)} Uacc[n, m],
//   Pre         = e^{i k f} dx^2 / (i lambda f)              (Eq. 2)
//
// K[n, j] = exp(2 pi i (A_j - n B_j)) with A_j = dj^2 kappa/2 + msh dj delta and
// B_j = dj delta (turns, dj = j - c).  A_j and B_j are reduced in FP64 once per
// row j; for the FP32 path B_j is split as hi + lo with hi a multiple of 2^-14
// so that n * hi is exact in FP32 for n < 1024.
#include <cmath>

#include "fzp_internal.cuh"

namespace fzp {
namespace {

constexpr int TN = 64, TM = 64, TJ = 16, JC = 2048;

struct ColArgs {
  int64_t c, j0, rows, c1_stride;
  int M;
  double kappa, delta;
  double msh;     // ROI shift in pitches: y_n = (n - msh) p
  double wr, wi;  // weight of this pass's field (1, 0 for a single-pass plate)
};

template <typename R> struct RowPhase;
template <> struct RowPhase<float> { float fa, hi, lo; };
template <> struct RowPhase<double> { double a, b; };

__device__ __forceinline__ void row_phase(const ColArgs& g, int64_t j, RowPhase<float>& rp) {
  const double dj = (double)(j - g.c);
  const double A = dj * dj * (0.5 * g.kappa) + g.msh * dj * g.delta;
  const double fb = frac_turns(dj * g.delta);
  const double hi = rint(fb * 16384.0) / 16384.0;
  rp.fa = (float)frac_turns(A);
  rp.hi = (float)hi;
  rp.lo = (float)(fb - hi);
}
__device__ __forceinline__ void row_phase(const ColArgs& g, int64_t j, RowPhase<double>& rp) {
  const double dj = (double)(j - g.c);
  rp.a = frac_turns(dj * dj * (0.5 * g.kappa) + g.msh * dj * g.delta);
  rp.b = frac_turns(dj * g.delta);
}

__device__ __forceinline__ float2 kern(const RowPhase<float>& rp, int n) {
  const float x = (float)n * rp.hi;
  const float t = rp.fa - (x - floorf(x)) - (float)n * rp.lo;
  float s, c;
  sincospif(2.0f * t, &s, &c);
  return make_float2(c, s);
}
__device__ __forceinline__ double2 kern(const RowPhase<double>& rp, int n) {
  return cis_turns_d(rp.a - (double)n * rp.b);
}

// grid (M/TM, M/TN, ceil(rows/JC)); 256 threads; each thread 4 n x 4 m outputs.
template <typename R>
__global__ void __launch_bounds__(256) k_colpass(ColArgs g, const R* __restrict__ C1, double2* __restrict__ Uacc) {
  using C = typename Cplx<R>::T;
  __shared__ C sK[TJ][TN + 1];
  __shared__ C sC[TJ][TM + 1];
  __shared__ RowPhase<R> sP[TJ];
  const int m0 = blockIdx.x * TM, n0 = blockIdx.y * TN;
  const int64_t jb = (int64_t)blockIdx.z * JC;
  const int64_t je = jb + JC < g.rows ? jb + JC : g.rows;
  const int tid = threadIdx.x;
  const int tn = tid >> 4, tm = tid & 15;  // 16 x 16 threads, 4 x 4 outputs each
  C acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) { acc[a][b].x = 0; acc[a][b].y = 0; }
  for (int64_t j = jb; j < je; j += TJ) {
    if (tid < TJ) {
      RowPhase<R> rp;
      row_phase(g, g.j0 + j + tid, rp);
      sP[tid] = rp;
    }
    // C tile: TJ rows x TM columns (j contiguous in C1)
    for (int t = tid; t < TJ * TM; t += 256) {
      const int jj = t % TJ, mm = t / TJ;
      const int m = m0 + mm;
      C v;
      v.x = 0; v.y = 0;
      if (j + jj < je) {
        v.x = C1[(int64_t)c1_row_re(m) * g.c1_stride + j + jj];
        v.y = C1[(int64_t)c1_row_im(m) * g.c1_stride + j + jj];
      }
      sC[jj][mm] = v;
    }
    __syncthreads();
    for (int t = tid; t < TJ * TN; t += 256) {
      const int jj = t / TN, nn = t % TN;
      C k;
      k.x = 0; k.y = 0;
      if (j + jj < je) k = kern(sP[jj], n0 + nn);
      sK[jj][nn] = k;
    }
    __syncthreads();
#pragma unroll 4
    for (int jj = 0; jj < TJ; ++jj) {
      C kv[4], cv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) kv[a] = sK[jj][tn + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) cv[b] = sC[jj][tm + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          acc[a][b].x = fma(kv[a].x, cv[b].x, fma(-kv[a].y, cv[b].y, acc[a][b].x));
          acc[a][b].y = fma(kv[a].x, cv[b].y, fma(kv[a].y, cv[b].x, acc[a][b].y));
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int n = n0 + tn + 16 * a, m = m0 + tm + 16 * b;
      const double ux = (double)acc[a][b].x, uy = (double)acc[a][b].y;
      atomicAdd(&Uacc[(int64_t)n * g.M + m].x, g.wr * ux - g.wi * uy);
      atomicAdd(&Uacc[(int64_t)n * g.M + m].y, g.wr * uy + g.wi * ux);
    }
}

__global__ void k_epilogue(int M, double msh, double p, double lf, double f_over_lambda, double amp,
                           const double2* __restrict__ Uacc, double2* __restrict__ out, int accumulate) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= M * M) return;
  const int n = t / M, m = t % M;
  const double xm = (double)m - msh, yn = (double)n - msh;
  // e^{ikf} (1/i) e^{i pi (x^2 + y^2)/(lambda f)}: turns f/lambda - 1/4 + (x^2 + y^2)/(2 lambda f)
  const double ph = frac_turns(f_over_lambda) - 0.25 + (xm * xm + yn * yn) * (p * p) / (2.0 * lf);
  double2 w = cis_turns_d(ph);
  w.x *= amp;
  w.y *= amp;
  const double2 u = Uacc[t];
  double2 v = make_double2(w.x * u.x - w.y * u.y, w.x * u.y + w.y * u.x);
  if (accumulate) {
    v.x += out[t].x;
    v.y += out[t].y;
  }
  out[t] = v;
}

__global__ void k_intensity(int64_t count, const double2* __restrict__ U, double* __restrict__ I) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < count) I[t] = U[t].x * U[t].x + U[t].y * U[t].y;
}

}  // namespace

fzp_status column_pass(Plan& P, int64_t j0, int64_t rows, cudaStream_t s) {
  ColArgs g{P.c, j0, rows, P.chunk_rows, P.M, P.kappa, P.delta, P.msh, 1.0, 0.0};
  if (P.pass_index >= 0) {
    g.wr = P.passes[P.pass_index].wr;
    g.wi = P.passes[P.pass_index].wi;
  }
  dim3 grid((unsigned)(P.M / TM), (unsigned)(P.M / TN), (unsigned)((rows + JC - 1) / JC));
  if (P.precision == FZP_PREC_FP64) k_colpass<double><<<grid, 256, 0, s>>>(g, P.d_C1d, P.d_Uacc);
  else k_colpass<float><<<grid, 256, 0, s>>>(g, P.d_C1, P.d_Uacc);
  P.launches += 1;
  FZP_CUDA_TRY(cudaGetLastError());
  return FZP_OK;
}

fzp_status epilogue(Plan& P, void* d_field, int accumulate, cudaStream_t s) {
  const double lf = P.lambda * P.f;
  const int count = P.M * P.M;
  k_epilogue<<<(count + 255) / 256, 256, 0, s>>>(P.M, P.msh, P.p, lf, P.f / P.lambda, P.dx2 / lf, P.d_Uacc,
                                                 reinterpret_cast<double2*>(d_field), accumulate);
  P.launches += 1;
  FZP_CUDA_TRY(cudaGetLastError());
  return FZP_OK;
}

fzp_status epilogue_z(Plan& P, void* d_field, int accumulate, double z, cudaStream_t s) {
  const double lz = P.lambda * z;
  const int count = P.M * P.M;
  k_epilogue<<<(count + 255) / 256, 256, 0, s>>>(P.M, P.msh, P.p, lz, P.f / P.lambda, P.dx2 / lz, P.d_Uacc,
                                                 reinterpret_cast<double2*>(d_field), accumulate);
  P.launches += 1;
  FZP_CUDA_TRY(cudaGetLastError());
  return FZP_OK;
}

fzp_status intensity(Plan& P, const void* d_field, void* d_I, cudaStream_t s) {
  const int64_t count = (int64_t)P.M * P.M;
  k_intensity<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(count, reinterpret_cast<const double2*>(d_field),
                                                               reinterpret_cast<double*>(d_I));
  P.launches += 1;
  FZP_CUDA_TRY(cudaGetLastError());
  return FZP_OK;
}

}  // namespace fzp
