// bluestein.cu -- form (a): row chirp-z transform by Bluestein's identity
// (Sec. 2.6; Eq. 9-10; Fig. 2 Stage 3; Fig. 18 Stage 3 "row Bluestein at fixed
// length nfft"), with FFTs written here.
//
// For aperture row j the row transform is
//   C[j, m] = sum_i x_i K[m, i],  x_i = T[j, i] e^{i phi[j, i]},
//   K[m, i] = exp(2 pi i theta(m, i)),  theta = di^2 kappa/2 - (m - msh) di delta
// (msh = -x0/p: M/2 for the ROI centred on the focus).
// With m i = (m^2 + i^2 - (m - i)^2) / 2 (Bluestein):
//   theta(m, i) = pre(i) + post(m) + delta (m - i)^2 / 2,
//   pre(i)  = di^2 kappa/2 - delta i^2/2 + delta msh i,
//   post(m) = -delta m^2/2 + delta m c - delta msh c,
// so C[j, .] = e^{2 pi i post} .* (y * h)[0..M) with y_i = x_i e^{2 pi i pre(i)} and
// the chirp h_k = e^{i pi delta k^2}, k in (-N, M): one linear convolution of
// length >= N + M - 1, done as FFT_L, pointwise product with FFT_L(h), IFFT_L.
//
// Large L is split four-step (Bailey, ref. [24] of the paper), L = L1 * L2,
// n = L2 n1 + n2, k = k1 + L1 k2:
//   pass F1 (L1 > 1): for each column n2 an L1-point FFT over n1, times e^{-2 pi i n2 k1 / L}
//   pass F2         : for each row k1 an L2-point FFT over n2 -> Y[k1 + L1 k2],
//                     times H, L2-point inverse FFT; only m < M outputs kept,
//                     times e^{+2 pi i k1 m / L}
//   pass F3 (L1 > 1): sum over k1, times e^{2 pi i post(m)} / L -> row intermediate.
// The mask and the input chirp are generated inside F1 (or F2 when L1 = 1):
// the aperture is never stored.
//
// FP32 default (fzp_params.conv): the same convolution partitioned into
// 4096-point blocks, each row on chip from its mask to its M outputs
// (k_seg, below); the four-step passes above remain the FP64 path and the
// single-convolution FP32 option.
#include <algorithm>
#include <cmath>

#include "fzp_internal.cuh"

namespace fzp {
namespace {

template <typename R> struct Traits;
template <> struct Traits<float> { static constexpr int L2MAX = 4096; };  // radix-16 pass kernel
template <> struct Traits<double> { static constexpr int L2MAX = 4096; };

__host__ __device__ inline int ilog2(int64_t v) { int r = 0; while ((1ll << r) < v) ++r; return r; }

__device__ __forceinline__ int brev(int v, int bits) { return (int)(__brev((unsigned)v) >> (32 - bits)); }

template <typename C> __device__ __forceinline__ C conjc(C a) { a.y = -a.y; return a; }

// Batched in-place radix-2 DIT: `batch` transforms of length n = 2^logn, column
// c at x + c * colstride; input in bit-reversed order, output natural; forward sign.
// tw[t] = e^{-2 pi i t / twN}.
template <typename C>
__device__ void dit(C* x, int logn, int batch, const C* __restrict__ tw, int twN, int colstride) {
  const int n = 1 << logn, nb = (n >> 1) * batch;
  for (int s = 1; s <= logn; ++s) {
    const int half = 1 << (s - 1);
    const int stride = twN >> s;
    for (int t = threadIdx.x; t < nb; t += blockDim.x) {
      const int col = t >> (logn - 1), b = t & ((n >> 1) - 1);
      const int k = b & (half - 1);
      const int i0 = col * colstride + ((b >> (s - 1)) << s) + k, i1 = i0 + half;
      const C w = tw[k * stride];
      const C a = x[i0], v = cmul(x[i1], w);
      x[i0] = cadd(a, v);
      x[i1] = csub(a, v);
    }
    __syncthreads();
  }
}

// The same transform with two radix-2 stages per pass (radix 2^2): each work
// item takes the four elements k, k + h, k + 2h, k + 3h of a group of 4h
// (h = 2^(s-1)), applies stage s to the pairs (0,1), (2,3) and stage s + 1 to
// (0,2), (1,3) in registers; a single radix-2 stage finishes odd lengths.
// tws[t] = e^{-2 pi i t / n} for t < n / 2, in shared memory.
template <typename C>
__device__ void dit22(C* x, int logn, int batch, const C* tws, int colstride) {
  const int n = 1 << logn;
  int s = 1;
  for (; s + 1 <= logn; s += 2) {
    const int h = 1 << (s - 1);
    const int items = (n >> 2) * batch;
    for (int t = threadIdx.x; t < items; t += blockDim.x) {
      const int col = t >> (logn - 2), g = t & ((n >> 2) - 1);
      const int k = g & (h - 1);
      const int i0 = col * colstride + ((g >> (s - 1)) << (s + 1)) + k;
      const C w1 = tws[k << (logn - s)];
      const C w2 = tws[k << (logn - s - 1)], w3 = tws[(k + h) << (logn - s - 1)];
      C a0 = x[i0], a1 = x[i0 + h], a2 = x[i0 + 2 * h], a3 = x[i0 + 3 * h];
      const C v1 = cmul(a1, w1), v3 = cmul(a3, w1);
      const C b0 = cadd(a0, v1), b1 = csub(a0, v1), b2 = cadd(a2, v3), b3 = csub(a2, v3);
      const C u2 = cmul(b2, w2), u3 = cmul(b3, w3);
      x[i0] = cadd(b0, u2);
      x[i0 + 2 * h] = csub(b0, u2);
      x[i0 + h] = cadd(b1, u3);
      x[i0 + 3 * h] = csub(b1, u3);
    }
    __syncthreads();
  }
  if (s == logn) {  // one radix-2 stage left
    const int h = 1 << (s - 1);
    const int items = (n >> 1) * batch;
    for (int t = threadIdx.x; t < items; t += blockDim.x) {
      const int col = t >> (logn - 1), b = t & ((n >> 1) - 1);
      const int k = b & (h - 1);
      const int i0 = col * colstride + ((b >> (s - 1)) << s) + k;
      const C w = tws[k << (logn - s)];
      const C a0 = x[i0], v = cmul(x[i0 + h], w);
      x[i0] = cadd(a0, v);
      x[i0 + h] = csub(a0, v);
    }
    __syncthreads();
  }
}

// In-place radix-2 DIF, natural input, bit-reversed output, inverse sign (no 1/n).
template <typename C>
__device__ void dif_inverse(C* x, int logn, const C* __restrict__ tw, int twN) {
  const int n = 1 << logn, nb = n >> 1;
  for (int s = logn; s >= 1; --s) {
    const int half = 1 << (s - 1);
    const int stride = twN >> s;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
      const int k = b & (half - 1);
      const int i0 = ((b >> (s - 1)) << s) + k, i1 = i0 + half;
      const C w = conjc(tw[k * stride]);
      const C a = x[i0], v = x[i1];
      x[i0] = cadd(a, v);
      x[i1] = cmul(csub(a, v), w);
    }
    __syncthreads();
  }
}

struct RowArgs {
  MaskGeom mg;
  int64_t N, L, L1, L2;
  int logL1, logL2, M;
  int64_t j0;        // first aperture row of this launch
  int64_t rows;      // rows in this launch
  int B, logB;       // columns per F1 block (a power of two)
  int has_deform;
  fzp_deform def;
  double dx, R, inv_lambda;
  // the deformation phase in turns, 2 w / lambda, as FP32 coefficients:
  //   amp2 sin(2 pi (di kx + dj ky)) (1 - tq (di^2 + dj^2)) + sum_k h2_k exp(-q_k d_k^2),
  //   d_k = (di - pi_k) nx_k + (dj - pj_k) ny_k  (sample units; (pi_k, pj_k) on the crease)
  DeformCoef df;
  const void* pre;   // N
  const void* H;     // [L1][L2]
  void* Z;           // [rows][L1][L2]
  void* G;           // [rows][L1][M]
  const void* post;  // M, includes 1/L
  const void* tw;    // twN entries: e^{-2 pi i t / twN}
  const void* twL;   // 4096 entries: e^{-2 pi i t / L}
  int twN;
  void* C1;          // [2M][c1_stride]
  int64_t c1_stride; // row length of C1
  int64_t c1_j0;     // aperture row of C1 column 0
  const void* vin;   // input sequence for the table-building mode (length L)
  int S;             // partitioned convolution: columns per block
  int64_t nseg;      // partitioned convolution: blocks per row (spectra in H)
};

// Aperture transmission of sample (j, i): T e^{i phi}, optional deformation.
template <typename R>
__device__ __forceinline__ typename Cplx<R>::T aperture(const RowArgs& a, int64_t j, int64_t i) {
  typename Cplx<R>::T v;
  v.x = 0; v.y = 0;
  if (i >= a.N) return v;
  const int64_t dj = j - a.mg.c, di = i - a.mg.c, s = dj * dj + di * di;
  if (s > a.mg.sR) return v;
  const int64_t z = zone_of(s, a.mg);
  if (a.mg.levels >= 2) {
    // L-level phase plate: e^{-2 pi i q / L}, q = zone mod L (Fig. 18 Stage 3)
    // fewer than 2^24 zone steps (a plan limit): a 32-bit remainder
    const int q = (int)((uint32_t)z % (uint32_t)a.mg.levels);
    if (sizeof(R) == 4) {
      // FP32 form: -q / L turns lies in (-1, 0], so FP32 carries it to within
      // an ulp without the FP64 reduction
      float sn, cs;
      sincospif(-2.0f * (float)q / (float)a.mg.levels, &sn, &cs);
      v.x = cs;
      v.y = sn;
    } else {
      v = cis_turns<R>(-(double)q / (double)a.mg.levels);
    }
    if (!a.has_deform) return v;
  } else {
    if (((z ^ a.mg.centre_open) & 1) == 0) return v;  // binary amplitude: odd zones open (even: positive-centred)
    v.x = 1;
    if (!a.has_deform) return v;
  }
  if (sizeof(R) == 4) {
    // FP32 form: the phase is at most about a turn, so FP32 coefficients
    // (relative error ~1e-7 of it) are far inside the form's tolerance
    const float fi = (float)di, fj = (float)dj;
    // turns of the wrinkle: |di| < 2^20 and kxh a multiple of 2^-14 with few
    // significant bits, so di kxh is exact and its integer part drops exactly
    const float th = fi * a.df.kxh + fj * a.df.kyh;
    const float tt = (th - rintf(th)) + (fi * a.df.kxl + fj * a.df.kyl);
    float wz = a.df.amp2 * sinpif(2.0f * (tt - rintf(tt))) * (1.0f - a.df.tq * (fi * fi + fj * fj));
    for (int k = 0; k < a.df.n; ++k) {
      const float d = (fi - a.df.pi_[k]) * a.df.nx[k] + (fj - a.df.pj[k]) * a.df.ny[k];
      wz += a.df.h2[k] * __expf(-a.df.q[k] * d * d);
    }
    // wz - rint(wz) is exact in FP32, so the reduction adds nothing to wz's
    // own rounding (the FP64 reduction of the same FP32 value gave the same)
    float sn, cs;
    sincospif(2.0f * (wz - rintf(wz)), &sn, &cs);
    typename Cplx<R>::T e;
    e.x = cs;
    e.y = sn;
    return cmul(v, e);
  }
  const double u = (double)(i - a.mg.c) * a.dx, w = (double)(j - a.mg.c) * a.dx;
  const fzp_deform& d = a.def;
  const double tt = (u * cos(d.theta) + w * sin(d.theta)) / d.period;  // turns
  const double r2 = (u * u + w * w) / (a.R * a.R);
  double wz = d.amp * sinpi(2.0 * frac_turns(tt)) * (1.0 - d.taper * r2);
  for (int k = 0; k < d.n_ridges; ++k) {
    const double dist = (u - d.ridge_px[k]) * (-sin(d.ridge_alpha[k])) + (w - d.ridge_py[k]) * cos(d.ridge_alpha[k]);
    const double sg = d.ridge_width[k] / (2.0 * sqrt(2.0 * log(2.0)));
    wz += d.ridge_h[k] * exp(-dist * dist / (2.0 * sg * sg));
  }
  return cmul(v, cis_turns<R>(2.0 * wz * a.inv_lambda));  // phi / (2 pi) = 2 w / lambda
}

// e^{sign 2 pi i t / L} for 0 <= t < L = L1 * L2 from two tables:
// t = th * 4096 + tl, W_L^t = W_{L1}^{th} W_L^{tl}, W_{L1}^{th} = tw[th * (twN / L1)].
template <typename R>
__device__ __forceinline__ typename Cplx<R>::T twiddle_L(const RowArgs& a, int64_t t, bool conj) {
  using C = typename Cplx<R>::T;
  if (a.L <= 4096) {
    C w = reinterpret_cast<const C*>(a.twL)[t];
    if (conj) w.y = -w.y;
    return w;
  }
  const int64_t th = t >> 12, tl = t & 4095;
  C w1 = reinterpret_cast<const C*>(a.tw)[th * (a.twN / a.L1)];
  C w2 = reinterpret_cast<const C*>(a.twL)[tl];
  C w = cmul(w1, w2);
  if (conj) w.y = -w.y;
  return w;
}

// mode 0: generate y = aperture * pre; mode 1: read the table input `vin`.
template <typename R>
__global__ void __launch_bounds__(256) k_f1(RowArgs a, int mode) {
  using C = typename Cplx<R>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* sm = reinterpret_cast<C*>(smem_raw);
  const int B = a.B;
  const int64_t r = blockIdx.y;
  const int64_t j = a.j0 + r;
  const int64_t n2_0 = (int64_t)blockIdx.x * B;
  const int L1 = (int)a.L1;
  const C* pre = reinterpret_cast<const C*>(a.pre);
  const C* vin = reinterpret_cast<const C*>(a.vin);
  C* tws = sm + (L1 + 1) * B;  // L1 / 2 twiddles of the column FFT
  for (int t = threadIdx.x; t < (L1 >> 1); t += blockDim.x)
    tws[t] = reinterpret_cast<const C*>(a.tw)[t * (a.twN / L1)];
  // load, bit-reversed within each column
  for (int t = threadIdx.x; t < L1 * B; t += blockDim.x) {
    const int n1 = t >> a.logB, b = t & (B - 1);
    const int64_t n = (int64_t)n1 * a.L2 + n2_0 + b;
    C x;
    if (mode == 0) {
      x = aperture<R>(a, j, n);
      if (x.x != 0 || x.y != 0) x = cmul(x, pre[n]);
    } else {
      x = vin[n];
    }
    sm[b * (L1 + 1) + brev(n1, a.logL1)] = x;  // odd column stride: no bank conflicts across columns
  }
  __syncthreads();
  dit22(sm, a.logL1, B, tws, L1 + 1);
  C* Z = reinterpret_cast<C*>(a.Z) + r * a.L;
  for (int t = threadIdx.x; t < L1 * B; t += blockDim.x) {
    const int k1 = t >> a.logB, b = t & (B - 1);
    const int64_t n2 = n2_0 + b;
    const C w = twiddle_L<R>(a, n2 * k1, false);
    Z[(int64_t)k1 * a.L2 + n2] = cmul(sm[b * (L1 + 1) + k1], w);
  }
}

// mode 0: full row transform; mode 1: forward FFT only, result -> Z as [k1][k2].
template <typename R>
__global__ void __launch_bounds__(512) k_f2(RowArgs a, int mode) {
  using C = typename Cplx<R>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* sm = reinterpret_cast<C*>(smem_raw);
  const int64_t k1 = blockIdx.x;
  const int64_t r = blockIdx.y;
  const int64_t j = a.j0 + r;
  const int L2 = (int)a.L2;
  const C* tw = reinterpret_cast<const C*>(a.tw);
  const C* pre = reinterpret_cast<const C*>(a.pre);
  if (a.L1 == 1) {
    const C* vin = reinterpret_cast<const C*>(a.vin);
    for (int n = threadIdx.x; n < L2; n += blockDim.x) {
      C x;
      if (mode == 0) {
        x = aperture<R>(a, j, n);
        if (x.x != 0 || x.y != 0) x = cmul(x, pre[n]);
      } else {
        x = vin[n];
      }
      sm[brev(n, a.logL2)] = x;
    }
  } else {
    const C* Z = reinterpret_cast<const C*>(a.Z) + r * a.L + k1 * a.L2;
    for (int n = threadIdx.x; n < L2; n += blockDim.x) sm[brev(n, a.logL2)] = Z[n];
  }
  __syncthreads();
  dit(sm, a.logL2, 1, tw, a.twN, (int)a.L2);
  if (mode == 1) {
    C* out = reinterpret_cast<C*>(a.Z) + r * a.L + k1 * a.L2;
    for (int k = threadIdx.x; k < L2; k += blockDim.x) out[k] = sm[k];
    return;
  }
  const C* H = reinterpret_cast<const C*>(a.H) + k1 * a.L2;
  for (int k = threadIdx.x; k < L2; k += blockDim.x) sm[k] = cmul(sm[k], H[k]);
  __syncthreads();
  dif_inverse(sm, a.logL2, tw, a.twN);
  if (a.L1 == 1) {
    // finalize directly: C = post(m) * z[m]  (post includes 1/L)
    const C* post = reinterpret_cast<const C*>(a.post);
    R* C1 = reinterpret_cast<R*>(a.C1);
    const int64_t jl = j - a.c1_j0;
    for (int m = threadIdx.x; m < a.M; m += blockDim.x) {
      const C v = cmul(sm[brev(m, a.logL2)], post[m]);
      C1[(int64_t)c1_row_re(m) * a.c1_stride + jl] = v.x;
      C1[(int64_t)c1_row_im(m) * a.c1_stride + jl] = v.y;
    }
    return;
  }
  C* G = reinterpret_cast<C*>(a.G) + (r * a.L1 + k1) * a.M;
  for (int m = threadIdx.x; m < a.M; m += blockDim.x) {
    G[m] = cmul(sm[brev(m, a.logL2)], twiddle_L<R>(a, (k1 * m) & (a.L - 1), true));
  }
}

// ---------------------------------------------------------------- FP32 pass F2, radix 16
constexpr int RL = 4096;  // inner FFT length of the FP32 four-step split

__device__ __forceinline__ void dft4(float2& a0, float2& a1, float2& a2, float2& a3, bool inv) {
  const float2 s02 = make_float2(a0.x + a2.x, a0.y + a2.y), d02 = make_float2(a0.x - a2.x, a0.y - a2.y);
  const float2 s13 = make_float2(a1.x + a3.x, a1.y + a3.y), d13 = make_float2(a1.x - a3.x, a1.y - a3.y);
  const float2 t = inv ? make_float2(-d13.y, d13.x) : make_float2(d13.y, -d13.x);  // (+/-i) d13
  a0 = make_float2(s02.x + s13.x, s02.y + s13.y);
  a2 = make_float2(s02.x - s13.x, s02.y - s13.y);
  a1 = make_float2(d02.x + t.x, d02.y + t.y);
  a3 = make_float2(d02.x - t.x, d02.y - t.y);
}

// ---------------------------------------------------------------- FP32 pass F2, radix 8
// L2 = 4096 = 8^4 points, 512 threads x 8 values in registers, Stockham
// order (pass s, Ns = 8^s: x_r = in[j + 512 r] times W_{8 Ns}^{r k}, k = j mod
// Ns, 8-point DFT, y_q -> out[(j / Ns) 8 Ns + q Ns + k]).  After the forward
// passes thread j holds Y[j + 512 q], the layout the inverse's first pass
// reads, so the product with H needs no exchange; the inverse's last pass
// (Ns = 512) evaluates only the outputs q < ceil(M / 512) it keeps.  Shared
// memory (padded one element per 8 against bank conflicts) carries the three
// exchanges of each transform.  Twiddles: W^k, W^{2k}, W^{4k} from the table,
// the other four by products.
constexpr int R8T = 512;
__device__ __forceinline__ int pidx8(int i) { return i + (i >> 3); }

__device__ __forceinline__ void dft8(float2 (&v)[8], bool inv) {
  // radix 2 x 4: two 4-point DFTs on the even and odd inputs, then W_8^q
  float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  float2 o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  dft4(e0, e1, e2, e3, inv);
  dft4(o0, o1, o2, o3, inv);
  const float h = 0.70710678118654752f;
  // o_q times W_8^{q} (forward e^{-2 pi i q / 8}; inverse conjugate)
  const float sg = inv ? 1.0f : -1.0f;
  float2 t1 = make_float2(h * (o1.x - sg * o1.y), h * (o1.y + sg * o1.x));  // W^1
  float2 t2 = make_float2(-sg * o2.y, sg * o2.x);                           // W^2 = -+i
  float2 t3 = make_float2(h * (-o3.x - sg * o3.y), h * (-o3.y + sg * o3.x)); // W^3
  v[0] = make_float2(e0.x + o0.x, e0.y + o0.y);
  v[4] = make_float2(e0.x - o0.x, e0.y - o0.y);
  v[1] = make_float2(e1.x + t1.x, e1.y + t1.y);
  v[5] = make_float2(e1.x - t1.x, e1.y - t1.y);
  v[2] = make_float2(e2.x + t2.x, e2.y + t2.y);
  v[6] = make_float2(e2.x - t2.x, e2.y - t2.y);
  v[3] = make_float2(e3.x + t3.x, e3.y + t3.y);
  v[7] = make_float2(e3.x - t3.x, e3.y - t3.y);
}

// v[r] *= W_{8 Ns}^{r k} (forward) or its conjugate; tw[t] = e^{-2 pi i t / 4096}.
__device__ __forceinline__ void twiddle8(float2 (&v)[8], int k, int step, const float2* __restrict__ tw, bool inv) {
  if (k == 0) return;
  float2 w1 = __ldg(tw + k * step), w2 = __ldg(tw + 2 * k * step), w4 = __ldg(tw + 4 * k * step);
  if (inv) { w1.y = -w1.y; w2.y = -w2.y; w4.y = -w4.y; }
  const float2 w3 = cmul(w1, w2), w5 = cmul(w1, w4), w6 = cmul(w2, w4), w7 = cmul(w3, w4);
  v[1] = cmul(v[1], w1); v[2] = cmul(v[2], w2); v[3] = cmul(v[3], w3); v[4] = cmul(v[4], w4);
  v[5] = cmul(v[5], w5); v[6] = cmul(v[6], w6); v[7] = cmul(v[7], w7);
}

// One Stockham pass with the exchange that feeds the next: twiddle, DFT,
// scatter to shared memory, gather the next pass's inputs.
__device__ __forceinline__ void r8_pass(float2 (&v)[8], float2* sm, int Ns, const float2* __restrict__ tw, bool inv) {
  const int j = threadIdx.x;
  const int k = j & (Ns - 1);
  twiddle8(v, k, 512 / Ns, tw, inv);
  dft8(v, inv);
  const int base = (j / Ns) * 8 * Ns + k;
#pragma unroll
  for (int q = 0; q < 8; ++q) sm[pidx8(base + q * Ns)] = v[q];
  __syncthreads();
#pragma unroll
  for (int q = 0; q < 8; ++q) v[q] = sm[pidx8(j + R8T * q)];
  __syncthreads();
}

// mode 0: row transform; mode 1: forward FFT only, natural order -> Z row (table build).
__global__ void __launch_bounds__(R8T, 2) k_f2_r8(RowArgs a, int mode) {
  __shared__ float2 sm[RL + RL / 8];
  const int j = threadIdx.x;
  const int64_t k1 = blockIdx.x, r = blockIdx.y, row = a.j0 + r;
  const float2* tw = reinterpret_cast<const float2*>(a.tw);
  float2 v[8];
  if (a.L1 == 1) {
    const float2* pre = reinterpret_cast<const float2*>(a.pre);
    const float2* vin = reinterpret_cast<const float2*>(a.vin);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int n = j + R8T * q;
      if (mode == 0) {
        float2 x = aperture<float>(a, row, n);
        if (x.x != 0.f || x.y != 0.f) x = cmul(x, pre[n]);
        v[q] = x;
      } else {
        v[q] = vin[n];
      }
    }
  } else {
    const float2* Z = reinterpret_cast<const float2*>(a.Z) + r * a.L + k1 * RL;
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = Z[j + R8T * q];
  }
  // forward: passes Ns = 1, 8, 64 with exchanges, then Ns = 512 in registers
  r8_pass(v, sm, 1, tw, false);
  r8_pass(v, sm, 8, tw, false);
  r8_pass(v, sm, 64, tw, false);
  twiddle8(v, j, 1, tw, false);
  dft8(v, false);  // thread j now holds Y[j + 512 q] in v[q]
  if (mode == 1) {
    float2* out = reinterpret_cast<float2*>(a.Z) + r * a.L + k1 * RL;
#pragma unroll
    for (int q = 0; q < 8; ++q) out[q * R8T + j] = v[q];
    return;
  }
  const float2* H = reinterpret_cast<const float2*>(a.H) + k1 * RL;
#pragma unroll
  for (int q = 0; q < 8; ++q) v[q] = cmul(v[q], __ldg(H + q * R8T + j));
  // inverse: passes Ns = 1, 8, 64, then the kept outputs of Ns = 512
  r8_pass(v, sm, 1, tw, true);
  r8_pass(v, sm, 8, tw, true);
  r8_pass(v, sm, 64, tw, true);
  twiddle8(v, j, 1, tw, true);
  // outputs m = q * 512 + j < M: y_q = sum_r v_r W_8^{-r q} (inverse sign)
  const int nq = (a.M + R8T - 1) / R8T;
  float2 y[2];
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    y[q] = make_float2(0.f, 0.f);
    if (q < nq) {
#pragma unroll
      for (int rr = 0; rr < 8; ++rr) {
        float sn, cs;
        // W_8^{-r q} = e^{+2 pi i r q / 8}: exact for r q mod 8 in {0, 2, 4, 6}; 1/sqrt(2) otherwise
        const int t = (rr * q) & 7;
        const float h = 0.70710678118654752f;
        const float ct[8] = {1.f, h, 0.f, -h, -1.f, -h, 0.f, h};
        const float st[8] = {0.f, h, 1.f, h, 0.f, -h, -1.f, -h};
        cs = ct[t];
        sn = st[t];
        y[q].x += v[rr].x * cs - v[rr].y * sn;
        y[q].y += v[rr].x * sn + v[rr].y * cs;
      }
    }
  }
  if (a.L1 == 1) {
    const float2* post = reinterpret_cast<const float2*>(a.post);
    float* C1 = reinterpret_cast<float*>(a.C1);
    const int64_t jl = row - a.c1_j0;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int m = q * R8T + j;
      if (q < nq && m < a.M) {
        const float2 z = cmul(y[q], post[m]);
        C1[(int64_t)c1_row_re(m) * a.c1_stride + jl] = z.x;
        C1[(int64_t)c1_row_im(m) * a.c1_stride + jl] = z.y;
      }
    }
    return;
  }
  float2* G = reinterpret_cast<float2*>(a.G) + (r * a.L1 + k1) * a.M;
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int m = q * R8T + j;
    if (q < nq && m < a.M) G[m] = cmul(y[q], twiddle_L<float>(a, (k1 * m) & (a.L - 1), true));
  }
}

// Sum over k1; tile of 32 rows x 32 m; writes C1 coalesced along rows.
template <typename R>
__global__ void __launch_bounds__(256) k_f3(RowArgs a) {
  using C = typename Cplx<R>::T;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 8 warps
  const int m0 = blockIdx.x * 32;
  const int64_t r0 = (int64_t)blockIdx.y * 32;
  __shared__ C tile[32][33];
  const C* G = reinterpret_cast<const C*>(a.G);
  for (int rr = ty; rr < 32; rr += 8) {
    const int64_t r = r0 + rr;
    C acc;
    acc.x = 0; acc.y = 0;
    if (r < a.rows)
      for (int64_t k1 = 0; k1 < a.L1; ++k1) acc = cadd(acc, G[(r * a.L1 + k1) * a.M + m0 + tx]);
    tile[rr][tx] = cmul(acc, reinterpret_cast<const C*>(a.post)[m0 + tx]);
  }
  __syncthreads();
  R* C1 = reinterpret_cast<R*>(a.C1);
  for (int mm = ty; mm < 32; mm += 8) {
    const int64_t r = r0 + tx;
    if (r >= a.rows) continue;
    const int m = m0 + mm;
    const int64_t jl = a.j0 + r - a.c1_j0;
    const C v = tile[tx][mm];
    C1[(int64_t)c1_row_re(m) * a.c1_stride + jl] = v.x;
    C1[(int64_t)c1_row_im(m) * a.c1_stride + jl] = v.y;
  }
}

// ---------------------------------------------------------------------------
// Partitioned convolution (FP32).  The row's convolution (y * h)[m], m < M, is
// a sum over blocks of S input columns, i in [i_s, i_s + S), i_s = s S.  With
// P = 4096 >= S + M - 1 a block's share is one P-point circular convolution of
// the zero-padded block with the chirp piece
//   g_s[q] = h_{q - i_s} (q < M),  g_s[q] = h_{q - P - i_s} (P - S < q < P),
// read at q = m < M: the two ranges hold every lag m - i the block needs and
// do not overlap.  The transform is linear, so a row needs one inverse
// transform of sum_s FFT_P(y_s) .* G_s, G_s = FFT_P(g_s) precomputed per block
// (the same for every row); blocks that miss the row's disc chord are skipped.
// A row's working set (the block, the spectrum sum, the transposes) stays in
// registers and shared memory.
//
// The P-point FFT: 256 threads, thread t holding elements t + 256 r, r < 16;
// P = 16 * 16 * 16 as three in-register 16-point DFTs with two shared-memory
// transposes (index t = a + 16 b + 256 r, frequency k = k0 + 16 c + 256 d):
//   pass A: over r -> k0, times e^{-2 pi i t k0 / P}
//   pass B: thread (a, k0) over b -> c, times e^{-2 pi i a c / 256}
//   pass C: thread (k0, c) over a -> d; thread t = k0 + 16 c then holds
//           X[t + 256 d], the same distribution as its input.
// ---------------------------------------------------------------------------
constexpr int SP = 4096;          // partition transform length
constexpr int STH = 256;          // threads per block
constexpr int SB0 = 256 * 17;     // transpose buffer A->B: [t][k0], row pitch 17
constexpr int SB1 = 16 * 273;     // transpose buffer B->C: [k0][c][a], pitches 273 and 17
constexpr int SBUF = SB1 > SB0 ? SB1 : SB0;
constexpr size_t SEG_SMEM = sizeof(float2) * (2 * SBUF + 15 * 256 + 256 + 64) + sizeof(uint32_t) * 512;
// row kernels: binary plate (chunk bits), phase plate (chunk zone steps),
// deformed binary plate (chunk bits and the membrane phasor), general
// transmission (a deformed phase plate)
enum { SEG_FLAT = 0, SEG_LEVELS = 1, SEG_MEMBRANE = 2, SEG_GENERAL = 3 };

// Membrane phasor e^{i phi} of the sample at (fi, fj) = (i - c, j - c) for the
// FP32 partitioned pass: phi / 2 pi = 2 w / lambda from the FP32 coefficients
// (the wrinkle's turns as in the transmission function: di kxh exact, its
// integer part dropped exactly), the wrinkle's turns and the total reduced to
// [-1/2, 1/2] before the hardware sine and cosine (absolute error below 4e-7
// each).  Row terms: fjkh = fj kyh, fjkl = fj kyl, fj2 = fj^2, cr[e] = (fj -
// pj_e) ny_e - pi_e nx_e, so a ridge's distance is fi nx_e + cr[e].
__device__ __forceinline__ float2 membrane_phasor(const DeformCoef& d, float fi, float fjkh, float fjkl, float fj2,
                                                  const float (&cr)[3]) {
  constexpr float TWO_PI = 6.28318530717958648f;
  const float th = fmaf(fi, d.kxh, fjkh);
  float tt = (th - rintf(th)) + fmaf(fi, d.kxl, fjkl);
  tt -= rintf(tt);
  float wz = d.amp2 * __sinf(TWO_PI * tt) * fmaf(-d.tq, fmaf(fi, fi, fj2), 1.0f);
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    if (e < d.n) {
      const float dd = fmaf(fi, d.nx[e], cr[e]);
      wz = fmaf(d.h2[e], __expf(-d.q[e] * dd * dd), wz);
    }
  }
  wz -= rintf(wz);
  float sn, cs;
  __sincosf(TWO_PI * wz, &sn, &cs);
  return make_float2(cs, sn);
}

// v e^{-2 pi i K / 16}
template <int K>
__device__ __forceinline__ float2 w16mul(float2 v) {
  constexpr float C1 = 0.923879532511286756f, S1 = 0.382683432365089772f, R2 = 0.707106781186547524f;
  if constexpr (K == 0) {
    return v;
  } else if constexpr (K == 4) {
    return make_float2(v.y, -v.x);
  } else if constexpr (K == 2) {
    return make_float2(R2 * (v.x + v.y), R2 * (v.y - v.x));
  } else if constexpr (K == 6) {
    return make_float2(R2 * (v.y - v.x), -R2 * (v.x + v.y));
  } else {
    constexpr float wr = K == 1 ? C1 : (K == 3 ? S1 : -C1);  // K = 1, 3, 9
    constexpr float wi = K == 1 ? -S1 : (K == 3 ? -C1 : S1);
    return make_float2(v.x * wr - v.y * wi, v.x * wi + v.y * wr);
  }
}

// Forward 4-point DFT in place.
__device__ __forceinline__ void dft4(float2& a0, float2& a1, float2& a2, float2& a3) {
  const float2 t0 = cadd(a0, a2), t1 = csub(a0, a2), t2 = cadd(a1, a3), t3 = csub(a1, a3);
  a0 = cadd(t0, t2);
  a2 = csub(t0, t2);
  a1 = make_float2(t1.x + t3.y, t1.y - t3.x);
  a3 = make_float2(t1.x - t3.y, t1.y + t3.x);
}

// x[k] <- sum_n x[n] e^{-2 pi i n k / 16}: n = q + 4 n1, k = p + 4 k1; 4-point
// DFTs over n1, twiddles e^{-2 pi i q p / 16}, 4-point DFTs over q.
__device__ __forceinline__ void dft16(float2 (&x)[16]) {
#pragma unroll
  for (int q = 0; q < 4; ++q) dft4(x[q], x[q + 4], x[q + 8], x[q + 12]);  // (q, p) at q + 4 p
  x[5] = w16mul<1>(x[5]);
  x[9] = w16mul<2>(x[9]);
  x[13] = w16mul<3>(x[13]);
  x[6] = w16mul<2>(x[6]);
  x[10] = w16mul<4>(x[10]);
  x[14] = w16mul<6>(x[14]);
  x[7] = w16mul<3>(x[7]);
  x[11] = w16mul<6>(x[11]);
  x[15] = w16mul<9>(x[15]);
#pragma unroll
  for (int p = 0; p < 4; ++p) dft4(x[4 * p], x[4 * p + 1], x[4 * p + 2], x[4 * p + 3]);  // (p, k1) at 4 p + k1
  float2 y[16];
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) y[p + 4 * k1] = x[4 * p + k1];
#pragma unroll
  for (int k = 0; k < 16; ++k) x[k] = y[k];
}

// Forward P-point DFT of the block distributed as v[r] = x[t + 256 r];
// on return v[d] = X[t + 256 d].  Two barriers; b0 and b1 alternate, so
// back-to-back calls need no further barrier.  twA[(k0 - 1) 256 + t] =
// e^{-2 pi i t k0 / P}, twB[c 16 + a] = e^{-2 pi i a c / 256}.
__device__ __forceinline__ void fft_p(float2 (&v)[16], float2* b0, float2* b1, const float2* twA,
                                      const float2* twB) {
  const int t = threadIdx.x;
  dft16(v);
#pragma unroll
  for (int k0 = 1; k0 < 16; ++k0) v[k0] = cmul(v[k0], twA[(k0 - 1) * 256 + t]);
#pragma unroll
  for (int k0 = 0; k0 < 16; ++k0) b0[t * 17 + k0] = v[k0];
  __syncthreads();
  {
    const int a = t & 15, k0 = t >> 4;
#pragma unroll
    for (int b = 0; b < 16; ++b) v[b] = b0[(a + 16 * b) * 17 + k0];
    dft16(v);
#pragma unroll
    for (int c = 1; c < 16; ++c) v[c] = cmul(v[c], twB[c * 16 + a]);
#pragma unroll
    for (int c = 0; c < 16; ++c) b1[k0 * 273 + c * 17 + a] = v[c];
  }
  __syncthreads();
  {
    const int k0 = t & 15, c = t >> 4;
#pragma unroll
    for (int a = 0; a < 16; ++a) v[a] = b1[k0 * 273 + c * 17 + a];
    dft16(v);
  }
}

__device__ __forceinline__ void seg_twiddles(float2* twA, float2* twB) {
  for (int e = threadIdx.x; e < 15 * 256; e += blockDim.x) {
    const int k0 = e / 256 + 1, th = e % 256;
    float sn, cs;
    sincospif(-(float)(th * k0) / 2048.0f, &sn, &cs);  // exact argument: th k0 < 2^12
    twA[e] = make_float2(cs, sn);
  }
  {
    const int c = threadIdx.x >> 4, a = threadIdx.x & 15;
    float sn, cs;
    sincospif(-(float)(a * c) / 128.0f, &sn, &cs);
    twB[threadIdx.x] = make_float2(cs, sn);
  }
  __syncthreads();
}

__device__ __forceinline__ int64_t isqrt_row(int64_t t) {
  int64_t b = (int64_t)sqrt((double)t);
  while (b > 0 && b * b > t) --b;
  while ((b + 1) * (b + 1) <= t) ++b;
  return b;
}

// Open bits of the 16 columns [x, x + 16) of a row (bit p: column x + p) of
// the binary plate, dj2 = dj^2.  Between the chunk's two ends the zone index
// steps through the boundaries m in (zn, zf] (zn, zf: the zones at the ends
// nearer to and farther from the axis, squared radius clamped into the
// disc); boundary m sits at distance a_m = ceil(sqrt(S_m - dj^2)) from the
// axis: at column c + a_m right of the axis (the zone reaches m there), at
// c - a_m + 1 left of it (the zone drops below m there).  With the chunk at
// distance d >= 128 from the axis, a_m = d + k, k in [1, 15] the smallest k
// with k (k + 2d) >= S_m - dj^2 - d^2 (below 30 d + 225: 32-bit); the
// estimate (S_m - dj^2 - d^2) / (2d) exceeds k by k^2 / (2d) < 1, and with
// FP32 rounding it lies within [k - 1, k + 2]: one step up and two down make
// k exact.  Chunks nearer the axis take the zone rule column by column.
// Columns outside the disc chord come out arbitrary (their input is zero).
__device__ __forceinline__ uint32_t chunk_bits(int64_t x, int64_t dj2, const MaskGeom& g) {
  const int64_t dr = x - g.c, dl = g.c - (x + 15);
  if (dr < 128 && dl < 128) {
    uint32_t bits = 0;
    for (int p = 0; p < 16; ++p) {
      const int64_t di = x + p - g.c, sq = dj2 + di * di;
      if (sq <= g.sR && ((zone_of(sq, g) ^ g.centre_open) & 1) != 0) bits |= 1u << p;
    }
    return bits;
  }
  const bool right = dr >= 128;
  const int64_t d = right ? dr : dl;
  const int64_t sn = dj2 + d * d, sf = dj2 + (d + 15) * (d + 15);
  const int64_t zn = zone_of(min(sn, g.sR), g), zf = zone_of(min(sf, g.sR), g);
  uint32_t bits = ((((right ? zn : zf) ^ g.centre_open) & 1) != 0) ? 0xFFFFu : 0u;  // parity at p = 0
  const float inv2d = 0.5f / (float)d;
  const int32_t td = (int32_t)(2 * d);
  for (int64_t m = zn + 1; m <= zf; ++m) {
    const int32_t D = (int32_t)(__ldg(g.thr + (m - 1)) - sn);
    int32_t k = __float2int_ru((float)D * inv2d);
    k += (k * (k + td) < D) ? 1 : 0;
    k -= (k > 0 && (k - 1) * (k - 1 + td) >= D) ? 1 : 0;
    k -= (k > 0 && (k - 1) * (k - 1 + td) >= D) ? 1 : 0;
    bits ^= (0xFFFFu << (right ? k : 16 - k)) & 0xFFFFu;
  }
  return bits;
}

// Zone steps of the 16 columns [x, x + 16) of a row of the phase plate:
// *z0 the zone at column x, *ud the columns at which the zone steps up
// (bits 0-15) or down (bits 16-31), so that z(x + p) = z0 + popc(up & m_p) -
// popc(down & m_p), m_p = bits 0..p.  Away from the axis the steps are the
// boundaries between the chunk's ends, placed by the window search of
// chunk_bits (all up right of the axis, all down left of it); within 128
// columns of it the zone rule runs column by column.  Returns false when two
// boundaries share a column (possible only at a sampling finer than one
// sample per level step); the caller then evaluates the zone rule per
// element.  Columns outside the disc come out arbitrary.
__device__ __forceinline__ bool chunk_zones(int64_t x, int64_t dj2, const MaskGeom& g, uint32_t* z0, uint32_t* ud) {
  const int64_t dr = x - g.c, dl = g.c - (x + 15);
  if (dr < 128 && dl < 128) {
    int64_t zp = zone_of(min(dj2 + dr * dr, g.sR), g);
    *z0 = (uint32_t)zp;
    uint32_t up = 0u, dn = 0u;
    for (int p = 1; p < 16; ++p) {
      const int64_t di = dr + p, z = zone_of(min(dj2 + di * di, g.sR), g);
      if (z == zp + 1) up |= 1u << p;
      else if (z == zp - 1) dn |= 1u << p;
      else if (z != zp) return false;
      zp = z;
    }
    *ud = up | (dn << 16);
    return true;
  }
  const bool right = dr >= 128;
  const int64_t d = right ? dr : dl;
  const int64_t sn = dj2 + d * d, sf = dj2 + (d + 15) * (d + 15);
  const int64_t zn = zone_of(min(sn, g.sR), g), zf = zone_of(min(sf, g.sR), g);
  const float inv2d = 0.5f / (float)d;
  const int32_t td = (int32_t)(2 * d);
  uint32_t ev = 0u;
  for (int64_t m = zn + 1; m <= zf; ++m) {
    const int32_t D = (int32_t)(__ldg(g.thr + (m - 1)) - sn);
    int32_t k = __float2int_ru((float)D * inv2d);
    k += (k * (k + td) < D) ? 1 : 0;
    k -= (k > 0 && (k - 1) * (k - 1 + td) >= D) ? 1 : 0;
    k -= (k > 0 && (k - 1) * (k - 1 + td) >= D) ? 1 : 0;
    ev |= 1u << (right ? k : 16 - k);
  }
  if ((int64_t)__popc(ev) != zf - zn) return false;
  *z0 = (uint32_t)(right ? zn : zf);
  *ud = right ? ev : (ev << 16);
  return true;
}

// G_s = FFT_P(g_s) for every block s (one CTA per block, grid-strided).
__global__ void __launch_bounds__(STH) k_seg_tables(int64_t nseg, int S, int M, double delta, float2* G) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* b0 = reinterpret_cast<float2*>(smem_raw);
  float2* b1 = b0 + SBUF;
  float2* twA = b1 + SBUF;
  float2* twB = twA + 15 * 256;
  seg_twiddles(twA, twB);
  const int t = threadIdx.x;
  for (int64_t s = blockIdx.x; s < nseg; s += gridDim.x) {
    const int64_t is = s * (int64_t)S;
    float2 v[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      const int q = t + 256 * r;
      v[r] = make_float2(0.0f, 0.0f);
      int64_t k = 0;
      bool have = false;
      if (q < M) { k = q - is; have = true; }
      else if (q > SP - S) { k = (int64_t)q - SP - is; have = true; }
      if (have) {
        const double kk = (double)k;  // |k| < 2^24: k^2 exact in FP64
        v[r] = cis_turns<float>(0.5 * delta * kk * kk);
      }
    }
    fft_p(v, b0, b1, twA, twB);
    float2* out = G + s * SP + t;
#pragma unroll
    for (int d = 0; d < 16; ++d) out[256 * d] = v[d];
  }
}

// Row pass of the partitioned convolution: rows j0 + r, r = blockIdx.x,
// blockIdx.x + gridDim.x, ... (interleaved, so every CTA gets rows from the
// whole range of chord lengths); writes C1 like k_f3.  The transmission of a
// block's samples: SEG_FLAT, binary amplitude plate without deformation, open
// bits per chunk of 16 columns (chunk_bits); SEG_LEVELS, phase plate without
// deformation, zone steps per chunk (chunk_zones) and the level's phasor from
// a table; SEG_GENERAL, the transmission function per sample (membrane
// phase).  A block's input chirp loads are issued together before the
// transmission is evaluated, and the spectra G_s before the last FFT pass,
// so each waits one memory latency.
template <int MODE>
__global__ void __launch_bounds__(STH, 2) k_seg(RowArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* b0 = reinterpret_cast<float2*>(smem_raw);
  float2* b1 = b0 + SBUF;
  float2* twA = b1 + SBUF;
  float2* twB = twA + 15 * 256;
  float2* phs = twB + 256;                             // SEG_LEVELS: e^{-2 pi i q / L}, q < L <= 64
  uint32_t* mk = reinterpret_cast<uint32_t*>(phs + 64);  // per chunk: open bits, or zone at its first column
  uint32_t* mk2 = mk + 256;                             // per chunk: zone steps up | down << 16
  const uint32_t nlev = (uint32_t)max(a.mg.levels, 1);
  const uint32_t lmagic = 0xFFFFFFFFu / nlev + 1u;     // z / L = umulhi(z, ceil(2^32 / L)) for z < 2^24
  if (MODE == SEG_LEVELS && threadIdx.x < nlev) {
    float sn, cs;
    sincospif(-2.0f * (float)threadIdx.x / (float)nlev, &sn, &cs);
    phs[threadIdx.x] = make_float2(cs, sn);
  }
  seg_twiddles(twA, twB);
  const int t = threadIdx.x;
  const float2* pre = reinterpret_cast<const float2*>(a.pre);
  const float2* Gs = reinterpret_cast<const float2*>(a.H);
  const float2* post = reinterpret_cast<const float2*>(a.post);
  float* C1 = reinterpret_cast<float*>(a.C1);
  const int S = a.S, RS = a.S / 256;
  const float scale = (float)a.L / (float)SP;  // post carries 1/L; the inverse below is unnormalised
  for (int64_t r = blockIdx.x; r < a.rows; r += gridDim.x) {
    const int64_t j = a.j0 + r;
    const int64_t dj = j - a.mg.c;
    const int64_t rem = a.mg.sR - dj * dj;
    float2 acc[16];
#pragma unroll
    for (int d = 0; d < 16; ++d) acc[d] = make_float2(0.0f, 0.0f);
    if (rem >= 0) {
      const int64_t bmax = isqrt_row(rem);
      // the row's disc chord, within the grid (a given N may cut the disc)
      const int64_t lo = max(a.mg.c - bmax, (int64_t)0), hi = min(a.mg.c + bmax, a.N - 1);
      const int64_t s1 = hi / S;
      for (int64_t s = lo / S; s <= s1; ++s) {
        const int64_t is = s * (int64_t)S;
        float2 v[16];
        if (MODE == SEG_FLAT || MODE == SEG_MEMBRANE) {
          // the block's chord [olo, ohi] in block offsets; loads clamped into
          // the grid, every element's value decided by its bit alone
          const int olo = (int)max(lo - is, (int64_t)0), ohi = (int)min(hi - is, (int64_t)(S - 1));
          const int lim = (int)min(a.N - 1 - is, (int64_t)(SP - 1));
          const float2* pb = pre + is;
#pragma unroll
          for (int q = 0; q < 16; ++q) v[q] = __ldg(pb + min(t + 256 * q, lim));
          // thread t < S/16 makes the bits of block offsets 16 t ... 16 t + 15
          // (zero outside the chord and beyond S); element (t, q) is offset
          // 256 q + t: word 16 q + t/16, bit t % 16
          {
            const int xo = 16 * t;
            uint32_t w = 0u;
            if (t < S / 16 && xo + 15 >= olo && xo <= ohi) {
              w = chunk_bits(is + xo, dj * dj, a.mg);
              const int p0 = max(olo - xo, 0), p1 = min(ohi - xo, 15);  // chord within the chunk
              w &= (0xFFFFu >> (15 - p1 + p0)) << p0;
            }
            mk[t] = w;
          }
          __syncthreads();
#pragma unroll
          for (int q = 0; q < 16; ++q)
            if (((mk[16 * q + (t >> 4)] >> (t & 15)) & 1u) == 0) v[q] = make_float2(0.0f, 0.0f);
          if (MODE == SEG_MEMBRANE) {
            const float fj = (float)dj;
            const float fjkh = fj * a.df.kyh, fjkl = fj * a.df.kyl, fj2 = fj * fj;
            float cr[3];
#pragma unroll
            for (int e = 0; e < 3; ++e) cr[e] = (fj - a.df.pj[e]) * a.df.ny[e] - a.df.pi_[e] * a.df.nx[e];
            const float fi0 = (float)(is + t - a.mg.c);
#pragma unroll
            for (int q = 0; q < 16; ++q)
              if (v[q].x != 0.0f || v[q].y != 0.0f)
                v[q] = cmul(v[q], membrane_phasor(a.df, fi0 + 256.0f * q, fjkh, fjkl, fj2, cr));
          }
        } else if (MODE == SEG_LEVELS) {
          const int olo = (int)max(lo - is, (int64_t)0), ohi = (int)min(hi - is, (int64_t)(S - 1));
          const int lim = (int)min(a.N - 1 - is, (int64_t)(SP - 1));
          const float2* pb = pre + is;
#pragma unroll
          for (int q = 0; q < 16; ++q) v[q] = __ldg(pb + min(t + 256 * q, lim));
          // chunk t: zone at its first column (bit 31: evaluate per element) and its steps
          {
            const int xo = 16 * t;
            uint32_t z0 = 0u, ud = 0u;
            if (t < S / 16 && xo + 15 >= olo && xo <= ohi)
              if (!chunk_zones(is + xo, dj * dj, a.mg, &z0, &ud)) z0 = 0x80000000u;
            mk[t] = z0;
            mk2[t] = ud;
          }
          __syncthreads();
          const uint32_t mp = (2u << (t & 15)) - 1u;  // steps at or before this thread's column of a chunk
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            const int o = t + 256 * q;
            if ((unsigned)(o - olo) > (unsigned)(ohi - olo)) {
              v[q] = make_float2(0.0f, 0.0f);  // outside the chord (and beyond S)
              continue;
            }
            const uint32_t z0 = mk[16 * q + (t >> 4)], ud = mk2[16 * q + (t >> 4)];
            uint32_t z;
            if (z0 & 0x80000000u) {
              const int64_t di = is + o - a.mg.c;
              z = (uint32_t)zone_of(min(dj * dj + di * di, a.mg.sR), a.mg);
            } else {
              z = z0 + __popc(ud & mp) - __popc((ud >> 16) & mp);
            }
            const uint32_t lv = z - nlev * __umulhi(z, lmagic);
            v[q] = cmul(v[q], phs[lv]);
          }
        } else {
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            const int64_t i = is + t + 256 * q;
            v[q] = (q < RS && i >= lo && i <= hi) ? __ldg(pre + i) : make_float2(0.0f, 0.0f);
          }
#pragma unroll
          for (int q = 0; q < 16; ++q) {
            const int64_t i = is + t + 256 * q;
            if (q < RS && i >= lo && i <= hi) v[q] = cmul(aperture<float>(a, j, i), v[q]);
          }
        }
        // forward FFT (passes A and B), spectrum loads, pass C, product-sum
        dft16(v);
#pragma unroll
        for (int k0 = 1; k0 < 16; ++k0) v[k0] = cmul(v[k0], twA[(k0 - 1) * 256 + t]);
#pragma unroll
        for (int k0 = 0; k0 < 16; ++k0) b0[t * 17 + k0] = v[k0];
        __syncthreads();
        {
          const int aa = t & 15, k0 = t >> 4;
#pragma unroll
          for (int b = 0; b < 16; ++b) v[b] = b0[(aa + 16 * b) * 17 + k0];
          dft16(v);
#pragma unroll
          for (int c = 1; c < 16; ++c) v[c] = cmul(v[c], twB[c * 16 + aa]);
#pragma unroll
          for (int c = 0; c < 16; ++c) b1[k0 * 273 + c * 17 + aa] = v[c];
        }
        __syncthreads();
        float2 g[16];
        const float2* G = Gs + s * SP + t;
#pragma unroll
        for (int d = 0; d < 16; ++d) g[d] = __ldg(G + 256 * d);
        {
          const int k0 = t & 15, c = t >> 4;
#pragma unroll
          for (int aa = 0; aa < 16; ++aa) v[aa] = b1[k0 * 273 + c * 17 + aa];
          dft16(v);
        }
#pragma unroll
        for (int d = 0; d < 16; ++d) {
          acc[d].x = fmaf(v[d].x, g[d].x, fmaf(-v[d].y, g[d].y, acc[d].x));
          acc[d].y = fmaf(v[d].x, g[d].y, fmaf(v[d].y, g[d].x, acc[d].y));
        }
      }
    }
    // inverse transform as conj(FFT(conj(.))), outputs m = t + 256 d < M
#pragma unroll
    for (int d = 0; d < 16; ++d) acc[d].y = -acc[d].y;
    fft_p(acc, b0, b1, twA, twB);
    const int64_t jl = j - a.c1_j0;
#pragma unroll
    for (int d = 0; d < 4; ++d) {
      const int m = t + 256 * d;
      if (m < a.M) {
        const float2 y = cmul(make_float2(acc[d].x * scale, -acc[d].y * scale), post[m]);
        C1[(int64_t)c1_row_re(m) * a.c1_stride + jl] = y.x;
        C1[(int64_t)c1_row_im(m) * a.c1_stride + jl] = y.y;
      }
    }
  }
}

// Tables: pre(i), post(m)/L, convolution chirp v (length L), twiddles.
template <typename R>
__global__ void k_tables(int64_t N, int M, double msh, int64_t L, int64_t c, double kappa, double delta, void* pre,
                         void* post,
                         void* v, void* tw, int twN, void* twL) {
  using C = typename Cplx<R>::T;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < L; t += stride) {
    if (t < N) {
      const double di = (double)(t - c), ti = (double)t;
      const double ph = di * di * (0.5 * kappa) - (0.5 * delta) * (ti * ti) + delta * msh * ti;
      reinterpret_cast<C*>(pre)[t] = cis_turns<R>(ph);
    }
    if (t < M) {
      const double tm = (double)t;
      const double ph = -(0.5 * delta) * tm * tm + delta * tm * (double)c - delta * msh * (double)c;
      C z = cis_turns<R>(ph);
      z.x /= (R)L; z.y /= (R)L;
      reinterpret_cast<C*>(post)[t] = z;
    }
    // chirp h_k = e^{i pi delta k^2}: index k for k < M, index L - k for 0 < k < N
    C h;
    h.x = 0; h.y = 0;
    int64_t k = -1;
    if (t < M) k = t;
    else if (t > L - N) k = L - t;
    if (k >= 0) {
      const double kk = (double)k;
      h = cis_turns<R>(0.5 * delta * kk * kk);
    }
    reinterpret_cast<C*>(v)[t] = h;
    if (t < twN) reinterpret_cast<C*>(tw)[t] = twiddle<R>(t, twN, -1.0f);
    if (t < 4096) reinterpret_cast<C*>(twL)[t] = twiddle<R>(t, L, -1.0f);
  }
}

template <typename R>
static size_t f1_smem(const RowArgs& a) {
  return sizeof(typename Cplx<R>::T) * (size_t)((a.L1 + 1) * a.B + a.L1 / 2);
}

}  // namespace

DeformCoef deform_coef(const Plan& P) {
  DeformCoef c{};
  const fzp_deform& d = P.deform;
  const double k2 = 2.0 / P.lambda;  // metres -> turns of phase (phi / 2 pi = 2 w / lambda)
  const double kx = std::cos(d.theta) * P.dx / d.period, ky = std::sin(d.theta) * P.dx / d.period;
  c.kxh = (float)(std::rint(kx * 16384.0) / 16384.0);
  c.kyh = (float)(std::rint(ky * 16384.0) / 16384.0);
  c.kxl = (float)(kx - (double)c.kxh);
  c.kyl = (float)(ky - (double)c.kyh);
  c.amp2 = (float)(d.amp * k2);
  c.tq = (float)(d.taper * P.dx * P.dx / (P.R * P.R));
  c.zc = (float)std::cos(2.0 * M_PI * kx);
  c.zs = (float)std::sin(2.0 * M_PI * kx);
  c.n = d.n_ridges;
  for (int k = 0; k < d.n_ridges && k < 3; ++k) {
    const double nx = -std::sin(d.ridge_alpha[k]), ny = std::cos(d.ridge_alpha[k]);
    const double sg = d.ridge_width[k] / (2.0 * std::sqrt(2.0 * std::log(2.0)));
    c.nx[k] = (float)nx;
    c.ny[k] = (float)ny;
    c.pi_[k] = (float)(d.ridge_px[k] / P.dx);
    c.pj[k] = (float)(d.ridge_py[k] / P.dx);
    c.q[k] = (float)(P.dx * P.dx / (2.0 * sg * sg));
    c.h2[k] = (float)(d.ridge_h[k] * k2);
    c.rho[k] = (float)std::exp(-2.0 * (P.dx * P.dx / (2.0 * sg * sg)) * nx * nx);
  }
  return c;
}

namespace {

static RowArgs make_args(const Plan& P) {
  const Bluestein& b = P.bs;
  RowArgs a{};
  a.mg = P.mg;
  a.N = P.N; a.L = b.L; a.L1 = b.L1; a.L2 = b.L2; a.logL1 = ilog2(b.L1); a.logL2 = ilog2(b.L2); a.M = P.M;
  // F1 columns per block: a power of two, at most 16, F1 tile <= 64 KiB
  {
    const int64_t csz = P.precision == FZP_PREC_FP64 ? 16 : 8;
    int64_t B = 16;
    while (B > 1 && (B * (b.L1 + 1) + b.L1 / 2) * csz > 65536) B >>= 1;
    a.B = (int)std::min<int64_t>(B, b.L2);
    a.logB = ilog2(a.B);
  }
  a.has_deform = P.has_deform ? 1 : 0;
  a.def = P.deform;
  a.dx = P.dx; a.R = P.R; a.inv_lambda = 1.0 / P.lambda;
  if (P.has_deform) a.df = deform_coef(P);
  a.pre = b.d_pre; a.H = b.d_H; a.Z = b.d_Z; a.G = b.d_G; a.post = b.d_post; a.tw = b.d_tw;
  a.twN = (int)b.L2;
  a.twL = b.d_twL;
  a.c1_stride = P.chunk_rows;
  a.C1 = P.precision == FZP_PREC_FP64 ? (void*)P.d_C1d : (void*)P.d_C1;
  a.vin = b.d_tab;
  a.S = b.S;
  a.nseg = b.nseg;
  return a;
}

template <typename R>
fzp_status layout_t(Plan& P, FormSizes* out) {
  using C = typename Cplx<R>::T;
  Bluestein& b = P.bs;
  b.L = 1;
  while (b.L < P.N + P.M - 1) b.L <<= 1;
  b.L2 = b.L < Traits<R>::L2MAX ? b.L : Traits<R>::L2MAX;
  b.L1 = b.L / b.L2;
  if (P.M > b.L2) return set_error(FZP_E_UNSUPPORTED, "M larger than the inner FFT length");
  // the F1 twiddles are read from the L2-entry table with stride L2 / L1
  if (b.L1 > b.L2) return set_error(FZP_E_UNSUPPORTED, "FFT length %lld above %lld", (long long)b.L,
                                    (long long)b.L2 * b.L2);
  b.seg = (sizeof(R) == 4 && P.conv_req != 1) ? 1 : 0;
  if (b.seg) {
    // partitioned convolution: S + M - 1 <= 4096, S a multiple of 256 (at most 15 x 256)
    b.S = 256 * std::min(15, (4097 - P.M) / 256);
    b.nseg = (P.N + b.S - 1) / b.S;
    b.rows = P.chunk_rows;
    out->pre = sizeof(C) * P.N;
    out->H = sizeof(C) * (size_t)SP * (size_t)b.nseg;
    out->tab = sizeof(C) * (b.L + (int)b.L2 + P.M + 4096);
    out->Z = 0;
    out->G = 0;
    static std::atomic<uint64_t> attr_seg{0}, attr_segt{0};
    static std::atomic<uint64_t> attr_segl{0}, attr_segm{0}, attr_segg{0};
    FZP_CUDA_TRY(smem_attr_once((const void*)k_seg<SEG_FLAT>, (int)SEG_SMEM, attr_seg));
    FZP_CUDA_TRY(smem_attr_once((const void*)k_seg<SEG_LEVELS>, (int)SEG_SMEM, attr_segl));
    FZP_CUDA_TRY(smem_attr_once((const void*)k_seg<SEG_MEMBRANE>, (int)SEG_SMEM, attr_segm));
    FZP_CUDA_TRY(smem_attr_once((const void*)k_seg<SEG_GENERAL>, (int)SEG_SMEM, attr_segg));
    FZP_CUDA_TRY(smem_attr_once((const void*)k_seg_tables, (int)SEG_SMEM, attr_segt));
    return FZP_OK;
  }
  // rows per pass: requested, else a transform workspace of about 1 GiB
  const int64_t zbytes = (int64_t)sizeof(C) * b.L;
  int64_t rows = P.row_batch_req > 0 ? P.row_batch_req : (1ll << 30) / zbytes;
  if (b.L1 == 1) rows = P.row_batch_req > 0 ? P.row_batch_req : P.chunk_rows;
  b.rows = std::max<int64_t>(1, std::min<int64_t>(std::min<int64_t>(rows, P.chunk_rows), 65535));
  const int twN = (int)b.L2;
  out->pre = sizeof(C) * P.N;
  out->H = sizeof(C) * b.L;
  out->tab = sizeof(C) * (b.L + twN + P.M + 4096);
  out->Z = sizeof(C) * b.L * (b.L1 > 1 ? b.rows : 1);  // row 0 also serves the table build
  out->G = b.L1 > 1 ? sizeof(C) * b.L1 * P.M * b.rows : 0;
  // 64 KiB covers every FP32 case; FP64 at L1 = 4096 needs ~96 KiB
  static std::atomic<uint64_t> attr_f1{0}, attr_f2{0};
  FZP_CUDA_TRY(smem_attr_once((const void*)k_f1<R>, 200 * 1024, attr_f1));
  FZP_CUDA_TRY(smem_attr_once((const void*)k_f2<R>, (int)(sizeof(C) * Traits<R>::L2MAX), attr_f2));
  return FZP_OK;
}

template <typename R>
fzp_status fill_tables_t(Plan& P, cudaStream_t s) {
  using C = typename Cplx<R>::T;
  Bluestein& b = P.bs;
  const int twN = (int)b.L2;
  b.d_tw = reinterpret_cast<C*>(b.d_tab) + b.L;
  b.d_post = reinterpret_cast<C*>(b.d_tw) + twN;
  b.d_twL = reinterpret_cast<C*>(b.d_post) + P.M;
  k_tables<R><<<1024, 256, 0, s>>>(P.N, P.M, P.msh, b.L, P.c, P.kappa, P.delta, b.d_pre, b.d_post, b.d_tab, b.d_tw, twN,
                                   b.d_twL);
  FZP_CUDA_TRY(cudaGetLastError());
  if (b.seg) {
    const unsigned g = (unsigned)std::min<int64_t>(b.nseg, 1024);
    k_seg_tables<<<g, STH, SEG_SMEM, s>>>(b.nseg, b.S, P.M, P.delta, reinterpret_cast<float2*>(b.d_H));
    FZP_CUDA_TRY(cudaGetLastError());
    P.launches += 2;
    return FZP_OK;
  }
  // H = FFT_L(v) in the [k1][k2] order: F1 (table mode) + F2 (forward only) into Z row 0, then copy.
  RowArgs a = make_args(P);
  a.j0 = 0;
  a.rows = 1;
  if (b.L1 > 1) k_f1<R><<<dim3((unsigned)(b.L2 / a.B), 1), 256, f1_smem<R>(a), s>>>(a, 1);
  if (sizeof(R) == 4 && b.L2 == RL) k_f2_r8<<<dim3((unsigned)b.L1, 1), R8T, 0, s>>>(a, 1);
  else k_f2<R><<<dim3((unsigned)b.L1, 1), 512, sizeof(C) * b.L2, s>>>(a, 1);
  FZP_CUDA_TRY(cudaGetLastError());
  FZP_CUDA_TRY(cudaMemcpyAsync(b.d_H, b.d_Z, sizeof(C) * b.L, cudaMemcpyDeviceToDevice, s));
  P.launches += b.L1 > 1 ? 3 : 2;
  return FZP_OK;
}

template <typename R>
fzp_status build_tables_t(Plan& P) {
  Bluestein& b = P.bs;
  FormSizes z;
  fzp_status st = layout_t<R>(P, &z);
  if (st != FZP_OK) return st;
  FZP_CUDA_TRY(cudaMalloc(&b.d_pre, z.pre));
  FZP_CUDA_TRY(cudaMalloc(&b.d_H, z.H));
  FZP_CUDA_TRY(cudaMalloc(&b.d_tab, z.tab));
  if (z.Z) FZP_CUDA_TRY(cudaMalloc(&b.d_Z, z.Z));
  if (z.G) FZP_CUDA_TRY(cudaMalloc(&b.d_G, z.G));
  P.device_bytes += z.pre + z.H + z.tab + z.Z + z.G;
  return fill_tables_t<R>(P, 0);
}

template <typename R>
fzp_status rows_t(Plan& P, int64_t j0, int64_t rows, cudaStream_t s) {
  using C = typename Cplx<R>::T;
  const Bluestein& b = P.bs;
  RowArgs a = make_args(P);
  a.c1_j0 = j0;
  if (b.seg) {
    // resident CTAs only: each takes every gridDim.x-th row of the range
    int ctas_per_sm = 0, sms = 0, dev = 0;
    FZP_CUDA_TRY(cudaGetDevice(&dev));
    FZP_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int mode = P.has_deform ? (P.levels >= 2 ? SEG_GENERAL : SEG_MEMBRANE) : (P.levels >= 2 ? SEG_LEVELS : SEG_FLAT);
    const void* kern = mode == SEG_FLAT ? (const void*)k_seg<SEG_FLAT>
                       : mode == SEG_LEVELS ? (const void*)k_seg<SEG_LEVELS>
                       : mode == SEG_MEMBRANE ? (const void*)k_seg<SEG_MEMBRANE>
                                              : (const void*)k_seg<SEG_GENERAL>;
    FZP_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ctas_per_sm, kern, STH, SEG_SMEM));
    if (ctas_per_sm < 1) ctas_per_sm = 1;
    a.j0 = j0;
    a.rows = rows;
    const int64_t grid = std::min<int64_t>(rows, (int64_t)ctas_per_sm * sms);
    prof_begin(P, s);
    if (mode == SEG_FLAT) k_seg<SEG_FLAT><<<(unsigned)grid, STH, SEG_SMEM, s>>>(a);
    else if (mode == SEG_LEVELS) k_seg<SEG_LEVELS><<<(unsigned)grid, STH, SEG_SMEM, s>>>(a);
    else if (mode == SEG_MEMBRANE) k_seg<SEG_MEMBRANE><<<(unsigned)grid, STH, SEG_SMEM, s>>>(a);
    else k_seg<SEG_GENERAL><<<(unsigned)grid, STH, SEG_SMEM, s>>>(a);
    prof_end(P, s);
    P.launches += 1;
    FZP_CUDA_TRY(cudaGetLastError());
    return FZP_OK;
  }
  for (int64_t r0 = 0; r0 < rows; r0 += b.rows) {
    const int64_t rb = std::min<int64_t>(b.rows, rows - r0);
    a.j0 = j0 + r0;
    a.rows = rb;
    if (b.L1 > 1) {
      k_f1<R><<<dim3((unsigned)(b.L2 / a.B), (unsigned)rb), 256, f1_smem<R>(a), s>>>(a, 0);
      prof_begin(P, s);
      if (sizeof(R) == 4 && b.L2 == RL) k_f2_r8<<<dim3((unsigned)b.L1, (unsigned)rb), R8T, 0, s>>>(a, 0);
      else k_f2<R><<<dim3((unsigned)b.L1, (unsigned)rb), 512, sizeof(C) * b.L2, s>>>(a, 0);
      prof_end(P, s);
      k_f3<R><<<dim3((unsigned)(P.M / 32), (unsigned)((rb + 31) / 32)), 256, 0, s>>>(a);
      P.launches += 3;
    } else {
      prof_begin(P, s);
      if (sizeof(R) == 4 && b.L2 == RL) k_f2_r8<<<dim3(1, (unsigned)rb), R8T, 0, s>>>(a, 0);
      else k_f2<R><<<dim3(1, (unsigned)rb), 512, sizeof(C) * b.L2, s>>>(a, 0);
      prof_end(P, s);
      P.launches += 1;
    }
  }
  FZP_CUDA_TRY(cudaGetLastError());
  return FZP_OK;
}

__global__ void k_mask(MaskGeom mg, int64_t N, int64_t j0, int64_t rows, uint8_t* out) {
  const int64_t total = rows * N;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t / N, i = t % N;
    const int64_t dj = j0 + r - mg.c, di = i - mg.c, sq = dj * dj + di * di;
    if (mg.levels >= 2) out[t] = sq > mg.sR ? 0 : (uint8_t)(1 + zone_of(sq, mg) % mg.levels);
    else out[t] = mask_open(dj, di, mg) ? 1 : 0;
  }
}

}  // namespace

fzp_status bluestein_mask(Plan& P, int64_t j0, int64_t rows, uint8_t* out, cudaStream_t s) {
  k_mask<<<1024, 256, 0, s>>>(P.mg, P.N, j0, rows, out);
  P.launches += 1;
  FZP_CUDA_TRY(cudaGetLastError());
  return FZP_OK;
}

fzp_status bluestein_build_tables(Plan& P) {
  return P.precision == FZP_PREC_FP64 ? build_tables_t<double>(P) : build_tables_t<float>(P);
}

fzp_status bluestein_layout(Plan& P, FormSizes* out) {
  return P.precision == FZP_PREC_FP64 ? layout_t<double>(P, out) : layout_t<float>(P, out);
}

fzp_status bluestein_fill_tables(Plan& P, cudaStream_t s) {
  return P.precision == FZP_PREC_FP64 ? fill_tables_t<double>(P, s) : fill_tables_t<float>(P, s);
}

fzp_status bluestein_rows(Plan& P, int64_t j0, int64_t rows, cudaStream_t stream) {
  P.dominant = P.precision == FZP_PREC_FP64 ? "bluestein_f2<double>"
                                             : (P.bs.seg ? "k_seg (partitioned convolution)" : "bluestein_f2<float>");
  return P.precision == FZP_PREC_FP64 ? rows_t<double>(P, j0, rows, stream) : rows_t<float>(P, j0, rows, stream);
}

}  // namespace fzp
