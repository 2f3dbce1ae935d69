// mlp.cu -- learned surrogate: a multilayer perceptron trained and evaluated by
// kernels written here (no counterpart in the paper; it learns the map from
// membrane-deformation parameters to the PSF and metrics that the CZT method
// computes, Sec. 7.2 / Sec. 9 name membrane deformation as the next input).
//
// Network: n_in -> hidden (x n_hidden_layers, SiLU) -> n_out (linear); loss =
// mean squared error over batch and outputs; optimiser AdamW (decoupled weight
// decay on weights, not biases).  Weights are kept as FP32 masters; every matrix
// product takes BF16 operands (weights, layer inputs, back-propagated errors)
// and accumulates in FP32 in tensor memory (tcgen05.mma kind::f16, M128 N128).
//
// Matrix products, all as C[M x N] = A[M x K] . B[N x K]^T with K contiguous:
//   forward  z_l   = h_{l-1} . W_l^T          (A = h, B = W)
//   backward dh    = g . W_l                  (A = g, B = W^T  kept transposed)
//            dW_l  = g^T . h_{l-1}            (A = g^T, B = h^T: transposed copies)
#include <cuda_bf16.h>

#include <cmath>
#include <new>
#include <vector>

#include "fzp_internal.cuh"
#include "tc_ptx.cuh"

namespace fzp {
namespace {

using namespace tc;

constexpr int GM = 128, GN = 128, GK = 64;  // GEMM tile; K step = one 128-byte swizzle row
constexpr int GEMM_THREADS = 128;
constexpr int GEMM_SMEM = 1024 + 2 * GM * GK * 2 + 64 + 16384;  // extra slack caps residency at 4 CTAs/SM

__host__ __device__ inline int64_t pad64(int64_t x) { return (x + 63) / 64 * 64; }

// K-major, 128-byte swizzle, 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t sdesc128(const void* p) {
  const uint64_t a = smem_u32(p);
  return ((a >> 4) & 0x3FFFull) | (1ull << 16) | ((uint64_t)(1024 >> 4) << 32) | (1ull << 46) | (2ull << 61);
}
constexpr uint32_t IDESC_G = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(GN >> 3) << 17) | ((uint32_t)(GM >> 4) << 24);

__device__ __forceinline__ void mma_g(uint32_t dtmem, uint64_t ad, uint64_t bd, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(
          dtmem),
      "l"(ad), "l"(bd), "r"(IDESC_G), "r"(acc)
      : "memory");
}

// Load a 128-row x 64-column BF16 tile (rows r0.., columns k0..) into the
// 128-byte-swizzled K-major layout; out-of-range elements are zero.
__device__ __forceinline__ void load_tile(uint8_t* s, const __nv_bfloat16* g, int64_t ld, int64_t rows, int64_t K,
                                          int64_t r0, int64_t k0) {
  for (int t = threadIdx.x; t < GM * 8; t += GEMM_THREADS) {
    const int r = t >> 3, ch = t & 7;
    const int64_t gr = r0 + r, gk = k0 + ch * 8;
    uint4 v = make_uint4(0, 0, 0, 0);
    if (gr < rows && gk < K) v = *reinterpret_cast<const uint4*>(g + gr * ld + gk);  // K, ld multiples of 8
    *reinterpret_cast<uint4*>(s + (r >> 3) * 1024 + (r & 7) * 128 + ((ch ^ (r & 7)) << 4)) = v;
  }
}

// C[M x N] (FP32, ldc) = A[M x K] . B[N x K]^T (+ bias[N]).  K must be a multiple of 8.
__global__ void __launch_bounds__(GEMM_THREADS) k_gemm_tn(int64_t M, int64_t N, int64_t K, const __nv_bfloat16* A,
                                                          int64_t lda, const __nv_bfloat16* B, int64_t ldb, float* C,
                                                          int64_t ldc, const float* bias, int* err) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = base;
  uint8_t* sB = base + GM * GK * 2;
  uint64_t* bar = reinterpret_cast<uint64_t*>(sB + GN * GK * 2);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(bar + 2);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t m0 = (int64_t)blockIdx.y * GM, n0 = (int64_t)blockIdx.x * GN;
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(GN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int64_t nk = (K + GK - 1) / GK;
  bool ok = true;
  for (int64_t kb = 0; kb < nk && ok; ++kb) {
    load_tile(sA, A, lda, M, K, m0, kb * GK);
    load_tile(sB, B, ldb, N, K, n0, kb * GK);
    fence_proxy_async();
    __syncthreads();
    if (threadIdx.x == 0) {
      tc_fence_after();
      const uint64_t ad = sdesc128(sA), bd = sdesc128(sB);
#pragma unroll
      for (int kk = 0; kk < GK / 16; ++kk)
        mma_g(tmem, ad + (uint64_t)((kk * 32) >> 4), bd + (uint64_t)((kk * 32) >> 4), (kb > 0 || kk > 0) ? 1u : 0u);
      mma_commit(bar);
    }
    // every thread waits for the MMAs of this step: the tile buffers are reused
    ok = mbar_wait(bar, (uint32_t)(kb & 1), abort_flag, err, 200);
    tc_fence_after();
    __syncthreads();
    ok = !*abort_flag;
  }
  if (ok) {
    const int64_t r = m0 + warp * 32 + lane;
#pragma unroll 1
    for (int c0 = 0; c0 < GN; c0 += 32) {
      float v[32];
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      if (r < M) {
#pragma unroll
        for (int q = 0; q < 32; ++q) {
          const int64_t n = n0 + c0 + q;
          if (n < N) C[r * ldc + n] = v[q] + (bias ? bias[n] : 0.f);
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(GN) : "memory");
  }
}

__device__ __forceinline__ float sigm(float z) { return 1.f / (1.f + expf(-z)); }

// dst[r][c] = bf16(act ? silu(src) : src) for r < R, c < Cn (ld in elements).
__global__ void k_to_bf16(int64_t R, int64_t Cn, const float* src, int64_t lds, __nv_bfloat16* dst, int64_t ldd,
                          int act) {
  const int64_t total = R * Cn;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t / Cn, c = t % Cn;
    float v = src[r * lds + c];
    if (act) v = v * sigm(v);
    dst[r * ldd + c] = __float2bfloat16_rn(v);
  }
}

// dst[c][r] = bf16(act ? silu(src[r][c]) : src[r][c])  (transposed copy).
__global__ void k_to_bf16_t(int64_t R, int64_t Cn, const float* src, int64_t lds, __nv_bfloat16* dst, int64_t ldd,
                            int act) {
  __shared__ float tile[32][33];
  const int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int64_t r = r0 + k, c = c0 + threadIdx.x;
    float v = 0.f;
    if (r < R && c < Cn) {
      v = src[r * lds + c];
      if (act) v = v * sigm(v);
    }
    tile[k][threadIdx.x] = v;
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int64_t c = c0 + k, r = r0 + threadIdx.x;
    if (r < R && c < Cn) dst[c * ldd + r] = __float2bfloat16_rn(tile[threadIdx.x][k]);
  }
}

// g = dh * silu'(z)
__global__ void k_silu_back(int64_t R, int64_t Cn, const float* dh, const float* z, int64_t ld, float* g) {
  const int64_t total = R * Cn;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t / Cn, c = t % Cn;
    const float zz = z[r * ld + c], s = sigm(zz);
    g[r * ld + c] = dh[r * ld + c] * (s * (1.f + zz * (1.f - s)));
  }
}

// g = 2 (yhat - y) / (B n); loss += mean((yhat - y)^2)
__global__ void k_mse(int64_t B, int64_t n, const float* yhat, int64_t ldy, const float* y, float* g, float* loss) {
  __shared__ float sh[256];
  float acc = 0.f;
  const float scale = 2.f / (float)(B * n);
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < B * n; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t / n, c = t % n;
    const float d = yhat[r * ldy + c] - y[r * n + c];
    g[r * ldy + c] = scale * d;
    acc += d * d;
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0 && loss) atomicAdd(loss, sh[0] / (float)(B * n));
}

// db[c] = sum_r g[r][c]
__global__ void k_colsum(int64_t R, int64_t Cn, const float* g, int64_t ld, float* db) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= Cn) return;
  float s = 0.f;
  for (int64_t r = 0; r < R; ++r) s += g[r * ld + c];
  db[c] = s;
}

// copy dW (FP32, [n_out][ld]) into the flat gradient vector
__global__ void k_pack(int64_t R, int64_t Cn, const float* src, int64_t ld, float* dst) {
  const int64_t total = R * Cn;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x)
    dst[t] = src[(t / Cn) * ld + t % Cn];
}

__global__ void k_adamw(int64_t n, float* p, const float* g, float* m, float* v, float lr, float wd, float b1, float b2,
                        float eps, float c1, float c2) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const float gg = g[t];
    const float mm = b1 * m[t] + (1.f - b1) * gg;
    const float vv = b2 * v[t] + (1.f - b2) * gg * gg;
    m[t] = mm;
    v[t] = vv;
    p[t] -= lr * ((mm / c1) / (sqrtf(vv / c2) + eps) + wd * p[t]);
  }
}

// Weights W (FP32 [n_out][n_in], row-major, inside the flat vector) -> BF16
// copies Wb [n_out][ld_in] and WTb [n_in][ld_out].
__global__ void k_weights_bf16(int64_t n_out, int64_t n_in, const float* W, __nv_bfloat16* Wb, int64_t ld_in,
                               __nv_bfloat16* WTb, int64_t ld_out) {
  const int64_t total = n_out * n_in;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o = t / n_in, i = t % n_in;
    const __nv_bfloat16 w = __float2bfloat16_rn(W[t]);
    Wb[o * ld_in + i] = w;
    WTb[i * ld_out + o] = w;
  }
}

__global__ void k_init_uniform(int64_t n, float* p, float scale, uint64_t seed) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    uint64_t z = seed + 0x9E3779B97F4A7C15ull * (uint64_t)(t + 1);  // splitmix64
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    p[t] = scale * (2.f * (float)((z >> 40) * (1.0 / 16777216.0)) - 1.f);
  }
}

}  // namespace

struct Layer {
  int64_t n_in, n_out, ld_in, ld_out;  // ld: padded to 64
  int64_t off_w, off_b;                // offsets in the flat parameter vector
  __nv_bfloat16 *Wb = nullptr, *WTb = nullptr;
};

}  // namespace fzp

using namespace fzp;

struct fzp_surrogate_s {
  std::vector<Layer> L;
  int64_t max_batch = 0, n_params = 0, step = 0;
  float *params = nullptr, *grads = nullptr, *m = nullptr, *v = nullptr;
  std::vector<float*> Z;             // pre-activations per layer [B][ld_out] FP32
  std::vector<__nv_bfloat16*> Hb;    // layer inputs, BF16 [B][ld_in]
  std::vector<__nv_bfloat16*> HTb;   // layer inputs transposed [ld_in... n_in][ldB]
  float *G = nullptr, *dH = nullptr, *dW = nullptr;
  __nv_bfloat16 *Gb = nullptr, *GTb = nullptr;
  int64_t ldB = 0, maxw = 0;
  int* err = nullptr;
  std::vector<void*> allocs;
};

namespace {

fzp_status gemm(fzp_surrogate_s& S, int64_t M, int64_t N, int64_t K, const __nv_bfloat16* A, int64_t lda,
                const __nv_bfloat16* B, int64_t ldb, float* C, int64_t ldc, const float* bias, cudaStream_t s) {
  dim3 grid((unsigned)((N + GN - 1) / GN), (unsigned)((M + GM - 1) / GM));
  k_gemm_tn<<<grid, GEMM_THREADS, GEMM_SMEM, s>>>(M, N, K, A, lda, B, ldb, C, ldc, bias, S.err);
  FZP_CUDA_TRY(cudaGetLastError());
  return FZP_OK;
}

unsigned blocks(int64_t n) { return (unsigned)std::min<int64_t>((n + 255) / 256, 4096); }

// Forward pass for a batch of B rows (x: FP32 [B][n_in0], contiguous).
fzp_status forward(fzp_surrogate_s& S, const float* x, int64_t B, cudaStream_t s) {
  const Layer& l0 = S.L[0];
  k_to_bf16<<<blocks(B * l0.n_in), 256, 0, s>>>(B, l0.n_in, x, l0.n_in, S.Hb[0], l0.ld_in, 0);
  for (size_t l = 0; l < S.L.size(); ++l) {
    const Layer& ly = S.L[l];
    fzp_status st = gemm(S, B, ly.n_out, ly.ld_in, S.Hb[l], ly.ld_in, ly.Wb, ly.ld_in, S.Z[l], ly.ld_out,
                         S.params + ly.off_b, s);
    if (st != FZP_OK) return st;
    if (l + 1 < S.L.size())
      k_to_bf16<<<blocks(B * ly.n_out), 256, 0, s>>>(B, ly.n_out, S.Z[l], ly.ld_out, S.Hb[l + 1], S.L[l + 1].ld_in, 1);
  }
  FZP_CUDA_TRY(cudaGetLastError());
  return FZP_OK;
}

// Loss and gradients into S.grads (flat, same layout as params).
// Requires forward() and transposed_inputs() for the same batch.
fzp_status backward(fzp_surrogate_s& S, const float* y, int64_t B, float* d_loss, cudaStream_t s) {
  fzp_status st = FZP_OK;
  const int nl = (int)S.L.size();
  const Layer& lo = S.L[nl - 1];
  if (d_loss) FZP_CUDA_TRY(cudaMemsetAsync(d_loss, 0, sizeof(float), s));
  k_mse<<<256, 256, 0, s>>>(B, lo.n_out, S.Z[nl - 1], lo.ld_out, y, S.G, d_loss);
  for (int l = nl - 1; l >= 0; --l) {
    const Layer& ly = S.L[l];
    // db = sum over batch of g; g in BF16 (row-major and transposed)
    k_colsum<<<(unsigned)((ly.n_out + 255) / 256), 256, 0, s>>>(B, ly.n_out, S.G, ly.ld_out, S.grads + ly.off_b);
    k_to_bf16<<<blocks(B * ly.n_out), 256, 0, s>>>(B, ly.n_out, S.G, ly.ld_out, S.Gb, S.maxw, 0);
    dim3 tg((unsigned)((ly.n_out + 31) / 32), (unsigned)((B + 31) / 32));
    k_to_bf16_t<<<tg, dim3(32, 8), 0, s>>>(B, ly.n_out, S.G, ly.ld_out, S.GTb, S.ldB, 0);
    // dW = g^T h  (M = n_out, N = n_in, K = B; B is a multiple of 8, so the
    // 8-element loads never reach columns a larger earlier batch left behind)
    st = gemm(S, ly.n_out, ly.n_in, B, S.GTb, S.ldB, S.HTb[l], S.ldB, S.dW, ly.ld_in, nullptr, s);
    if (st != FZP_OK) return st;
    k_pack<<<blocks(ly.n_out * ly.n_in), 256, 0, s>>>(ly.n_out, ly.n_in, S.dW, ly.ld_in, S.grads + ly.off_w);
    if (l > 0) {
      // dh = g W  (M = B, N = n_in, K = n_out), then g = dh silu'(z_{l-1})
      st = gemm(S, B, ly.n_in, ly.ld_out, S.Gb, S.maxw, ly.WTb, ly.ld_out, S.dH, S.L[l - 1].ld_out, nullptr, s);
      if (st != FZP_OK) return st;
      k_silu_back<<<blocks(B * ly.n_in), 256, 0, s>>>(B, ly.n_in, S.dH, S.Z[l - 1], S.L[l - 1].ld_out, S.G);
    }
  }
  FZP_CUDA_TRY(cudaGetLastError());
  return FZP_OK;
}

// h^T copies are needed by the weight gradient: refresh them from Hb after forward.
fzp_status transposed_inputs(fzp_surrogate_s& S, const float* x, int64_t B, cudaStream_t s) {
  for (size_t l = 0; l < S.L.size(); ++l) {
    const Layer& ly = S.L[l];
    const float* src = l == 0 ? x : S.Z[l - 1];
    const int64_t lds = l == 0 ? ly.n_in : S.L[l - 1].ld_out;
    dim3 tg((unsigned)((ly.n_in + 31) / 32), (unsigned)((B + 31) / 32));
    k_to_bf16_t<<<tg, dim3(32, 8), 0, s>>>(B, ly.n_in, src, lds, S.HTb[l], S.ldB, l == 0 ? 0 : 1);
  }
  FZP_CUDA_TRY(cudaGetLastError());
  return FZP_OK;
}

fzp_status refresh_weights(fzp_surrogate_s& S, cudaStream_t s) {
  for (const Layer& ly : S.L)
    k_weights_bf16<<<blocks(ly.n_out * ly.n_in), 256, 0, s>>>(ly.n_out, ly.n_in, S.params + ly.off_w, ly.Wb,
                                                              ly.ld_in, ly.WTb, ly.ld_out);
  FZP_CUDA_TRY(cudaGetLastError());
  return FZP_OK;
}

fzp_status grad_all(fzp_surrogate_s& S, const float* x, const float* y, int64_t B, float* d_loss, cudaStream_t s) {
  fzp_status st = forward(S, x, B, s);
  if (st == FZP_OK) st = transposed_inputs(S, x, B, s);
  if (st == FZP_OK) st = backward(S, y, B, d_loss, s);
  return st;
}

void surrogate_release(fzp_surrogate_s* S) {
  if (!S) return;
  cudaDeviceSynchronize();
  for (void* p : S->allocs)
    if (p) cudaFree(p);
  delete S;
}

}  // namespace

extern "C" {

fzp_status fzp_surrogate_create(int n_in, int hidden, int n_hidden_layers, int n_out, int max_batch, uint64_t seed,
                                fzp_surrogate_t* out) {
  if (!out) return set_error(FZP_E_INVALID, "out is NULL");
  *out = nullptr;
  if (n_in < 1 || hidden < 1 || n_hidden_layers < 1 || n_out < 1 || max_batch < 1 || n_in > 65536 ||
      hidden > 65536 || n_out > 65536 || max_batch > 65536)
    return set_error(FZP_E_INVALID, "surrogate sizes must be in [1, 65536]");
  fzp_surrogate_s* S = new (std::nothrow) fzp_surrogate_s();
  if (!S) return set_error(FZP_E_OOM, "host allocation failed");
  std::vector<int64_t> dims;
  dims.push_back(n_in);
  for (int k = 0; k < n_hidden_layers; ++k) dims.push_back(hidden);
  dims.push_back(n_out);
  int64_t off = 0, maxw = 0;
  for (size_t l = 0; l + 1 < dims.size(); ++l) {
    Layer ly;
    ly.n_in = dims[l];
    ly.n_out = dims[l + 1];
    ly.ld_in = pad64(ly.n_in);
    ly.ld_out = pad64(ly.n_out);
    ly.off_w = off;
    off += ly.n_in * ly.n_out;
    ly.off_b = off;
    off += ly.n_out;
    maxw = std::max(maxw, std::max(ly.ld_in, ly.ld_out));
    S->L.push_back(ly);
  }
  S->n_params = off;
  S->max_batch = max_batch;
  S->ldB = pad64(max_batch);
  S->maxw = maxw;
  auto alloc = [&](size_t bytes) -> void* {
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) return nullptr;
    S->allocs.push_back(p);
    cudaMemset(p, 0, bytes);  // padding must read as zero
    return p;
  };
  bool ok = true;
  auto A = [&](size_t bytes) {
    void* p = alloc(bytes);
    ok = ok && p;
    return p;
  };
  S->params = (float*)A(sizeof(float) * off);
  S->grads = (float*)A(sizeof(float) * off);
  S->m = (float*)A(sizeof(float) * off);
  S->v = (float*)A(sizeof(float) * off);
  S->err = (int*)A(sizeof(int));
  for (Layer& ly : S->L) {
    ly.Wb = (__nv_bfloat16*)A(sizeof(__nv_bfloat16) * ly.n_out * ly.ld_in);
    ly.WTb = (__nv_bfloat16*)A(sizeof(__nv_bfloat16) * ly.n_in * ly.ld_out);
    S->Z.push_back((float*)A(sizeof(float) * max_batch * ly.ld_out));
    S->Hb.push_back((__nv_bfloat16*)A(sizeof(__nv_bfloat16) * max_batch * ly.ld_in));
    S->HTb.push_back((__nv_bfloat16*)A(sizeof(__nv_bfloat16) * ly.ld_in * S->ldB));
  }
  S->G = (float*)A(sizeof(float) * max_batch * maxw);
  S->dH = (float*)A(sizeof(float) * max_batch * maxw);
  S->dW = (float*)A(sizeof(float) * maxw * maxw);
  S->Gb = (__nv_bfloat16*)A(sizeof(__nv_bfloat16) * max_batch * maxw);
  S->GTb = (__nv_bfloat16*)A(sizeof(__nv_bfloat16) * maxw * S->ldB);
  if (!ok) {
    cudaGetLastError();
    surrogate_release(S);
    return set_error(FZP_E_OOM, "surrogate allocation failed");
  }
  static std::atomic<uint64_t> attr{0};
  if (smem_attr_once((const void*)k_gemm_tn, GEMM_SMEM, attr) != cudaSuccess) {
    surrogate_release(S);
    return set_error(FZP_E_CUDA, "cudaFuncSetAttribute(k_gemm_tn)");
  }
  // weights ~ U(-1/sqrt(fan_in), 1/sqrt(fan_in)); biases zero
  for (const Layer& ly : S->L)
    k_init_uniform<<<blocks(ly.n_in * ly.n_out), 256>>>(ly.n_in * ly.n_out, S->params + ly.off_w,
                                                       1.f / sqrtf((float)ly.n_in), seed + (uint64_t)ly.off_w);
  fzp_status st = refresh_weights(*S, 0);
  if (st == FZP_OK && cudaDeviceSynchronize() != cudaSuccess) st = set_error(FZP_E_CUDA, "surrogate init failed");
  if (st != FZP_OK) {
    surrogate_release(S);
    return st;
  }
  *out = S;
  return FZP_OK;
}

size_t fzp_surrogate_param_count(fzp_surrogate_t S) { return S ? (size_t)S->n_params : 0; }

fzp_status fzp_surrogate_params(fzp_surrogate_t S, float* h_buf, size_t count, int set) {
  if (!S || !h_buf || count != (size_t)S->n_params) return set_error(FZP_E_INVALID, "bad surrogate or count");
  if (set) {
    FZP_CUDA_TRY(cudaMemcpy(S->params, h_buf, count * sizeof(float), cudaMemcpyHostToDevice));
    fzp_status st = refresh_weights(*S, 0);
    if (st != FZP_OK) return st;
    FZP_CUDA_TRY(cudaDeviceSynchronize());
  } else {
    FZP_CUDA_TRY(cudaMemcpy(h_buf, S->params, count * sizeof(float), cudaMemcpyDeviceToHost));
  }
  return FZP_OK;
}

fzp_status fzp_surrogate_infer(fzp_surrogate_t S, const float* d_x, int batch, float* d_y, void* stream) {
  if (!S || !d_x || !d_y || batch < 1 || batch > S->max_batch) return set_error(FZP_E_INVALID, "bad infer arguments");
  cudaStream_t s = (cudaStream_t)stream;
  fzp_status st = forward(*S, d_x, batch, s);
  if (st != FZP_OK) return st;
  const Layer& lo = S->L.back();
  FZP_CUDA_TRY(cudaMemcpy2DAsync(d_y, lo.n_out * sizeof(float), S->Z.back(), lo.ld_out * sizeof(float),
                                 lo.n_out * sizeof(float), batch, cudaMemcpyDeviceToDevice, s));
  return FZP_OK;
}

fzp_status fzp_surrogate_grad(fzp_surrogate_t S, const float* d_x, const float* d_y, int batch, float* d_grad,
                              float* d_loss, void* stream) {
  if (!S || !d_x || !d_y || batch < 8 || batch > S->max_batch || (batch % 8) != 0)
    return set_error(FZP_E_INVALID, "bad grad arguments (batch must be a multiple of 8)");
  cudaStream_t s = (cudaStream_t)stream;
  fzp_status st = grad_all(*S, d_x, d_y, batch, d_loss, s);
  if (st != FZP_OK) return st;
  if (d_grad) FZP_CUDA_TRY(cudaMemcpyAsync(d_grad, S->grads, S->n_params * sizeof(float), cudaMemcpyDeviceToDevice, s));
  return FZP_OK;
}

fzp_status fzp_surrogate_train_step(fzp_surrogate_t S, const float* d_x, const float* d_y, int batch, float lr,
                                    float weight_decay, float* d_loss, void* stream) {
  if (!S || !d_x || !d_y || batch < 8 || batch > S->max_batch || (batch % 8) != 0 || !(lr > 0))
    return set_error(FZP_E_INVALID, "bad train arguments (batch must be a multiple of 8, lr > 0)");
  cudaStream_t s = (cudaStream_t)stream;
  fzp_status st = grad_all(*S, d_x, d_y, batch, d_loss, s);
  if (st != FZP_OK) return st;
  S->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)S->step), c2 = 1.f - powf(b2, (float)S->step);
  for (const Layer& ly : S->L) {
    k_adamw<<<blocks(ly.n_in * ly.n_out), 256, 0, s>>>(ly.n_in * ly.n_out, S->params + ly.off_w,
                                                       S->grads + ly.off_w, S->m + ly.off_w, S->v + ly.off_w, lr,
                                                       weight_decay, b1, b2, 1e-8f, c1, c2);
    k_adamw<<<blocks(ly.n_out), 256, 0, s>>>(ly.n_out, S->params + ly.off_b, S->grads + ly.off_b, S->m + ly.off_b,
                                             S->v + ly.off_b, lr, 0.f, b1, b2, 1e-8f, c1, c2);
  }
  FZP_CUDA_TRY(cudaGetLastError());
  return refresh_weights(*S, s);
}

fzp_status fzp_surrogate_destroy(fzp_surrogate_t S) {
  surrogate_release(S);
  return FZP_OK;
}

}  // extern "C"
