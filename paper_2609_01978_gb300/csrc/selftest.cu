// selftest.cu -- exercises the failure path every kernel of the library shares:
// a bounded mbarrier wait that runs out.  No counterpart in the paper.
//
// One thread waits on a shared-memory mbarrier that nothing arrives at, with
// the same helper (and try-wait suspend hint) as the production kernels but a
// caller-chosen limit; when the limit passes it records the timeout code in
// the error word and returns, and the host turns the word into FZP_E_TIMEOUT,
// as fzp_metrics does for a propagation.  Nothing else is in flight, so the
// context stays usable (the test propagates afterwards).
#include <cstdint>
#include <mutex>

#include "fzp_internal.cuh"
#include "tc_ptx.cuh"

namespace fzp {
namespace {

constexpr int SELFTEST_CODE = 901;
__device__ int g_selftest_err;

__global__ void k_wait_timeout(uint64_t limit_ns, int* err) {
  __shared__ uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) tc::mbar_wait_for(&bar, 0, &abort_flag, err, SELFTEST_CODE, limit_ns);
}

}  // namespace
}  // namespace fzp

using namespace fzp;

extern "C" fzp_status fzp_selftest_wait_timeout(uint32_t limit_us, void* stream) {
  if (limit_us < 1 || limit_us > 2000000) return set_error(FZP_E_INVALID, "limit_us must be in [1, 2000000]");
  int* err = nullptr;
  FZP_CUDA_TRY(cudaGetSymbolAddress(reinterpret_cast<void**>(&err), g_selftest_err));
  cudaStream_t s = (cudaStream_t)stream;
  FZP_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), s));
  k_wait_timeout<<<1, 32, 0, s>>>((uint64_t)limit_us * 1000ull, err);
  FZP_CUDA_TRY(cudaGetLastError());
  int h = 0;
  FZP_CUDA_TRY(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s));
  FZP_CUDA_TRY(cudaStreamSynchronize(s));
  if (h == SELFTEST_CODE)
    return set_error(FZP_E_TIMEOUT, "a device-side wait timed out (code %d) after %u us, as designed", h, limit_us);
  return set_error(FZP_E_CUDA, "the self-test wait did not report its timeout (error word %d)", h);
}
