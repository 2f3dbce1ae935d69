// dense.cu -- form (b) placeholder until the tensor-core contraction lands.
#include "fzp_internal.cuh"
namespace fzp {
fzp_status dense_build_tables(Plan&) { return set_error(FZP_E_UNSUPPORTED, "dense form not built yet"); }
fzp_status dense_rows(Plan&, int64_t, int64_t, cudaStream_t) { return set_error(FZP_E_UNSUPPORTED, "dense form not built yet"); }
}  // namespace fzp
