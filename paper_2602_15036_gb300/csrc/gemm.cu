// Placeholder until the tcgen05 DFT-GEMM kernels land.
#include "gemm.h"

namespace litho {

size_t gemm_workspace_bytes(const litho_kernels*, litho_precision) { return 0; }
litho_status gemm_supported(const litho_kernels*, litho_precision) {
  set_error("tensor-core path not built yet");
  return LITHO_EUNSUPPORTED;
}
litho_status gemm_aerial_clip(const litho_kernels*, const float2*, float, litho_precision, float*, void*,
                              cudaStream_t) {
  set_error("tensor-core path not built yet");
  return LITHO_EUNSUPPORTED;
}
void gemm_free_operands(litho_kernels*) {}

}  // namespace litho
