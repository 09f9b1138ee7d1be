// Tensor-core (tcgen05) DFT-GEMM path: stage 2 of the SOCS image as dense GEMMs.
#pragma once

#include "litho_internal.h"

namespace litho {

// Device scratch the GEMM path needs for one clip (all focus planes).
size_t gemm_workspace_bytes(const litho_kernels* h, litho_precision prec);
// LITHO_OK when the precision can run for this kernel set and device, else
// EUNSUPPORTED with a message.
litho_status gemm_supported(const litho_kernels* h, litho_precision prec);
// I[f][y][x] = dose sum_k lam_fk |E_fk|^2 for one clip given its band spectrum.
litho_status gemm_aerial_clip(const litho_kernels* h, const float2* mhat, float dose, litho_precision prec, float* img,
                              void* ws, cudaStream_t st);
void gemm_free_operands(litho_kernels* h);

}  // namespace litho
