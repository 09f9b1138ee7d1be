// Tensor-core (tcgen05) DFT-GEMM path: stage 2 of the SOCS image as dense GEMMs.
#pragma once

#include "litho_internal.h"

namespace litho {

// Device scratch the GEMM path needs for a batch of b clips (it images clips
// in groups of gemm_group_clips()).
// `coarse` evaluates on the grid h->nc instead of h->n.
size_t gemm_workspace_bytes(const litho_kernels* h, litho_precision prec, int b, bool coarse);
int gemm_group_clips();
// LITHO_OK when the precision can run for this kernel set, grid and device
// (and builds its constant operands on first use), else EUNSUPPORTED.
litho_status gemm_supported(const litho_kernels* h, litho_precision prec, bool coarse);
// I[c][f][y][x] = dose sum_k lam_fk |E_fk|^2 on the full (or coarse) grid for
// `clips` clips given their band spectra mhat[c][C][C].
litho_status gemm_aerial_group(const litho_kernels* h, const float2* mhat, int clips, float dose,
                               litho_precision prec, bool coarse, float* img, void* ws, cudaStream_t st);
// Waits for `st` and reports ETIMEOUT if a device-side pipeline wait gave up.
litho_status gemm_check_device(const litho_kernels* h, cudaStream_t st);
// Runs the bounded-wait self-test kernel (a wait nothing completes, limited to
// limit_ms) and returns what gemm_check_device reports (ETIMEOUT when it works).
litho_status gemm_wait_selftest(const litho_kernels* h, double limit_ms, cudaStream_t st);
void gemm_free_operands(litho_kernels* h);

}  // namespace litho
