// rewhiten.h -- the re-solve of the whitened states after a factor change, BF16 mode (rewhiten_tc.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace diam {

// z = Lq^{-1}(X - x_ref) per chain (X, Z: P x d FP32, chain-major; Lq: d x ldk BF16 lower triangle, zero
// padding), q = |z|^2 inv_infl2 / 2 per chain and, for the reference target, lp_ref = -q. FP32 arithmetic with
// the panel updates on the tensor cores. status receives DEV_TIMEOUT if a bounded wait expired.
bool rewhiten_tc_fits(int d, int ldk);
size_t rewhiten_tc_smem(int d);
cudaError_t rewhiten_tc_setup(int d);   // once, outside any graph capture
cudaError_t rewhiten_tc(int d, int P, const uint16_t* Lq, int ldk, const float* X, const float* xref, float* Z,
                        double* q, double inv_infl2, double* lp_ref, int* status, cudaStream_t st);

}  // namespace diam
