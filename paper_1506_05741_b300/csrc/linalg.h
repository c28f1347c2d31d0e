// linalg.h -- host entry points of the FP64 dense kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace diam {

// Workspace of the tensor-core (Ozaki-split) updates: BF16 slices of the operands' rows and row exponents.
struct OzakiWs {
    uint16_t* SL = nullptr;    // cap_rows x 448: first operand
    int* ex = nullptr;         // cap_rows
    int cap_rows = 0;
    uint16_t* SL2 = nullptr;   // cap2 x 448: second operand of a general update (triangular solves)
    int* ex2 = nullptr;        // cap2
    int cap2 = 0;
};

// C[n][m] -= sum_k P[n][k] P[m][k] for n >= m (k < 64), FP64-accurate on the BF16 tensor cores; P (rows x 64,
// stride lda) and C (stride ldc) FP64. status_dev receives DEV_TIMEOUT if a bounded wait expired.
cudaError_t ozaki_trailing_update(const double* P, int lda, int rows, double* C, int ldc, OzakiWs& ws, int* status_dev,
                                  cudaStream_t st);

// C[n][m] -= sum_k A[m][k] B[n][k] for m < Ma, n < Nb (k < 64), FP64-accurate on the BF16 tensor cores; A
// (Ma x 64, stride lda), B (Nb x 64, stride ldb) and C (stride ldc) FP64; needs Ma <= cap_rows, Nb <= cap2.
cudaError_t ozaki_gemm_update(const double* A, int lda, int Ma, const double* B, int ldb, int Nb, double* C, int ldc,
                              OzakiWs& ws, int* status_dev, cudaStream_t st);

// In-place lower Cholesky of the n x n lower triangle of A (row-major, stride lda); the strict upper
// triangle is zeroed. *info_dev receives (first failing pivot + 1) if the matrix is not positive
// definite; it is never cleared here.
// oz (optional): run the trailing updates on the tensor cores (Ozaki splitting, FP64-accurate).
cudaError_t cholesky_f64(double* A, int n, int lda, int* info_dev, cudaStream_t st, OzakiWs* oz = nullptr,
                         int* status_dev = nullptr);

// For nrows right-hand sides stored as rows of B (row r at B + r*ldb, n entries): B_r <- L^{-1} B_r.
// oz (optional, with cap_rows >= n and cap2 >= nrows): run the block updates on the tensor cores.
cudaError_t trsm_lower_f64(const double* L, int ldl, int n, double* B, int ldb, int nrows, cudaStream_t st,
                           OzakiWs* oz = nullptr, int* status_dev = nullptr);

}  // namespace diam
