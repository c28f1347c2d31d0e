// linalg.h -- host entry points of the FP64 dense kernels.
#pragma once
#include <cuda_runtime.h>

namespace diam {

// In-place lower Cholesky of the n x n lower triangle of A (row-major, stride lda); the strict upper
// triangle is zeroed. *info_dev receives (first failing pivot + 1) if the matrix is not positive
// definite; it is never cleared here.
cudaError_t cholesky_f64(double* A, int n, int lda, int* info_dev, cudaStream_t st);

// For nrows right-hand sides stored as rows of B (row r at B + r*ldb, n entries): B_r <- L^{-1} B_r.
cudaError_t trsm_lower_f64(const double* L, int ldl, int n, double* B, int ldb, int nrows, cudaStream_t st);

}  // namespace diam
