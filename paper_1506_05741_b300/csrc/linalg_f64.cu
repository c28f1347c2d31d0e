// linalg_f64.cu -- FP64 Cholesky factorisation and triangular solves on the GPU.
//
// Algorithm 1 refreshes the proposal factor with A_n = Cholesky(C_n) every n_lag steps. Here that is a
// blocked right-looking factorisation (block 64): the diagonal block is factored unblocked in shared
// memory, the panel below it is solved row by row (one warp per row), and the trailing lower triangle
// takes a DFMA rank-64 update. The same row solve, applied to many right-hand sides, gives
// z = A_n^{-1}(x - x_ref) for every chain when the factor changes.
#include "linalg.h"
#include "gemm_f64.cuh"

namespace diam {

constexpr int CH_NB = 64;

// Unblocked Cholesky of the nb x nb diagonal block at (k0, k0); lower part in, L out, upper part zeroed.
// 256 threads as 8 x 32: the rank-1 update of pivot j touches rows j+1+ty, ... and columns j+1+tx, ...
__global__ void __launch_bounds__(256) chol_diag_kernel(double* __restrict__ A, int lda, int k0, int nb, int* info) {
    __shared__ double a[CH_NB][CH_NB + 1];
    __shared__ double s_inv;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int i = ty; i < nb; i += 8)
        for (int j = tx; j < nb; j += 32) a[i][j] = (j <= i) ? A[(size_t)(k0 + i) * lda + k0 + j] : 0.0;
    __syncthreads();
    for (int j = 0; j < nb; ++j) {
        if (threadIdx.x == 0) {
            double piv = a[j][j];
            if (!(piv > 0.0) && info) atomicCAS(info, 0, k0 + j + 1);
            double dj = sqrt(piv);    // NaN on failure: it propagates and the caller discards the result
            a[j][j] = dj;
            s_inv = 1.0 / dj;
        }
        __syncthreads();
        const double inv = s_inv;
        for (int i = j + 1 + threadIdx.x; i < nb; i += blockDim.x) a[i][j] *= inv;
        __syncthreads();
        for (int i = j + 1 + ty; i < nb; i += 8) {
            const double aij = a[i][j];
            for (int l = j + 1 + tx; l <= i; l += 32) a[i][l] = fma(-aij, a[l][j], a[i][l]);
        }
        __syncthreads();
    }
    for (int i = ty; i < nb; i += 8)
        for (int j = tx; j < nb; j += 32) A[(size_t)(k0 + i) * lda + k0 + j] = (j <= i) ? a[i][j] : 0.0;
}

// For each of nrows rows r: solve L y = b in place, b = B[r*ldb + 0 .. nb), L the nb x nb lower triangle
// at Lkk (row stride ldl). One warp per row; lane l holds entries l and l + 32. The diagonal enters as
// reciprocals computed once per block.
__global__ void __launch_bounds__(256) trsv_rows_kernel(const double* __restrict__ Lkk, int ldl, int nb,
                                                         double* __restrict__ B, int ldb, int nrows) {
    __shared__ double L[CH_NB][CH_NB + 1];
    __shared__ double invd[CH_NB];
    for (int idx = threadIdx.x; idx < CH_NB * CH_NB; idx += blockDim.x) {
        int i = idx >> 6, j = idx & 63;
        L[i][j] = (i < nb && j <= i) ? Lkk[(size_t)i * ldl + j] : 0.0;
    }
    __syncthreads();
    if (threadIdx.x < nb) invd[threadIdx.x] = 1.0 / L[threadIdx.x][threadIdx.x];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int warps = blockDim.x >> 5;
    for (int r = blockIdx.x * warps + (threadIdx.x >> 5); r < nrows; r += gridDim.x * warps) {
        double* b = B + (size_t)r * ldb;
        double v0 = lane < nb ? b[lane] : 0.0;
        double v1 = lane + 32 < nb ? b[lane + 32] : 0.0;
        for (int j = 0; j < nb; ++j) {
            double bj = __shfl_sync(0xffffffffu, j < 32 ? v0 : v1, j & 31);
            double yj = bj * invd[j];
            if (lane == (j & 31)) {
                if (j < 32) v0 = yj; else v1 = yj;
            }
            if (lane > j) v0 = fma(-L[lane][j], yj, v0);
            if (lane + 32 > j) v1 = fma(-L[lane + 32][j], yj, v1);
        }
        if (lane < nb) b[lane] = v0;
        if (lane + 32 < nb) b[lane + 32] = v1;
    }
}

__global__ void zero_upper_kernel(double* A, int lda, int n) {
    int i = blockIdx.y;
    for (int j = i + 1 + blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
        A[(size_t)i * lda + j] = 0.0;
}

static int row_blocks(int nrows) { return max(1, min((nrows + 7) / 8, 148 * 8)); }

cudaError_t cholesky_f64(double* A, int n, int lda, int* info_dev, cudaStream_t st, OzakiWs* oz, int* status_dev) {
    for (int k0 = 0; k0 < n; k0 += CH_NB) {
        int nb = min(CH_NB, n - k0);
        { chol_diag_kernel<<<1, 256, 0, st>>>(A, lda, k0, nb, info_dev); count_launch(); }
        int k1 = k0 + nb, rest = n - k1;
        if (rest <= 0) break;
        // panel rows solve x L_kk^T = a, i.e. L_kk x^T = a^T
        { trsv_rows_kernel<<<row_blocks(rest), 256, 0, st>>>(A + (size_t)k0 * lda + k0, lda, nb,
                                                             A + (size_t)k1 * lda + k0, lda, rest); count_launch(); }
        // trailing lower triangle: A[k1+n][k1+m] -= sum_k L[k1+m][k0+k] L[k1+n][k0+k]
        cudaError_t e;
        if (oz && nb == CH_NB && rest >= 128) {
            e = ozaki_trailing_update(A + (size_t)k1 * lda + k0, lda, rest, A + (size_t)k1 * lda + k1, lda, *oz,
                                      status_dev, st);
        } else {
            EpiStore epi{A + (size_t)k1 * lda + k1, lda, -1.0, nullptr, 1.0};
            e = gemm_f64<true, true>(rest, rest, nb, A + (size_t)k1 * lda + k0, lda, A + (size_t)k1 * lda + k0, lda,
                                     TileRange{0, 1}, epi, st);
        }
        if (e != cudaSuccess) return e;
    }
    dim3 g(max(1, min(32, (n + 255) / 256)), n);
    { zero_upper_kernel<<<g, 256, 0, st>>>(A, lda, n); count_launch(); }
    return cudaGetLastError();
}

cudaError_t trsm_lower_f64(const double* L, int ldl, int n, double* B, int ldb, int nrows, cudaStream_t st) {
    if (nrows <= 0 || n <= 0) return cudaSuccess;
    for (int k0 = 0; k0 < n; k0 += CH_NB) {
        int nb = min(CH_NB, n - k0);
        { trsv_rows_kernel<<<row_blocks(nrows), 256, 0, st>>>(L + (size_t)k0 * ldl + k0, ldl, nb, B + k0, ldb, nrows); count_launch(); }
        int k1 = k0 + nb;
        if (k1 >= n) break;
        // B[r][k1 + i] -= sum_k L[k1 + i][k0 + k] Y[r][k0 + k]
        EpiStore epi{B + k1, ldb, -1.0, nullptr, 1.0};
        cudaError_t e = gemm_f64<true, true>(n - k1, nrows, nb, L + (size_t)k1 * ldl + k0, ldl, B + k0, ldb,
                                             TileRange{0, 0}, epi, st);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

}  // namespace diam
