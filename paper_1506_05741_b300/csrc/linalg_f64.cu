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

// 1/D by the Newton-Raphson iteration y <- y + y (1 - D y) from an FP32 seed (two steps: relative error
// below 2^-46 after the first, at rounding level after the second); outside the FP32 range, a division.
__device__ __forceinline__ double recip_newton(double D) {
    const double aD = fabs(D);
    if (!(aD > 1e-30 && aD < 1e30)) return 1.0 / D;
    double y = (double)__frcp_rn((float)D);
    double e = fma(-D, y, 1.0);
    y = fma(y, e, y);
    e = fma(-D, y, 1.0);
    return fma(y, e, y);
}

// Owner warp of column j of the diagonal block: broadcast D_j, take its reciprocal on one lane, publish the
// column a_ij (i > j) and its scaled copy a_ij / D_j into buffer j & 1.
__device__ __forceinline__ void diag_publish(int j, double v0, double v1, int lane, int k0, int* info, double* dpiv,
                                             double (*colb)[64], double (*scol)[64]) {
    const double D = __shfl_sync(0xffffffffu, j < 32 ? v0 : v1, j & 31);
    double r = 0.0;
    if (lane == 0) {
        if (D > 0.0) {
            r = recip_newton(D);
        } else {   // not positive definite: NaN propagates and the caller discards the factor
            r = __longlong_as_double(0x7ff8000000000000ll);
            if (info) atomicCAS(info, 0, k0 + j + 1);
        }
        dpiv[j] = D;
    }
    r = __shfl_sync(0xffffffffu, r, 0);
    const int b = j & 1;
    if (lane > j) {
        colb[b][lane] = v0;
        scol[b][lane] = v0 * r;
    }
    if (lane + 32 > j) {
        colb[b][lane + 32] = v1;
        scol[b][lane + 32] = v1 * r;
    }
}

// Cholesky of the nb x nb diagonal block at (k0, k0), nb <= 64: lower part in, L out, upper part zeroed.
// Right-looking LDL^T in registers: pivot j subtracts a_ij (a_lj / D_j) from every a_il with j < l <= i,
// leaving a_ij = L_ij sqrt(D_j); the square roots are taken once at the end. Warp w owns the columns
// l = w, w + 8, ..., w + 56 and lane t the rows t and t + 32. After its own update, the warp that owns
// column j + 1 publishes it (and its scaled copy a_i,j+1 / D_j+1) into a double-buffered shared column, so
// each pivot costs one barrier.
__global__ void __launch_bounds__(256) chol_diag_kernel(double* __restrict__ A, int lda, int k0, int nb, int* info) {
    __shared__ double colb[2][CH_NB];   // a_ij, i > j (column j of the current pivot)
    __shared__ double scol[2][CH_NB];   // a_lj / D_j
    __shared__ double dpiv[CH_NB];      // D_j
    __shared__ double dsq[CH_NB], dinv[CH_NB];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double a[8][2];
#pragma unroll
    for (int c = 0; c < 8; ++c)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int l = w + 8 * c, i = lane + 32 * h;
            a[c][h] = (l <= i && i < nb) ? A[(size_t)(k0 + i) * lda + k0 + l] : 0.0;
        }
    if (w == 0) diag_publish(0, a[0][0], a[0][1], lane, k0, info, dpiv, colb, scol);
    __syncthreads();
    for (int j = 0; j < nb; ++j) {
        const int b = j & 1, jn = j + 1;
        const double ci0 = colb[b][lane], ci1 = colb[b][lane + 32];
        const bool owner = jn < nb && w == (jn & 7);
        if (owner) {   // the next pivot's column first: it is on the critical path
            const double s = scol[b][jn];
            double v0 = 0.0, v1 = 0.0;
#pragma unroll
            for (int c = 0; c < 8; ++c) {   // register arrays need compile-time indices
                if (w + 8 * c == jn) {
                    if (jn < 32 && lane >= jn) a[c][0] = fma(-ci0, s, a[c][0]);
                    if (lane + 32 >= jn) a[c][1] = fma(-ci1, s, a[c][1]);
                    v0 = a[c][0];
                    v1 = a[c][1];
                }
            }
            diag_publish(jn, v0, v1, lane, k0, info, dpiv, colb, scol);
        }
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int l = w + 8 * c;
            if (l <= j || l >= nb || (owner && l == jn)) continue;   // warp-uniform
            const double s = scol[b][l];
            if (l < 32) {
                if (lane >= l) a[c][0] = fma(-ci0, s, a[c][0]);
            }
            if (lane + 32 >= l) a[c][1] = fma(-ci1, s, a[c][1]);
        }
        __syncthreads();
    }
    if (threadIdx.x < nb) {
        const double q = sqrt(dpiv[threadIdx.x]);
        dsq[threadIdx.x] = q;
        dinv[threadIdx.x] = 1.0 / q;
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < 8; ++c)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int l = w + 8 * c, i = lane + 32 * h;
            if (i < nb && l < nb)
                A[(size_t)(k0 + i) * lda + k0 + l] = (l < i) ? a[c][h] * dinv[l] : (l == i ? dsq[l] : 0.0);
        }
}

// For each of nrows rows r: solve L y = b in place, b = B[r*ldb + 0 .. nb), L the nb x nb lower triangle
// at Lkk (row stride ldl). With L = U D (U unit lower, D = diag L): U w = b by forward substitution, then
// y = D^{-1} w. One warp per row; lane l holds entries l and l + 32.
__global__ void __launch_bounds__(256) trsv_rows_kernel(const double* __restrict__ Lkk, int ldl, int nb,
                                                         double* __restrict__ B, int ldb, int nrows) {
    __shared__ double U[CH_NB][CH_NB + 1];
    __shared__ double invd[CH_NB];
    if (threadIdx.x < CH_NB) invd[threadIdx.x] = threadIdx.x < nb ? 1.0 / Lkk[(size_t)threadIdx.x * ldl + threadIdx.x] : 0.0;
    __syncthreads();
    for (int idx = threadIdx.x; idx < CH_NB * CH_NB; idx += blockDim.x) {
        int i = idx >> 6, j = idx & 63;
        U[i][j] = (i < nb && j < i) ? Lkk[(size_t)i * ldl + j] * invd[j] : 0.0;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int warps = blockDim.x >> 5;
    const double id0 = invd[lane], id1 = invd[lane + 32];
    for (int r = blockIdx.x * warps + (threadIdx.x >> 5); r < nrows; r += gridDim.x * warps) {
        double* b = B + (size_t)r * ldb;
        double v0 = lane < nb ? b[lane] : 0.0;
        double v1 = lane + 32 < nb ? b[lane + 32] : 0.0;
        const int n0 = min(nb, 32);
        for (int j = 0; j < n0; ++j) {
            const double wj = __shfl_sync(0xffffffffu, v0, j);
            if (lane > j) v0 = fma(-U[lane][j], wj, v0);
            v1 = fma(-U[lane + 32][j], wj, v1);
        }
        for (int j = 32; j < nb; ++j) {
            const double wj = __shfl_sync(0xffffffffu, v1, j - 32);
            if (lane + 32 > j) v1 = fma(-U[lane + 32][j], wj, v1);
        }
        if (lane < nb) b[lane] = v0 * id0;
        if (lane + 32 < nb) b[lane + 32] = v1 * id1;
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

cudaError_t trsm_lower_f64(const double* L, int ldl, int n, double* B, int ldb, int nrows, cudaStream_t st,
                           OzakiWs* oz, int* status_dev) {
    if (nrows <= 0 || n <= 0) return cudaSuccess;
    for (int k0 = 0; k0 < n; k0 += CH_NB) {
        int nb = min(CH_NB, n - k0);
        { trsv_rows_kernel<<<row_blocks(nrows), 256, 0, st>>>(L + (size_t)k0 * ldl + k0, ldl, nb, B + k0, ldb, nrows); count_launch(); }
        int k1 = k0 + nb;
        if (k1 >= n) break;
        // B[r][k1 + i] -= sum_k L[k1 + i][k0 + k] Y[r][k0 + k]
        cudaError_t e;
        if (oz && nb == CH_NB && n - k1 <= oz->cap_rows && nrows <= oz->cap2) {
            e = ozaki_gemm_update(L + (size_t)k1 * ldl + k0, ldl, n - k1, B + k0, ldb, nrows, B + k1, ldb, *oz,
                                  status_dev, st);
        } else {
            EpiStore epi{B + k1, ldb, -1.0, nullptr, 1.0};
            e = gemm_f64<true, true>(n - k1, nrows, nb, L + (size_t)k1 * ldl + k0, ldl, B + k0, ldb, TileRange{0, 0},
                                     epi, st);
        }
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

}  // namespace diam
