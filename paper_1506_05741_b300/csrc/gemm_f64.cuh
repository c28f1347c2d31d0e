// gemm_f64.cuh -- register-tiled FP64 (DFMA) GEMM with pluggable epilogues.
//
//   acc(n, m) = sum_k A(m, k) * B(n, k),   k in [0, K) (or [0, min(K, m0 + 64)) for a lower-triangular A)
//   A(m, k) = A_K ? A[m*lda + k] : A[k*lda + m]      B(n, k) = B_K ? B[n*ldb + k] : B[k*ldb + n]
//
// Output (n, m) follows the chain-major layout of the sampler (row n, column m). 64 x 64 output tile per
// 256-thread block, 4 x 4 per thread, K in steps of 16 through shared memory. B300's FP64 rate (about
// 1 TFLOP/s for the whole GPU) is far below what shared memory and HBM can feed, so the kernel is
// DFMA-issue bound by construction.
#pragma once
#include "common.cuh"

namespace diam {

constexpr int GF_BM = 64, GF_BN = 64, GF_BK = 16;

struct TileRange {
    int a_lower;    // A(m, k) = 0 for k > m: the K loop of an m-tile stops at m0 + 64
    int out_lower;  // only n >= m is produced: tiles strictly above the diagonal are skipped
};

template <bool A_K, bool B_K, class Epi>
__global__ void __launch_bounds__(256) gemm_f64_kernel(int M, int N, int K, const double* __restrict__ A, int lda,
                                                       const double* __restrict__ B, int ldb, TileRange tr, Epi epi) {
    __shared__ double As[GF_BK][GF_BM + 1];
    __shared__ double Bs[GF_BK][GF_BN + 1];
    const int m0 = blockIdx.x * GF_BM, n0 = blockIdx.y * GF_BN;
    if (tr.out_lower && n0 + GF_BN - 1 < m0) return;  // uniform per block: every (n, m) has n < m
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    int kend = K;
    if (tr.a_lower) kend = min(K, m0 + GF_BM);
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

    for (int k0 = 0; k0 < kend; k0 += GF_BK) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            int idx = threadIdx.x + r * 256;
            int mm, kk;
            if (A_K) { mm = idx >> 4; kk = idx & 15; } else { kk = idx >> 6; mm = idx & 63; }
            int gm = m0 + mm, gk = k0 + kk;
            double v = 0.0;
            if (gm < M && gk < kend) v = A_K ? A[(size_t)gm * lda + gk] : A[(size_t)gk * lda + gm];
            As[kk][mm] = v;
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            int idx = threadIdx.x + r * 256;
            int nn, kk;
            if (B_K) { nn = idx >> 4; kk = idx & 15; } else { kk = idx >> 6; nn = idx & 63; }
            int gn = n0 + nn, gk = k0 + kk;
            double v = 0.0;
            if (gn < N && gk < kend) v = B_K ? B[(size_t)gn * ldb + gk] : B[(size_t)gk * ldb + gn];
            Bs[kk][nn] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GF_BK; ++kk) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][tx + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][ty + 16 * j];
#pragma unroll
            for (int j = 0; j < 4; ++j)
#pragma unroll
                for (int i = 0; i < 4; ++i) acc[j][i] = fma(a[i], b[j], acc[j][i]);
        }
        __syncthreads();
    }
    epi.apply(acc, m0, n0, tx, ty, M, N, tr.out_lower);
}

// ---------------------------------------------------------------------------------------------
// Epilogues. acc[j][i] is output (n0 + ty + 16 j, m0 + tx + 16 i).

// D[n*ldd + m] = alpha * (*alpha_dev) * acc + beta_d * D
struct EpiStore {
    double* D;
    int ldd;
    double alpha;
    const double* alpha_dev;
    double beta_d;
    __device__ void apply(double (&acc)[4][4], int m0, int n0, int tx, int ty, int M, int N, int out_lower) const {
        double a = alpha * (alpha_dev ? *alpha_dev : 1.0);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int n = n0 + ty + 16 * j;
            if (n >= N) continue;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                int m = m0 + tx + 16 * i;
                if (m >= M || (out_lower && n < m)) continue;
                double* p = D + (size_t)n * ldd + m;
                *p = (beta_d == 0.0) ? a * acc[j][i] : fma(a, acc[j][i], beta_d * *p);
            }
        }
    }
};

// Per-chain partial log-density of a linear-map target, one value per (m-tile, chain n):
//   DENSE: sum_m -u^2 / 2;   TANH: sum_m -(y_m - tanh u)^2 inv2s2;   u = acc(n, m)
struct EpiTargetReduce {
    double* partial;    // [gridDim.x][N]
    const double* y;
    double inv2s2;
    int tanh_mode;
    __device__ void apply(double (&acc)[4][4], int m0, int n0, int tx, int ty, int M, int N, int) const {
        __shared__ double red[16][GF_BN + 1];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            double s = 0.0;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                int m = m0 + tx + 16 * i;
                if (m < M) {
                    double u = acc[j][i];
                    if (tanh_mode) {
                        double r = y[m] - tanh(u);
                        s -= r * r * inv2s2;
                    } else {
                        s -= 0.5 * u * u;
                    }
                }
            }
            red[tx][ty + 16 * j] = s;
        }
        __syncthreads();
        if (threadIdx.x < GF_BN) {
            int nn = threadIdx.x;
            double s = 0.0;
            for (int q = 0; q < 16; ++q) s += red[q][nn];
            if (n0 + nn < N) partial[(size_t)blockIdx.x * N + n0 + nn] = s;
        }
    }
};

// Moment fold of one interval (pairwise update of Chan, Golub and LeVeque), lower triangle n >= m:
//   M2[n][m] += acc - s_n s_m / nb + delta_n delta_m w
struct EpiFold {
    double* M2;
    int ld;
    const double* s;      // sums of the centred samples of the interval
    const double* delta;  // interval mean - running mean
    double inb;           // 1 / nb
    double w;             // n nb / (n + nb)
    __device__ void apply(double (&acc)[4][4], int m0, int n0, int tx, int ty, int M, int N, int) const {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int n = n0 + ty + 16 * j;
            if (n >= N) continue;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                int m = m0 + tx + 16 * i;
                if (m >= M || n < m) continue;
                double v = acc[j][i] - s[n] * s[m] * inb + delta[n] * delta[m] * w;
                M2[(size_t)n * ld + m] += v;
            }
        }
    }
};

template <bool A_K, bool B_K, class Epi>
inline cudaError_t gemm_f64(int M, int N, int K, const double* A, int lda, const double* B, int ldb, TileRange tr,
                            const Epi& epi, cudaStream_t st) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    dim3 grid((M + GF_BM - 1) / GF_BM, (N + GF_BN - 1) / GF_BN);
    { gemm_f64_kernel<A_K, B_K, Epi><<<grid, 256, 0, st>>>(M, N, K, A, lda, B, ldb, tr, epi); count_launch(); }
    return cudaGetLastError();
}

}  // namespace diam
