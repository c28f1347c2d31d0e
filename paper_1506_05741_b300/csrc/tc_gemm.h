// tc_gemm.h -- BF16 tensor-core (tcgen05, sm_103a) GEMM used by the BF16 mode of the sampler.
//
//   acc(n, m) = sum_k A[m*lda + k] * B[n*ldb + k]   (+ B2[n*ldb + k] accumulated into the same acc)
//
// A and B are BF16, K-contiguous (row-major with K the fastest index), K a multiple of 64 and the row
// strides multiples of 8 elements; accumulation is FP32 in tensor memory. Tiles are 128 (m) x BN (n).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

struct CUtensorMap_st;

namespace diam {

// 2D BF16 tensor map over rows x ld (ld = padded row length, multiple of 64), box 64 x box_rows, 128-byte
// swizzle; cached per (pointer, rows, ld, box_rows).
bool make_map(struct CUtensorMap_st* map, const void* ptr, int rows, int ld, int box_rows);

enum TcMode : int {
    TC_STORE = 0,   // D[n*ldd + m] = scale * acc (FP32), scale = *scale_dev
    TC_TARGET = 1,  // partial[m_tile * N + n] = sum_m f(acc(n, m)): -(y_m - tanh acc)^2 inv2s2 or -acc^2/2
    TC_FOLD = 2,    // lower triangle n >= m: M2[n*ldm + m] += acc - s_n s_m inb + delta_n delta_m w
    TC_GELU = 3     // z = acc + bias[m]: Zout[n*ldz + m] = z (FP32, optional), Hout[n*ldo + m] = bf16(GELU(z))
};

struct TcEpi {
    int mode;
    float* D;
    int ldd;
    const double* scale_dev;
    double* partial;
    const double* y;
    double inv2s2;
    int tanh_mode;
    double* M2;
    int ldm;
    const double* s;
    const double* delta;
    double inb, w;
    size_t split_stride;   // TC_STORE with split K: distance between partial planes (elements)
    uint16_t* Hout;        // TC_GELU
    int ldo;
    float* Zout;
    int ldz;
    const float* bias;
    const int* n_dev;      // optional: the product uses only the first *n_dev rows of B (n-tiles past it exit)
};

// a_lower: A is lower triangular (A[m][k] = 0 for k > m), K blocks past the m-tile are skipped.
// status_dev: receives a non-zero code if a bounded wait inside the kernel expired.
// bn: tile width over N (32, 64, 128 or 256; see tc_autotune).
cudaError_t tc_gemm_bf16(int M, int N, int K, const uint16_t* A, int lda, const uint16_t* B, const uint16_t* B2,
                         int ldb, int a_lower, const TcEpi& epi, int* status_dev, cudaStream_t st, int bn = 128);

// D = op(A + A2, B): the product with a second A operand (same layout as A) summed in, as a second pass over
// K (A2 with B). No B2.
cudaError_t tc_gemm_bf16_a2(int M, int N, int K, const uint16_t* A, const uint16_t* A2, int lda, const uint16_t* B,
                            int ldb, int a_lower, const TcEpi& epi, int* status_dev, cudaStream_t st, int bn = 128);

// Split-K TC_STORE: grid z = splits, K blocks divided evenly; *used receives the number of partial planes.
cudaError_t tc_gemm_bf16_splitk(int M, int N, int K, const uint16_t* A, int lda, const uint16_t* B, const uint16_t* B2,
                                int ldb, int splits, const TcEpi& epi, int* status_dev, cudaStream_t st, int* used,
                                int bn = 128);

// Tile autotuner: the fastest tile width (32, 64, 128) for this product, timed on the given buffers once
// per shape (cached); best_ms (optional) receives its launch time. Must not be called during capture.
int tc_autotune(int M, int N, int K, const uint16_t* A, int lda, const uint16_t* B, const uint16_t* B2, int ldb,
                int splits, int a_lower, const TcEpi& epi, int* status_dev, cudaStream_t st, float* best_ms);

// out[c*ldo + r] = bf16(in[r*ldi + c]) (round to nearest even) for r < rows, c < cols; out[c*ldo + r] = 0 for
// rows <= r < ldo, so the K padding of the transposed operand is zero
cudaError_t transpose_f32_bf16(const float* in, int ldi, int rows, int cols, uint16_t* out, int ldo, cudaStream_t st);

}  // namespace diam
