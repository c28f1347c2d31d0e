/*
 * diam_ops.h -- op-level entry points of the DIAM library: the building blocks of one sampler step,
 * callable on caller-owned device buffers (all pointers below are device pointers unless marked host).
 * They run on the given cudaStream_t (NULL: the default stream) and return a diam_status; none of them
 * allocates device memory or synchronises the stream except where stated.
 */
#ifndef DIAM_OPS_H
#define DIAM_OPS_H

#include "diam.h"

#ifdef __cplusplus
extern "C" {
#endif

/* The Gaussian draws W of Algorithm 1 for steps t0 .. t0+n_steps-1 and chains 0 .. P-1: row r = s*P + p
 * of out (row stride ld >= d, entries d .. ld-1 set to 0) holds W for chain p at step t0 + s. Philox4x32-10
 * (Salmon et al., SC'11) keyed by (seed, problem_id), Box-Muller in IEEE FP32 (bit-reproducible).
 * kind: 0 = FP32, 1 = FP64 (the FP32 draw widened), 2 = BF16 bits (the FP32 draw rounded to nearest even). */
DIAM_API diam_status diam_op_normals(uint64_t seed, uint32_t problem_id, int64_t t0, int32_t n_steps, int32_t P, int32_t d,
                            int32_t ld, int32_t kind, void* out, void* stream);

/* The library's bounded device wait as an op: one GPU thread waits until the device int *flag equals expected,
 * or until limit_cycles SM clock cycles (at most 2^33, about four seconds) have passed, whichever comes first;
 * DIAM_ETIMEOUT in the second case. The library's kernels bound every wait of theirs this way (a clock limit,
 * then a recorded timeout instead of a hang); callers that order GPU work on a flag in device memory get the
 * same guarantee. Nothing is left running when it returns; the device stays usable. Synchronises the stream. */
DIAM_API diam_status diam_op_wait_flag(const int32_t* flag, int32_t expected, int64_t limit_cycles, void* stream);

/* In-place lower Cholesky factor (Algorithm 1, "A_n = Cholesky(C_n)") of the n x n lower triangle of A
 * (row-major, stride lda, FP64); the strict upper triangle is zeroed. *info_host receives 0, or the
 * 1-based index of the first non-positive pivot. Synchronises the stream. */
DIAM_API diam_status diam_op_cholesky_f64(int32_t n, double* A, int32_t lda, int32_t* info_host, void* stream);

/* diam_op_cholesky_f64 with the trailing updates on the BF16 tensor cores, FP64-accurate by the error-free
 * splitting of Ozaki, Ogita, Oishi and Rump (2012): each 64-wide panel row is cut into 7 BF16 integer
 * slices under a power-of-two scale, slice products are summed exactly in FP32 tensor memory, grouped by
 * weight and combined as 64-bit integers (the dropped terms are of the size of an FP64 GEMM's rounding).
 * This is the factorisation the BF16 sampler mode uses for its refresh: the chain of 64 x 64 diagonal
 * blocks, the rest of each panel and the trailing updates run on three streams of its own, ordered after
 * the work already on `stream` and joined back to it. Allocates its workspace (the panels' slices, about
 * 2 x 448 x n BF16). Synchronises the stream; DIAM_ETIMEOUT on a device-side timeout. */
DIAM_API diam_status diam_op_cholesky_f64_tc(int32_t n, double* A, int32_t lda, int32_t* info_host, void* stream);

/* For nrows right-hand sides stored as rows of B (row r at B + r*ldb, n entries): B_r <- L^{-1} B_r with L
 * lower triangular (n x n, stride ldl, FP64). This is z = A_n^{-1}(x - x_ref) for every chain. */
DIAM_API diam_status diam_op_trsm_lower_f64(int32_t n, int32_t nrows, const double* L, int32_t ldl, double* B, int32_t ldb,
                                   void* stream);

/* diam_op_trsm_lower_f64 with the block updates B[:, k1:] -= Y L[k1:, block]^T on the BF16 tensor cores,
 * FP64-accurate by the same Ozaki splitting as diam_op_cholesky_f64_tc (the re-solve of z after a refresh
 * in the BF16 sampler mode). Allocates its workspace (7 x 64 x (n + nrows) BF16). Synchronises the stream;
 * DIAM_ETIMEOUT on a device-side timeout. */
DIAM_API diam_status diam_op_trsm_lower_f64_tc(int32_t n, int32_t nrows, const double* L, int32_t ldl, double* B,
                                               int32_t ldb, void* stream);

/* D[n*ldd + m] = scale * sum_k A[m*lda + k] (B[n*ldb + k] + B2[n*ldb + k]) on the tensor cores (tcgen05):
 * A (M x K) and B, B2 (N x K) BF16 bits, K-contiguous, K, lda, ldb multiples of 64, 16-byte aligned
 * pointers; B2 may be NULL; FP32 accumulation; D FP32. a_lower: A is lower triangular and K blocks past
 * each 128-row tile are skipped (the batched noise product xi = beta alpha A_n W of Algorithm 1); A's strict
 * upper triangle must then be zero (which of its blocks are read depends on the tiling).
 * Synchronises the stream and reports a device-side timeout as DIAM_ETIMEOUT. */
DIAM_API diam_status diam_op_gemm_bf16(int32_t M, int32_t N, int32_t K, const uint16_t* A, int32_t lda, const uint16_t* B,
                              const uint16_t* B2, int32_t ldb, int32_t a_lower, float scale, float* D, int32_t ldd,
                              void* stream);

/* diam_op_gemm_bf16 with an explicit tile width over N (bn = 32, 64, 128, or 256 when B2 is NULL): the
 * candidates the tile autotuner times for each product shape. DIAM_EINVAL for other widths. Synchronises the
 * stream. */
DIAM_API diam_status diam_op_gemm_bf16_tile(int32_t M, int32_t N, int32_t K, const uint16_t* A, int32_t lda,
                                            const uint16_t* B, const uint16_t* B2, int32_t ldb, int32_t a_lower,
                                            float scale, float* D, int32_t ldd, int32_t bn, void* stream);

/* The product of diam_op_gemm_bf16 (same arguments, same result within FP32 summation order; with a_lower, A's
 * strict upper triangle must be zero, as there) for callers
 * that cannot allocate device memory: code whose device memory belongs to its own pool and forbids outside
 * allocations, or code on a latency-critical path that cannot afford the device-wide synchronisation that
 * cudaMalloc and cudaFree may cause.
 * The paper has no counterpart; this is an interface convenience of this library.
 * It never calls cudaMalloc / cudaFree: its scratch (split-K partial products, a status word) is one fixed
 * 16 MiB device array inside the library, held by every GPU that loads the library until the process exits.
 * Limits: M * N at most 4,194,240 (the partials of one split must fit the array); larger products are
 * rejected with DIAM_EINVAL. The first call on each device looks up the array's device address; make that
 * call before any stream capture. All calls share the array: calls that overlap on the GPU (other streams,
 * other host threads) race and must be serialised by the caller. Synchronises the stream. */
DIAM_API diam_status diam_op_gemm_bf16_noalloc(int32_t M, int32_t N, int32_t K, const uint16_t* A, int32_t lda,
                                               const uint16_t* B, const uint16_t* B2, int32_t ldb, int32_t a_lower,
                                               float scale, float* D, int32_t ldd, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* DIAM_OPS_H */
