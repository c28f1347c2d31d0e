// linalg.h -- host entry points of the FP64 dense kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace diam {

// Workspace of the tensor-core (Ozaki-split) updates: BF16 slices of the operands' rows and row exponents.
struct OzakiWs {
    uint16_t* SL = nullptr;    // 2 x cap_rows x 448: first operand (two buffers: the factorisation's lookahead)
    int* ex = nullptr;         // 2 x cap_rows
    int cap_rows = 0;
    uint16_t* SL2 = nullptr;   // 2 x cap2 x 448: right-hand sides of the triangular solve (two buffers)
    int* ex2 = nullptr;        // 2 x cap2
    int cap2 = 0;
    uint16_t* SLP = nullptr;   // capP x 448: every 64-column panel below the diagonal of the solve's factor
    int* exP = nullptr;        // capP
    int64_t capP = 0;
    // streams and events of the factorisation's lookahead, created on first use (ozaki_ws_release frees them):
    // hi carries the chain of diagonal blocks, mid the rest of each panel, lo the trailing updates. The chain
    // runs at the highest stream priority, mid just below it, the trailing updates at the lowest unless
    // lo_high is set (a factorisation running beside other work, whose chain waits on those updates)
    bool lo_high = false;
    cudaStream_t hi = nullptr, mid = nullptr, lo = nullptr;
    cudaEvent_t ev_in = nullptr, ev_slice = nullptr, ev_rest = nullptr, ev_lo = nullptr, ev_diag = nullptr,
                ev_mid = nullptr;
};

// Bytes of the slice buffers a workspace for rows / rows2 needs (SL: both buffers).
inline size_t ozaki_sl_bytes(int rows) { return sizeof(uint16_t) * 2 * (size_t)rows * 448; }
inline size_t ozaki_ex_bytes(int rows) { return sizeof(int) * 2 * (size_t)rows; }

// Rows of all 64-column panels below the diagonal blocks of an n x n lower triangle:
// sum over k of max(0, n - 64 (k + 1)).
inline int64_t ozaki_panel_rows(int n) {
    int64_t r = 0;
    for (int k1 = 64; k1 < n; k1 += 64) r += n - k1;
    return r;
}

// Destroy the workspace's streams and events (device buffers belong to the caller).
void ozaki_ws_release(OzakiWs& ws);

// C[n][m] -= sum_k P[n][k] P[m][k] for n >= m (k < 64), FP64-accurate on the BF16 tensor cores; P (rows x 64,
// stride lda) and C (stride ldc) FP64. status_dev receives DEV_TIMEOUT if a bounded wait expired.
cudaError_t ozaki_trailing_update(const double* P, int lda, int rows, double* C, int ldc, OzakiWs& ws, int* status_dev,
                                  cudaStream_t st);

// Slice the rows x 64 panel P (stride lda) into buffer buf (0 or 1) of the workspace.
cudaError_t ozaki_slice_panel(const double* P, int lda, int rows, int buf, OzakiWs& ws, cudaStream_t st);

// C[n][m] -= sum_k P[r0 + m][k] P[c0 + n][k] for m < Ma, n < Nb (and n >= m when lower), P the panel sliced
// into buffer buf.
cudaError_t ozaki_update_sliced(int buf, int r0, int Ma, int c0, int Nb, double* C, int ldc, int lower, OzakiWs& ws,
                                int* status_dev, cudaStream_t st);

// Slices of every panel of the lower triangle L (n x n, stride ldl) into ws.SLP / ws.exP: panel k (rows
// 64 (k + 1) .. n - 1 of columns 64 k .. 64 k + 63) follows the panels before it.
cudaError_t ozaki_slice_panels(const double* L, int ldl, int n, OzakiWs& ws, cudaStream_t st);

// C[n][m] -= sum_k A[m][k] B[n][k] from slices already made: A rows SA (Ma rows, exponents exA), B rows SB
// (Nb rows, exponents exB); lower: only n >= m.
cudaError_t ozaki_update_raw(const uint16_t* SA, int Ma, const int* exA, const uint16_t* SB, int Nb, const int* exB,
                             double* C, int ldc, int lower, int* status_dev, cudaStream_t st);

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
