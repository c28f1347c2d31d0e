// linalg_f64.cu -- FP64 Cholesky factorisation and triangular solves on the GPU.
//
// Algorithm 1 refreshes the proposal factor with A_n = Cholesky(C_n) every n_lag steps. Here that is a
// blocked right-looking factorisation (block 64): the diagonal block is factored unblocked in shared
// memory, the panel below it is solved row by row (one warp per row), and the trailing lower triangle
// takes a DFMA rank-64 update. The same row solve, applied to many right-hand sides, gives
// z = A_n^{-1}(x - x_ref) for every chain when the factor changes.
#include "linalg.h"
#include "gemm_f64.cuh"
#include "ozaki_slice.cuh"

namespace diam {

constexpr int CH_NB = 64;

// 1/D for the pivot chain, with as few FP64 instructions as possible (on B300 each one costs about 64
// cycles of latency, one lane or thirty-two): the seed y0 ~ 1/D (relative error below 2^-21) comes from an
// FP32 reciprocal of D's leading 23 mantissa bits, assembled and taken apart with integer operations; one
// cubic Newton-Raphson step y = y0 (1 + e + e^2), e = 1 - D y0, leaves a relative error of e^3 < 2^-63 plus
// the rounding of its two fused multiply-adds. Outside the exponents where that holds, a division.
__device__ __forceinline__ double recip_pivot(double D) {
    const long long b = __double_as_longlong(D);
    const int e = (int)((b >> 52) & 0x7ff);
    if (e < 2 || e > 2044) return 1.0 / D;
    const float m = __uint_as_float(0x3F800000u | (unsigned)((b >> 29) & 0x7FFFFF));   // [1, 2)
    const unsigned rb = __float_as_uint(__frcp_rn(m));                                 // (0.5, 1]
    const int er = (int)((rb >> 23) & 0xff) - 127;                                     // -1 or 0
    const double y0 = __longlong_as_double(((long long)(er + 2046 - e) << 52) | ((long long)(rb & 0x7FFFFF) << 29));
    const double eps = fma(-D, y0, 1.0);
    return fma(y0, fma(eps, eps, eps), y0);
}

// D > 0 and finite, from the bits (no FP64 comparison on the pivot chain).
__device__ __forceinline__ bool positive_finite(double D) {
    const long long b = __double_as_longlong(D);
    return b > 0 && ((b >> 52) & 0x7ff) != 0x7ff;
}

// Cholesky of the nb x nb diagonal block at (k0, k0), nb <= 64: lower part in, L out, upper part zeroed.
// LDL^T in shared memory, in sub-panels of 16 columns: pivot j subtracts a_ij (a_lj / D_j) from a_il, leaving
// a_ij = L_ij sqrt(D_j); the square roots are taken once at the end. Inside a sub-panel, per pivot j:
//   - warp 0 (the critical path) updates column j + 1, takes 1 / D_{j+1} and publishes that column and its
//     scaled copy (double-buffered shared columns, and the sub-panel's scaled columns for the rank update);
//   - the warps on the other three schedulers update the sub-panel's columns j + 2 .. (a packed table lists
//     the lower triangle column by column from the last one, so any run of columns is one contiguous range);
// then one barrier. After the sub-panel's pivots every thread takes part in its rank-16 update of the
// columns to its right, so the pivot steps carry only the small in-panel updates.
constexpr int DIAG_THREADS = 512, DIAG_SB = 16;

__device__ __forceinline__ void diag_publish(int c, int q0, double v0, double v1, int lane, int nb, int k0, int* info,
                                             double* dpiv, double (*colb)[CH_NB], double (*scol)[CH_NB],
                                             double (*scp)[CH_NB + 1]) {
    double r = 0.0;
    if (lane == 0) {
        if (positive_finite(v0)) {
            r = recip_pivot(v0);
        } else {   // not positive definite: NaN propagates and the caller discards the factor
            r = __longlong_as_double(0x7ff8000000000000ll);
            if (info) atomicCAS(info, 0, k0 + c + 1);
        }
        dpiv[c] = v0;
    }
    r = __shfl_sync(0xffffffffu, r, 0);
    const int b = c & 1;
    if (c + lane < nb) {
        const double sv = v0 * r;
        colb[b][c + lane] = v0;
        scol[b][c + lane] = sv;
        scp[c - q0][c + lane] = sv;
    }
    if (c + 32 < nb) {   // warp-uniform: the second half exists
        if (c + 32 + lane < nb) {
            const double sv = v1 * r;
            colb[b][c + 32 + lane] = v1;
            scol[b][c + 32 + lane] = sv;
            scp[c - q0][c + 32 + lane] = sv;
        }
    }
}

// pre (a panel follows, so column k0 + nb exists): the panel solve's operands are left in places the
// factorisation does not read and clears at its end -- U = L D^{-1} (the unit factor, U_ij = L_ij / L_jj)
// transposed in the block's strict upper triangle, 1 / L_jj in row k0 + j, column k0 + nb -- computed with
// the operations the panel solve would use, so every CTA of it loads them instead of recomputing them.
__global__ void __launch_bounds__(DIAG_THREADS) chol_diag_kernel(double* __restrict__ A, int lda, int k0, int nb,
                                                                 int* info, int pre) {
    __shared__ double a[CH_NB][CH_NB + 1];
    __shared__ double colb[2][CH_NB];          // a_ij, i > j, of the current pivot j
    __shared__ double scol[2][CH_NB];          // a_ij / D_j
    __shared__ double scp[DIAG_SB][CH_NB + 1]; // the current sub-panel's scaled columns
    __shared__ double dpiv[CH_NB];             // D_j
    __shared__ double dsq[CH_NB], dinv[CH_NB];
    __shared__ uint16_t tab[CH_NB * (CH_NB + 1) / 2];   // (i << 8) | l, columns nb-1 down to 0
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    for (int idx = tid; idx < nb * nb; idx += DIAG_THREADS) {
        const int i = idx / nb, l = idx - i * nb;
        a[i][l] = (l <= i) ? A[(size_t)(k0 + i) * lda + k0 + l] : 0.0;
    }
    if (tid < nb) {   // column l = tid: its nb - l elements follow those of the columns right of it
        const int l = tid, off = (nb - l - 1) * (nb - l) / 2;
        for (int r = 0; r < nb - l; ++r) tab[off + r] = (uint16_t)(((l + r) << 8) | l);
    }
    __syncthreads();
    // bulk warps (the three schedulers other than warp 0's, warp w issuing on sub-partition w % 4)
    constexpr int NB_T = (DIAG_THREADS / 32) / 4 * 3 * 32;
    const int bt = (w - (w >> 2) - 1) * 32 + lane;
    auto col_start = [&](int l) { return (nb - l - 1) * (nb - l) / 2; };   // first table entry of column l
    for (int q0 = 0; q0 < nb; q0 += DIAG_SB) {
        const int q1 = min(nb, q0 + DIAG_SB);
        if (w == 0)
            diag_publish(q0, q0, q0 + lane < nb ? a[q0 + lane][q0] : 0.0, q0 + 32 + lane < nb ? a[q0 + 32 + lane][q0] : 0.0,
                         lane, nb, k0, info, dpiv, colb, scol, scp);
        __syncthreads();
        for (int j = q0; j < q1; ++j) {
            const int b = j & 1, jn = j + 1;
            if (w == 0) {
                if (jn < q1) {
                    const double s = scol[b][jn];
                    const int i0 = jn + lane, i1 = jn + lane + 32;
                    double v0 = 0.0, v1 = 0.0;
                    if (i0 < nb) {
                        v0 = fma(-colb[b][i0], s, a[i0][jn]);
                        a[i0][jn] = v0;
                    }
                    if (jn + 32 < nb) {   // warp-uniform, so no FP64 instruction is issued for an empty half
                        if (i1 < nb) {
                            v1 = fma(-colb[b][i1], s, a[i1][jn]);
                            a[i1][jn] = v1;
                        }
                    }
                    diag_publish(jn, q0, v0, v1, lane, nb, k0, info, dpiv, colb, scol, scp);
                }
            } else if ((w & 3) && j + 2 < q1) {
                // columns j + 2 .. q1 - 1 of the sub-panel: table entries [start(q1 - 1), start(j + 1))
                const int e0 = col_start(q1 - 1), e1 = col_start(j + 1);
                for (int e = e0 + bt; e < e1; e += NB_T) {
                    const int t = tab[e], i = t >> 8, l = t & 255;
                    a[i][l] = fma(-colb[b][i], scol[b][l], a[i][l]);
                }
            }
            __syncthreads();
        }
        if (q1 < nb) {   // rank-(q1 - q0) update of the columns q1 .. nb - 1: table entries [0, start(q1 - 1))
            const int e1 = col_start(q1 - 1), kn = q1 - q0;
            for (int e = tid; e < e1; e += DIAG_THREADS) {
                const int t = tab[e], i = t >> 8, l = t & 255;
                double s0 = 0.0, s1 = 0.0;   // two partial sums: half the dependent FP64 chain
                for (int k = 0; k + 1 < kn; k += 2) {
                    s0 = fma(a[i][q0 + k], scp[k][l], s0);
                    s1 = fma(a[i][q0 + k + 1], scp[k + 1][l], s1);
                }
                if (kn & 1) s0 = fma(a[i][q1 - 1], scp[kn - 1][l], s0);
                a[i][l] -= s0 + s1;
            }
            __syncthreads();
        }
    }
    if (tid < nb) {
        const double qv = sqrt(dpiv[tid]);
        dsq[tid] = qv;
        dinv[tid] = 1.0 / qv;
    }
    __syncthreads();
    for (int idx = tid; idx < nb * nb; idx += DIAG_THREADS) {
        const int i = idx / nb, l = idx - i * nb;
        double v = 0.0;
        if (l < i) v = a[i][l] * dinv[l];
        else if (l == i) v = dsq[l];
        else if (pre) v = (a[l][i] * dinv[i]) * dinv[i];   // U_li = L_li (1 / L_ii), at (i, l)
        A[(size_t)(k0 + i) * lda + k0 + l] = v;
    }
    if (pre && tid < nb) A[(size_t)(k0 + tid) * lda + k0 + nb] = dinv[tid];
}

// For each of nrows rows r: solve L y = b in place, b = B[r*ldb + 0 .. nb), L the nb x nb lower triangle
// at Lkk (row stride ldl). With L = U D (U unit lower, D = diag L): U w = b by forward substitution, then
// y = D^{-1} w. One warp per row; lane l holds entries l and l + 32.
// With SL != nullptr (nb = 64), each solved row is also cut into its Ozaki slices (row r at SL + r * 448,
// exponent in ex[r]) for the tensor-core update that follows.
// pre: U and 1 / L_jj were left by chol_diag_kernel (U transposed above the block, the reciprocals in the
// column right of it) and are loaded; otherwise they are computed here.
__global__ void __launch_bounds__(256) trsv_rows_kernel(const double* __restrict__ Lkk, int ldl, int nb,
                                                         double* __restrict__ B, int ldb, int nrows,
                                                         uint16_t* __restrict__ SL = nullptr, int* __restrict__ ex = nullptr,
                                                         int pre = 0) {
    __shared__ double U[CH_NB][CH_NB + 1];
    __shared__ double invd[CH_NB];
    if (pre) {
        if (threadIdx.x < CH_NB) invd[threadIdx.x] = threadIdx.x < nb ? Lkk[(size_t)threadIdx.x * ldl + nb] : 0.0;
        for (int idx = threadIdx.x; idx < CH_NB * CH_NB; idx += blockDim.x) {   // row j of the stored U^T
            const int j = idx >> 6, i = idx & 63;
            U[i][j] = (i < nb && j < i) ? Lkk[(size_t)j * ldl + i] : 0.0;
        }
        __syncthreads();
    } else {
        if (threadIdx.x < CH_NB) invd[threadIdx.x] = threadIdx.x < nb ? 1.0 / Lkk[(size_t)threadIdx.x * ldl + threadIdx.x] : 0.0;
        __syncthreads();
        for (int idx = threadIdx.x; idx < CH_NB * CH_NB; idx += blockDim.x) {
            int i = idx >> 6, j = idx & 63;
            U[i][j] = (i < nb && j < i) ? Lkk[(size_t)i * ldl + j] * invd[j] : 0.0;
        }
        __syncthreads();
    }
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
        v0 *= id0;
        v1 *= id1;
        if (lane < nb) b[lane] = v0;
        if (lane + 32 < nb) b[lane + 32] = v1;
        if (SL) {
            const int e = ozaki_slice_row(v0, v1, lane, SL + (size_t)r * OZ_LD);
            if (lane == 0) ex[r] = e;
        }
    }
}

// The panel's top rows on the factorisation's critical path: trsv_rows_kernel's solve (pre: U and 1 / L_jj as
// chol_diag_kernel left them) with one warp per CTA and U read from global memory (L2) as the substitution goes,
// so that each row has an SM's FP64 pipe to itself and no CTA waits for a shared-memory copy of U. Slices as
// trsv_rows_kernel's (nb = 64).
__global__ void __launch_bounds__(32) trsv_top_kernel(const double* __restrict__ Lkk, int ldl, double* __restrict__ B,
                                                      int ldb, int nrows, uint16_t* __restrict__ SL, int* __restrict__ ex) {
    const int r = blockIdx.x, lane = threadIdx.x;
    if (r >= nrows) return;
    const double id0 = Lkk[(size_t)lane * ldl + CH_NB], id1 = Lkk[(size_t)(lane + 32) * ldl + CH_NB];
    double* b = B + (size_t)r * ldb;
    double v0 = b[lane], v1 = b[lane + 32];
#pragma unroll 8
    for (int j = 0; j < 32; ++j) {   // U_ij for i > j is stored at (j, i)
        const double u0 = Lkk[(size_t)j * ldl + lane], u1 = Lkk[(size_t)j * ldl + lane + 32];
        const double wj = __shfl_sync(0xffffffffu, v0, j);
        if (lane > j) v0 = fma(-u0, wj, v0);
        v1 = fma(-u1, wj, v1);
    }
#pragma unroll 8
    for (int j = 32; j < CH_NB; ++j) {
        const double u1 = Lkk[(size_t)j * ldl + lane + 32];
        const double wj = __shfl_sync(0xffffffffu, v1, j - 32);
        if (lane + 32 > j) v1 = fma(-u1, wj, v1);
    }
    v0 *= id0;
    v1 *= id1;
    b[lane] = v0;
    b[lane + 32] = v1;
    const int e = ozaki_slice_row(v0, v1, lane, SL + (size_t)r * OZ_LD);
    if (lane == 0) ex[r] = e;
}

__global__ void zero_upper_kernel(double* A, int lda, int n) {
    int i = blockIdx.y;
    for (int j = i + 1 + blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
        A[(size_t)i * lda + j] = 0.0;
}

static int row_blocks(int nrows) { return max(1, min((nrows + 7) / 8, 148 * 8)); }

static cudaError_t ensure_streams(OzakiWs& ws) {
    if (ws.hi) return cudaSuccess;
    int lo_pri = 0, hi_pri = 0;
    cudaError_t e = cudaDeviceGetStreamPriorityRange(&lo_pri, &hi_pri);   // numerically lower = higher priority
    const int next = hi_pri < lo_pri ? hi_pri + 1 : hi_pri;
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&ws.hi, cudaStreamNonBlocking, hi_pri);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&ws.mid, cudaStreamNonBlocking, next);
    const int lo_use = ws.lo_high ? next : lo_pri;
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&ws.lo, cudaStreamNonBlocking, lo_use);
    for (cudaEvent_t* ev : {&ws.ev_in, &ws.ev_slice, &ws.ev_rest, &ws.ev_lo, &ws.ev_diag, &ws.ev_mid})
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    if (e != cudaSuccess) ozaki_ws_release(ws);
    return e;
}

#define LA_CK(x)                          \
    do {                                  \
        cudaError_t e_ = (x);             \
        if (e_ != cudaSuccess) return e_; \
    } while (0)

// DFMA form: diagonal block, panel solve, DFMA rank-64 update of the trailing lower triangle, in order.
static cudaError_t cholesky_dfma(double* A, int n, int lda, int* info_dev, cudaStream_t st) {
    for (int k0 = 0; k0 < n; k0 += CH_NB) {
        int nb = min(CH_NB, n - k0);
        { chol_diag_kernel<<<1, DIAG_THREADS, 0, st>>>(A, lda, k0, nb, info_dev, k0 + nb < n); count_launch(); }
        int k1 = k0 + nb, rest = n - k1;
        if (rest <= 0) break;
        // panel rows solve x L_kk^T = a, i.e. L_kk x^T = a^T
        { trsv_rows_kernel<<<row_blocks(rest), 256, 0, st>>>(A + (size_t)k0 * lda + k0, lda, nb,
                                                             A + (size_t)k1 * lda + k0, lda, rest, nullptr, nullptr, 1); count_launch(); }
        // trailing lower triangle: A[k1+n][k1+m] -= sum_k L[k1+m][k0+k] L[k1+n][k0+k]
        EpiStore epi{A + (size_t)k1 * lda + k1, lda, -1.0, nullptr, 1.0};
        LA_CK((gemm_f64<true, true>(rest, rest, nb, A + (size_t)k1 * lda + k0, lda, A + (size_t)k1 * lda + k0, lda,
                                    TileRange{0, 1}, epi, st)));
    }
    return cudaGetLastError();
}

// Tensor-core form with lookahead, on three streams. Per 64-column block k (panel P = the rows below the
// diagonal block, T = the trailing triangle):
//   hi:  diagonal block k; solve of P's top 64 rows (the rows of block k + 1, with their Ozaki slices); the
//        update of diagonal block k + 1 by those rows -- all that diagonal block k + 1 needs from block k;
//   mid: solve of the rest of P (with slices); the update of the rest of T's first 64 columns, the panel
//        of block k + 1 (it runs while diagonal block k + 1 is factored; block k + 1's top solve waits on it);
//   lo:  the update of T right of its first 64 columns.
// A region written by the trailing update of block k - 1 is updated for block k only after it (hi and mid
// wait for that update first); a slice buffer (two, alternating by block) is rewritten only after every
// update that reads it.
static cudaError_t cholesky_ozaki(double* A, int n, int lda, int* info_dev, cudaStream_t st, OzakiWs& oz,
                                  int* status_dev) {
    LA_CK(ensure_streams(oz));
    cudaStream_t hi = oz.hi, mid = oz.mid, lo = oz.lo;
    LA_CK(cudaEventRecord(oz.ev_in, st));
    LA_CK(cudaStreamWaitEvent(hi, oz.ev_in, 0));
    LA_CK(cudaStreamWaitEvent(mid, oz.ev_in, 0));
    LA_CK(cudaStreamWaitEvent(lo, oz.ev_in, 0));
    bool rest_pending = false, mid_pending = false;
    for (int k0 = 0; k0 < n; k0 += CH_NB) {
        int nb = min(CH_NB, n - k0);
        { chol_diag_kernel<<<1, DIAG_THREADS, 0, hi>>>(A, lda, k0, nb, info_dev, k0 + nb < n); count_launch(); }
        int k1 = k0 + nb, rest = n - k1;
        if (rest <= 0) break;
        double* T = A + (size_t)k1 * lda + k1;          // trailing block
        const double* Lkk = A + (size_t)k0 * lda + k0;
        double* Pn = A + (size_t)k1 * lda + k0;         // the panel
        const bool tc = nb == CH_NB && rest >= 2 * CH_NB && rest <= oz.cap_rows;
        if (tc) {
            const int buf = (k0 / CH_NB) & 1, rr = rest - CH_NB;
            uint16_t* SLb = oz.SL + (size_t)buf * oz.cap_rows * OZ_LD;
            int* exb = oz.ex + (size_t)buf * oz.cap_rows;
            // hi: the top rows of the panel (updated for this block by the previous block's mid work)
            if (mid_pending) LA_CK(cudaStreamWaitEvent(hi, oz.ev_mid, 0));
            { trsv_top_kernel<<<CH_NB, 32, 0, hi>>>(Lkk, lda, Pn, lda, CH_NB, SLb, exb); count_launch(); }
            LA_CK(cudaEventRecord(oz.ev_diag, hi));
            // mid: the rest of the panel, then the rest of the next 64 columns
            LA_CK(cudaStreamWaitEvent(mid, oz.ev_diag, 0));
            { trsv_rows_kernel<<<row_blocks(rr), 256, 0, mid>>>(Lkk, lda, nb, Pn + (size_t)CH_NB * lda, lda, rr,
                                                                SLb + (size_t)CH_NB * OZ_LD, exb + CH_NB, 1); count_launch(); }
            LA_CK(cudaEventRecord(oz.ev_slice, mid));
            if (rest_pending) LA_CK(cudaStreamWaitEvent(mid, oz.ev_rest, 0));
            LA_CK(ozaki_update_sliced(buf, 0, CH_NB, CH_NB, rr, T + (size_t)CH_NB * lda, lda, 0, oz, status_dev, mid));
            LA_CK(cudaEventRecord(oz.ev_mid, mid));
            mid_pending = true;
            // hi: the next diagonal block
            if (rest_pending) LA_CK(cudaStreamWaitEvent(hi, oz.ev_rest, 0));
            LA_CK(ozaki_update_sliced(buf, 0, CH_NB, 0, CH_NB, T, lda, 1, oz, status_dev, hi));
            // lo: the rest of the trailing triangle
            LA_CK(cudaStreamWaitEvent(lo, oz.ev_slice, 0));
            LA_CK(ozaki_update_sliced(buf, CH_NB, rr, CH_NB, rr, T + (size_t)CH_NB * lda + CH_NB, lda, 1, oz, status_dev,
                                      lo));
            LA_CK(cudaEventRecord(oz.ev_rest, lo));
            rest_pending = true;
        } else {   // the last blocks, in order on hi
            if (mid_pending) LA_CK(cudaStreamWaitEvent(hi, oz.ev_mid, 0));
            if (rest_pending) LA_CK(cudaStreamWaitEvent(hi, oz.ev_rest, 0));
            mid_pending = rest_pending = false;
            { trsv_rows_kernel<<<row_blocks(rest), 256, 0, hi>>>(Lkk, lda, nb, Pn, lda, rest, nullptr, nullptr, 1); count_launch(); }
            EpiStore epi{T, lda, -1.0, nullptr, 1.0};
            LA_CK((gemm_f64<true, true>(rest, rest, nb, Pn, lda, Pn, lda, TileRange{0, 1}, epi, hi)));
        }
    }
    if (mid_pending) LA_CK(cudaStreamWaitEvent(hi, oz.ev_mid, 0));
    if (rest_pending) LA_CK(cudaStreamWaitEvent(hi, oz.ev_rest, 0));
    dim3 g(max(1, min(32, (n + 255) / 256)), n);
    { zero_upper_kernel<<<g, 256, 0, hi>>>(A, lda, n); count_launch(); }
    LA_CK(cudaEventRecord(oz.ev_lo, hi));
    LA_CK(cudaStreamWaitEvent(st, oz.ev_lo, 0));
    return cudaGetLastError();
}

cudaError_t cholesky_f64(double* A, int n, int lda, int* info_dev, cudaStream_t st, OzakiWs* oz, int* status_dev) {
    if (oz) return cholesky_ozaki(A, n, lda, info_dev, st, *oz, status_dev);
    LA_CK(cholesky_dfma(A, n, lda, info_dev, st));
    dim3 g(max(1, min(32, (n + 255) / 256)), n);
    { zero_upper_kernel<<<g, 256, 0, st>>>(A, lda, n); count_launch(); }
    return cudaGetLastError();
}

// DFMA form of the blocked solve: panel solve of the right-hand sides, DFMA update of the columns right
// of the block.
static cudaError_t trsm_dfma(const double* L, int ldl, int n, double* B, int ldb, int nrows, cudaStream_t st) {
    for (int k0 = 0; k0 < n; k0 += CH_NB) {
        int nb = min(CH_NB, n - k0);
        { trsv_rows_kernel<<<row_blocks(nrows), 256, 0, st>>>(L + (size_t)k0 * ldl + k0, ldl, nb, B + k0, ldb, nrows); count_launch(); }
        int k1 = k0 + nb;
        if (k1 >= n) break;
        // B[r][k1 + i] -= sum_k L[k1 + i][k0 + k] Y[r][k0 + k]
        EpiStore epi{B + k1, ldb, -1.0, nullptr, 1.0};
        LA_CK((gemm_f64<true, true>(n - k1, nrows, nb, L + (size_t)k1 * ldl + k0, ldl, B + k0, ldb, TileRange{0, 0},
                                    epi, st)));
    }
    return cudaGetLastError();
}

// Tensor-core form with lookahead: the panels of L are sliced once up front; per block, on the
// high-priority stream, the panel solve of the right-hand sides (which also slices them) and the update of
// the next 64 columns; the update of the columns right of those runs on the second stream and overlaps the
// next block's solve.
static cudaError_t trsm_ozaki(const double* L, int ldl, int n, double* B, int ldb, int nrows, cudaStream_t st,
                              OzakiWs& oz, int* status_dev) {
    LA_CK(ensure_streams(oz));
    cudaStream_t hi = oz.hi, lo = oz.lo;
    LA_CK(cudaEventRecord(oz.ev_in, st));
    LA_CK(cudaStreamWaitEvent(hi, oz.ev_in, 0));
    LA_CK(cudaStreamWaitEvent(lo, oz.ev_in, 0));
    LA_CK(ozaki_slice_panels(L, ldl, n, oz, hi));
    bool rest_pending = false;
    int64_t off = 0;   // first row of panel k in the panel slices
    for (int k0 = 0; k0 < n; k0 += CH_NB) {
        const int nb = min(CH_NB, n - k0), k1 = k0 + nb, rows = n - k1;
        const int buf = (k0 / CH_NB) & 1;
        const bool tc = nb == CH_NB && rows > 0;
        uint16_t* SY = oz.SL2 + (size_t)buf * oz.cap2 * OZ_LD;
        int* eY = oz.ex2 + (size_t)buf * oz.cap2;
        { trsv_rows_kernel<<<row_blocks(nrows), 256, 0, hi>>>(L + (size_t)k0 * ldl + k0, ldl, nb, B + k0, ldb, nrows,
                                                              tc ? SY : nullptr, tc ? eY : nullptr); count_launch(); }
        if (rows <= 0) break;
        const uint16_t* SA = oz.SLP + (size_t)off * OZ_LD;
        const int* eA = oz.exP + off;
        LA_CK(cudaEventRecord(oz.ev_slice, hi));
        if (rest_pending) LA_CK(cudaStreamWaitEvent(hi, oz.ev_rest, 0));
        // next 64 columns: B[r][k1 + i] -= sum_k L[k1 + i][k0 + k] Y[r][k0 + k], i < 64
        LA_CK(ozaki_update_raw(SA, min(CH_NB, rows), eA, SY, nrows, eY, B + k1, ldb, 0, status_dev, hi));
        if (rows > CH_NB) {
            LA_CK(cudaStreamWaitEvent(lo, oz.ev_slice, 0));
            LA_CK(ozaki_update_raw(SA + (size_t)CH_NB * OZ_LD, rows - CH_NB, eA + CH_NB, SY, nrows, eY, B + k1 + CH_NB,
                                   ldb, 0, status_dev, lo));
            LA_CK(cudaEventRecord(oz.ev_rest, lo));
            rest_pending = true;
        }
        off += rows;
    }
    if (rest_pending) LA_CK(cudaStreamWaitEvent(hi, oz.ev_rest, 0));
    LA_CK(cudaEventRecord(oz.ev_lo, hi));
    LA_CK(cudaStreamWaitEvent(st, oz.ev_lo, 0));
    return cudaGetLastError();
}

cudaError_t trsm_lower_f64(const double* L, int ldl, int n, double* B, int ldb, int nrows, cudaStream_t st,
                           OzakiWs* oz, int* status_dev) {
    if (nrows <= 0 || n <= 0) return cudaSuccess;
    if (oz && nrows <= oz->cap2 && ozaki_panel_rows(n) <= oz->capP && oz->SLP)
        return trsm_ozaki(L, ldl, n, B, ldb, nrows, st, *oz, status_dev);
    return trsm_dfma(L, ldl, n, B, ldb, nrows, st);
}

}  // namespace diam
