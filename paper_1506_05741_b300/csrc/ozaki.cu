// ozaki.cu -- FP64-accurate rank-64 updates C -= A B^T on the BF16 tensor cores.
//
// The refresh factors C_n = A_n A_n^T in FP64 (Algorithm 1) and then re-solves z = A_n^{-1}(x - x_ref) for
// every chain; the rank-64 updates of the blocked factorisation and of the blocked triangular solve hold
// nearly all of their flops, and B300 runs FP64 at about 1/1500 of its BF16 tensor rate. The updates are
// computed here by the error-free splitting of Ozaki, Ogita, Oishi and Rump (Numer. Algorithms 59, 2012),
// with BF16 slices:
//   - each operand row i (64 entries) is scaled by 2^-e_i (e_i: max_k |P_ik| < 2^e_i), rounded to the
//     integer R_ik = round(P_ik 2^(55 - e_i)) (|R| <= 2^55) and cut into 7 signed base-256 digits
//     |S_a| <= 128: P_ik = 2^(e_i - 7) sum_a S_a[i][k] 2^(-8a) up to 2^(e_i - 56);
//   - slice products are grouped by g = a + b: T_g = sum_{a+b=g} sum_k S_a[m][k] S_b[n][k] is an integer
//     below 7 * 64 * 2^14 < 2^23, so its FP32 accumulation in tensor memory is exact;
//   - the epilogue adds the T_g as 64-bit integers, I = sum_{g<6} T_g 2^(40-8g) + floor(T_6 / 2^8)
//     (|I| < 2^61), and subtracts I 2^(e_m + e_n - 54) with one FP64 fused multiply-add.
// Terms with g >= 7 and the low bits of T_6 are dropped; their size, about 64 * 2^-56 |P_m| |P_n|, is that
// of an FP64 GEMM's own rounding bound. Only one conversion and one FMA per output touch the FP64 pipe.
// One CTA per 128 x 16 output tile keeps the 7 B slices in shared memory, streams the 7 A slices through
// two stages and holds the 7 group accumulators in tensor memory (112 of 128 columns); four CTAs share an SM.
#include "linalg.h"
#include "ozaki_slice.cuh"
#include "tc_common.cuh"
#include "tc_gemm.h"

namespace diam {

constexpr int OZ_BN = 16, OZ_TMEM = 128;   // tile width; tensor-memory columns (7 x 16 used)

// One warp per operand row: exponent and the 7 BF16 slices (exact integers) of the row's 64 entries.
__global__ void ozaki_slice_kernel(const double* __restrict__ P, int lda, int rows, uint16_t* __restrict__ SL,
                                   int* __restrict__ ex) {
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= rows) return;
    const int e = ozaki_slice_row(P[(size_t)row * lda + lane], P[(size_t)row * lda + lane + 32], lane,
                                  SL + (size_t)row * OZ_LD);
    if (lane == 0) ex[row] = e;
}

// C[n][m] -= sum_k A[m][k] B[n][k] for m < Ma, n < Nb (and n >= m when lower), from the slices of A
// (tensor map tmA, 128-row boxes) and of B (tmB, 16-row boxes). A 128 x 16 tile per CTA: the 7 B slices stay
// in shared memory, the A slices stream through a two-stage ring in slice order (slice a meets B slices
// 0 .. 6 - a, so each group's first product comes with a = 0), the 7 groups take 112 tensor-memory columns.
// With 47 KB of shared memory and 128 columns four CTAs share an SM, their epilogues beside others' loads.
__global__ void __launch_bounds__(128, 4) ozaki_update_kernel(const __grid_constant__ CUtensorMap tmA,
                                                              const __grid_constant__ CUtensorMap tmB, int Ma, int Nb,
                                                              const int* __restrict__ exA, const int* __restrict__ exB,
                                                              double* __restrict__ Cm, int ldc, int lower,
                                                              int* status) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    constexpr uint32_t A_BYTES = 128 * OZ_K * 2, B_BYTES = OZ_BN * OZ_K * 2;
    uint8_t* sB = smem;                                 // 7 x 4 KB
    uint8_t* sA = smem + OZ_S * B_BYTES;                // 2 x 16 KB ring
    uint64_t* fullB = (uint64_t*)(sA + 2 * A_BYTES);
    uint64_t* fullA = fullB + 1;                        // 2
    uint64_t* emptyA = fullA + 2;                       // 2
    uint64_t* done = emptyA + 2;
    uint32_t* tmem_slot = (uint32_t*)(done + 1);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

    const int m0 = blockIdx.x * 128, n0 = blockIdx.y * OZ_BN;
    if ((lower && n0 + OZ_BN - 1 < m0) || n0 >= Nb || m0 >= Ma) return;   // nothing of this tile is updated
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __shared__ int sex[OZ_BN];   // exponents of this tile's B rows
    if (threadIdx.x < OZ_BN) sex[threadIdx.x] = (n0 + (int)threadIdx.x < Nb) ? exB[n0 + threadIdx.x] : 0;
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(fullB), 1);
        for (int s = 0; s < 2; ++s) {
            mbar_init(smem_u32(&fullA[s]), 1);
            mbar_init(smem_u32(&emptyA[s]), 1);
        }
        mbar_init(smem_u32(done), 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"((uint32_t)OZ_TMEM));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // producer: the B slices, then the A slices through the ring
        mbar_expect_tx(smem_u32(fullB), OZ_S * B_BYTES);
        for (int b = 0; b < OZ_S; ++b) tma_load_2d(smem_u32(sB + b * B_BYTES), &tmB, smem_u32(fullB), b * OZ_K, n0);
        int issued = 0;
        for (int a = 0; a < OZ_S; ++a) {
            const int st = a & 1;
            if (a >= 2 && !mbar_wait(smem_u32(&emptyA[st]), ((a >> 1) - 1) & 1, abort_flag)) break;
            mbar_expect_tx(smem_u32(&fullA[st]), A_BYTES);
            tma_load_2d(smem_u32(sA + st * A_BYTES), &tmA, smem_u32(&fullA[st]), a * OZ_K, m0);
            issued = a + 1;
        }
        if (*abort_flag) {   // every issued copy lands before the CTA may exit (bounded)
            for (int a = (issued > 2 ? issued - 2 : 0); a < issued; ++a) {
                const long long t0 = clock64();
                while (!mbar_try(smem_u32(&fullA[a & 1]), (a >> 1) & 1) && clock64() - t0 < TC_WAIT_CYCLES) {
                }
            }
            const long long t0 = clock64();
            while (!mbar_try(smem_u32(fullB), 0) && clock64() - t0 < TC_WAIT_CYCLES) {
            }
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer: slice a of A against B slices 0 .. 6 - a, product (a, b) into group a + b
        constexpr uint32_t idesc = idesc_bf16(OZ_BN);
        bool ok = mbar_wait(smem_u32(fullB), 0, abort_flag);
        for (int a = 0; ok && a < OZ_S; ++a) {
            const int st = a & 1;
            if (!mbar_wait(smem_u32(&fullA[st]), (a >> 1) & 1, abort_flag)) break;
            tc_fence_after();
            const uint32_t pa = smem_u32(sA + st * A_BYTES);
            for (int b = 0; a + b < OZ_S; ++b) {
                const uint32_t pb = smem_u32(sB + b * B_BYTES);
#pragma unroll
                for (int kk = 0; kk < OZ_K / 16; ++kk)
                    umma_bf16(tmem + (uint32_t)((a + b) * OZ_BN), sdesc_sw128(pa + kk * 32), sdesc_sw128(pb + kk * 32),
                              idesc, (a | kk) ? 1u : 0u);
            }
            umma_commit(smem_u32(&emptyA[st]));   // the stage is free once these products are done
        }
        umma_commit(smem_u32(done));
    }
    __syncwarp();
    mbar_wait(smem_u32(done), 0, abort_flag);
    __syncthreads();
    const bool ok = (*abort_flag == 0);
    tc_fence_after();
    if (ok) {
        const int row = warp * 32 + lane;
        const int m = m0 + row;
        const bool vm = m < Ma;
        const int em = vm ? exA[m] : 0;
        const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
        {
            // issue the tile's 16 loads of C first: their latency hides behind the tensor-memory reads
            double cv[OZ_BN];
#pragma unroll
            for (int j = 0; j < OZ_BN; ++j) {
                const int n = n0 + j;
                cv[j] = (vm && n < Nb && (!lower || n >= m)) ? Cm[(size_t)n * ldc + m] : 0.0;
            }
            long long acc[OZ_BN];
#pragma unroll
            for (int j = 0; j < OZ_BN; ++j) acc[j] = 0;
#pragma unroll 1
            for (int g = 0; g < OZ_S; ++g) {
                uint32_t r[OZ_BN];
                tmem_ld16(trow + (uint32_t)(g * OZ_BN), r);
                if (g < OZ_S - 1) {
                    const int sh = 40 - 8 * g;
#pragma unroll
                    for (int j = 0; j < OZ_BN; ++j) acc[j] += (long long)__float2int_rn(__uint_as_float(r[j])) * (1ll << sh);
                } else {
#pragma unroll
                    for (int j = 0; j < OZ_BN; ++j) acc[j] += (long long)(__float2int_rn(__uint_as_float(r[j])) >> 8);
                }
            }
#pragma unroll
            for (int j = 0; j < OZ_BN; ++j) {
                const int n = n0 + j;
                if (vm && n < Nb && (!lower || n >= m))
                    Cm[(size_t)n * ldc + m] = fma(-(double)acc[j], pow2(em + sex[j] - 54), cv[j]);
            }
        }
    } else if (threadIdx.x == 0) {
        set_status(status, DEV_TIMEOUT);   // the producer has waited for its copies in flight
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)OZ_TMEM));
}

static size_t update_smem() { return 1024 + (size_t)OZ_S * OZ_BN * OZ_K * 2 + 2 * (size_t)128 * OZ_K * 2 + 256; }

static cudaError_t launch_update(const uint16_t* SA, int Ma, const int* exA, const uint16_t* SB, int Nb,
                                 const int* exB, double* Cm, int ldc, int lower, int* status, cudaStream_t st) {
    CUtensorMap mA, mB;
    if (!make_map(&mA, SA, Ma, OZ_LD, 128) || !make_map(&mB, SB, Nb, OZ_LD, OZ_BN)) return cudaErrorInvalidValue;
    static bool attr = false;
    if (!attr) {
        cudaError_t e =
            cudaFuncSetAttribute(ozaki_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)update_smem());
        if (e != cudaSuccess) return e;
        attr = true;
    }
    dim3 grid((Ma + 127) / 128, (Nb + OZ_BN - 1) / OZ_BN);
    { ozaki_update_kernel<<<grid, 128, update_smem(), st>>>(mA, mB, Ma, Nb, exA, exB, Cm, ldc, lower, status); count_launch(); }
    return cudaGetLastError();
}

static void slice(const double* P, int lda, int rows, uint16_t* SL, int* ex, cudaStream_t st) {
    ozaki_slice_kernel<<<(rows + 7) / 8, 256, 0, st>>>(P, lda, rows, SL, ex);
    count_launch();
}

cudaError_t ozaki_trailing_update(const double* Pnl, int lda, int rows, double* Cm, int ldc, OzakiWs& ws, int* status,
                                  cudaStream_t st) {
    if (rows <= 0) return cudaSuccess;
    if (rows > ws.cap_rows) return cudaErrorInvalidValue;
    slice(Pnl, lda, rows, ws.SL, ws.ex, st);
    return launch_update(ws.SL, rows, ws.ex, ws.SL, rows, ws.ex, Cm, ldc, 1, status, st);
}

cudaError_t ozaki_slice_panel(const double* Pnl, int lda, int rows, int buf, OzakiWs& ws, cudaStream_t st) {
    if (rows > ws.cap_rows) return cudaErrorInvalidValue;
    slice(Pnl, lda, rows, ws.SL + (size_t)buf * ws.cap_rows * OZ_LD, ws.ex + (size_t)buf * ws.cap_rows, st);
    return cudaGetLastError();
}

cudaError_t ozaki_update_sliced(int buf, int r0, int Ma, int c0, int Nb, double* Cm, int ldc, int lower, OzakiWs& ws,
                                int* status, cudaStream_t st) {
    if (Ma <= 0 || Nb <= 0) return cudaSuccess;
    const uint16_t* S = ws.SL + (size_t)buf * ws.cap_rows * OZ_LD;
    const int* e = ws.ex + (size_t)buf * ws.cap_rows;
    return launch_update(S + (size_t)r0 * OZ_LD, Ma, e + r0, S + (size_t)c0 * OZ_LD, Nb, e + c0, Cm, ldc, lower, status, st);
}

__global__ void ozaki_slice_panels_kernel(const double* __restrict__ L, int ldl, int n, int64_t total,
                                          uint16_t* __restrict__ SL, int* __restrict__ ex) {
    const int64_t g = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (g >= total) return;
    int k = 0;
    int64_t off = 0;
    while (g >= off + (n - OZ_K * (k + 1))) {   // the panel holding row g (warp-uniform)
        off += n - OZ_K * (k + 1);
        ++k;
    }
    const double* row = L + (size_t)(OZ_K * (k + 1) + (g - off)) * ldl + OZ_K * k;
    const int e = ozaki_slice_row(row[lane], row[lane + 32], lane, SL + (size_t)g * OZ_LD);
    if (lane == 0) ex[g] = e;
}

cudaError_t ozaki_slice_panels(const double* L, int ldl, int n, OzakiWs& ws, cudaStream_t st) {
    const int64_t total = ozaki_panel_rows(n);
    if (total > ws.capP) return cudaErrorInvalidValue;
    if (total == 0) return cudaSuccess;
    { ozaki_slice_panels_kernel<<<(unsigned)((total + 7) / 8), 256, 0, st>>>(L, ldl, n, total, ws.SLP, ws.exP); count_launch(); }
    return cudaGetLastError();
}

cudaError_t ozaki_update_raw(const uint16_t* SA, int Ma, const int* exA, const uint16_t* SB, int Nb, const int* exB,
                             double* C, int ldc, int lower, int* status, cudaStream_t st) {
    if (Ma <= 0 || Nb <= 0) return cudaSuccess;
    return launch_update(SA, Ma, exA, SB, Nb, exB, C, ldc, lower, status, st);
}

void ozaki_ws_release(OzakiWs& ws) {
    if (ws.hi) cudaStreamDestroy(ws.hi);
    if (ws.lo) cudaStreamDestroy(ws.lo);
    for (cudaEvent_t e : {ws.ev_in, ws.ev_slice, ws.ev_rest, ws.ev_lo})
        if (e) cudaEventDestroy(e);
    ws.hi = ws.lo = nullptr;
    ws.ev_in = ws.ev_slice = ws.ev_rest = ws.ev_lo = nullptr;
}

cudaError_t ozaki_gemm_update(const double* A, int lda, int Ma, const double* B, int ldb, int Nb, double* Cm, int ldc,
                              OzakiWs& ws, int* status, cudaStream_t st) {
    if (Ma <= 0 || Nb <= 0) return cudaSuccess;
    if (Ma > ws.cap_rows || Nb > ws.cap2) return cudaErrorInvalidValue;
    slice(A, lda, Ma, ws.SL, ws.ex, st);
    slice(B, ldb, Nb, ws.SL2, ws.ex2, st);
    return launch_update(ws.SL, Ma, ws.ex, ws.SL2, Nb, ws.ex2, Cm, ldc, 0, status, st);
}

}  // namespace diam
