// ozaki.cu -- FP64-accurate rank-64 trailing update of the Cholesky refresh on the BF16 tensor cores.
//
// The refresh factors C_n = A_n A_n^T in FP64 (Algorithm 1); its trailing updates C[n][m] -= sum_k P_nk P_mk
// (P the 64-wide panel) hold nearly all of its d^3/3 flops, and B300 runs FP64 at about 1/1500 of its BF16
// tensor rate. The update is computed here by the error-free splitting of Ozaki, Ogita, Oishi and Rump
// (Numer. Algorithms 59, 2012), with BF16 slices:
//   - each panel row i is scaled by 2^-e_i (e_i: max_k |P_ik| < 2^e_i) and cut into 7 slices of integers
//     |S_a| <= 128, P_ik = 2^e_i sum_a S_a[i][k] 2^(-7-8a) + (a remainder below 2^(e_i-63));
//   - slice products are grouped by g = a + b: T_g = sum_{a+b=g} sum_k S_a[m][k] S_b[n][k] is an integer
//     below 7 * 64 * 2^14 < 2^23, so its FP32 accumulation in tensor memory is exact;
//   - the epilogue forms sum_g 2^(-8g) T_g in FP64 and subtracts 2^(e_m + e_n - 14) times it.
// Terms with g >= 7 are dropped; their size, about 64 * 2^-56 |P_m| |P_n|, is that of an FP64 GEMM's
// rounding bound. One CTA per 128 x 64 tile of the lower triangle keeps all 14 slice tiles in shared memory
// and the 7 group accumulators in tensor memory (448 of its 512 columns).
#include "linalg.h"
#include "tc_common.cuh"
#include "tc_gemm.h"

namespace diam {

constexpr int OZ_S = 7, OZ_K = 64, OZ_LD = OZ_S * OZ_K, OZ_BN = 64;

// One warp per panel row: exponent and the 7 BF16 slices (exact integers) of the row's 64 entries.
__global__ void ozaki_slice_kernel(const double* __restrict__ P, int lda, int rows, uint16_t* __restrict__ SL,
                                   int* __restrict__ ex) {
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= rows) return;
    double v[2] = {P[(size_t)row * lda + lane], P[(size_t)row * lda + lane + 32]};
    double m = fmax(fabs(v[0]), fabs(v[1]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    const int e = (m > 0.0) ? ilogb(m) + 1 : 0;   // m < 2^e
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        double r = ldexp(v[h], 7 - e);            // |r| < 128, exact scaling
#pragma unroll
        for (int a = 0; a < OZ_S; ++a) {
            const double s = rint(r);             // |s| <= 128: exact in BF16
            SL[(size_t)row * OZ_LD + a * OZ_K + lane + 32 * h] = (uint16_t)(__float_as_uint((float)s) >> 16);
            r = (r - s) * 256.0;                  // exact: |r - s| <= 1/2
        }
    }
    if (lane == 0) ex[row] = e;
}

__global__ void __launch_bounds__(128, 1) ozaki_update_kernel(const __grid_constant__ CUtensorMap tmA,
                                                              const __grid_constant__ CUtensorMap tmB, int rows,
                                                              const int* __restrict__ ex, double* __restrict__ Cm,
                                                              int ldc, int* status) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    constexpr uint32_t A_BYTES = 128 * OZ_K * 2, B_BYTES = OZ_BN * OZ_K * 2;
    uint8_t* sA = smem;                                 // 7 x 16 KB
    uint8_t* sB = smem + OZ_S * A_BYTES;                // 7 x 8 KB
    uint64_t* full = (uint64_t*)(smem + OZ_S * (A_BYTES + B_BYTES));
    uint64_t* done = full + 1;
    uint32_t* tmem_slot = (uint32_t*)(done + 1);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

    const int m0 = blockIdx.x * 128, n0 = blockIdx.y * OZ_BN;
    if (n0 + OZ_BN - 1 < m0 || n0 >= rows) return;    // tile strictly above the diagonal, or past the rows
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(full), 1);
        mbar_init(smem_u32(done), 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(512u));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        const uint32_t fb = smem_u32(full);
        mbar_expect_tx(fb, OZ_S * (A_BYTES + B_BYTES));
        for (int a = 0; a < OZ_S; ++a) {
            tma_load_2d(smem_u32(sA + a * A_BYTES), &tmA, fb, a * OZ_K, m0);
            tma_load_2d(smem_u32(sB + a * B_BYTES), &tmB, fb, a * OZ_K, n0);
        }
    } else if (warp == 1 && lane == 0) {
        constexpr uint32_t idesc = idesc_bf16(OZ_BN);
        if (mbar_wait(smem_u32(full), 0, abort_flag)) {
            tc_fence_after();
            for (int g = 0; g < OZ_S; ++g) {
                for (int a = 0; a <= g; ++a) {
                    const int b = g - a;
                    const uint32_t pa = smem_u32(sA + a * A_BYTES), pb = smem_u32(sB + b * B_BYTES);
#pragma unroll
                    for (int kk = 0; kk < OZ_K / 16; ++kk)
                        umma_bf16(tmem + (uint32_t)(g * OZ_BN), sdesc_sw128(pa + kk * 32), sdesc_sw128(pb + kk * 32),
                                  idesc, (a | kk) ? 1u : 0u);
                }
            }
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
        const bool vm = m < rows;
        const int em = vm ? ex[m] : 0;
        const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
        for (int c = 0; c < OZ_BN / 32; ++c) {
            double acc[32];
#pragma unroll
            for (int j = 0; j < 32; ++j) acc[j] = 0.0;
#pragma unroll 1
            for (int g = OZ_S - 1; g >= 0; --g) {     // small groups first
                uint32_t r[32];
                tmem_ld32(trow + (uint32_t)(g * OZ_BN + c * 32), r);
#pragma unroll
                for (int j = 0; j < 32; ++j) acc[j] += ldexp((double)__uint_as_float(r[j]), -8 * g);
            }
            if (vm) {
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int n = n0 + c * 32 + j;
                    if (n < rows && n >= m) Cm[(size_t)n * ldc + m] -= ldexp(acc[j], em + ex[n] - 14);
                }
            }
        }
    } else if (threadIdx.x == 0) {
        set_status(status, DEV_TIMEOUT);
        // the loads were issued on one barrier: let them land before the CTA exits (bounded)
        long long t0 = clock64();
        while (!mbar_try(smem_u32(full), 0) && clock64() - t0 < TC_WAIT_CYCLES) {
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512u));
}

cudaError_t ozaki_trailing_update(const double* Pnl, int lda, int rows, double* Cm, int ldc, OzakiWs& ws, int* status,
                                  cudaStream_t st) {
    if (rows <= 0) return cudaSuccess;
    if (rows > ws.cap_rows) return cudaErrorInvalidValue;
    { ozaki_slice_kernel<<<(rows + 7) / 8, 256, 0, st>>>(Pnl, lda, rows, ws.SL, ws.ex); count_launch(); }
    CUtensorMap mA, mB;
    if (!make_map(&mA, ws.SL, rows, OZ_LD, 128) || !make_map(&mB, ws.SL, rows, OZ_LD, OZ_BN)) return cudaErrorInvalidValue;
    const size_t smem = 1024 + (size_t)OZ_S * (128 * OZ_K * 2 + OZ_BN * OZ_K * 2) + 256;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(ozaki_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    dim3 grid((rows + 127) / 128, (rows + OZ_BN - 1) / OZ_BN);
    { ozaki_update_kernel<<<grid, 128, smem, st>>>(mA, mB, rows, ws.ex, Cm, ldc, status); count_launch(); }
    return cudaGetLastError();
}

}  // namespace diam
