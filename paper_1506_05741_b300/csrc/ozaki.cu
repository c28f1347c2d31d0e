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
// A CTA keeps the 7 B slices of a 16-row tile in shared memory and walks a run of 128-row tiles of A, whose
// slices stream through a four-stage ring; slice a of A meets B slices 0 .. 6 - a in one product of width
// 16 (7 - a), and the 7 group accumulators of a tile fill one of two tensor-memory buffers.
#include <mutex>
#include "linalg.h"
#include "ozaki_slice.cuh"
#include "tc_common.cuh"
#include "tc_gemm.h"

namespace diam {

constexpr int OZ_BN = 16, OZ_TMEM = 256;   // tile width; tensor-memory columns (two buffers of 7 x 16)

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

// Work units of the update: one 16-row tile of B (n0 .. n0 + 15) with a run of 128-row tiles of A
// (mt0 .. mt1 - 1), at most ch of them. With lower, A tile mt takes part only if 128 mt <= n0 + 15; the
// n-tiles come in groups of eight with the same number of A tiles (g + 1 for group g, up to the last A tile).
// Unit u counts from the largest units down, so the longest-running CTAs start first.
struct OzUnit {
    int n0, mt0, mt1;
};

__host__ __device__ inline int oz_units(int Ma, int Nb, int lower, int ch, int u, OzUnit* w) {
    const int NT = (Nb + OZ_BN - 1) / OZ_BN, MT = (Ma + 127) / 128;
    int total = 0;
    if (!lower) {
        const int nch = (MT + ch - 1) / ch;
        total = NT * nch;
        if (w && u < total) {
            const int v = total - 1 - u, nt = v / nch, c = v % nch;
            *w = OzUnit{nt * OZ_BN, c * ch, min(MT, c * ch + ch)};
        }
        return total;
    }
    for (int g = 0; 8 * g < NT; ++g) total += min(8, NT - 8 * g) * ((min(MT, g + 1) + ch - 1) / ch);
    if (w && u < total) {
        int v = total - 1 - u;
        for (int g = 0; 8 * g < NT; ++g) {
            const int cnt = min(MT, g + 1), nch = (cnt + ch - 1) / ch, units = min(8, NT - 8 * g) * nch;
            if (v < units) {
                const int nt = 8 * g + v / nch, c = v % nch;
                *w = OzUnit{nt * OZ_BN, c * ch, min(cnt, c * ch + ch)};
                break;
            }
            v -= units;
        }
    }
    return total;
}

constexpr int OZ_STAGES = 4;            // A slices in flight
constexpr int OZ_THREADS = 320;         // warp 0: TMA, warp 1: MMA issue, warps 2-9: epilogue
constexpr int OZ_EPI_WARPS = 8;         // two per tensor-memory lane quarter, 8 of the 16 columns each
constexpr uint32_t OZ_ABYTES = 128 * OZ_K * 2, OZ_BBYTES = OZ_BN * OZ_K * 2;

// C[n][m] -= sum_k A[m][k] B[n][k] for m < Ma, n < Nb (and n >= m when lower), from the slices of A
// (tensor map tmA, 128-row boxes) and of B (tmB, 16-row boxes). One CTA per work unit: the 7 B slices of
// its n-tile stay in shared memory; the A slices of its m-tiles stream through a four-stage ring in slice
// order (slice a meets B slices 0 .. 6 - a in one product, so each group's first product comes with a = 0);
// each tile's 7 group accumulators take 112 columns of one of two tensor-memory buffers (128 columns apart),
// so the epilogue of one tile overlaps the products of the next. The epilogue warps read a tile's groups, release
// its buffer, then combine and subtract (eight epilogue warps, two per lane quarter, split the 16 columns).
// With 78 KB of shared memory and 256 columns two CTAs share an SM.
__global__ void __launch_bounds__(OZ_THREADS, 2) ozaki_update_kernel(const __grid_constant__ CUtensorMap tmA,
                                                                     const __grid_constant__ CUtensorMap tmB, int Ma,
                                                                     int Nb, const int* __restrict__ exA,
                                                                     const int* __restrict__ exB,
                                                                     double* __restrict__ Cm, int ldc, int lower,
                                                                     int ch, int* status) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* sB = smem;                                  // 7 x 2 KB
    uint8_t* sA = smem + OZ_S * OZ_BBYTES;               // OZ_STAGES x 16 KB
    uint64_t* fullB = (uint64_t*)(sA + OZ_STAGES * OZ_ABYTES);
    uint64_t* fullA = fullB + 1;                         // OZ_STAGES
    uint64_t* emptyA = fullA + OZ_STAGES;                // OZ_STAGES
    uint64_t* tfull = emptyA + OZ_STAGES;                // 2: a tile's accumulators are complete
    uint64_t* tempty = tfull + 2;                        // 2: the epilogue has read them
    uint64_t* done = tempty + 2;
    uint32_t* tmem_slot = (uint32_t*)(done + 1);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
    __shared__ OzUnit su;
    __shared__ int sex[OZ_BN];   // exponents of the n-tile's B rows
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        OzUnit w{0, 0, 0};
        oz_units(Ma, Nb, lower, ch, blockIdx.x, &w);
        su = w;
    }
    __syncthreads();
    const OzUnit w = su;
    const int ntiles = w.mt1 - w.mt0;
    if (ntiles <= 0) return;
    const int n0 = w.n0;
    if (threadIdx.x < OZ_BN) sex[threadIdx.x] = (n0 + (int)threadIdx.x < Nb) ? exB[n0 + threadIdx.x] : 0;
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(fullB), 1);
        for (int s = 0; s < OZ_STAGES; ++s) {
            mbar_init(smem_u32(&fullA[s]), 1);
            mbar_init(smem_u32(&emptyA[s]), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&tfull[b]), 1);
            mbar_init(smem_u32(&tempty[b]), OZ_EPI_WARPS);   // one arrival per epilogue warp
        }
        mbar_init(smem_u32(done), 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"((uint32_t)OZ_TMEM));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int nq = ntiles * OZ_S;   // A slices of the unit, in order (tile i, slice a) -> q = 7 i + a

    if (warp == 0 && lane == 0) {
        // producer: the B slices, then every A slice of the unit through the ring
        mbar_expect_tx(smem_u32(fullB), OZ_S * OZ_BBYTES);
        for (int b = 0; b < OZ_S; ++b) tma_load_2d(smem_u32(sB + b * OZ_BBYTES), &tmB, smem_u32(fullB), b * OZ_K, n0);
        int issued = 0;
        for (int q = 0; q < nq; ++q) {
            const int st = q % OZ_STAGES;
            if (q >= OZ_STAGES && !mbar_wait(smem_u32(&emptyA[st]), ((q / OZ_STAGES) - 1) & 1, abort_flag)) break;
            mbar_expect_tx(smem_u32(&fullA[st]), OZ_ABYTES);
            tma_load_2d(smem_u32(sA + st * OZ_ABYTES), &tmA, smem_u32(&fullA[st]), (q % OZ_S) * OZ_K,
                        (w.mt0 + q / OZ_S) * 128);
            issued = q + 1;
        }
        if (*abort_flag) {   // every issued copy lands before the CTA may exit (bounded)
            for (int q = (issued > OZ_STAGES ? issued - OZ_STAGES : 0); q < issued; ++q) {
                const long long t0 = clock64();
                while (!mbar_try(smem_u32(&fullA[q % OZ_STAGES]), (q / OZ_STAGES) & 1) && clock64() - t0 < TC_WAIT_CYCLES) {
                }
            }
            const long long t0 = clock64();
            while (!mbar_try(smem_u32(fullB), 0) && clock64() - t0 < TC_WAIT_CYCLES) {
            }
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer: tile i into buffer i & 1; slice a of A against B slices 0 .. 6 - a as one product of
        // width 16 (7 - a): the B slices lie one after another with the same 1024-byte group stride, and block b
        // of the result lands in columns 16 (a + b) of the buffer, the accumulator of group a + b
        bool ok = mbar_wait(smem_u32(fullB), 0, abort_flag);
        for (int i = 0; ok && i < ntiles; ++i) {
            const int buf = i & 1;
            if (i >= 2 && !mbar_wait(smem_u32(&tempty[buf]), ((i >> 1) - 1) & 1, abort_flag)) break;
            tc_fence_after();
            const uint32_t tb = tmem + (uint32_t)(buf * 128);
            for (int a = 0; a < OZ_S; ++a) {
                const int q = i * OZ_S + a, st = q % OZ_STAGES;
                if (!mbar_wait(smem_u32(&fullA[st]), (q / OZ_STAGES) & 1, abort_flag)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t pa = smem_u32(sA + st * OZ_ABYTES), pb = smem_u32(sB);
                const uint32_t idesc = idesc_bf16(OZ_BN * (OZ_S - a));
#pragma unroll
                for (int kk = 0; kk < OZ_K / 16; ++kk)
                    umma_bf16(tb + (uint32_t)(a * OZ_BN), sdesc_sw128(pa + kk * 32), sdesc_sw128(pb + kk * 32), idesc,
                              (a | kk) ? 1u : 0u);
                umma_commit(smem_u32(&emptyA[st]));   // the stage is free once these products are done
            }
            if (ok) umma_commit(smem_u32(&tfull[buf]));
        }
        umma_commit(smem_u32(done));   // arrives once every product issued here has completed
    } else if (warp >= 2) {
        // epilogue: warp w reads tensor-memory lanes 32 (w % 4) .. + 31, i.e. rows of the A tile, and columns
        // 8 h .. 8 h + 7 of every group (h = 0 for warps 2-5, 1 for warps 6-9)
        constexpr int NJ = OZ_BN / 2;
        const int rq = warp & 3, row = rq * 32 + lane, j0 = (warp - 2) / 4 * NJ;
        int sx[NJ];
#pragma unroll
        for (int j = 0; j < NJ; ++j) sx[j] = sex[j0 + j];
        for (int i = 0; i < ntiles; ++i) {
            const int m = (w.mt0 + i) * 128 + row;
            const bool vm = m < Ma;
            const int em = vm ? exA[m] : 0;
            // the loads of C first: their latency hides behind the wait and the tensor-memory reads
            double cv[NJ];
#pragma unroll
            for (int j = 0; j < NJ; ++j) {
                const int n = n0 + j0 + j;
                cv[j] = (vm && n < Nb && (!lower || n >= m)) ? Cm[(size_t)n * ldc + m] : 0.0;
            }
            const int buf = i & 1;
            if (!mbar_wait(smem_u32(&tfull[buf]), (i >> 1) & 1, abort_flag)) break;
            tc_fence_after();
            const uint32_t trow = tmem + (uint32_t)(buf * 128 + j0) + ((uint32_t)(rq * 32) << 16);
            long long acc[NJ];
#pragma unroll
            for (int j = 0; j < NJ; ++j) acc[j] = 0;
#pragma unroll
            for (int g = 0; g < OZ_S; ++g) {   // constant shifts: one or two integer operations per term
                uint32_t r[NJ];
                tmem_ld8(trow + (uint32_t)(g * OZ_BN), r);
#pragma unroll
                for (int j = 0; j < NJ; ++j) {
                    const int v = __float2int_rn(__uint_as_float(r[j]));
                    if (g < OZ_S - 1) acc[j] += (long long)v * (1ll << (40 - 8 * g));
                    else acc[j] += (long long)(v >> 8);
                }
            }
            tc_fence_before();   // the buffer goes back to the MMA issuer
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&tempty[buf]));
#pragma unroll
            for (int j = 0; j < NJ; ++j) {
                const int n = n0 + j0 + j;
                if (vm && n < Nb && (!lower || n >= m))
                    Cm[(size_t)n * ldc + m] = fma(-(double)acc[j], pow2(em + sx[j] - 54), cv[j]);
            }
        }
    }
    __syncwarp();
    {   // no thread leaves before the products it depends on are complete (bounded)
        const long long t0 = clock64();
        while (!mbar_try(smem_u32(done), 0) && clock64() - t0 < TC_WAIT_CYCLES) {
        }
    }
    __syncthreads();
    if (*abort_flag && threadIdx.x == 0) set_status(status, DEV_TIMEOUT);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)OZ_TMEM));
}

static size_t update_smem() {
    return 1024 + (size_t)OZ_S * OZ_BBYTES + (size_t)OZ_STAGES * OZ_ABYTES + (OZ_STAGES * 2 + 6) * 8 + 16;
}

static cudaError_t launch_update(const uint16_t* SA, int Ma, const int* exA, const uint16_t* SB, int Nb,
                                 const int* exB, double* Cm, int ldc, int lower, int* status, cudaStream_t st) {
    CUtensorMap mA, mB;
    if (!make_map(&mA, SA, Ma, OZ_LD, 128) || !make_map(&mB, SB, Nb, OZ_LD, OZ_BN)) return cudaErrorInvalidValue;
    // the dynamic shared-memory attribute applies to the current device only: set once per device
    static std::mutex attr_mu;
    static bool attr[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    {
        std::lock_guard<std::mutex> g(attr_mu);
        if (!attr[dev]) {
            cudaError_t e =
                cudaFuncSetAttribute(ozaki_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)update_smem());
            if (e != cudaSuccess) return e;
            attr[dev] = true;
        }
    }
    // A tiles per unit: about one wave of units over the SMs (two resident per SM), at most 16 tiles (a unit's
    // B load, pipeline fill and drain cost about as much as two tiles; longer runs unbalance the triangle)
    const int tiles = oz_units(Ma, Nb, lower, 1, 0, nullptr);
    const int ch = std::max(1, std::min(16, (tiles + 2 * 148 - 1) / (2 * 148)));
    const int units = oz_units(Ma, Nb, lower, ch, 0, nullptr);
    { ozaki_update_kernel<<<units, OZ_THREADS, update_smem(), st>>>(mA, mB, Ma, Nb, exA, exB, Cm, ldc, lower, ch, status); count_launch(); }
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
    for (cudaStream_t s : {ws.hi, ws.mid, ws.lo})
        if (s) cudaStreamDestroy(s);
    for (cudaEvent_t e : {ws.ev_in, ws.ev_slice, ws.ev_rest, ws.ev_lo, ws.ev_diag, ws.ev_mid})
        if (e) cudaEventDestroy(e);
    ws.hi = ws.mid = ws.lo = nullptr;
    ws.ev_in = ws.ev_slice = ws.ev_rest = ws.ev_lo = ws.ev_diag = ws.ev_mid = nullptr;
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
