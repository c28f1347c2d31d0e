// rewhiten_tc.cu -- re-solve of the whitened states after a factor change (BF16 mode), with the panel updates
// of the blocked forward substitution on the 5th-generation tensor cores.
//
// z = Lq^{-1}(x - x_ref) for every chain (the z of the proposal quadratic, Algorithm 1), in FP32: Lq is the
// BF16 factor, exact in FP32. One CTA per G <= 4 chains keeps their right-hand sides in shared memory. Per
// 64-column block k: the block's diagonal factor arrives by TMA (the next one's while this one is used) and
// warp g solves chain g's 64
// unknowns y (the 64-step chain on lane shuffles); then every row below the block is updated, r -= L_panel y,
// as one tensor-core product per 128-row tile: the panel tile (BF16, TMA, 128-byte swizzle) times the block's
// solution split into three BF16 terms per chain (y = hi + mid + lo to 2^-24, so every product is exact and the
// FP32 accumulation is the only rounding: the accuracy of an FP32 update), 12 of the 16 columns of N. Each
// tile's 16 result columns have their own tensor-memory range (up to 32 tiles: d <= 4160); the TMA ring runs
// ahead of the products, and four warps subtract the results from the right-hand sides.
// Every wait is clock-bounded; on expiry the CTA records DEV_TIMEOUT, lets its copies land and returns.
#include <cuda.h>
#include <cuda_runtime.h>

#include "common.cuh"
#include "rewhiten.h"
#include "tc_common.cuh"
#include "tc_gemm.h"

namespace diam {

namespace {

constexpr int RWT_G = 4;          // chains per CTA
constexpr int RWT_THREADS = 192;  // warps 0-3: solves and epilogue; warp 4: TMA; warp 5: MMA issue
constexpr int RWT_STAGES = 6;     // panel tiles in flight
constexpr int RWT_MAXT = 32;      // tiles of one panel (16 tensor-memory columns each)
constexpr uint32_t RWT_ABYTES = 128 * 64 * 2, RWT_BBYTES = 16 * 64 * 2;

struct RwtSmem {   // offsets (bytes) into the 1024-aligned dynamic shared memory
    static constexpr size_t A = 0;                                   // RWT_STAGES x 16 KB panel tiles
    static constexpr size_t LD = A + (size_t)RWT_STAGES * RWT_ABYTES; // 2 x 8 KB: diagonal blocks (BF16, SW128)
    static constexpr size_t B = LD + 2 * 8192;                       // 2 KB: the split solution (SW128)
    static constexpr size_t RD = B + RWT_BBYTES;                     // 64 floats: reciprocals of the diagonal
    static constexpr size_t Y = RD + 64 * 4;                         // 4 x 64 floats: the block's solution
    static constexpr size_t BAR = Y + RWT_G * 64 * 4;                // mbarriers: full, empty (stages), done, ld (2), groups (4)
    static constexpr size_t MISC = BAR + (2 * RWT_STAGES + 7) * 8;   // tensor-memory slot, abort flag
    static constexpr size_t RW = (MISC + 16 + 15) / 16 * 16;         // G x d floats: right-hand sides
};

// Byte offset of element (n, k) of a 16-row, 64-column BF16 operand in the 128-byte-swizzled layout the
// shared-memory descriptor expects (8-row groups of 1024 bytes; 16-byte chunk c of row r at c ^ (r % 8)).
__device__ __forceinline__ uint32_t sw128_off(int n, int k) {
    const int c = (k * 2) >> 4;
    return (uint32_t)((n >> 3) * 1024 + (n & 7) * 128 + ((c ^ (n & 7)) << 4) + ((k * 2) & 15));
}

__global__ void __launch_bounds__(RWT_THREADS, 1) rewhiten_tc_kernel(const __grid_constant__ CUtensorMap tmL,
                                                                     const __grid_constant__ CUtensorMap tmD, int d, int P,
                                                                     const uint16_t* __restrict__ Lq, int ldk,
                                                                     const float* __restrict__ X,
                                                                     const float* __restrict__ xref, float* __restrict__ Zs,
                                                                     double* __restrict__ qout, double inv_infl2,
                                                                     double* __restrict__ lp_ref, int* status) {
    extern __shared__ uint8_t rwt_raw[];
    uint8_t* sm = (uint8_t*)(((uintptr_t)rwt_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* sA = sm + RwtSmem::A;
    uint8_t* sB = sm + RwtSmem::B;
    uint8_t* sD = sm + RwtSmem::LD;
    float* rdiag = (float*)(sm + RwtSmem::RD);
    float* yv = (float*)(sm + RwtSmem::Y);
    uint64_t* full = (uint64_t*)(sm + RwtSmem::BAR);
    uint64_t* empty = full + RWT_STAGES;
    uint64_t* done = empty + RWT_STAGES;
    uint64_t* ldfull = done + 1;   // 2: the diagonal block's tile landed
    uint64_t* tgrp = ldfull + 2;   // 4: the products of tiles 8 q .. 8 q + 7 of the block are complete
    uint32_t* tmem_slot = (uint32_t*)(sm + RwtSmem::MISC);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
    float* rw = (float*)(sm + RwtSmem::RW);
    __shared__ double sh[32];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int p0 = blockIdx.x * RWT_G, ng = min(RWT_G, P - p0);
    if (tid == 0) {
        for (int s = 0; s < RWT_STAGES; ++s) {
            mbar_init(smem_u32(&full[s]), 1);
            mbar_init(smem_u32(&empty[s]), 1);
        }
        mbar_init(smem_u32(done), 1);
        mbar_init(smem_u32(&ldfull[0]), 1);
        mbar_init(smem_u32(&ldfull[1]), 1);
        for (int q = 0; q < RWT_MAXT / 8; ++q) mbar_init(smem_u32(&tgrp[q]), 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(512u));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    for (int g = 0; g < ng; ++g)
        for (int i = tid; i < d; i += RWT_THREADS) rw[(size_t)g * d + i] = X[(size_t)(p0 + g) * d + i] - xref[i];
    for (int e = tid; e < RWT_BBYTES / 4; e += RWT_THREADS) ((uint32_t*)sB)[e] = 0u;   // rows 12 .. 15 stay zero
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    constexpr uint32_t idesc = idesc_bf16(16);
    long long tile_count = 0;   // panel tiles of the blocks done so far (the ring's position across blocks)
    long long issued = 0;       // the TMA thread's copies issued so far
    const int nblk = (d + 63) / 64;
    int ld_issued = 0;          // diagonal-block tiles issued (TMA thread)
    // element (r, c) of a 64 x 64 BF16 tile in the 128-byte-swizzled layout of a TMA copy
    auto dl = [&](const uint8_t* t, int r, int c) { return bf16_bits_to_f32(*(const uint16_t*)(t + sw128_off(r, c))); };
    if (warp == 4 && lane == 0) {   // the first diagonal block
        mbar_expect_tx(smem_u32(&ldfull[0]), 8192);
        tma_load_2d(smem_u32(sD), &tmD, smem_u32(&ldfull[0]), 0, 0);
        ld_issued = 1;
    }

    for (int k0 = 0, kb = 0; k0 < d; k0 += 64, ++kb) {
        const int nb = min(64, d - k0);
        const uint8_t* tD = sD + (kb & 1) * 8192;
        if (warp == 4 && lane == 0 && kb + 1 < nblk) {   // the next block's diagonal tile, while this one is used
            mbar_expect_tx(smem_u32(&ldfull[(kb + 1) & 1]), 8192);
            tma_load_2d(smem_u32(sD + ((kb + 1) & 1) * 8192), &tmD, smem_u32(&ldfull[(kb + 1) & 1]), k0 + 64, k0 + 64);
            ld_issued = kb + 2;
        }
        mbar_wait(smem_u32(&ldfull[kb & 1]), (uint32_t)((kb >> 1) & 1), abort_flag);
        __syncthreads();
        if (*abort_flag) break;   // uniform after the barrier
        if (tid < nb) rdiag[tid] = 1.0f / dl(tD, tid, tid);
        __syncthreads();
        if (warp < ng) {   // chain warp: forward substitution within the block
            float* rg = rw + (size_t)warp * d + k0;
            float v0 = lane < nb ? rg[lane] : 0.f, v1 = lane + 32 < nb ? rg[lane + 32] : 0.f;
            for (int j = 0; j < nb; ++j) {
                const float vj = __shfl_sync(0xffffffffu, j < 32 ? v0 : v1, j & 31);
                const float yj = vj * rdiag[j];
                if (lane > j && lane < nb) v0 = fmaf(-dl(tD, lane, j), yj, v0);
                if (lane + 32 > j && lane + 32 < nb) v1 = fmaf(-dl(tD, lane + 32, j), yj, v1);
                if (lane == (j & 31)) {
                    if (j < 32) v0 = yj;
                    else v1 = yj;
                }
            }
            if (lane < nb) rg[lane] = v0;
            if (lane + 32 < nb) rg[lane + 32] = v1;
            yv[warp * 64 + lane] = lane < nb ? v0 : 0.f;
            yv[warp * 64 + lane + 32] = lane + 32 < nb ? v1 : 0.f;
        }
        const int r0 = k0 + nb, nt = (d - r0 + 127) / 128;   // rows below the block, in 128-row tiles
        if (nt <= 0) break;                                   // uniform: the last block
        __syncthreads();
        // the solution as three BF16 terms per chain: operand row 3 g + s, column c
        for (int e = tid; e < ng * 64; e += RWT_THREADS) {
            const int g = e >> 6, c = e & 63;
            const float y = yv[g * 64 + c];
            const uint16_t h = f32_to_bf16_bits(y);
            const float r1 = y - bf16_bits_to_f32(h);
            const uint16_t m = f32_to_bf16_bits(r1);
            const uint16_t l = f32_to_bf16_bits(r1 - bf16_bits_to_f32(m));
            *(uint16_t*)(sB + sw128_off(3 * g, c)) = h;
            *(uint16_t*)(sB + sw128_off(3 * g + 1, c)) = m;
            *(uint16_t*)(sB + sw128_off(3 * g + 2, c)) = l;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic writes -> the tensor core's reads
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (warp == 4 && lane == 0) {   // TMA: the panel's tiles through the ring
            for (int t = 0; t < nt; ++t) {
                const long long tt = tile_count + t;
                const int s = (int)(tt % RWT_STAGES);
                if (tt >= RWT_STAGES && !mbar_wait(smem_u32(&empty[s]), (uint32_t)(((tt / RWT_STAGES) - 1) & 1), abort_flag))
                    break;
                mbar_expect_tx(smem_u32(&full[s]), RWT_ABYTES);
                tma_load_2d(smem_u32(sA + (size_t)s * RWT_ABYTES), &tmL, smem_u32(&full[s]), k0, r0 + 128 * t);
                issued = tt + 1;
            }
        } else if (warp == 5 && lane == 0) {   // MMA: tile t into tensor-memory columns 16 t .. 16 t + 15
            for (int t = 0; t < nt; ++t) {
                const long long tt = tile_count + t;
                const int s = (int)(tt % RWT_STAGES);
                if (!mbar_wait(smem_u32(&full[s]), (uint32_t)((tt / RWT_STAGES) & 1), abort_flag)) break;
                tc_fence_after();
                const uint32_t pa = smem_u32(sA + (size_t)s * RWT_ABYTES), pb = smem_u32(sB);
#pragma unroll
                for (int kk = 0; kk < 4; ++kk)
                    umma_bf16(tmem + (uint32_t)(16 * t), sdesc_sw128(pa + kk * 32), sdesc_sw128(pb + kk * 32), idesc,
                              kk ? 1u : 0u);
                umma_commit(smem_u32(&empty[s]));
                if ((t & 7) == 7 || t == nt - 1) umma_commit(smem_u32(&tgrp[t >> 3]));   // a group of 8 tiles done
            }
            umma_commit(smem_u32(done));
        }
        __syncwarp();
        if (warp < 4) {   // each warp its 32 rows of every tile: r -= hi + mid + lo, per chain, a group of 8 tiles at a
                          // time as soon as its products are complete (the later groups' copies and products go on)
            for (int q = 0; q * 8 < nt; ++q) {
                // a group is committed in every block whose panel reaches it, and panels only shrink: phase kb & 1
                if (!mbar_wait(smem_u32(&tgrp[q]), (uint32_t)(kb & 1), abort_flag)) break;
                tc_fence_after();
                const int tq0 = 8 * q, tq1 = min(nt, tq0 + 8);
                uint32_t v[4][32];
#pragma unroll
                for (int pp = 0; pp < 4; ++pp)
                    if (tq0 + 2 * pp < tq1)
                        tmem_ld32_nowait(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(16 * (tq0 + 2 * pp)), v[pp]);
                tmem_wait_ld();
#pragma unroll
                for (int pp = 0; pp < 4; ++pp) {
                    tmem_regs_ready(v[pp]);
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int t = tq0 + 2 * pp + h, row = r0 + 128 * t + 32 * warp + lane;
                        if (t < tq1 && row < d) {
#pragma unroll
                            for (int g = 0; g < RWT_G; ++g)
                                if (g < ng)
                                    rw[(size_t)g * d + row] -= __uint_as_float(v[pp][16 * h + 3 * g]) +
                                                               __uint_as_float(v[pp][16 * h + 3 * g + 1]) +
                                                               __uint_as_float(v[pp][16 * h + 3 * g + 2]);
                        }
                    }
                }
            }
        }
        mbar_wait(smem_u32(done), (uint32_t)(kb & 1), abort_flag);   // every product of the block is complete
        tile_count += nt;
        tc_fence_before();
        __syncthreads();
        if (*abort_flag) break;   // uniform after the barrier
    }
    __syncthreads();   // the last block's solve
    if (*abort_flag) {
        if (tid == 0) set_status(status, DEV_TIMEOUT);
        if (warp == 4 && lane == 0) {   // the copies still in flight target this CTA's shared memory (bounded)
            for (int b = ld_issued > 2 ? ld_issued - 2 : 0; b < ld_issued; ++b) {
                const long long t0 = clock64();
                while (!mbar_try(smem_u32(&ldfull[b & 1]), (uint32_t)((b >> 1) & 1)) && clock64() - t0 < TC_WAIT_CYCLES) {
                }
            }
            for (long long tt = issued > RWT_STAGES ? issued - RWT_STAGES : 0; tt < issued; ++tt) {
                const long long t0 = clock64();
                while (!mbar_try(smem_u32(&full[tt % RWT_STAGES]), (uint32_t)((tt / RWT_STAGES) & 1)) &&
                       clock64() - t0 < TC_WAIT_CYCLES) {
                }
            }
        }
    } else {
        for (int g = 0; g < ng; ++g) {
            double acc = 0.0;
            for (int i = tid; i < d; i += RWT_THREADS) {
                const float v = rw[(size_t)g * d + i];
                Zs[(size_t)(p0 + g) * d + i] = v;
                acc += (double)v * (double)v;
            }
            acc = block_sum(acc, sh);
            if (tid == 0) {
                const double qq = 0.5 * acc * inv_infl2;
                qout[p0 + g] = qq;
                if (lp_ref) lp_ref[p0 + g] = -qq;
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512u));
}

}  // namespace

size_t rewhiten_tc_smem(int d) { return 1024 + RwtSmem::RW + sizeof(float) * RWT_G * (size_t)d; }

bool rewhiten_tc_fits(int d, int ldk) { return d > 0 && d <= 64 + 128 * RWT_MAXT && ldk % 64 == 0 && rewhiten_tc_smem(d) <= 227 * 1024; }

cudaError_t rewhiten_tc_setup(int d) {
    if (rewhiten_tc_smem(d) > 227 * 1024) return cudaErrorInvalidValue;
    return allow_max_dynamic_smem((const void*)rewhiten_tc_kernel);
}

cudaError_t rewhiten_tc(int d, int P, const uint16_t* Lq, int ldk, const float* X, const float* xref, float* Z,
                        double* q, double inv_infl2, double* lp_ref, int* status, cudaStream_t st) {
    CUtensorMap m, md;
    if (!rewhiten_tc_fits(d, ldk) || !make_map(&m, Lq, d, ldk, 128) || !make_map(&md, Lq, d, ldk, 64))
        return cudaErrorInvalidValue;
    { rewhiten_tc_kernel<<<(P + RWT_G - 1) / RWT_G, RWT_THREADS, rewhiten_tc_smem(d), st>>>(m, md, d, P, Lq, ldk, X, xref, Z, q,
                                                                                       inv_infl2, lp_ref, status); count_launch(); }
    return cudaGetLastError();
}

}  // namespace diam
