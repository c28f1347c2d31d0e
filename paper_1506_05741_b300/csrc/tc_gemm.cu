// tc_gemm.cu -- BF16 x BF16 -> FP32 GEMM on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// One CTA per 128 x BN output tile (cta_group::1). K advances in blocks of 64 BF16 (128 bytes): a TMA
// thread stages the A and B tiles (128-byte swizzle) into a shared-memory ring (4 stages, fewer when they
// do not fit), one elected thread issues tcgen05.mma into an FP32 accumulator in tensor memory and
// releases each stage with tcgen05.commit, and all four warps read the accumulator back (tcgen05.ld) for
// the epilogue:
//   - store (the noise product xi = beta alpha Lq W of Algorithm 1's batch update),
//   - per-chain reduction of the target's log-likelihood terms (linear-map targets),
//   - the FP64 moment fold of a lower-triangle SYRK (eq. (sampcov) as a pairwise centred update).
// Every wait is bounded by the clock; on expiry the kernel records DEV_TIMEOUT, drains what it issued,
// frees its tensor memory and returns.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>

#include "common.cuh"
#include "tc_common.cuh"
#include "tc_gemm.h"

namespace diam {

template <int BN>
__global__ void __launch_bounds__(128, 1) tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA,
                                                         const __grid_constant__ CUtensorMap tmB,
                                                         const __grid_constant__ CUtensorMap tmB2,
                                                         const __grid_constant__ CUtensorMap tmA2, int M, int N, int nkb,
                                                         int a_lower, int has_b2, int has_a2, int kb_split, int stages,
                                                         TcEpi epi, int* status) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    constexpr uint32_t A_BYTES = TC_BM * TC_BK * 2, B_BYTES = BN * TC_BK * 2;
    // B2 up to 128 wide: both B tiles share a stage with one A tile; 256 wide: a second pass over K (two
    // 256-row B tiles per stage would leave room for two stages only). A2: always a second pass (A2 with B).
    constexpr bool kext = BN == 256;
    const bool inst_b2 = has_b2 && !kext && !has_a2;
    const bool two_pass = (has_b2 && !inst_b2) || has_a2;
    const uint32_t stage_bytes = A_BYTES + B_BYTES * (inst_b2 ? 2u : 1u);
    uint64_t* bars = (uint64_t*)(smem + stages * stage_bytes);
    uint64_t* full = bars;
    uint64_t* empty = bars + stages;
    uint64_t* done = bars + 2 * stages;
    uint32_t* tmem_slot = (uint32_t*)(done + 1);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

    const int mt = blockIdx.x, nt = blockIdx.y;
    const int m0 = mt * TC_BM, n0 = nt * BN;
    if (epi.mode == TC_FOLD && n0 + BN - 1 < m0) return;  // every (n, m) of the tile has n < m
    if (epi.n_dev) N = min(N, *epi.n_dev);                // device-side row count of B (compacted rows)
    if (n0 >= N) return;                                  // uniform per CTA, before any barrier or TMEM use
    // K blocks of A this tile needs (a_lower: none past the tile's last row); with B2 the loop runs over them
    // twice, the second pass pairing A's block with B2's
    const int cap = a_lower ? min(nkb, (m0 + TC_BM + TC_BK - 1) / TC_BK) : nkb;
    int kb_end = two_pass ? 2 * cap : cap;
    // split K (grid z): this CTA sums K blocks [kb_begin, kb_end) into its own partial plane
    int kb_begin = 0;
    if (kb_split > 0) {
        kb_begin = blockIdx.z * kb_split;
        kb_end = min(kb_end, kb_begin + kb_split);
    }
    const int nk = max(kb_end - kb_begin, 0);   // the launcher guarantees nk >= 1
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) {
            mbar_init(smem_u32(&full[s]), 1);
            mbar_init(smem_u32(&empty[s]), 1);
        }
        mbar_init(smem_u32(done), 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"((uint32_t)BN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // TMA producer
        int issued = 0;
        for (int it = 0; it < nk; ++it) {
            const int kb = kb_begin + it;
            const int s = it % stages;
            if (it >= stages && !mbar_wait(smem_u32(&empty[s]), ((it / stages) & 1) ^ 1, abort_flag)) break;
            uint8_t* st = smem + s * stage_bytes;
            const uint32_t fb = smem_u32(&full[s]);
            const bool second = kb >= cap;
            const int ka = second ? kb - cap : kb;
            mbar_expect_tx(fb, stage_bytes);
            tma_load_2d(smem_u32(st), (second && has_a2) ? &tmA2 : &tmA, fb, ka * TC_BK, m0);
            tma_load_2d(smem_u32(st + A_BYTES), (second && has_b2) ? &tmB2 : &tmB, fb, ka * TC_BK, n0);
            if (inst_b2) tma_load_2d(smem_u32(st + A_BYTES + B_BYTES), &tmB2, fb, ka * TC_BK, n0);
            issued = it + 1;
        }
        if (*abort_flag) {
            // drain: every issued stage must land before the CTA may exit
            for (int kb = max(0, issued - stages); kb < issued; ++kb) {
                long long t0 = clock64();
                while (!mbar_try(smem_u32(&full[kb % stages]), (kb / stages) & 1) && clock64() - t0 < TC_WAIT_CYCLES) {
                }
            }
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        constexpr uint32_t idesc = idesc_bf16(BN);
        for (int it = 0; it < nk; ++it) {
            const int s = it % stages;
            if (!mbar_wait(smem_u32(&full[s]), (it / stages) & 1, abort_flag)) break;
            tc_fence_after();
            const uint32_t sa = smem_u32(smem + s * stage_bytes);
            const uint32_t sb = sa + A_BYTES;
#pragma unroll
            for (int kk = 0; kk < TC_BK / 16; ++kk) {
                const uint64_t ad = sdesc_sw128(sa + kk * 32);
                umma_bf16(tmem, ad, sdesc_sw128(sb + kk * 32), idesc, (it | kk) ? 1u : 0u);
                if (inst_b2) umma_bf16(tmem, ad, sdesc_sw128(sb + B_BYTES + kk * 32), idesc, 1u);
            }
            umma_commit(smem_u32(&empty[s]));
        }
        umma_commit(smem_u32(done));
    }
    __syncwarp();

    // epilogue: wait for the accumulator (bounded; after an abort too, for the MMAs issued so far to complete
    // before tensor memory is read or freed), then every warp reads its 32 TMEM lanes
    mbar_wait_drain(smem_u32(done), 0);
    __syncthreads();
    const bool ok = (*abort_flag == 0);
    tc_fence_after();
    if (ok) {
        const int row = warp * 32 + lane;
        const int m = m0 + row;
        const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
        if (epi.mode == TC_TARGET) {
            float* red = (float*)smem;  // the staging ring is free once the accumulator is complete
#pragma unroll 1
            for (int c = 0; c < BN / 32; ++c) {
                uint32_t r[32];
                tmem_ld32(trow + c * 32, r);
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int n = n0 + c * 32 + j;
                    float f = 0.f;
                    if (m < M && n < N) {
                        float u = __uint_as_float(r[j]);
                        if (epi.tanh_mode) {
                            double rr = epi.y[m] - (double)tanhf(u);
                            f = (float)(-rr * rr * epi.inv2s2);
                        } else {
                            f = -0.5f * u * u;
                        }
                    }
                    red[row * (BN + 1) + c * 32 + j] = f;
                }
            }
            __syncthreads();
            for (int col = threadIdx.x; col < BN; col += blockDim.x) {
                double s = 0.0;
                for (int rr = 0; rr < TC_BM; ++rr) s += (double)red[rr * (BN + 1) + col];
                if (n0 + col < N) epi.partial[(size_t)mt * N + n0 + col] = s;
            }
        } else {
            // the scale as two floats (beta alpha of the noise product: the same value the z recursion uses)
            const F2 scale = split_f2((epi.mode == TC_STORE && epi.scale_dev) ? *epi.scale_dev : 1.0);
#pragma unroll 1
            for (int c = 0; c < BN / 32; ++c) {
                uint32_t r[32];
                tmem_ld32(trow + c * 32, r);
                if (m < M) {
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const int n = n0 + c * 32 + j;
                        if (n >= N) continue;
                        const float v = __uint_as_float(r[j]);
                        if (epi.mode == TC_STORE) {
                            epi.D[(size_t)blockIdx.z * epi.split_stride + (size_t)n * epi.ldd + m] = mul_f2(scale, v, 0.f);
                        } else if (epi.mode == TC_GELU) {
                            const float zf = v + epi.bias[m];
                            if (epi.Zout) epi.Zout[(size_t)n * epi.ldz + m] = zf;
                            const float g = 0.5f * zf * (1.0f + erff(zf * 0.70710678118654752f));
                            epi.Hout[(size_t)n * epi.ldo + m] = f32_to_bf16_bits(g);
                        } else if (n >= m) {
                            double add = (double)v - epi.s[n] * epi.s[m] * epi.inb + epi.delta[n] * epi.delta[m] * epi.w;
                            epi.M2[(size_t)n * epi.ldm + m] += add;
                        }
                    }
                }
            }
        }
    } else if (threadIdx.x == 0) {
        set_status(status, DEV_TIMEOUT);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)BN));
}

// Persistent form of the wide products (BN = 256, store and fold epilogues, no split K): the interval's noise
// product, its map and the fold's SYRK. One CTA per SM walks a static list of output tiles (tile t = blockIdx.x +
// i gridDim.x, m fastest, so each CTA's tiles mix short and long triangular K ranges). Warp 0 stages the A and B
// tiles through the shared-memory ring without stopping at tile boundaries; warp 1 issues the products; warps 2-9
// (two per 32-lane quarter of tensor memory, 128 columns each) sum them.
//
// Accumulation in chunks: the tensor cores add each product into the FP32 accumulator after aligning it to the
// running sum and dropping the bits below (a truncation: a bias toward zero that grows with the number of products
// summed in one accumulator, measured on B300 at -8e-6 relative for K = 4096 on products like the noise product's,
// -4.7e-7 for chunks of 256 and -1e-7 for chunks of 64 summed outside in round-to-nearest). So each chunk of
// `chunk` K blocks goes into a fresh accumulator, one of two (2 x 256 columns, all of tensor memory), and the
// epilogue warps add the chunk sums in FP32 registers (round to nearest) while the next chunk's products run; a
// tile's result is written from the registers after its last chunk, while the products run up to two chunks
// ahead. The launcher sizes the chunk so that those two chunks cover the tile's write: 8 K blocks (K = 512) for
// the FP32 store, 32 (K = 2048) for the fold's FP64 read-modify-write of M2.
//
// Barriers: full / empty per ring stage, tfull (MMA -> epilogue) and tempty (epilogue -> MMA, 256 arrivals) per
// accumulator. Every wait is clock-bounded; on expiry the CTA records DEV_TIMEOUT, lets its TMA loads land and its
// issued MMAs complete (one commit tracks them all), frees its tensor memory and returns.
constexpr int PT_THREADS = 320, PT_BN = 256, PT_CHUNK_STORE = 8, PT_CHUNK_FOLD = 32;

__global__ void __launch_bounds__(PT_THREADS, 1) tc_gemm_persist_kernel(
    const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
    const __grid_constant__ CUtensorMap tmB2, const __grid_constant__ CUtensorMap tmA2, int M, int N, int nkb,
    int a_lower, int has_b2, int has_a2, int stages, int mtiles, int ntiles, int chunk, TcEpi epi, int* status) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    constexpr uint32_t A_BYTES = TC_BM * TC_BK * 2, B_BYTES = PT_BN * TC_BK * 2, STAGE = A_BYTES + B_BYTES;
    const bool two_pass = has_b2 || has_a2;
    uint64_t* full = (uint64_t*)(smem + stages * STAGE);
    uint64_t* empty = full + stages;
    uint64_t* tfull = empty + stages;   // [2]
    uint64_t* tempty = tfull + 2;       // [2]
    uint64_t* drain = tempty + 2;
    uint32_t* tmem_slot = (uint32_t*)(drain + 1);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (epi.n_dev) N = min(N, *epi.n_dev);   // device-side row count of B: tiles past it are skipped by every role
    // The tile list, n-column by n-column (the m-tiles of one column share its B tile in L2). The fold lists only
    // the tiles that meet the lower triangle (n0 + 255 >= m0): column j holds the first min(mtiles, fold_rows(j)).
    const bool fold = epi.mode == TC_FOLD;
    auto fold_rows = [&](int j) { return min(mtiles, (j * PT_BN + PT_BN - 1) / TC_BM + 1); };
    int T = mtiles * ntiles;
    if (fold) {
        T = 0;
        for (int j = 0; j < ntiles; ++j) T += fold_rows(j);
    }
    auto tile_of = [&](int t, int& m0, int& n0) {
        if (!fold) {
            m0 = (t % mtiles) * TC_BM;
            n0 = (t / mtiles) * PT_BN;
            return;
        }
        int j = 0;
        while (t >= fold_rows(j)) t -= fold_rows(j++);
        m0 = t * TC_BM;
        n0 = j * PT_BN;
    };
    // Round k of the CTAs takes tiles k G .. k G + G - 1, in reverse CTA order on odd rounds: with the noise
    // product's triangular K ranges (m-tile i carries i + 1 units) every CTA then gets close to the mean work.
    const int G = (int)gridDim.x, bx = (int)blockIdx.x;
    auto tile_at = [&](int k) { return k * G + ((k & 1) ? G - 1 - bx : bx); };
    auto valid = [&](int m0, int n0) { return n0 < N && !(epi.mode == TC_FOLD && n0 + PT_BN - 1 < m0); };
    auto cap_of = [&](int m0) { return a_lower ? min(nkb, (m0 + TC_BM + TC_BK - 1) / TC_BK) : nkb; };
    auto kend_of = [&](int m0) { return two_pass ? 2 * cap_of(m0) : cap_of(m0); };

    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) {
            mbar_init(smem_u32(&full[s]), 1);
            mbar_init(smem_u32(&empty[s]), 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(smem_u32(&tfull[a]), 1);
            mbar_init(smem_u32(&tempty[a]), 256);
        }
        mbar_init(smem_u32(drain), 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(2u * PT_BN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {   // TMA producer: a global k-block count across the CTA's tiles
            // the store products' A operand (the factor, the map: tens of MB, read by every n-column of tiles) is
            // kept in L2 while B (the interval's noise, hundreds of MB) streams through it
            const uint64_t pol_a = l2_policy_evict_last();
            const bool hint_a = epi.mode == TC_STORE;
            int it = 0;
            for (int k = 0; k * G < T && !*abort_flag; ++k) {
                const int t = tile_at(k);
                if (t >= T) continue;
                int m0, n0;
                tile_of(t, m0, n0);
                if (!valid(m0, n0)) continue;
                const int cap = cap_of(m0), kend = kend_of(m0);
                for (int kb = 0; kb < kend; ++kb, ++it) {
                    const int s = it % stages;
                    if (it >= stages && !mbar_wait(smem_u32(&empty[s]), ((it / stages) & 1) ^ 1, abort_flag)) break;
                    uint8_t* st = smem + s * STAGE;
                    const uint32_t fb = smem_u32(&full[s]);
                    const bool second = kb >= cap;
                    const int ka = second ? kb - cap : kb;
                    mbar_expect_tx(fb, STAGE);
                    const CUtensorMap* ma = (second && has_a2) ? &tmA2 : &tmA;
                    if (hint_a) tma_load_2d_hint(smem_u32(st), ma, fb, ka * TC_BK, m0, pol_a);
                    else tma_load_2d(smem_u32(st), ma, fb, ka * TC_BK, m0);
                    tma_load_2d(smem_u32(st + A_BYTES), (second && has_b2) ? &tmB2 : &tmB, fb, ka * TC_BK, n0);
                }
            }
            if (*abort_flag) {   // every issued load lands before the CTA may exit
                for (int k = max(0, it - stages); k < it; ++k) {
                    const long long t0 = clock64();
                    while (!mbar_try(smem_u32(&full[k % stages]), (k / stages) & 1) && clock64() - t0 < TC_WAIT_CYCLES) {
                    }
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {   // MMA issuer: a global chunk count picks the accumulator
            constexpr uint32_t idesc = idesc_bf16(PT_BN);
            int it = 0, cc = 0;
            bool ok = true;
            for (int k = 0; k * G < T && ok && !*abort_flag; ++k) {
                const int t = tile_at(k);
                if (t >= T) continue;
                int m0, n0;
                tile_of(t, m0, n0);
                if (!valid(m0, n0)) continue;
                const int kend = kend_of(m0);
                for (int kb0 = 0; kb0 < kend; kb0 += chunk, ++cc) {
                    const int acc = cc & 1;
                    // the epilogue has taken the chunk two back out of this accumulator
                    if (cc >= 2 && !mbar_wait(smem_u32(&tempty[acc]), ((cc >> 1) - 1) & 1, abort_flag)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t tacc = tmem + (uint32_t)(acc * PT_BN);
                    const int kb1 = min(kend, kb0 + chunk);
                    for (int kb = kb0; kb < kb1; ++kb, ++it) {
                        const int s = it % stages;
                        if (!mbar_wait(smem_u32(&full[s]), (it / stages) & 1, abort_flag)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t sa = smem_u32(smem + s * STAGE), sb = sa + A_BYTES;
#pragma unroll
                        for (int kk = 0; kk < TC_BK / 16; ++kk)
                            umma_bf16(tacc, sdesc_sw128(sa + kk * 32), sdesc_sw128(sb + kk * 32), idesc,
                                      (kb > kb0 || kk) ? 1u : 0u);
                        umma_commit(smem_u32(&empty[s]));
                    }
                    if (!ok) break;
                    umma_commit(smem_u32(&tfull[acc]));
                }
            }
            umma_commit(smem_u32(drain));   // completes once every MMA this thread issued has
        }
    } else {   // epilogue warps 2-9: lanes 32 (warp % 4) .. + 31 of tensor memory, columns 128 h .. + 127
        const int quarter = warp & 3, h = (warp - 2) >> 2, row = quarter * 32 + lane;
        const F2 scale = split_f2((epi.mode == TC_STORE && epi.scale_dev) ? *epi.scale_dev : 1.0);
        float sum[128];
        int cc = 0;
        bool ok = true;
        for (int k = 0; k * G < T && ok; ++k) {
            const int t = tile_at(k);
            if (t >= T) continue;
            int m0, n0;
            tile_of(t, m0, n0);
            if (!valid(m0, n0)) continue;
            const int nch = (kend_of(m0) + chunk - 1) / chunk;
            for (int c = 0; c < nch; ++c, ++cc) {
                const int acc = cc & 1;
                if (!mbar_wait(smem_u32(&tfull[acc]), (cc >> 1) & 1, abort_flag)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t tb = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(acc * PT_BN + h * 128);
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    uint32_t r[16];
                    tmem_ld16(tb + i * 16, r);
#pragma unroll
                    for (int j = 0; j < 16; ++j) sum[i * 16 + j] = (c ? sum[i * 16 + j] : 0.f) + __uint_as_float(r[j]);
                }
                tc_fence_before();
                mbar_arrive(smem_u32(&tempty[acc]));
            }
            if (!ok) break;
            const int m = m0 + row;
            if (m < M) {
#pragma unroll
                for (int j = 0; j < 128; ++j) {
                    const int n = n0 + h * 128 + j;
                    if (n >= N) continue;
                    if (epi.mode == TC_STORE) {
                        epi.D[(size_t)n * epi.ldd + m] = mul_f2(scale, sum[j], 0.f);
                    } else if (n >= m) {
                        const double add = (double)sum[j] - epi.s[n] * epi.s[m] * epi.inb + epi.delta[n] * epi.delta[m] * epi.w;
                        epi.M2[(size_t)n * epi.ldm + m] += add;
                    }
                }
            }
        }
    }
    __syncwarp();
    // every MMA issued has completed (bounded, even after an abort) before tensor memory is freed
    mbar_wait_drain(smem_u32(drain), 0);
    if (threadIdx.x == 0 && *abort_flag) set_status(status, DEV_TIMEOUT);
    tc_fence_before();
    __syncthreads();
    if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2u * PT_BN));
}

// ---------------------------------------------------------------------------------------------------- host
constexpr int kAttrDevices = 64;   // devices a process can drive (per-device launch attributes)
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    });
    return fn;
}

// 2D BF16 map over rows x ld (ld the padded row length, a multiple of 64), box 64 x box_rows, 128B swizzle.
bool make_map(CUtensorMap* map, const void* ptr, int rows, int ld, int box_rows) {
    static std::mutex mu;
    static std::map<std::tuple<const void*, int, int, int>, CUtensorMap> cache;
    std::lock_guard<std::mutex> g(mu);
    auto key = std::make_tuple(ptr, rows, ld, box_rows);
    auto it = cache.find(key);
    if (it != cache.end()) {
        *map = it->second;
        return true;
    }
    EncodeTiledFn enc = encode_fn();
    if (!enc) return false;
    cuuint64_t dims[2] = {(cuuint64_t)ld, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    cuuint32_t box[2] = {(cuuint32_t)TC_BK, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return false;
    if (cache.size() > 4096) cache.clear();
    cache[key] = *map;
    return true;
}

template <int BN>
static cudaError_t launch_bn(int M, int N, int K, const uint16_t* A, int lda, const uint16_t* B, const uint16_t* B2,
                             int ldb, int a_lower, const TcEpi& epi, int* status, cudaStream_t st, int splits = 1,
                             const uint16_t* A2 = nullptr) {
    CUtensorMap mA, mB, mB2, mA2;
    if (B2 && A2) return cudaErrorInvalidValue;
    if (!make_map(&mA, A, M, lda, TC_BM) || !make_map(&mB, B, N, ldb, BN) ||
        !make_map(&mB2, B2 ? B2 : B, N, ldb, BN) || !make_map(&mA2, A2 ? A2 : A, M, lda, TC_BM))
        return cudaErrorInvalidValue;
    const int has_b2 = B2 != nullptr, has_a2 = A2 != nullptr;
    const bool kext = BN == 256;
    const bool inst_b2 = has_b2 && !kext && !has_a2, two_pass = (has_b2 && !inst_b2) || has_a2;
    const size_t stage = (size_t)TC_BM * TC_BK * 2 + (size_t)BN * TC_BK * 2 * (inst_b2 ? 2 : 1);
    // 4 stages where they fit (measured: deeper rings only add L2 traffic in flight at the same rate)
    const int stages = (int)std::min<size_t>(TC_MAX_STAGES, (227 * 1024 - 1024 - 256) / stage);
    size_t smem = 1024 + stages * stage + 256;
    const size_t red = (size_t)TC_BM * (BN + 1) * 4;
    if (smem < 1024 + red + 256) smem = 1024 + red + 256;
    // the 227 KB dynamic shared-memory attribute applies to the current device only: set once per device
    static std::mutex attr_mu;
    static bool attr_set[kAttrDevices] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kAttrDevices) return cudaErrorInvalidDevice;
    {
        std::lock_guard<std::mutex> g(attr_mu);
        if (!attr_set[dev]) {
            cudaError_t e = cudaFuncSetAttribute(tc_gemm_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
            if (e != cudaSuccess) return e;
            attr_set[dev] = true;
        }
    }
    const int nkb = K / TC_BK, ktot = two_pass ? 2 * nkb : nkb;
    int kb_split = 0;
    if (splits > 1) {
        kb_split = (ktot + splits - 1) / splits;
        splits = (ktot + kb_split - 1) / kb_split;   // every split gets at least one K block
    } else {
        splits = 1;
    }
    dim3 grid((M + TC_BM - 1) / TC_BM, (N + BN - 1) / BN, splits);
    if (BN == PT_BN && splits == 1 && (epi.mode == TC_STORE || epi.mode == TC_FOLD)) {
        // the wide store / fold products: persistent, one CTA per SM, epilogues beside the next tile's products
        static bool pattr_set[kAttrDevices] = {};
        static int sms[kAttrDevices] = {};
        {
            std::lock_guard<std::mutex> g(attr_mu);
            if (!pattr_set[dev]) {
                cudaError_t e = cudaFuncSetAttribute(tc_gemm_persist_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                     227 * 1024);
                if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms[dev], cudaDevAttrMultiProcessorCount, dev);
                if (e != cudaSuccess) return e;
                pattr_set[dev] = true;
            }
        }
        const size_t pstage = (size_t)TC_BM * TC_BK * 2 + (size_t)PT_BN * TC_BK * 2;
        const int pst = (int)std::min<size_t>(TC_MAX_STAGES, (227 * 1024 - 1024 - 256) / pstage);
        const size_t psmem = 1024 + pst * pstage + 256;
        int tiles = (int)grid.x * (int)grid.y;
        if (epi.mode == TC_FOLD) {   // the tiles that meet the lower triangle (the kernel's list)
            tiles = 0;
            for (int j = 0; j < (int)grid.y; ++j) tiles += std::min((int)grid.x, (j * PT_BN + PT_BN - 1) / TC_BM + 1);
        }
        const int ctas = std::max(1, std::min(tiles, sms[dev]));
        const int chunk = epi.mode == TC_FOLD ? PT_CHUNK_FOLD : PT_CHUNK_STORE;
        { tc_gemm_persist_kernel<<<ctas, PT_THREADS, psmem, st>>>(mA, mB, mB2, mA2, M, N, nkb, a_lower, has_b2, has_a2,
                                                                 pst, (int)grid.x, (int)grid.y, chunk, epi, status); count_launch(); }
        return cudaGetLastError();
    }
    { tc_gemm_kernel<BN><<<grid, 128, smem, st>>>(mA, mB, mB2, mA2, M, N, nkb, a_lower, has_b2, has_a2, kb_split, stages,
                                                  epi, status); count_launch(); }
    return cudaGetLastError();
}

static cudaError_t launch_any(int bn, int M, int N, int K, const uint16_t* A, int lda, const uint16_t* B,
                              const uint16_t* B2, int ldb, int a_lower, const TcEpi& epi, int* status, cudaStream_t st,
                              int splits, const uint16_t* A2 = nullptr) {
    switch (bn) {
        case 32: return launch_bn<32>(M, N, K, A, lda, B, B2, ldb, a_lower, epi, status, st, splits, A2);
        case 64: return launch_bn<64>(M, N, K, A, lda, B, B2, ldb, a_lower, epi, status, st, splits, A2);
        case 256: return launch_bn<256>(M, N, K, A, lda, B, B2, ldb, a_lower, epi, status, st, splits, A2);
        default: return launch_bn<128>(M, N, K, A, lda, B, B2, ldb, a_lower, epi, status, st, splits, A2);
    }
}

static bool args_ok(int K, int lda, int ldb, const uint16_t* A, const uint16_t* B, const uint16_t* B2) {
    if (K <= 0 || K % TC_BK || lda % TC_BK || ldb % TC_BK || K > lda || K > ldb) return false;
    return ((((uintptr_t)A | (uintptr_t)B | (uintptr_t)(B2 ? B2 : B)) & 15) == 0);
}

cudaError_t tc_gemm_bf16(int M, int N, int K, const uint16_t* A, int lda, const uint16_t* B, const uint16_t* B2, int ldb,
                         int a_lower, const TcEpi& epi, int* status_dev, cudaStream_t st, int bn) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    if (!args_ok(K, lda, ldb, A, B, B2)) return cudaErrorInvalidValue;
    return launch_any(bn, M, N, K, A, lda, B, B2, ldb, a_lower, epi, status_dev, st, 1);
}

cudaError_t tc_gemm_bf16_a2(int M, int N, int K, const uint16_t* A, const uint16_t* A2, int lda, const uint16_t* B,
                            int ldb, int a_lower, const TcEpi& epi, int* status_dev, cudaStream_t st, int bn) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    if (!A2 || (((uintptr_t)A2) & 15) || !args_ok(K, lda, ldb, A, B, nullptr)) return cudaErrorInvalidValue;
    return launch_any(bn, M, N, K, A, lda, B, nullptr, ldb, a_lower, epi, status_dev, st, 1, A2);
}

// Split-K form: K blocks divided over `splits` CTAs per tile; each writes its FP32 partial product to
// D + z * split_stride (TC_STORE only, no triangular skip). Returns the number of partial planes in *used.
cudaError_t tc_gemm_bf16_splitk(int M, int N, int K, const uint16_t* A, int lda, const uint16_t* B, const uint16_t* B2,
                                int ldb, int splits, const TcEpi& epi, int* status_dev, cudaStream_t st, int* used, int bn) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    if (epi.mode != TC_STORE || splits < 1) return cudaErrorInvalidValue;
    if (!args_ok(K, lda, ldb, A, B, B2)) return cudaErrorInvalidValue;
    const int ktot = (K / TC_BK) * ((B2 && bn == 256) ? 2 : 1);
    splits = std::min(splits, ktot);
    const int per = (ktot + splits - 1) / splits;
    *used = (ktot + per - 1) / per;
    return launch_any(bn, M, N, K, A, lda, B, B2, ldb, 0, epi, status_dev, st, *used);
}

// Tile autotuner: times BN = 32, 64, 128 (one warm-up and two timed launches each, CUDA events on st)
// for this product on the caller's buffers and keeps the fastest per shape.
int tc_autotune(int M, int N, int K, const uint16_t* A, int lda, const uint16_t* B, const uint16_t* B2, int ldb,
                int splits, int a_lower, const TcEpi& epi, int* status_dev, cudaStream_t st, float* best_ms) {
    static std::mutex mu;
    static std::map<std::tuple<int, int, int, int, int, int, int>, std::pair<int, float>> cache;
    const auto key = std::make_tuple(M, N, K, B2 ? 1 : 0, splits, a_lower, epi.mode);
    {
        std::lock_guard<std::mutex> g(mu);
        auto it = cache.find(key);
        if (it != cache.end()) {
            if (best_ms) *best_ms = it->second.second;
            return it->second.first;
        }
    }
    int best = 128;
    float best_t = 1e30f;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return best;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return best;
    }
    for (int bn : {32, 64, 128, 256}) {
        if (bn > 32 && N <= bn / 2) continue;   // a tile at least twice as wide as N only wastes MMA work
        int used = 1;
        auto go = [&]() {
            return splits > 1 ? tc_gemm_bf16_splitk(M, N, K, A, lda, B, B2, ldb, splits, epi, status_dev, st, &used, bn)
                              : tc_gemm_bf16(M, N, K, A, lda, B, B2, ldb, a_lower, epi, status_dev, st, bn);
        };
        if (go() != cudaSuccess) continue;
        cudaEventRecord(e0, st);
        bool ok = go() == cudaSuccess && go() == cudaSuccess;
        cudaEventRecord(e1, st);
        if (!ok || cudaEventSynchronize(e1) != cudaSuccess) continue;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_t) {
            best_t = ms;
            best = bn;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    {
        std::lock_guard<std::mutex> g(mu);
        cache[key] = {best, best_t / 2};
    }
    if (best_ms) *best_ms = best_t / 2;
    return best;
}

// ---------------------------------------------------------------------------------------------------- transpose
__global__ void transpose_f32_bf16_kernel(const float* __restrict__ in, int ldi, int rows, int cols,
                                          uint16_t* __restrict__ out, int ldo) {
    __shared__ uint16_t tile[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        int r = r0 + k, c = c0 + threadIdx.x;
        tile[k][threadIdx.x] = (r < rows && c < cols) ? f32_to_bf16_bits(in[(size_t)r * ldi + c]) : (uint16_t)0;
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        int c = c0 + k, r = r0 + threadIdx.x;
        if (c < cols && r < ldo) out[(size_t)c * ldo + r] = tile[threadIdx.x][k];
    }
}

cudaError_t transpose_f32_bf16(const float* in, int ldi, int rows, int cols, uint16_t* out, int ldo, cudaStream_t st) {
    dim3 grid((cols + 31) / 32, (ldo + 31) / 32);
    { transpose_f32_bf16_kernel<<<grid, dim3(32, 8), 0, st>>>(in, ldi, rows, cols, out, ldo); count_launch(); }
    return cudaGetLastError();
}

}  // namespace diam
