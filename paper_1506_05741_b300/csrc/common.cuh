// common.cuh -- device helpers shared by the DIAM kernels (sm_103a).
//
// Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) with the counter layout
//   key = (seed lo, seed hi ^ problem_id * 0x9E3779B9), ctr = (j, step lo, chain, tag | step hi << 8),
// and Gaussian pairs by the Box-Muller transform evaluated in IEEE FP32 with log / sin / cos written out
// from their series. Every operation is an explicitly rounded intrinsic (__fmaf_rn, __fmul_rn, ...), so
// the compiler cannot contract or reorder it and each draw is fixed by IEEE arithmetic alone.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

namespace diam {

// Host side: every kernel launch of the library is counted (diam_kernel_launches).
void count_launch();

enum : uint32_t { TAG_W = 0, TAG_U = 1, TAG_X0 = 2, TAG_UDA = 3 };

struct Key {
    uint32_t k0, k1;
};

__host__ __device__ inline Key make_key(uint64_t seed, uint32_t problem_id) {
    Key k;
    k.k0 = (uint32_t)seed;
    k.k1 = (uint32_t)(seed >> 32) ^ (uint32_t)(problem_id * 0x9E3779B9u);
    return k;
}

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, Key k) {
    uint32_t k0 = k.k0, k1 = k.k1;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

__device__ __forceinline__ uint4 draw(Key k, uint32_t j, int64_t t, uint32_t p, uint32_t tag) {
    uint4 c = make_uint4(j, (uint32_t)t, p, tag | ((uint32_t)((uint64_t)t >> 32) << 8));
    return philox4x32_10(c, k);
}

// ln(u1), u1 = ((a >> 8) + 1) 2^-24: ln m = 2 atanh(s), s = (m-1)/(m+1), m in [1/sqrt2, sqrt2].
__device__ __forceinline__ float ln_u24(uint32_t a) {
    uint32_t kk = (a >> 8) + 1u;
    int e = 31 - __clz(kk);
    float m = __fmul_rn(__uint2float_rn(kk), __int_as_float((127 - e) << 23));  // exact scaling by 2^-e
    if (m > 0x1.6a09e6p+0f) {
        m = __fmul_rn(m, 0.5f);
        e += 1;
    }
    float s = __fdiv_rn(__fsub_rn(m, 1.0f), __fadd_rn(m, 1.0f));
    float w = __fmul_rn(s, s);
    float poly = 0x1.c71c72p-4f;
    poly = __fmaf_rn(poly, w, 0x1.24924ap-3f);
    poly = __fmaf_rn(poly, w, 0x1.99999ap-3f);
    poly = __fmaf_rn(poly, w, 0x1.555556p-2f);
    poly = __fmaf_rn(poly, w, 1.0f);
    float lnm = __fmul_rn(__fmul_rn(2.0f, s), poly);
    return __fmaf_rn((float)(e - 24), 0x1.62e430p-1f, lnm);
}

// (cos, sin)(2 pi u2), u2 = (b >> 8) 2^-24: quadrant from the top two bits; Taylor series on [0, pi/4].
__device__ __forceinline__ void cossin_u24(uint32_t b, float& co, float& si) {
    uint32_t q = b >> 30;
    uint32_t f = (b >> 8) & 0x3FFFFFu;
    bool swap = f > (1u << 21);
    uint32_t fw = swap ? ((1u << 22) - f) : f;
    float phi = __fmul_rn(__fmul_rn(__uint2float_rn(fw), 0x1p-22f), 0x1.921fb6p+0f);
    float p2 = __fmul_rn(phi, phi);
    float ts = 0x1.71de3ap-19f;
    ts = __fmaf_rn(ts, p2, -0x1.a01a02p-13f);
    ts = __fmaf_rn(ts, p2, 0x1.111112p-7f);
    ts = __fmaf_rn(ts, p2, -0x1.555556p-3f);
    ts = __fmaf_rn(ts, p2, 1.0f);
    float sphi = __fmul_rn(phi, ts);
    float tc = -0x1.27e4fcp-22f;
    tc = __fmaf_rn(tc, p2, 0x1.a01a02p-16f);
    tc = __fmaf_rn(tc, p2, -0x1.6c16c2p-10f);
    tc = __fmaf_rn(tc, p2, 0x1.555556p-5f);
    tc = __fmaf_rn(tc, p2, -0.5f);
    tc = __fmaf_rn(tc, p2, 1.0f);
    float s = swap ? tc : sphi;
    float c = swap ? sphi : tc;
    switch (q) {
        case 0: co = c; si = s; break;
        case 1: co = -s; si = c; break;
        case 2: co = -c; si = -s; break;
        default: co = s; si = -c; break;
    }
}

__device__ __forceinline__ float2 boxmuller(uint32_t a, uint32_t b) {
    float r = __fsqrt_rn(__fmul_rn(-2.0f, ln_u24(a)));
    float c, s;
    cossin_u24(b, c, s);
    return make_float2(__fmul_rn(r, c), __fmul_rn(r, s));
}

// Four consecutive components 4j .. 4j+3 of W for chain p at step t.
__device__ __forceinline__ float4 normals4(Key k, uint32_t j, int64_t t, uint32_t p) {
    uint4 r = draw(k, j, t, p, TAG_W);
    float2 a = boxmuller(r.x, r.y);
    float2 b = boxmuller(r.z, r.w);
    return make_float4(a.x, a.y, b.x, b.y);
}

// u in (0, 1], 53 bits: u = (u53 + 1) 2^-53.
__device__ __forceinline__ double uniform53(Key k, int64_t t, uint32_t p, uint32_t tag) {
    uint4 r = draw(k, 0u, t, p, tag);
    uint64_t u53 = ((uint64_t)(r.x >> 11) << 32) | (uint64_t)r.y;
    return (double)(u53 + 1ull) * 0x1p-53;
}

// Round to nearest even at BF16 precision (8 significant bits), FP64 in, FP64 out.
__host__ __device__ inline double round_bf16(double v) {
    unsigned long long bits;
#ifdef __CUDA_ARCH__
    bits = (unsigned long long)__double_as_longlong(v);
#else
    memcpy(&bits, &v, 8);
#endif
    if (((bits >> 52) & 0x7FFull) == 0x7FFull) return v;
    unsigned long long lsb = (bits >> 45) & 1ull;
    bits += (1ull << 44) - 1ull + lsb;
    bits &= ~((1ull << 45) - 1ull);
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)bits);
#else
    double r;
    memcpy(&r, &bits, 8);
    return r;
#endif
}

// FP32 -> BF16 bits, round to nearest even.
__device__ __forceinline__ uint16_t f32_to_bf16_bits(float v) {
    uint32_t b = __float_as_uint(v);
    if ((b & 0x7F800000u) == 0x7F800000u) return (uint16_t)(b >> 16);
    b += 0x7FFFu + ((b >> 16) & 1u);
    return (uint16_t)(b >> 16);
}

// TF32: 11 significant bits (FP32's exponent range), round to nearest, ties to even, from FP64.
__host__ __device__ inline double round_tf32(double v) {
    unsigned long long bits;
#ifdef __CUDA_ARCH__
    bits = (unsigned long long)__double_as_longlong(v);
#else
    memcpy(&bits, &v, 8);
#endif
    if (((bits >> 52) & 0x7FFull) == 0x7FFull) return v;
    const unsigned long long lsb = (bits >> 42) & 1ull;
    bits += (1ull << 41) - 1ull + lsb;
    bits &= ~((1ull << 42) - 1ull);
    double r;
#ifdef __CUDA_ARCH__
    r = __longlong_as_double((long long)bits);
#else
    memcpy(&r, &bits, 8);
#endif
    return r;
}

// An FP64 value already at BF16 precision, as BF16 bits (exact).
__device__ __forceinline__ uint16_t bf16_bits_of_rounded(double v) {
    return (uint16_t)(__float_as_uint((float)v) >> 16);
}

__device__ __forceinline__ float bf16_bits_to_f32(uint16_t h) { return __uint_as_float(((uint32_t)h) << 16); }

// Device status word (one per context): the first error wins.
enum : int { DEV_OK = 0, DEV_TIMEOUT = 1, DEV_BADARG = 2 };

__device__ __forceinline__ void set_status(int* st, int code) {
    if (st) atomicCAS(st, 0, code);
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide sum (blockDim.x a multiple of 32); result valid in every thread. sh: >= 32 elements.
template <typename T>
__device__ __forceinline__ T block_sum(T v, T* sh) {
    v = warp_sum(v);
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    int nw = blockDim.x >> 5;
    T r = (threadIdx.x < (unsigned)nw) ? sh[threadIdx.x] : (T)0;
    if (w == 0) r = warp_sum(r);
    if (threadIdx.x == 0) sh[0] = r;
    __syncthreads();
    r = sh[0];
    __syncthreads();
    return r;
}

// An FP64 scalar as the unevaluated sum of two floats (hi + lo equals it to about 2^-48 relative). The FP32
// updates of BF16 mode take the proposal's rho and beta alpha this way: rounded to one float each, rho^2 + beta^2
// would miss 1 by up to ~1e-7, a different proposal whose density the z recursion no longer gives exactly, and x*
// would leave the FP64 proposal by a coherent rho-rounding times x (its log-density change by ~1e-7 d); with the
// pair, x* and z* differ from the FP64 proposal only by the FP32 rounding of each result.
struct F2 {
    float hi, lo;
};
__host__ __device__ __forceinline__ F2 split_f2(double v) {
    const float h = (float)v;
    return F2{h, (float)(v - (double)h)};
}
// a x + add, with a given as hi + lo
__device__ __forceinline__ float mul_f2(F2 a, float x, float add) { return fmaf(a.hi, x, fmaf(a.lo, x, add)); }

// A kernel's dynamic shared-memory limit is a property of the kernel (per device), shared by every context in the
// process whatever its size: raise it once to all the device allows next to the kernel's static shared memory, so
// no context lowers it below what another launches with.
inline cudaError_t allow_max_dynamic_smem(const void* kernel) {
    cudaFuncAttributes fa;
    int dev = 0, optin = 0;
    cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
    return e;
}

}  // namespace diam
