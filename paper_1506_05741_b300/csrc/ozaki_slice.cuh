// ozaki_slice.cuh -- the row splitting of the Ozaki scheme, shared by the kernels that produce panels.
//
// A row of 64 FP64 entries (lane l holds entries l and l + 32) is scaled by 2^-e (max |entry| < 2^e),
// rounded once to the integer R = round(entry 2^(55 - e)) (|R| <= 2^55) and cut into 7 signed base-256
// digits |S_a| <= 128, entry = 2^(e - 7) sum_a S_a 2^(-8a) up to 2^(e - 56). Each digit is an integer of at
// most 8 significant bits and so exact in BF16; digit a of entry k goes to SLrow[a * 64 + k].
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace diam {

constexpr int OZ_S = 7, OZ_K = 64, OZ_LD = OZ_S * OZ_K;

// 2^e as a double (exact for normal exponents).
__device__ __forceinline__ double pow2(int e) {
    return (e >= -1022 && e <= 1023) ? __hiloint2double((e + 1023) << 20, 0) : ldexp(1.0, e);
}

// Whole warp: slices of the row (v0, v1) into SLrow; returns e (lane 0 stores it where the caller says).
__device__ __forceinline__ int ozaki_slice_row(double v0, double v1, int lane, uint16_t* __restrict__ SLrow) {
    double m = fmax(fabs(v0), fabs(v1));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    const int e = (m > 0.0) ? ilogb(m) + 1 : 0;   // m < 2^e
    const double sc = pow2(55 - e);
    uint16_t* out = SLrow + lane;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        long long R = __double2ll_rn((h ? v1 : v0) * sc);   // exact scaling, then one rounding
#pragma unroll
        for (int a = 0; a < OZ_S; ++a) {
            const int s = 48 - 8 * a;
            const long long S = (s > 0) ? ((R + (1ll << (s - 1))) >> s) : R;   // |S| <= 128
            R -= S * (1ll << s);                                                 // |R| <= 2^(s-1)
            out[a * OZ_K + 32 * h] = (uint16_t)(__float_as_uint((float)S) >> 16);
        }
    }
    return e;
}

}  // namespace diam
