// rec.cuh -- the linear map of the target carried through the proposal (BF16 mode, linear-map targets).
//
// The target's expensive term is a linear map u = A x (tanh regression: u_m = a_m . x; dense Gaussian:
// u = G x). The proposal of eq. (diam), x* = x_ref + rho (x - x_ref) + xi with xi = beta alpha A_n W, is
// linear in x, so A x* = rho (A x) + (1 - rho) (A x_ref) + (A A_n) (beta alpha W): with M = A A_n formed once
// per refresh and the products M W of a whole interval in one GEMM (Algorithm 1's batching of the noise
// product, extended to the map), each step needs only O(d_y) work per chain instead of a d_y x d product.
// A x of the current states is recomputed at every interval start from the states split into three BF16
// terms (hi + lo + lo2 = x exactly; FP32 accumulation); accepted chains copy A x*. M is kept as a two-term
// BF16 split (hi + lo, relative error ~2^-17): its error enters each step's map through beta alpha M W only.
#pragma once
#include "common.cuh"

namespace diam {
namespace {

// hi = bf16(F), lo = bf16(F - hi) for rows x cols of F (stride ld); the padding columns stay zero.
__global__ void split_hi_lo_kernel(int rows, int cols, int ld, const float* __restrict__ F, uint16_t* __restrict__ hi,
                                   uint16_t* __restrict__ lo) {
    const int r = blockIdx.y;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < cols; c += gridDim.x * blockDim.x) {
        const float v = F[(size_t)r * ld + c];
        const uint16_t h = f32_to_bf16_bits(v);
        hi[(size_t)r * ld + c] = h;
        lo[(size_t)r * ld + c] = f32_to_bf16_bits(v - bf16_bits_to_f32(h));
    }
}

// D[i] += E[i] for i < n (the last term of a product split over K passes)
__global__ void add_f32_kernel(size_t n, float* __restrict__ D, const float* __restrict__ E) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) D[i] += E[i];
}

// axref[m] = sum_k A[m][k] x_ref[k] (A the BF16 map, stride ld), FP64 sums; one block per row.
__global__ void __launch_bounds__(256) axref_kernel(int d, int ld, const uint16_t* __restrict__ A,
                                                     const float* __restrict__ xref, float* __restrict__ axref) {
    __shared__ double sh[32];
    const int m = blockIdx.x;
    double s = 0.0;
    for (int k = threadIdx.x; k < d; k += blockDim.x)
        s += (double)bf16_bits_to_f32(A[(size_t)m * ld + k]) * (double)xref[k];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) axref[m] = (float)s;
}

// One block per chain: u = rho Ax + (1 - rho) Axref + AXi[step], stored as the proposal's map values, and
// the linear-map terms of log pi summed in FP32 (tanh regression: -(y - tanh u)^2 inv2s2; dense: -u^2 / 2).
__global__ void __launch_bounds__(256) rec_map_kernel(int P, int dy, const Ctl* ctl, const float* __restrict__ Ax,
                                                       const float* __restrict__ axref, const float* __restrict__ AXi,
                                                       float* __restrict__ Axp, const float* __restrict__ y32,
                                                       float inv2s2, int tanh_mode, double* __restrict__ lmap) {
    __shared__ float shf[32];
    const int p = blockIdx.x;
    const F2 rho = split_f2(ctl->rho);
    const float om = (float)(1.0 - ctl->rho);
    const float* ax = Ax + (size_t)p * dy;
    const float* xi = AXi + ((size_t)ctl->s_cur * P + p) * dy;
    float* axp = Axp + (size_t)p * dy;
    float acc = 0.f;
    for (int m = threadIdx.x; m < dy; m += blockDim.x) {
        const float u = mul_f2(rho, ax[m], fmaf(om, axref[m], xi[m]));
        axp[m] = u;
        if (tanh_mode) {
            const float r = y32[m] - tanhf(u);
            acc -= r * r * inv2s2;
        } else {
            acc -= 0.5f * u * u;
        }
    }
    acc = block_sum(acc, shf);
    if (threadIdx.x == 0) lmap[p] = (double)acc;
}

}  // namespace
}  // namespace diam
