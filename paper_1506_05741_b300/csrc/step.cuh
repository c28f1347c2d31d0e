// step.cuh -- per-step and per-interval kernels of the DIAM sampler.
//
// T is the chain-state type: double (FP64 mode) or float (BF16 mode, where the factor, the noise and the
// target's linear map are BF16 and the states FP32). One thread block per chain for the O(d) work; the
// products (noise, linear-map targets, moments) are separate GEMM launches.
#pragma once
#include <type_traits>

#include "common.cuh"
#include "tc_common.cuh"

namespace diam {
namespace {  // internal linkage: each translation unit that launches these gets its own copy

// Device-resident scalars of one context.
struct Ctl {
    double beta, rho, ba, inv_infl2;   // beta, sqrt(1 - beta^2), beta * alpha, 1 / alpha^2 (in effect)
    unsigned long long acc_block;      // accepted moves in the current interval
    unsigned long long nonfinite;      // proposals with a non-finite log-density
    int status;                        // DEV_* code, first error wins
    int chol_info;                     // Cholesky failure (pivot + 1)
    double trace;                      // tr(M2) at the last refresh
    long long t_cur;                   // global step the step kernels are working on
    int s_cur;                         // its index within the interval
    unsigned done_blocks;              // blocks of the step's last kernel that have finished (0 between steps)
};

// End of one step: the step counters move on (the step kernels read them, so a captured graph of the
// interval's steps replays unchanged).
__global__ void advance_kernel(Ctl* ctl) {
    ctl->t_cur += 1;
    ctl->s_cur += 1;
}

__global__ void set_step_kernel(Ctl* ctl, long long t, int s) {
    ctl->t_cur = t;
    ctl->s_cur = s;
}

enum : int { TK_DIAG = 0, TK_DENSE = 1, TK_TANH = 2, TK_BANANA = 3, TK_REF = 4, TK_CALLBACK = 5, TK_TWIST = 6 };

struct TargetDev {
    int kind;
    int d_y;
    const double* inv_lam;     // d, 1 / lambda_i
    const float* inv_lam32;    // the same in FP32 (BF16 mode: FP32 states)
    double ban_a, ban_b, ban_c;
};

// O(d) part of log pi at x (terms that need no matrix): the diagonal Gaussian, the tanh-regression prior,
// the banana tail. Returns this thread's share over i = tid, tid + nthreads, ...
template <typename T>
__device__ __forceinline__ double od_term(const TargetDev& tg, int i, T x) {
    if (tg.kind == TK_DIAG || tg.kind == TK_TANH || (tg.kind == TK_BANANA && i >= 2)) {
        double xd = (double)x;
        return -0.5 * xd * xd * tg.inv_lam[i];
    }
    return 0.0;
}

__device__ __forceinline__ double banana_head(const TargetDev& tg, double x1, double x2) {
    double v = x2 + tg.ban_b * x1 * x1 - tg.ban_c;
    return -x1 * x1 / (2.0 * tg.ban_a) - 0.5 * v * v;
}

// ---------------------------------------------------------------------------------------------------
// W for n_steps steps starting at t0 and P chains: row r = s P + p holds W (d entries, zero-padded to ld).
template <typename OutT>
__device__ __forceinline__ OutT cvt_w(float v);
template <>
__device__ __forceinline__ double cvt_w<double>(float v) { return (double)v; }
template <>
__device__ __forceinline__ float cvt_w<float>(float v) { return v; }
template <>
__device__ __forceinline__ uint16_t cvt_w<uint16_t>(float v) { return f32_to_bf16_bits(v); }

// Four entries of a W row, one vector store where the row allows it (BF16: 8 bytes, FP32: 16 bytes).
template <typename OutT>
__device__ __forceinline__ void store_w4(OutT* o, float4 w, int left, bool vec) {
    const float v[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) o[q] = (q < left) ? cvt_w<OutT>(v[q]) : cvt_w<OutT>(0.f);
}
template <>
__device__ __forceinline__ void store_w4<uint16_t>(uint16_t* o, float4 w, int left, bool vec) {
    if (vec && left >= 4) {
        *reinterpret_cast<uint2*>(o) = make_uint2((uint32_t)f32_to_bf16_bits(w.x) | ((uint32_t)f32_to_bf16_bits(w.y) << 16),
                                                  (uint32_t)f32_to_bf16_bits(w.z) | ((uint32_t)f32_to_bf16_bits(w.w) << 16));
        return;
    }
    const float v[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) o[q] = (q < left) ? f32_to_bf16_bits(v[q]) : (uint16_t)0;
}
template <>
__device__ __forceinline__ void store_w4<float>(float* o, float4 w, int left, bool vec) {
    if (vec && left >= 4) {
        *reinterpret_cast<float4*>(o) = w;
        return;
    }
    const float v[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) o[q] = (q < left) ? v[q] : 0.f;
}

// W rows r = s P + p (step s of the interval, chain p), entries 0 .. ld - 1 (zero from d on): grid (rows,
// column blocks), every thread draws four entries per Philox call and loops over the row.
template <typename OutT>
__global__ void gen_w_kernel(Key key, int64_t t0, int P, int d, int ld, OutT* __restrict__ out) {
    const int64_t r = blockIdx.x;
    const int s = (int)(r / P), p = (int)(r % P);
    const int64_t t = t0 + s;
    const bool vec = (ld % 4) == 0 && ((uintptr_t)out % 16) == 0;
    for (int j = blockIdx.y * blockDim.x + threadIdx.x; 4 * j < ld; j += gridDim.y * blockDim.x) {
        float4 w = make_float4(0.f, 0.f, 0.f, 0.f);
        if (4 * j < d) w = normals4(key, (uint32_t)j, t, (uint32_t)p);
        store_w4<OutT>(out + r * ld + 4 * j, w, d - 4 * j, vec);
    }
}

template <typename WT>
__device__ __forceinline__ float w_as_f32(WT v);
template <>
__device__ __forceinline__ float w_as_f32<uint16_t>(uint16_t v) { return bf16_bits_to_f32(v); }
template <>
__device__ __forceinline__ float w_as_f32<float>(float v) { return v; }

// ---------------------------------------------------------------------------------------------------
// Proposal of eq. (diamnl) for every chain, with the whitened state carried along:
//   x* = x_ref + rho (x - x_ref) + xi,   z* = rho z + beta alpha W,   q* = |z*|^2 / (2 alpha^2)
// (z = A_n^{-1}(x - x_ref) is exact in exact arithmetic: applying A_n^{-1} to the proposal gives the
// z recursion, so q* needs no triangular solve). The O(d) part of log pi(x*) is summed on the way.
// BF16 mode also writes x* as a two-term BF16 split (hi + lo) for the tensor-core target product.
// Grid (P, chunks): block (p, c) covers entries [c CHUNK, (c+1) CHUNK) of chain p and writes its partial
// sums of |z*|^2 and of the O(d) log-density terms to qpart[c P + p], lpart[c P + p].
constexpr int CHUNK = 1024;

template <typename T, typename WT>
__global__ void __launch_bounds__(256) propose_kernel(int d, int P, const T* __restrict__ X, const T* __restrict__ Z,
                                                      const T* __restrict__ Xi, const WT* __restrict__ W, int ldw,
                                                      const T* __restrict__ xref, T* __restrict__ Xp, T* __restrict__ Zp,
                                                      double* __restrict__ qpart, double* __restrict__ lpart,
                                                      const Ctl* ctl, TargetDev tg, uint16_t* __restrict__ op_hi,
                                                      uint16_t* __restrict__ op_lo, int ldk) {
    __shared__ double sh[32];
    __shared__ float shf[32];
    const int p = blockIdx.x, c = blockIdx.y;
    const int i0 = c * CHUNK, i1 = min(d, i0 + CHUNK);
    const T rho = (T)ctl->rho, ba = (T)ctl->ba;
    const F2 rho2 = split_f2(ctl->rho), ba2 = split_f2(ctl->ba);   // the FP32 updates' rho and beta alpha
    const size_t row = (size_t)ctl->s_cur * P + p;   // this step's row of the interval's noise buffers
    const T* x = X + (size_t)p * d;
    const T* z = Z + (size_t)p * d;
    const T* xi = Xi + row * d;
    const WT* w = W + row * ldw;
    T* xp = Xp + (size_t)p * d;
    T* zp = Zp + (size_t)p * d;
    double qacc = 0.0, lacc = 0.0;
    bool vec_done = false;
    if constexpr (std::is_same<T, float>::value && std::is_same<WT, uint16_t>::value) {
        // BF16 mode, d a multiple of 4: four entries per thread through 16-byte loads; the per-thread
        // partial sums of a handful of terms stay in FP32 (B300's FP64 rate is ~1/60 of its FP32 rate)
        if ((d & 3) == 0) {
            float qf = 0.f, lf = 0.f;
            const bool prior = tg.kind == TK_DIAG || tg.kind == TK_TANH || tg.kind == TK_BANANA;
            for (int i = i0 + 4 * threadIdx.x; i < i1; i += 4 * blockDim.x) {
                const float4 xr = *reinterpret_cast<const float4*>(xref + i);
                const float4 xv = *reinterpret_cast<const float4*>(x + i);
                const float4 zv = *reinterpret_cast<const float4*>(z + i);
                const float4 xiv = *reinterpret_cast<const float4*>(xi + i);
                const uint2 wb = *reinterpret_cast<const uint2*>(w + i);
                const float wv[4] = {bf16_bits_to_f32((uint16_t)(wb.x & 0xFFFFu)), bf16_bits_to_f32((uint16_t)(wb.x >> 16)),
                                     bf16_bits_to_f32((uint16_t)(wb.y & 0xFFFFu)), bf16_bits_to_f32((uint16_t)(wb.y >> 16))};
                const float xa[4] = {xv.x, xv.y, xv.z, xv.w}, ra[4] = {xr.x, xr.y, xr.z, xr.w};
                const float za[4] = {zv.x, zv.y, zv.z, zv.w}, ia[4] = {xiv.x, xiv.y, xiv.z, xiv.w};
                float vo[4], uo[4];
                uint16_t ho[4], lo[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    vo[k] = ra[k] + mul_f2(rho2, xa[k] - ra[k], ia[k]);
                    uo[k] = mul_f2(rho2, za[k], mul_f2(ba2, wv[k], 0.f));
                    qf += uo[k] * uo[k];
                    if (prior && (tg.kind != TK_BANANA || i + k >= 2)) lf -= 0.5f * vo[k] * vo[k] * tg.inv_lam32[i + k];
                    ho[k] = f32_to_bf16_bits(vo[k]);
                    lo[k] = f32_to_bf16_bits(vo[k] - bf16_bits_to_f32(ho[k]));
                }
                *reinterpret_cast<float4*>(xp + i) = make_float4(vo[0], vo[1], vo[2], vo[3]);
                *reinterpret_cast<float4*>(zp + i) = make_float4(uo[0], uo[1], uo[2], uo[3]);
                if (op_hi) {
                    *reinterpret_cast<uint2*>(op_hi + (size_t)p * ldk + i) =
                        make_uint2((uint32_t)ho[0] | ((uint32_t)ho[1] << 16), (uint32_t)ho[2] | ((uint32_t)ho[3] << 16));
                    *reinterpret_cast<uint2*>(op_lo + (size_t)p * ldk + i) =
                        make_uint2((uint32_t)lo[0] | ((uint32_t)lo[1] << 16), (uint32_t)lo[2] | ((uint32_t)lo[3] << 16));
                }
            }
            // block sums in FP32 too: FP64 adds run at about 1/64 of the FP32 rate on B300, and a tree of
            // 256 partial sums loses about 8 ulps of FP32 (relative 5e-7), far inside the BF16-mode bounds
            qf = block_sum(qf, shf);
            lf = block_sum(lf, shf);
            if (threadIdx.x == 0) {
                double la = (double)lf;
                if (tg.kind == TK_BANANA && c == 0) la += banana_head(tg, (double)xp[0], d > 1 ? (double)xp[1] : 0.0);
                qpart[(size_t)c * P + p] = (double)qf;
                lpart[(size_t)c * P + p] = la;
            }
            return;
        }
    }
    for (int i = i0 + threadIdx.x; !vec_done && i < i1; i += blockDim.x) {
        T xr = xref[i];
        T wz;
        if constexpr (sizeof(WT) == sizeof(T)) wz = (T)w[i];
        else wz = (T)w_as_f32<WT>(w[i]);
        T v, u;
        if constexpr (std::is_same<T, float>::value) {
            v = xr + mul_f2(rho2, x[i] - xr, xi[i]);
            u = mul_f2(rho2, z[i], mul_f2(ba2, wz, 0.f));
        } else {
            v = xr + rho * (x[i] - xr) + xi[i];
            u = rho * z[i] + ba * wz;
        }
        xp[i] = v;
        zp[i] = u;
        qacc += (double)u * (double)u;
        lacc += od_term<T>(tg, i, v);
        if (op_hi) {
            uint16_t h = f32_to_bf16_bits((float)v);
            float hv = bf16_bits_to_f32(h);
            op_hi[(size_t)p * ldk + i] = h;
            op_lo[(size_t)p * ldk + i] = f32_to_bf16_bits((float)v - hv);
        }
    }
    qacc = block_sum(qacc, sh);
    lacc = block_sum(lacc, sh);
    if (threadIdx.x == 0) {
        if (tg.kind == TK_BANANA && c == 0) lacc += banana_head(tg, (double)xp[0], d > 1 ? (double)xp[1] : 0.0);
        qpart[(size_t)c * P + p] = qacc;
        lpart[(size_t)c * P + p] = lacc;
    }
}

// O(d) part of log pi for any state buffer (initial state, imported state); BF16 operand planes if asked:
// x = hi + lo to 16 bits of x's mantissa, and with op_lo2 also lo2 = bf16(x - hi - lo), so hi + lo + lo2 = x
// exactly (FP32 x: 24 bits in three 8-bit pieces, each difference exact in FP32).
template <typename T>
__global__ void __launch_bounds__(256) od_terms_kernel(int d, const T* __restrict__ Xs, double* __restrict__ lpo,
                                                       TargetDev tg, uint16_t* __restrict__ op_hi,
                                                       uint16_t* __restrict__ op_lo, int ldk,
                                                       uint16_t* __restrict__ op_lo2 = nullptr) {
    __shared__ double sh[32];
    const int p = blockIdx.x;
    const T* x = Xs + (size_t)p * d;
    double lacc = 0.0;
    for (int i = threadIdx.x; i < d; i += blockDim.x) {
        T v = x[i];
        lacc += od_term<T>(tg, i, v);
        if (op_hi) {
            uint16_t h = f32_to_bf16_bits((float)v);
            op_hi[(size_t)p * ldk + i] = h;
            const float r = (float)v - bf16_bits_to_f32(h);
            const uint16_t l = f32_to_bf16_bits(r);
            op_lo[(size_t)p * ldk + i] = l;
            if (op_lo2) op_lo2[(size_t)p * ldk + i] = f32_to_bf16_bits(r - bf16_bits_to_f32(l));
        }
    }
    lacc = block_sum(lacc, sh);
    if (threadIdx.x == 0) {
        if (tg.kind == TK_BANANA) lacc += banana_head(tg, (double)x[0], d > 1 ? (double)x[1] : 0.0);
        lpo[p] = lacc;
    }
}

// The twisted Gaussians of Sec. 3.1 (pi_5, pi_6): from u = G x of chain p (row p of U, d_y entries),
// log pi = -1/2 sum_j (u_j + c_j u_{j-1}^2)^2 / lambda_j (c_0 = 0), summed in FP64 in a fixed order (per thread,
// then the block tree). One block per chain.
template <typename UT>
__global__ void __launch_bounds__(256) twisted_lp_kernel(int dy, const UT* __restrict__ U, int ldu,
                                                         const double* __restrict__ inv_lam, const double* __restrict__ cw,
                                                         double* __restrict__ out) {
    __shared__ double sh[32];
    const int p = blockIdx.x;
    const UT* u = U + (size_t)p * ldu;
    double acc = 0.0;
    for (int j = threadIdx.x; j < dy; j += blockDim.x) {
        const double uj = (double)u[j];
        const double ph = j > 0 ? uj + cw[j] * (double)u[j - 1] * (double)u[j - 1] : uj;
        acc += ph * ph * inv_lam[j];
    }
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) out[p] = -0.5 * acc;
}

// lp[p] = lpo[p] + sum over m-tiles of the linear-map partials (fixed order), or the external value.
__global__ void sum_lp_kernel(int P, const double* __restrict__ lpo, const double* __restrict__ partial, int nparts,
                              const double* __restrict__ ext, double* __restrict__ lp) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    double v;
    if (ext) {
        v = ext[p];
    } else {
        v = lpo[p];
        for (int m = 0; m < nparts; ++m) v += partial[(size_t)m * P + p];
    }
    lp[p] = v;
}

// ---------------------------------------------------------------------------------------------------
// Metropolis-Hastings test of Algorithm 1 (finish kernels) and the select / record step.
struct TraceDev {
    double *lp, *q, *qc, *loga;
    int8_t* acc;
    int64_t steps;
};

// Metropolis-Hastings test of Algorithm 1 for chain p, given log pi(x*) and q(x*):
//   log a = log pi(x*) + q(x*) - log pi(x) - q(x);  accept iff log u < log a, u = Philox uniform (tag U).
// Updates lp, q and the counters; records the decision for the select step and returns it.
__device__ __forceinline__ int decide(int p, int P, Key key, int64_t t, double lpp, double qpp, double* lp, double* q,
                                       int8_t* accf, Ctl* ctl, const TraceDev& tr) {
    const double lpc = lp[p], qc = q[p];
    const double loga = lpp - lpc + qpp - qc;
    const bool finite = isfinite(lpp) && isfinite(qpp);
    const double u = uniform53(key, t, (uint32_t)p, TAG_U);
    const int a = finite && (log(u) < loga);
    if (t < tr.steps) {
        size_t k = (size_t)t * P + p;
        tr.lp[k] = lpp; tr.q[k] = qpp; tr.qc[k] = qc; tr.loga[k] = loga; tr.acc[k] = (int8_t)a;
    }
    if (a) {
        lp[p] = lpp;
        q[p] = qpp;
        atomicAdd(&ctl->acc_block, 1ull);
    }
    if (!finite) atomicAdd(&ctl->nonfinite, 1ull);
    accf[p] = (int8_t)a;
    return a;
}

// One thread per chain: log pi(x*) = O(d) partials + linear-map partials (FP64 GEMM epilogue), or an
// externally evaluated value; q(x*) from the proposal's partials; then the decision.
__global__ void finish_kernel(int P, int nchunk, Key key, const double* __restrict__ qpart,
                              const double* __restrict__ lpart, const double* __restrict__ partial, int nparts,
                              const double* __restrict__ ext, double inv_infl2, double* lp, double* q, int8_t* accf,
                              Ctl* ctl, TraceDev tr) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    const int64_t t = ctl->t_cur;
    double lpp = 0.0, qs = 0.0;
    for (int c = 0; c < nchunk; ++c) qs += qpart[(size_t)c * P + p];
    if (ext) {
        lpp = ext[p];
    } else {
        for (int c = 0; c < nchunk; ++c) lpp += lpart[(size_t)c * P + p];
        for (int m = 0; m < nparts; ++m) lpp += partial[(size_t)m * P + p];
    }
    decide(p, P, key, t, lpp, 0.5 * qs * inv_infl2, lp, q, accf, ctl, tr);
}

// One block per chain, for a linear-map target computed as split-K FP32 partial products ws[s][p][m]
// (m < d_y): u_m = sum_s ws (fixed order), log-likelihood -(y_m - tanh u_m)^2 inv2s2 or -u_m^2 / 2, summed
// in FP32 (relative error ~1e-6 of the sum, inside the BF16-mode bounds); then the O(d) partials and q(x*)
// in FP64, and the decision.
__global__ void __launch_bounds__(256) finish_linear_kernel(int P, int dy, int nsplit, const float* __restrict__ ws,
                                                             const float* __restrict__ y32, float inv2s2, int tanh_mode,
                                                             int nchunk, Key key,
                                                             const double* __restrict__ qpart,
                                                             const double* __restrict__ lpart, double inv_infl2,
                                                             double* lp, double* q, int8_t* accf, Ctl* ctl,
                                                             TraceDev tr) {
    __shared__ float shf[32];
    const int p = blockIdx.x;
    const int64_t t = ctl->t_cur;
    const size_t plane = (size_t)P * dy;
    float accf32 = 0.f;
    for (int m = threadIdx.x; m < dy; m += blockDim.x) {
        float u = 0.f;
        for (int s = 0; s < nsplit; ++s) u += ws[s * plane + (size_t)p * dy + m];
        if (tanh_mode) {
            const float r = y32[m] - tanhf(u);
            accf32 -= r * r * inv2s2;
        } else {
            accf32 -= 0.5f * u * u;
        }
    }
    double acc = (double)block_sum(accf32, shf);
    if (threadIdx.x == 0) {
        double qs = 0.0;
        for (int c = 0; c < nchunk; ++c) {
            qs += qpart[(size_t)c * P + p];
            acc += lpart[(size_t)c * P + p];
        }
        decide(p, P, key, t, acc, 0.5 * qs * inv_infl2, lp, q, accf, ctl, tr);
    }
}

// Select / record, grid (P, chunks): x, z <- x*, z* for accepted chains; the post-step state (centred in FP64
// mode)
// x_{n+1} - c goes to the interval record (moment fold) and to the per-chain interval sums.
template <typename T, typename HT>
__device__ __forceinline__ HT to_hist(T v);
template <>
__device__ __forceinline__ double to_hist<double, double>(double v) { return v; }
template <>
__device__ __forceinline__ float to_hist<float, float>(float v) { return v; }

// Counters of the delayed-acceptance screen and of its ring buffer of exactly evaluated pairs.
struct DaCounters {
    unsigned long long tested, passed, exact;
    int count;           // survivors of the current step
    int pad;
    long long head, filled;   // ring buffer
};

// The ring head moves past this step's exactly evaluated pairs.
__device__ __forceinline__ void ring_advance_step(DaCounters* cnt, long long cap) {
    cnt->head = (cnt->head + cnt->count) % cap;
    cnt->filled = min(cap, cnt->filled + (long long)cnt->count);
}

template <typename T, typename HT>
__global__ void __launch_bounds__(256) select_kernel(int d, int P, int nl, Ctl* ctl, const int8_t* __restrict__ accf,
                                                     T* __restrict__ X, T* __restrict__ Z, const T* __restrict__ Xp,
                                                     const T* __restrict__ Zp, HT* __restrict__ hist_base, int ldh,
                                                     const T* __restrict__ cen, HT* __restrict__ bsum_base,
                                                     HT* __restrict__ bsq_base,
                                                     double* __restrict__ lpsum_base, const double* __restrict__ lp,
                                                     float* __restrict__ Ax, const float* __restrict__ Axp, int dy,
                                                     DaCounters* dacnt, long long ring_cap) {
    const int p = blockIdx.x, c = blockIdx.y;
    const long long blk = ctl->t_cur / nl;
    HT* hist = hist_base ? hist_base + (size_t)ctl->s_cur * P * ldh : nullptr;
    HT* bsum = bsum_base ? bsum_base + (size_t)blk * P * d : nullptr;
    HT* bsq = bsq_base ? bsq_base + (size_t)blk * P * d : nullptr;   // per-chain interval sums of x^2
    double* lpsum = lpsum_base ? lpsum_base + (size_t)blk * P : nullptr;
    const int i0 = c * CHUNK, i1 = min(d, i0 + CHUNK);
    const int a = accf[p];
    T* x = X + (size_t)p * d;
    T* z = Z + (size_t)p * d;
    const T* xp = Xp + (size_t)p * d;
    const T* zp = Zp + (size_t)p * d;
    HT* h = hist ? hist + (size_t)p * ldh : nullptr;
    HT* bs = bsum ? bsum + (size_t)p * d : nullptr;
    HT* bq = bsq ? bsq + (size_t)p * d : nullptr;
    bool vec_done = false;
    if constexpr (std::is_same<T, float>::value && std::is_same<HT, float>::value) {
        if ((d & 3) == 0 && (ldh & 3) == 0 && h) {
            for (int i = i0 + 4 * threadIdx.x; i < i1; i += 4 * blockDim.x) {
                float4 v = a ? *reinterpret_cast<const float4*>(xp + i) : *reinterpret_cast<const float4*>(x + i);
                if (a) {
                    *reinterpret_cast<float4*>(x + i) = v;
                    *reinterpret_cast<float4*>(z + i) = *reinterpret_cast<const float4*>(zp + i);
                }
                *reinterpret_cast<float4*>(h + i) = v;   // BF16 mode: the fold subtracts the centre
                if (bs) {   // BF16 mode keeps the per-chain interval sums in FP32 (128-step sums, ~1e-5 relative)
                    float4 b = *reinterpret_cast<float4*>(bs + i);
                    *reinterpret_cast<float4*>(bs + i) = make_float4(b.x + v.x, b.y + v.y, b.z + v.z, b.w + v.w);
                }
            }
            vec_done = true;
        }
    }
    for (int i = i0 + threadIdx.x; !vec_done && i < i1; i += blockDim.x) {
        T v = a ? xp[i] : x[i];
        if (a) {
            x[i] = v;
            z[i] = zp[i];
        }
        if (h) {   // FP64 mode records x - c; BF16 mode records x (its fold subtracts c in FP32)
            if constexpr (std::is_same<HT, float>::value) h[i] = (float)v;
            else h[i] = to_hist<T, HT>(v - cen[i]);
        }
        if (bs) bs[i] += (HT)v;
        if (bq) bq[i] += (HT)v * (HT)v;
    }
    if (Ax && a) {   // the carried map: accepted chains take A x*, block c its share of the row
        const int per = (dy + gridDim.y - 1) / gridDim.y;
        for (int m = c * per + threadIdx.x; m < min(dy, (c + 1) * per); m += blockDim.x)
            Ax[(size_t)p * dy + m] = Axp[(size_t)p * dy + m];
    }
    if (lpsum && c == 0 && threadIdx.x == 0) lpsum[p] += lp[p];
    // the last block of the step moves the step counters (and the ring head) on
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&ctl->done_blocks, 1u) == gridDim.x * gridDim.y - 1) {
            if (dacnt) ring_advance_step(dacnt, ring_cap);
            ctl->t_cur += 1;
            ctl->s_cur += 1;
            ctl->done_blocks = 0;
        }
    }
}

// The test of Algorithm 1 in the fused kernels, from the block's FP32 sums. Absolute sums (|z*|^2, the prior
// terms, the likelihood terms of the map) give log pi(x*) = prior + likelihood and q* = |z*|^2 / (2 alpha^2), the
// values kept for x* when it is accepted. log a = (log pi(x*) - log pi(x)) + (q* - q(x)) is formed from the sums
// of the per-coordinate differences instead (dq = sum (z*_i - z_i)(z*_i + z_i), the prior's and the likelihood's
// differences likewise): each difference term is of the size of the move, so the FP32 sums carry rounding of
// the size of log a's terms rather than of |log pi| (about 3e3 at d = 4096, where absolute FP32 sums lose
// 1e-3 nats). The same quantity in exact arithmetic. log u < log a is decided as in FP64: the FP32 log of u
// (within 1e-5 of log u: u's rounding to FP32 and a few ulps of logf, |log u| <= 37) decides unless log a lies
// within 1e-4 of it; then the FP64 log does. Writes the trace entry of (t, p) when it is kept.
__device__ __forceinline__ int rec_test(float sm, float dsq, float dsl, float dsm, double dextra, double inv_infl2,
                                        double lpc, double qc, double u, float lu32, long long t, int p, int P,
                                        const TraceDev& tr, double& lmap, double& lpp, double& qpp, bool& finite) {
    lmap = (double)sm;
    const double dlp = ((double)dsl + (double)dsm) + dextra, dq = 0.5 * (double)dsq * inv_infl2;
    lpp = lpc + dlp;   // the proposal's values carried from the current state's by the differences
    qpp = qc + dq;
    const double loga = dlp + dq;
    finite = isfinite(lpp) && isfinite(qpp) && isfinite(loga);
    const double l32 = (double)lu32;
    int a = 0;
    if (finite) a = loga > l32 + 1e-4 ? 1 : loga < l32 - 1e-4 ? 0 : (log(u) < loga);
    if (t < tr.steps) {
        const size_t k = (size_t)t * P + p;
        tr.lp[k] = lpp; tr.q[k] = qpp; tr.qc[k] = qc; tr.loga[k] = loga; tr.acc[k] = (int8_t)a;
    }
    return a;
}

// ---------------------------------------------------------------------------------------------------
// One whole step of every chain in one launch, for a target whose expensive term is a linear map carried
// through the proposal (BF16 mode; no surrogate screen in force). Block p holds chain p's proposal from the
// draw to the record:
//   x* = x_ref + rho (x - x_ref) + xi,  z* = rho z + beta alpha W   (eq. (diamnl), z-recursion)
//   u  = rho (A x) + (1 - rho) (A x_ref) + A xi                     (the map of x*, A xi from the interval GEMM)
//   log pi(x*) = prior terms of x* + likelihood terms of u,  q* = |z*|^2 / (2 alpha^2)
// then the Metropolis-Hastings test of Algorithm 1, x, z, A x <- x*, z*, u when accepted, the record row (the
// post-step state; the fold centres it), the log pi sums and, with a surrogate attached, the (bf16(x*),
// likelihood terms) training pair in
// ring slot head + p. The last block to finish moves the step counters (and the ring head) on.
// Only x*, u and W stay in registers across the test; the second pass reads x (rejected) or z (accepted, z*
// recomputed by the same fused multiply-add) again, from the staged rows (or L2), and issues no other load.
// Sums are FP32, one tree per block.
// Element layout of thread tid: VEC (d, d_y multiples of 4): entries 4 (tid + g FT) + j of group g < NV (NM);
// otherwise entries tid + (4 g + j) FT. So d <= 4 NV FT and d_y <= 4 NM FT.
// STAGE (with VEC): the chain's x, z and xi rows (12 d bytes of dynamic shared memory) arrive by three bulk
// copies issued at the start, so the whole row is requested at once; the map terms are computed while they
// are in flight, and the second pass reads x or z from shared memory. The copy wait is clock-bounded.
constexpr int FUSED_THREADS = 256;

// Resident blocks per SM the fused kernels are compiled for: four (64 registers a thread) while a chain's vectors
// fit the small instances; two (128 registers) for the instances with eight element groups per thread (d or d_y
// past 4096), whose shared memory allows at most two or three blocks per SM anyway and whose register arrays would
// otherwise spill.
constexpr int fused_min_blocks(int nv, int nm) { return (nv >= 8 || nm >= 8) ? 2 : 4; }

template <int NV, int NM, bool VEC, bool STAGE = false>
__global__ void __launch_bounds__(FUSED_THREADS, fused_min_blocks(NV, NM)) step_rec_kernel(
    int d, int P, int nl, int dy, Ctl* ctl, Key key, TargetDev tg, double inv_infl2,
    float* __restrict__ X, float* __restrict__ Z, const float* __restrict__ Xi, const uint16_t* __restrict__ W, int ldw,
    const float* __restrict__ xref, float* __restrict__ Ax,
    const float* __restrict__ axref, const float* __restrict__ AXi, const float* __restrict__ y32, float inv2s2,
    int tanh_mode, double* lp, double* q, int8_t* accf, TraceDev tr, float* __restrict__ hist_base, int ldh,
    float* __restrict__ bsum_base, double* __restrict__ lpsum_base, DaCounters* dacnt, uint16_t* __restrict__ ring_x,
    float* __restrict__ ring_lp, long long ring_cap, int ldk) {
    static_assert(!STAGE || VEC, "staging reads 16-byte vectors");
    constexpr int FT = FUSED_THREADS;
    extern __shared__ float4 stage_smem[];   // STAGE: x, z, xi of the chain (d floats each)
    __shared__ float red[4][FT / 32];
    __shared__ double s_u, s_lpc, s_qc;
    __shared__ float s_lu32;
    __shared__ int s_acc;
    __shared__ uint64_t s_bar;
    const int p = blockIdx.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const F2 rho = split_f2(ctl->rho), ba = split_f2(ctl->ba);
    const float om = (float)(1.0 - ctl->rho);
    const int s = ctl->s_cur;
    const long long t = ctl->t_cur;
    const size_t row = (size_t)s * P + p;
    float* x = X + (size_t)p * d;
    float* z = Z + (size_t)p * d;
    const float* xi = Xi + row * d;
    const uint16_t* w = W + row * ldw;
    float* sx = reinterpret_cast<float*>(stage_smem);
    float* sz = sx + d;
    float* sxi = sz + d;
    if (STAGE) {
        if (tid == 0) {
            mbar_init(smem_u32(&s_bar), 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        }
        __syncthreads();
        if (tid == 0) {
            const uint32_t bar = smem_u32(&s_bar), bytes = (uint32_t)d * 4u;
            mbar_expect_tx(bar, 3u * bytes);
            bulk_load_1d(smem_u32(sx), x, bytes, bar);
            bulk_load_1d(smem_u32(sz), z, bytes, bar);
            bulk_load_1d(smem_u32(sxi), xi, bytes, bar);
        }
    }
    const float* xsrc = STAGE ? sx : x;
    const float* zsrc = STAGE ? sz : z;
    const float* isrc = STAGE ? sxi : xi;
    // the O(d) terms: the tanh regression's prior, the diagonal Gaussian, the banana's coordinates past its head
    // (their 1 / lambda are zero at 0 and 1); the dense Gaussian's whole density is its map
    const bool prior = tg.kind == TK_TANH || tg.kind == TK_DIAG || tg.kind == TK_BANANA;
    auto idx = [&](int g, int j) { return VEC ? 4 * (tid + g * FT) + j : tid + (4 * g + j) * FT; };
    if (tid == FT - 32) {   // the test's other inputs, off the path of the sums: u, its FP32 log, log pi(x), q(x)
        const double u = uniform53(key, t, (uint32_t)p, TAG_U);
        s_u = u;
        s_lu32 = logf((float)u);
        s_lpc = lp[p];
        s_qc = q[p];
    }
    // differences of q, of the prior terms and of the map terms (rec_test); the map terms of x* themselves only
    // for the surrogate's ring
    float mf = 0.f, dqf = 0.f, dlf = 0.f, dmf = 0.f;
    const bool want_map = ring_x != nullptr;
    // the map of x* and its likelihood terms first (they need none of the chain's d-vectors)
    float uv[4 * NM];
    const float* ax = Ax + (size_t)p * dy;
    const float* axi = AXi + row * dy;
    // u = (A x*)_m, uc = (A x)_m: the term of x* and its difference from x's
    auto map_term = [&](float u, float uc, float yv) {
        if (tanh_mode) {
            const float tn = tanhf(u), tc = tanhf(uc);
            if (want_map) {
                const float r = yv - tn;
                mf -= r * r * inv2s2;
            }
            dmf -= (tc - tn) * (2.f * yv - tn - tc) * inv2s2;
        } else {
            if (want_map) mf -= 0.5f * u * u;
            dmf -= 0.5f * (u - uc) * (u + uc);
        }
    };
#pragma unroll
    for (int g = 0; g < NM; ++g) {
        if (VEC) {
            const int m = idx(g, 0);
            if (m < dy) {
                const float4 a4 = *reinterpret_cast<const float4*>(ax + m);
                const float4 r4 = *reinterpret_cast<const float4*>(axref + m);
                const float4 i4 = *reinterpret_cast<const float4*>(axi + m);
                const float4 y4 = tanh_mode ? *reinterpret_cast<const float4*>(y32 + m) : make_float4(0.f, 0.f, 0.f, 0.f);
                uv[4 * g] = mul_f2(rho, a4.x, fmaf(om, r4.x, i4.x));
                uv[4 * g + 1] = mul_f2(rho, a4.y, fmaf(om, r4.y, i4.y));
                uv[4 * g + 2] = mul_f2(rho, a4.z, fmaf(om, r4.z, i4.z));
                uv[4 * g + 3] = mul_f2(rho, a4.w, fmaf(om, r4.w, i4.w));
                map_term(uv[4 * g], a4.x, y4.x);
                map_term(uv[4 * g + 1], a4.y, y4.y);
                map_term(uv[4 * g + 2], a4.z, y4.z);
                map_term(uv[4 * g + 3], a4.w, y4.w);
            }
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int m = idx(g, j);
                if (m < dy) {
                    uv[4 * g + j] = mul_f2(rho, ax[m], fmaf(om, axref[m], axi[m]));
                    map_term(uv[4 * g + j], ax[m], tanh_mode ? y32[m] : 0.f);
                }
            }
        }
    }
    if (STAGE) {   // every thread waits for the staged rows (bounded; on expiry the step is abandoned)
        const uint32_t bar = smem_u32(&s_bar);
        long long t0 = clock64();
        bool ok = true;
        while (!mbar_try(bar, 0)) {
            if (clock64() - t0 > TC_WAIT_CYCLES) {
                ok = false;
                break;
            }
        }
        if (!ok) {
            if (tid == 0) set_status(&ctl->status, DEV_TIMEOUT);
            t0 = clock64();   // the copies still in flight target this CTA's shared memory: wait for them
            while (!mbar_try(bar, 0) && clock64() - t0 < TC_WAIT_CYCLES) {
            }
            return;
        }
    }

    float xs[4 * NV];
    uint2 wreg[NV];   // VEC: this thread's W, kept for z* of an accepted chain
#pragma unroll
    for (int g = 0; g < NV; ++g) {
        if (VEC) {
            const int i = idx(g, 0);
            wreg[g] = make_uint2(0u, 0u);
            if (i < d) {
                const float4 xr = *reinterpret_cast<const float4*>(xref + i);
                const float4 xa = *reinterpret_cast<const float4*>(xsrc + i);
                const float4 za = *reinterpret_cast<const float4*>(zsrc + i);
                const float4 ia = *reinterpret_cast<const float4*>(isrc + i);
                const uint2 wb = *reinterpret_cast<const uint2*>(w + i);
                wreg[g] = wb;
                const float r4[4] = {xr.x, xr.y, xr.z, xr.w}, x4[4] = {xa.x, xa.y, xa.z, xa.w};
                const float z4[4] = {za.x, za.y, za.z, za.w}, i4[4] = {ia.x, ia.y, ia.z, ia.w};
                const float w4[4] = {bf16_bits_to_f32((uint16_t)(wb.x & 0xFFFFu)), bf16_bits_to_f32((uint16_t)(wb.x >> 16)),
                                     bf16_bits_to_f32((uint16_t)(wb.y & 0xFFFFu)), bf16_bits_to_f32((uint16_t)(wb.y >> 16))};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float xv = xs[4 * g + j] = r4[j] + mul_f2(rho, x4[j] - r4[j], i4[j]);
                    const float zs = mul_f2(rho, z4[j], mul_f2(ba, w4[j], 0.f));
                    dqf += (zs - z4[j]) * (zs + z4[j]);
                    if (prior) dlf -= 0.5f * (xv - x4[j]) * (xv + x4[j]) * tg.inv_lam32[i + j];
                }
            }
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int i = idx(g, j);
                if (i < d) {
                    const float xr = xref[i], xc = x[i], zc = z[i];
                    const float xv = xs[4 * g + j] = xr + mul_f2(rho, xc - xr, xi[i]);
                    const float zs = mul_f2(rho, zc, mul_f2(ba, bf16_bits_to_f32(w[i]), 0.f));
                    dqf += (zs - zc) * (zs + zc);
                    if (prior) dlf -= 0.5f * (xv - xc) * (xv + xc) * tg.inv_lam32[i];
                }
            }
        }
    }
    // the four sums over the block, then the test (Algorithm 1) in thread 0
    mf = warp_sum(mf);
    dqf = warp_sum(dqf);
    dlf = warp_sum(dlf);
    dmf = warp_sum(dmf);
    if (lane == 0) {
        red[0][wid] = mf;
        red[1][wid] = dqf;
        red[2][wid] = dlf;
        red[3][wid] = dmf;
    }
    __syncthreads();
    if (wid == 0) {
        float sum4[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) sum4[k] = warp_sum(lane < FT / 32 ? red[k][lane] : 0.f);
        if (lane == 0) {
            double lmap, lpp, qpp;
            bool finite;
            // the banana's head (coordinates 0 and 1, both this thread's in the 16-byte layout) in FP64
            const double dhead = tg.kind == TK_BANANA
                                     ? banana_head(tg, (double)xs[0], (double)xs[1]) - banana_head(tg, (double)xsrc[0], (double)xsrc[1])
                                     : 0.0;
            const int a = rec_test(sum4[0], sum4[1], sum4[2], sum4[3], dhead, inv_infl2, s_lpc, s_qc, s_u, s_lu32, t, p, P,
                                   tr, lmap, lpp, qpp, finite);
            if (a) {
                lp[p] = lpp;
                q[p] = qpp;
                atomicAdd(&ctl->acc_block, 1ull);
            }
            if (!finite) atomicAdd(&ctl->nonfinite, 1ull);
            accf[p] = (int8_t)a;
            s_acc = a;
            if (ring_x) ring_lp[(dacnt->head + p) % ring_cap] = (float)lmap;
            if (lpsum_base) lpsum_base[(size_t)(t / nl) * P + p] += a ? lpp : s_lpc;
        }
    }
    __syncthreads();
    const int a = s_acc;
    float* h = hist_base ? hist_base + row * ldh : nullptr;
    float* bs = bsum_base ? bsum_base + ((size_t)(t / nl) * P + p) * d : nullptr;
    uint16_t* rx = ring_x ? ring_x + (size_t)((dacnt->head + p) % ring_cap) * ldk : nullptr;
#pragma unroll
    for (int g = 0; g < NV; ++g) {
        if (VEC) {
            const int i = idx(g, 0);
            if (i < d) {
                float v[4];
                if (a) {
                    const float4 za = *reinterpret_cast<const float4*>(zsrc + i);
                    const uint2 wb = wreg[g];
                    const float z4[4] = {za.x, za.y, za.z, za.w};
                    const float w4[4] = {bf16_bits_to_f32((uint16_t)(wb.x & 0xFFFFu)), bf16_bits_to_f32((uint16_t)(wb.x >> 16)),
                                         bf16_bits_to_f32((uint16_t)(wb.y & 0xFFFFu)), bf16_bits_to_f32((uint16_t)(wb.y >> 16))};
                    float zn[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        v[j] = xs[4 * g + j];
                        zn[j] = mul_f2(rho, z4[j], mul_f2(ba, w4[j], 0.f));
                    }
                    *reinterpret_cast<float4*>(x + i) = make_float4(v[0], v[1], v[2], v[3]);
                    *reinterpret_cast<float4*>(z + i) = make_float4(zn[0], zn[1], zn[2], zn[3]);
                } else {
                    const float4 xa = *reinterpret_cast<const float4*>(xsrc + i);
                    v[0] = xa.x; v[1] = xa.y; v[2] = xa.z; v[3] = xa.w;
                }
                if (h) *reinterpret_cast<float4*>(h + i) = make_float4(v[0], v[1], v[2], v[3]);
                if (bs) {
                    const float4 b = *reinterpret_cast<const float4*>(bs + i);
                    *reinterpret_cast<float4*>(bs + i) = make_float4(b.x + v[0], b.y + v[1], b.z + v[2], b.w + v[3]);
                }
                if (rx) {
                    const uint32_t lo = (uint32_t)f32_to_bf16_bits(xs[4 * g]) | ((uint32_t)f32_to_bf16_bits(xs[4 * g + 1]) << 16);
                    const uint32_t hi = (uint32_t)f32_to_bf16_bits(xs[4 * g + 2]) | ((uint32_t)f32_to_bf16_bits(xs[4 * g + 3]) << 16);
                    *reinterpret_cast<uint2*>(rx + i) = make_uint2(lo, hi);
                }
            }
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int i = idx(g, j);
                if (i < d) {
                    float v;
                    if (a) {
                        v = xs[4 * g + j];
                        x[i] = v;
                        z[i] = mul_f2(rho, z[i], mul_f2(ba, bf16_bits_to_f32(w[i]), 0.f));
                    } else {
                        v = x[i];
                    }
                    if (h) h[i] = v;
                    if (bs) bs[i] += v;
                    if (rx) rx[i] = f32_to_bf16_bits(xs[4 * g + j]);
                }
            }
        }
    }
    if (rx)   // the row's padding stays zero (the network's input width is ldk)
        for (int i = d + tid; i < ldk; i += FT) rx[i] = 0;
    if (a) {
        float* axw = Ax + (size_t)p * dy;
#pragma unroll
        for (int g = 0; g < NM; ++g) {
            if (VEC) {
                const int m = idx(g, 0);
                if (m < dy) *reinterpret_cast<float4*>(axw + m) = make_float4(uv[4 * g], uv[4 * g + 1], uv[4 * g + 2], uv[4 * g + 3]);
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int m = idx(g, j);
                    if (m < dy) axw[m] = uv[4 * g + j];
                }
            }
        }
    }
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        if (atomicAdd(&ctl->done_blocks, 1u) == gridDim.x - 1) {
            if (dacnt) {   // every proposal was evaluated exactly and went to the ring
                dacnt->count = P;
                dacnt->exact += (unsigned long long)P;
                ring_advance_step(dacnt, ring_cap);
            }
            ctl->t_cur += 1;
            ctl->s_cur += 1;
            ctl->done_blocks = 0;
        }
    }
}

// ---------------------------------------------------------------------------------------------------
// ns consecutive steps of chain p in one block (the steps of step_rec_kernel, in the same arithmetic). Within
// an interval the chains share nothing that changes: the factor, x_ref, rho, beta alpha and the interval's
// noise W, its product xi and the map of xi are fixed before the first step (Algorithm 1 changes the factor
// only between intervals). So each block walks its chain through the steps on its own, x, z and A x held in
// shared memory throughout: per step it reads the chain's xi, W and A xi rows and writes the record row (and
// the ring row); the state, log pi and q go back to memory after the last step, and the last block to finish
// moves the counters on by ns. No block waits on another, so the blocks drift apart and the loads of some
// overlap the reductions and tests of others. The caller keeps steps s0 .. s0 + ns - 1 inside one interval.
// VEC layout (entries 4 (tid + g FT) + j); dynamic shared memory (2 d + 2 d_y) floats: x, z, A x and, for the tanh
// regression, tanh(A x) (the current state's terms in log a's likelihood difference). pf_l2 (rows
// 16-byte aligned): thread 0 asks for the next step's xi, W and A xi rows to be brought into L2 at the start
// of each step, so the HBM reads of a step overlap the previous step's reductions, test and stores.
template <int NV, int NM>
__global__ void __launch_bounds__(FUSED_THREADS, fused_min_blocks(NV, NM)) interval_rec_kernel(
    int d, int P, int nl, int dy, int ns, Ctl* ctl, Key key, TargetDev tg, double inv_infl2,
    float* __restrict__ X, float* __restrict__ Z, const float* __restrict__ Xi, const uint16_t* __restrict__ W, int ldw,
    const float* __restrict__ xref, float* __restrict__ Ax, const float* __restrict__ axref,
    const float* __restrict__ AXi, const float* __restrict__ y32, float inv2s2, int tanh_mode, double* lp, double* q,
    int8_t* accf, TraceDev tr, float* __restrict__ hist_base, int ldh, double* __restrict__ lpsum_base,
    DaCounters* dacnt, uint16_t* __restrict__ ring_x, float* __restrict__ ring_lp, long long ring_cap, int ldk,
    int pf_l2) {
    constexpr int FT = FUSED_THREADS;
    extern __shared__ float4 ival_smem[];
    __shared__ float red[4][FT / 32];
    __shared__ double s_u;
    __shared__ float s_lu32;
    __shared__ int s_acc;
    const int p = blockIdx.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const F2 rho = split_f2(ctl->rho), ba = split_f2(ctl->ba);
    const float om = (float)(1.0 - ctl->rho);
    const int s0 = ctl->s_cur;
    const long long t0 = ctl->t_cur;
    const long long head0 = dacnt ? dacnt->head : 0;
    float* sx = reinterpret_cast<float*>(ival_smem);
    float* sz = sx + d;
    float* su = sz + d;
    float* st = su + dy;   // tanh of su (tanh mode)
    const bool prior = tg.kind == TK_TANH || tg.kind == TK_DIAG || tg.kind == TK_BANANA;   // as step_rec_kernel
    auto idx = [&](int g) { return 4 * (tid + g * FT); };
    // the chain's state: every thread loads (and later stores) only its own entries, so no barrier is needed
#pragma unroll
    for (int g = 0; g < NV; ++g) {
        const int i = idx(g);
        if (i < d) {
            *reinterpret_cast<float4*>(sx + i) = *reinterpret_cast<const float4*>(X + (size_t)p * d + i);
            *reinterpret_cast<float4*>(sz + i) = *reinterpret_cast<const float4*>(Z + (size_t)p * d + i);
        }
    }
#pragma unroll
    for (int g = 0; g < NM; ++g) {
        const int m = idx(g);
        if (m < dy) {
            const float4 a4 = *reinterpret_cast<const float4*>(Ax + (size_t)p * dy + m);
            *reinterpret_cast<float4*>(su + m) = a4;
            if (tanh_mode) *reinterpret_cast<float4*>(st + m) = make_float4(tanhf(a4.x), tanhf(a4.y), tanhf(a4.z), tanhf(a4.w));
        }
    }
    // thread 0 carries log pi(x), q(x), the interval's log pi sum and the counts from step to step (in shared
    // memory: registers of every thread would hold them otherwise)
    __shared__ double lpc, qc, lps;
    __shared__ unsigned long long nacc, nnf;
    __shared__ int a_last;
    const size_t lps_at = (size_t)(t0 / nl) * P + p;
    if (tid == 0) {
        lpc = lp[p];
        qc = q[p];
        lps = lpsum_base ? lpsum_base[lps_at] : 0.0;
        nacc = 0;
        nnf = 0;
        a_last = 0;
    }
    // u = (A x*)_m; uc = (A x)_m and tc = tanh(uc) of the current state: the term of x* and its difference
    const bool want_map = ring_x != nullptr;   // the map terms of x* themselves: only for the surrogate's ring
    auto map_term = [&](float u, float uc, float tc, float yv, float& tn, float& mf, float& dmf) {
        if (tanh_mode) {
            tn = tanhf(u);
            if (want_map) {
                const float r = yv - tn;
                mf -= r * r * inv2s2;
            }
            dmf -= (tc - tn) * (2.f * yv - tn - tc) * inv2s2;
        } else {
            if (want_map) mf -= 0.5f * u * u;
            dmf -= 0.5f * (u - uc) * (u + uc);
        }
    };
    for (int k = 0; k < ns; ++k) {
        const int s = s0 + k;
        const long long t = t0 + k;
        const size_t row = (size_t)s * P + p;
        const float* xi = Xi + row * d;
        const uint16_t* w = W + row * ldw;
        const float* axi = AXi + row * dy;
        if (tid == FT - 32) {   // u and its FP32 log, off the path of the sums
            const double u = uniform53(key, t, (uint32_t)p, TAG_U);
            s_u = u;
            s_lu32 = logf((float)u);
        }
        if (pf_l2 && tid == 0 && k + 1 < ns) {   // the next step's rows into L2 while this step runs
            const size_t rn = row + (size_t)P;
            l2_prefetch(Xi + rn * d, (uint32_t)d * 4u);
            l2_prefetch(W + rn * ldw, (uint32_t)ldw * 2u);
            l2_prefetch(AXi + rn * dy, (uint32_t)dy * 4u);
        }
        float mf = 0.f, dqf = 0.f, dlf = 0.f, dmf = 0.f;   // the map terms of x* (ring only); differences
        float uv[4 * NM], tnv[4 * NM];   // u = (A x*)_m and, tanh mode, tanh(u) (kept for an accepted step)
#pragma unroll
        for (int g = 0; g < NM; ++g) {
            const int m = idx(g);
            if (m < dy) {
                const float4 a4 = *reinterpret_cast<const float4*>(su + m);
                const float4 r4 = *reinterpret_cast<const float4*>(axref + m);
                const float4 i4 = *reinterpret_cast<const float4*>(axi + m);
                const float4 y4 = tanh_mode ? *reinterpret_cast<const float4*>(y32 + m) : make_float4(0.f, 0.f, 0.f, 0.f);
                const float4 t4 = tanh_mode ? *reinterpret_cast<const float4*>(st + m) : make_float4(0.f, 0.f, 0.f, 0.f);
                uv[4 * g] = mul_f2(rho, a4.x, fmaf(om, r4.x, i4.x));
                uv[4 * g + 1] = mul_f2(rho, a4.y, fmaf(om, r4.y, i4.y));
                uv[4 * g + 2] = mul_f2(rho, a4.z, fmaf(om, r4.z, i4.z));
                uv[4 * g + 3] = mul_f2(rho, a4.w, fmaf(om, r4.w, i4.w));
                map_term(uv[4 * g], a4.x, t4.x, y4.x, tnv[4 * g], mf, dmf);
                map_term(uv[4 * g + 1], a4.y, t4.y, y4.y, tnv[4 * g + 1], mf, dmf);
                map_term(uv[4 * g + 2], a4.z, t4.z, y4.z, tnv[4 * g + 2], mf, dmf);
                map_term(uv[4 * g + 3], a4.w, t4.w, y4.w, tnv[4 * g + 3], mf, dmf);
            }
        }
        float xs[4 * NV];
        uint2 wreg[NV];
#pragma unroll
        for (int g = 0; g < NV; ++g) {
            const int i = idx(g);
            wreg[g] = make_uint2(0u, 0u);
            if (i < d) {
                const float4 xr = *reinterpret_cast<const float4*>(xref + i);
                const float4 xa = *reinterpret_cast<const float4*>(sx + i);
                const float4 za = *reinterpret_cast<const float4*>(sz + i);
                const float4 ia = *reinterpret_cast<const float4*>(xi + i);
                const uint2 wb = *reinterpret_cast<const uint2*>(w + i);
                wreg[g] = wb;
                const float r4[4] = {xr.x, xr.y, xr.z, xr.w}, x4[4] = {xa.x, xa.y, xa.z, xa.w};
                const float z4[4] = {za.x, za.y, za.z, za.w}, i4[4] = {ia.x, ia.y, ia.z, ia.w};
                const float w4[4] = {bf16_bits_to_f32((uint16_t)(wb.x & 0xFFFFu)), bf16_bits_to_f32((uint16_t)(wb.x >> 16)),
                                     bf16_bits_to_f32((uint16_t)(wb.y & 0xFFFFu)), bf16_bits_to_f32((uint16_t)(wb.y >> 16))};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const float xv = xs[4 * g + j] = r4[j] + mul_f2(rho, x4[j] - r4[j], i4[j]);
                    const float zs = mul_f2(rho, z4[j], mul_f2(ba, w4[j], 0.f));
                    dqf += (zs - z4[j]) * (zs + z4[j]);
                    if (prior) dlf -= 0.5f * (xv - x4[j]) * (xv + x4[j]) * tg.inv_lam32[i + j];
                }
            }
        }
        mf = warp_sum(mf);
        dqf = warp_sum(dqf);
        dlf = warp_sum(dlf);
        dmf = warp_sum(dmf);
        if (lane == 0) {
            red[0][wid] = mf;
            red[1][wid] = dqf;
            red[2][wid] = dlf;
            red[3][wid] = dmf;
        }
        __syncthreads();
        if (wid == 0) {
            float sum4[4];
#pragma unroll
            for (int k2 = 0; k2 < 4; ++k2) sum4[k2] = warp_sum(lane < FT / 32 ? red[k2][lane] : 0.f);
            if (lane == 0) {
                double lmap, lpp, qpp;
                bool finite;
                const double dhead = tg.kind == TK_BANANA   // the banana's head (coordinates 0 and 1: this thread's)
                                         ? banana_head(tg, (double)xs[0], (double)xs[1]) - banana_head(tg, (double)sx[0], (double)sx[1])
                                         : 0.0;
                const int a = rec_test(sum4[0], sum4[1], sum4[2], sum4[3], dhead, inv_infl2, lpc, qc, s_u, s_lu32, t, p, P,
                                       tr, lmap, lpp, qpp, finite);
                if (a) {
                    lpc = lpp;
                    qc = qpp;
                    ++nacc;
                }
                if (!finite) ++nnf;
                if (ring_x) ring_lp[(head0 + (long long)k * P + p) % ring_cap] = (float)lmap;
                lps += lpc;   // log pi after the step: log pi(x*) if accepted, else log pi(x)
                s_acc = a;
                a_last = a;
            }
        }
        __syncthreads();
        const int a = s_acc;
        float* h = hist_base ? hist_base + row * ldh : nullptr;
        uint16_t* rx = ring_x ? ring_x + (size_t)((head0 + (long long)k * P + p) % ring_cap) * ldk : nullptr;
#pragma unroll
        for (int g = 0; g < NV; ++g) {
            const int i = idx(g);
            if (i < d) {
                float v[4];
                if (a) {
                    const float4 za = *reinterpret_cast<const float4*>(sz + i);
                    const uint2 wb = wreg[g];
                    const float z4[4] = {za.x, za.y, za.z, za.w};
                    const float w4[4] = {bf16_bits_to_f32((uint16_t)(wb.x & 0xFFFFu)), bf16_bits_to_f32((uint16_t)(wb.x >> 16)),
                                         bf16_bits_to_f32((uint16_t)(wb.y & 0xFFFFu)), bf16_bits_to_f32((uint16_t)(wb.y >> 16))};
                    float zn[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        v[j] = xs[4 * g + j];
                        zn[j] = mul_f2(rho, z4[j], mul_f2(ba, w4[j], 0.f));
                    }
                    *reinterpret_cast<float4*>(sx + i) = make_float4(v[0], v[1], v[2], v[3]);
                    *reinterpret_cast<float4*>(sz + i) = make_float4(zn[0], zn[1], zn[2], zn[3]);
                } else {
                    const float4 xa = *reinterpret_cast<const float4*>(sx + i);
                    v[0] = xa.x; v[1] = xa.y; v[2] = xa.z; v[3] = xa.w;
                }
                if (h) *reinterpret_cast<float4*>(h + i) = make_float4(v[0], v[1], v[2], v[3]);
                if (rx) {
                    const uint32_t lo = (uint32_t)f32_to_bf16_bits(xs[4 * g]) | ((uint32_t)f32_to_bf16_bits(xs[4 * g + 1]) << 16);
                    const uint32_t hi = (uint32_t)f32_to_bf16_bits(xs[4 * g + 2]) | ((uint32_t)f32_to_bf16_bits(xs[4 * g + 3]) << 16);
                    *reinterpret_cast<uint2*>(rx + i) = make_uint2(lo, hi);
                }
            }
        }
        if (rx)   // the row's padding stays zero (the network's input width is ldk)
            for (int i = d + tid; i < ldk; i += FT) rx[i] = 0;
        if (a) {
#pragma unroll
            for (int g = 0; g < NM; ++g) {
                const int m = idx(g);
                if (m < dy) {
                    *reinterpret_cast<float4*>(su + m) = make_float4(uv[4 * g], uv[4 * g + 1], uv[4 * g + 2], uv[4 * g + 3]);
                    if (tanh_mode)
                        *reinterpret_cast<float4*>(st + m) = make_float4(tnv[4 * g], tnv[4 * g + 1], tnv[4 * g + 2],
                                                                         tnv[4 * g + 3]);
                }
            }
        }
    }
#pragma unroll
    for (int g = 0; g < NV; ++g) {
        const int i = idx(g);
        if (i < d) {
            *reinterpret_cast<float4*>(X + (size_t)p * d + i) = *reinterpret_cast<const float4*>(sx + i);
            *reinterpret_cast<float4*>(Z + (size_t)p * d + i) = *reinterpret_cast<const float4*>(sz + i);
        }
    }
#pragma unroll
    for (int g = 0; g < NM; ++g) {
        const int m = idx(g);
        if (m < dy) *reinterpret_cast<float4*>(Ax + (size_t)p * dy + m) = *reinterpret_cast<const float4*>(su + m);
    }
    if (tid == 0) {
        lp[p] = lpc;
        q[p] = qc;
        accf[p] = (int8_t)a_last;
        if (lpsum_base) lpsum_base[lps_at] = lps;
        if (nacc) atomicAdd(&ctl->acc_block, nacc);
        if (nnf) atomicAdd(&ctl->nonfinite, nnf);
        __threadfence();
        if (atomicAdd(&ctl->done_blocks, 1u) == gridDim.x - 1) {
            if (dacnt) {   // every proposal was evaluated exactly and went to the ring, P per step
                const long long n = (long long)ns * P;
                dacnt->count = P;
                dacnt->exact += (unsigned long long)n;
                dacnt->head = (head0 + n) % ring_cap;
                dacnt->filled = min(ring_cap, dacnt->filled + n);
            }
            ctl->t_cur += ns;
            ctl->s_cur += ns;
            ctl->done_blocks = 0;
        }
    }
}

// ---------------------------------------------------------------------------------------------------
// Interval moment fold: column sums of the centred samples (two-pass, fixed order).
template <typename HT>
__device__ __forceinline__ double hist_val(HT v);
template <>
__device__ __forceinline__ double hist_val<double>(double v) { return v; }
template <>
__device__ __forceinline__ double hist_val<float>(float v) { return (double)v; }

template <typename HT>
__global__ void colsum_partial_kernel(const HT* __restrict__ H, int ldh, int rows, int d, double* __restrict__ part) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d) return;
    if constexpr (std::is_same<HT, float>::value) {
        // FP32 records: compensated FP32 summation (Kahan 1965), error ~2 ulps of FP32 on the sum whatever the
        // number of rows, at FP32 rate
        float s = 0.f, comp = 0.f;
        for (int r = blockIdx.y; r < rows; r += gridDim.y) {
            const float yv = H[(size_t)r * ldh + i] - comp;
            const float tv = s + yv;
            comp = (tv - s) - yv;
            s = tv;
        }
        part[(size_t)blockIdx.y * d + i] = (double)s - (double)comp;
        return;
    }
    double s = 0.0;
    for (int r = blockIdx.y; r < rows; r += gridDim.y) s += hist_val<HT>(H[(size_t)r * ldh + i]);
    part[(size_t)blockIdx.y * d + i] = s;
}

// s = sum of the partials; delta = (c + s / nb) - mean
__global__ void fold_prep_kernel(int d, int nparts, const double* __restrict__ part, const double* __restrict__ cen64,
                                 const double* __restrict__ mean, double inb, double* __restrict__ s,
                                 double* __restrict__ delta) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d) return;
    double v = 0.0;
    for (int c = 0; c < nparts; ++c) v += part[(size_t)c * d + i];
    s[i] = v;
    delta[i] = (cen64[i] + v * inb) - mean[i];
}

// The interval's FP32 records of x (row s P + p: step s < n_lag, chain p < P; stride ldh), centred here by
// c (cen) as they are read, once, by blocks of
// 32 chains x 32 coordinates that walk the interval's steps (the next step's records loaded ahead):
//   - rows of the steps s >= s0 (past the burn-in): their BF16 transpose HT[c][(s - s0) P + p] (the SYRK
//     operand) and, per (step, chain block) tile, the FP32 sums of the records and of their BF16 values
//     (psum, pbf: tile (s - s0) gridDim.y + blockIdx.y, d entries each); HT == nullptr skips this part;
//   - xs != nullptr: every chain's sum over all n_lag steps, xs[p][c] = sum_s (H - cen[c]) + n_lag cen[c],
//     the per-interval, per-chain sums of x, and its scatter about its interval mean,
//     xm2[p][c] = sum_s H^2 - (sum_s H)^2 / n_lag (the PSRF's within-chain terms).
__global__ void __launch_bounds__(256) fold_records_kernel(const float* __restrict__ H, int ldh, int P, int nl, int s0,
                                                           int d, const float* __restrict__ cen,
                                                           uint16_t* __restrict__ HT, int ldt, float* __restrict__ psum,
                                                           float* __restrict__ pbf, float* __restrict__ xs,
                                                           float* __restrict__ xm2) {
    __shared__ uint16_t tile[32][33];
    __shared__ float sx[8][33], sb[8][33];
    const int c0 = blockIdx.x * 32, p0 = blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int c = c0 + tx;
    float acc[4] = {0.f, 0.f, 0.f, 0.f}, acc2[4] = {0.f, 0.f, 0.f, 0.f}, cur[4], nxt[4];
    const float cc0 = c < d ? cen[c] : 0.f;
    auto load = [&](int st, float* v) {   // the centred record x - c
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int p = p0 + ty + 8 * k;
            v[k] = (p < P && c < d) ? H[((size_t)st * P + p) * ldh + c] - cc0 : 0.f;
        }
    };
    load(0, cur);
    for (int st = 0; st < nl; ++st) {
        if (st + 1 < nl) load(st + 1, nxt);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            acc[k] += cur[k];
            acc2[k] = fmaf(cur[k], cur[k], acc2[k]);
        }
        if (HT && st >= s0) {
            float ax = 0.f, ab = 0.f;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const uint16_t b = f32_to_bf16_bits(cur[k]);
                tile[ty + 8 * k][tx] = b;
                ax += cur[k];
                ab += bf16_bits_to_f32(b);
            }
            sx[ty][tx] = ax;
            sb[ty][tx] = ab;
            __syncthreads();
            if (ty == 0 && c < d) {
                float tsx = 0.f, tsb = 0.f;
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    tsx += sx[k][tx];
                    tsb += sb[k][tx];
                }
                const size_t tl = (size_t)(st - s0) * gridDim.y + blockIdx.y;
                psum[tl * d + c] = tsx;
                pbf[tl * d + c] = tsb;
            }
            const size_t r0 = (size_t)(st - s0) * P + p0;
            for (int k = ty; k < 32; k += 8) {
                const int cc = c0 + k;
                if (cc < d && p0 + tx < P) HT[(size_t)cc * ldt + r0 + tx] = tile[tx][k];
            }
            __syncthreads();
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) cur[k] = nxt[k];
    }
    if (xs && c < d) {
        const float cn = (float)nl * cen[c];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int p = p0 + ty + 8 * k;
            if (p < P) {
                xs[(size_t)p * d + c] = acc[k] + cn;
                if (xm2) xm2[(size_t)p * d + c] = fmaxf(0.f, acc2[k] - acc[k] * acc[k] / (float)nl);
            }
        }
    }
}

// fold_records_kernel with 16-byte loads: blocks of 32 chains x 128 coordinates (d, ldh multiples of 4, P a
// multiple of 8, so every 8 chains' BF16 values of one coordinate are one 16-byte store of the transpose).
// Thread (ty, tx) loads coordinates 4 tx .. 4 tx + 3 of chains ty + 8 k; the tile is kept chain-major in shared
// memory and read across chains for the transposed stores. Same outputs as fold_records_kernel.
__global__ void __launch_bounds__(256) fold_records4_kernel(const float* __restrict__ H, int ldh, int P, int nl, int s0,
                                                            int d, const float* __restrict__ cen,
                                                            uint16_t* __restrict__ HT, int ldt, float* __restrict__ psum,
                                                            float* __restrict__ pbf, float* __restrict__ xs,
                                                            float* __restrict__ xm2) {
    __shared__ __align__(16) uint16_t tile[32][136];   // [chain][coordinate], 272-byte rows
    __shared__ float sx[8][132], sb[8][132];
    const int c0 = blockIdx.x * 128, p0 = blockIdx.y * 32;
    const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
    const int c = c0 + 4 * tx;
    const bool cv = c < d;
    float4 acc[4], acc2[4], cur[4], nxt[4];
    const float4 cc4 = cv ? *reinterpret_cast<const float4*>(cen + c) : make_float4(0.f, 0.f, 0.f, 0.f);
    auto load = [&](int st, float4* v) {   // the centred records x - c
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int p = p0 + ty + 8 * k;
            if (p < P && cv) {
                const float4 r = *reinterpret_cast<const float4*>(H + ((size_t)st * P + p) * ldh + c);
                v[k] = make_float4(r.x - cc4.x, r.y - cc4.y, r.z - cc4.z, r.w - cc4.w);
            } else {
                v[k] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
    };
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        acc[k] = make_float4(0.f, 0.f, 0.f, 0.f);
        acc2[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    load(0, cur);
    for (int st = 0; st < nl; ++st) {
        if (st + 1 < nl) load(st + 1, nxt);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            acc[k].x += cur[k].x; acc[k].y += cur[k].y; acc[k].z += cur[k].z; acc[k].w += cur[k].w;
            acc2[k].x = fmaf(cur[k].x, cur[k].x, acc2[k].x);
            acc2[k].y = fmaf(cur[k].y, cur[k].y, acc2[k].y);
            acc2[k].z = fmaf(cur[k].z, cur[k].z, acc2[k].z);
            acc2[k].w = fmaf(cur[k].w, cur[k].w, acc2[k].w);
        }
        if (HT && st >= s0) {
            float ax[4] = {0.f, 0.f, 0.f, 0.f}, ab[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float v[4] = {cur[k].x, cur[k].y, cur[k].z, cur[k].w};
                uint16_t b[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    b[j] = f32_to_bf16_bits(v[j]);
                    ax[j] += v[j];
                    ab[j] += bf16_bits_to_f32(b[j]);
                }
                *reinterpret_cast<uint2*>(&tile[ty + 8 * k][4 * tx]) =
                    make_uint2((uint32_t)b[0] | ((uint32_t)b[1] << 16), (uint32_t)b[2] | ((uint32_t)b[3] << 16));
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                sx[ty][4 * tx + j] = ax[j];
                sb[ty][4 * tx + j] = ab[j];
            }
            __syncthreads();
            const size_t tl = (size_t)(st - s0) * gridDim.y + blockIdx.y;
            if (tid < 128 && c0 + tid < d) {
                float tsx = 0.f, tsb = 0.f;
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    tsx += sx[k][tid];
                    tsb += sb[k][tid];
                }
                psum[tl * d + c0 + tid] = tsx;
                pbf[tl * d + c0 + tid] = tsb;
            }
            {   // transposed stores: coordinate cc, chains 16 h .. 16 h + 15 as two 16-byte stores
                const int cc = tid >> 1, h = tid & 1;
                const size_t r0 = (size_t)(st - s0) * P + p0 + 16 * h;
                if (c0 + cc < d) {
#pragma unroll
                    for (int q = 0; q < 2; ++q) {
                        if (p0 + 16 * h + 8 * q < P) {
                            uint32_t w[4];
#pragma unroll
                            for (int i = 0; i < 4; ++i)
                                w[i] = (uint32_t)tile[16 * h + 8 * q + 2 * i][cc] |
                                       ((uint32_t)tile[16 * h + 8 * q + 2 * i + 1][cc] << 16);
                            *reinterpret_cast<uint4*>(HT + (size_t)(c0 + cc) * ldt + r0 + 8 * q) =
                                make_uint4(w[0], w[1], w[2], w[3]);
                        }
                    }
                }
            }
            __syncthreads();
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) cur[k] = nxt[k];
    }
    if (xs && cv) {
        const float4 cn = *reinterpret_cast<const float4*>(cen + c);
        const float fn = (float)nl;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int p = p0 + ty + 8 * k;
            if (p < P) {
                *reinterpret_cast<float4*>(xs + (size_t)p * d + c) =
                    make_float4(acc[k].x + fn * cn.x, acc[k].y + fn * cn.y, acc[k].z + fn * cn.z, acc[k].w + fn * cn.w);
                if (xm2)
                    *reinterpret_cast<float4*>(xm2 + (size_t)p * d + c) =
                        make_float4(fmaxf(0.f, acc2[k].x - acc[k].x * acc[k].x / (float)nl),
                                    fmaxf(0.f, acc2[k].y - acc[k].y * acc[k].y / (float)nl),
                                    fmaxf(0.f, acc2[k].z - acc[k].z * acc[k].z / (float)nl),
                                    fmaxf(0.f, acc2[k].w - acc[k].w * acc[k].w / (float)nl));
            }
        }
    }
}

// Potential scale reduction factor of eq. (winco), (btwco), (psrf) over the intervals [b0, b0 + nb) of the
// per-chain interval sums (n = nb n_lag samples per chain). Stage 1, thread (p, i): the window's mean of
// chain p and its scatter, the intervals combined pairwise (Chan, Golub & LeVeque 1979); q holds per interval
// the scatter about the interval mean (raw = 0) or the raw sum of squares (raw = 1).
template <typename HT>
__global__ void psrf_chain_kernel(int d, int P, int nl, long long b0, int nb, const HT* __restrict__ bsum,
                                  const HT* __restrict__ bq, int raw, double* __restrict__ cmean,
                                  double* __restrict__ cvar) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x, p = blockIdx.y;
    if (i >= d) return;
    double m = 0.0, M2 = 0.0;
    for (int k = 0; k < nb; ++k) {
        const size_t o = ((size_t)(b0 + k) * P + p) * d + i;
        const double s = (double)bsum[o], q = (double)bq[o];
        const double mk = s / nl, m2k = raw ? fmax(0.0, q - s * mk) : q;
        const double delta = mk - m;
        m += delta / (k + 1);
        M2 += m2k + delta * delta * ((double)k * nl / (k + 1));
    }
    cmean[(size_t)p * d + i] = m;
    cvar[(size_t)p * d + i] = M2 / ((double)nb * nl);   // (C^p)_ii with the 1/n of eq. (sampcov)
}

// Stage 2, thread i: B_i, W_i of eq. (btwco) over the P chains and sqrt(R_i) of eq. (psrf).
__global__ void psrf_final_kernel(int d, int P, double n, const double* __restrict__ cmean,
                                  const double* __restrict__ cvar, double* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d) return;
    double mg = 0.0, w = 0.0;
    for (int p = 0; p < P; ++p) {
        mg += cmean[(size_t)p * d + i];
        w += cvar[(size_t)p * d + i];
    }
    mg /= P;
    double b = 0.0;
    for (int p = 0; p < P; ++p) {
        const double e = cmean[(size_t)p * d + i] - mg;
        b += e * e;
    }
    const double B = n / (P - 1) * b, W = n / ((n - 1.0) * P) * w;
    out[i] = sqrt((n - 1.0) / n + (P + 1.0) / (P * n) * B / W);
}

// Column totals of the tile sums (compensated FP32 per thread, Kahan 1965; FP64 across threads), then the
// interval's centring terms: s = sum of the records, delta = (c + s / nb) - mean, s16 = sum of their BF16
// values. One block per 32 coordinates, 8 threads per coordinate.
__global__ void __launch_bounds__(256) fold_sums_kernel(int d, int ntile, const float* __restrict__ psum,
                                                        const float* __restrict__ pbf, const double* __restrict__ cen64,
                                                        const double* __restrict__ mean, double inb,
                                                        double* __restrict__ s, double* __restrict__ delta,
                                                        double* __restrict__ s16) {
    __shared__ double rx[8][32], rb[8][32];
    const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
    const int i = blockIdx.x * 32 + lane;
    float sx = 0.f, cx = 0.f, sb = 0.f, cb = 0.f;
    if (i < d) {
        for (int t = g; t < ntile; t += 8) {
            const float yx = psum[(size_t)t * d + i] - cx, yb = pbf[(size_t)t * d + i] - cb;
            const float tx = sx + yx, tb = sb + yb;
            cx = (tx - sx) - yx;
            cb = (tb - sb) - yb;
            sx = tx;
            sb = tb;
        }
    }
    rx[g][lane] = (double)sx - (double)cx;
    rb[g][lane] = (double)sb - (double)cb;
    __syncthreads();
    if (g == 0 && i < d) {
        double vx = 0.0, vb = 0.0;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            vx += rx[k][lane];
            vb += rb[k][lane];
        }
        s[i] = vx;
        delta[i] = (cen64[i] + vx * inb) - mean[i];
        s16[i] = vb;
    }
}

// out = s * M with M symmetric and only its lower triangle stored (both d x d, stride d): 32 x 32 tiles,
// the upper tiles through a shared-memory transpose of their lower mirror.
__global__ void symmetrize_kernel(int d, const double* __restrict__ M, double s, double* __restrict__ out) {
    __shared__ double t[32][33];
    const int bi = blockIdx.y, bj = blockIdx.x;   // output tile (rows bi, columns bj)
    const int si = max(bi, bj), sj = min(bi, bj);  // source tile in the lower triangle
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int r = si * 32 + k, c = sj * 32 + threadIdx.x;
        t[k][threadIdx.x] = (r < d && c < d && c <= r) ? M[(size_t)r * d + c] : 0.0;
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int r = bi * 32 + k, c = bj * 32 + threadIdx.x;
        if (r >= d || c >= d) continue;
        // element (r, c) = M[max][min]: in the source tile at (r - 32 si, c - 32 sj) or its transpose
        const double v = (c <= r) ? ((bi == si) ? t[k][threadIdx.x] : t[threadIdx.x][k])
                                  : ((bi == si) ? t[threadIdx.x][k] : t[threadIdx.x][k]);
        out[(size_t)r * d + c] = s * v;
    }
}

// s16[i] = sum over the interval's samples of the BF16-rounded centred records (row i of the transposed
// record): the sums of exactly the values the tensor-core SYRK multiplies, so that G - s16 s16^T / nb is
// the scatter matrix of those values (positive semi-definite up to the FP32 accumulation).
__global__ void __launch_bounds__(256) rowsum_bf16_kernel(const uint16_t* __restrict__ HT_, int ldt, int rows,
                                                          double* __restrict__ s16) {
    __shared__ double sh[32];
    const int i = blockIdx.x;
    float s = 0.f, comp = 0.f;   // compensated FP32 summation per thread (Kahan 1965), FP64 across threads
    for (int r = threadIdx.x; r < rows; r += blockDim.x) {
        const float yv = bf16_bits_to_f32(HT_[(size_t)i * ldt + r]) - comp;
        const float tv = s + yv;
        comp = (tv - s) - yv;
        s = tv;
    }
    double acc = block_sum((double)s - (double)comp, sh);
    if (threadIdx.x == 0) s16[i] = acc;
}

// mean += delta nb / (n + nb); the next interval is centred at the new mean (cen64 exact copy of cenT).
template <typename T>
__global__ void mean_update_kernel(int d, double frac, const double* __restrict__ delta, double* __restrict__ mean,
                                   double* __restrict__ cen64, T* __restrict__ cenT) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d) return;
    double m = mean[i] + delta[i] * frac;
    mean[i] = m;
    T c = (T)m;
    cenT[i] = c;
    cen64[i] = (double)c;
}

// Centre of the coming interval's records: the mean of the chains' current states (a close predictor of
// the interval's mean, so the centred sums stay small and the FP32 tensor-core SYRK loses little to
// cancellation). cen64 holds exactly the values subtracted (in the state type).
template <typename T>
__global__ void centre_kernel(int d, int P, const T* __restrict__ X, T* __restrict__ cenT, double* __restrict__ cen64) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d) return;
    double s = 0.0;
    for (int p = 0; p < P; ++p) s += (double)X[(size_t)p * d + i];
    T c = (T)(s / P);
    cenT[i] = c;
    cen64[i] = (double)c;
}

// ---------------------------------------------------------------------------------------------------
// Refresh helpers.
__global__ void trace_kernel(int d, const double* __restrict__ M2, int ld, Ctl* ctl) {
    __shared__ double sh[32];
    double s = 0.0;
    for (int i = threadIdx.x; i < d; i += blockDim.x) s += M2[(size_t)i * ld + i];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) ctl->trace = s;
}

// C = M2 / n with its diagonal loaded by (1 + eps) (lower triangle)
__global__ void build_c_kernel(int d, const double* __restrict__ M2, int ld, double inv_n, double eps,
                               double* __restrict__ Cm) {
    int i = blockIdx.y;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j <= i; j += gridDim.x * blockDim.x) {
        double v = M2[(size_t)i * ld + j] * inv_n;
        if (i == j) v *= 1.0 + eps;
        Cm[(size_t)i * ld + j] = v;
    }
}

// Quantised factor: Lq64 = round_bf16(L) and its BF16 bits (row-major, ldk columns, zero padded).
// Lq = the factor rounded to BF16 (Lq16 its bits), or, with Lq16lo, to TF32: 11 significant bits, exactly the
// sum of two BF16 values (Lq16 = the BF16 rounding of the TF32 value, Lq16lo = the rest, at most 3 bits).
__global__ void quantise_factor_kernel(int d, const double* __restrict__ L, int ld, double* __restrict__ Lq64,
                                       uint16_t* __restrict__ Lq16, int ldk, uint16_t* __restrict__ Lq16lo) {
    int i = blockIdx.y;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < ldk; j += gridDim.x * blockDim.x) {
        const double l = (j < d) ? L[(size_t)i * ld + j] : 0.0;
        const double v = Lq16lo ? round_tf32(l) : round_bf16(l);
        if (j < d) Lq64[(size_t)i * ld + j] = v;
        const double h = round_bf16(v);
        Lq16[(size_t)i * ldk + j] = bf16_bits_of_rounded(h);
        if (Lq16lo) Lq16lo[(size_t)i * ldk + j] = bf16_bits_of_rounded(v - h);   // exact: v - h has <= 3 bits
    }
}

// work = x - x_ref in FP64 (for the whitening solve z = Lq^{-1}(x - x_ref))
template <typename T>
__global__ void diff_kernel(int d, const T* __restrict__ Xs, const T* __restrict__ xref, double* __restrict__ work) {
    int p = blockIdx.y;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d; i += gridDim.x * blockDim.x)
        work[(size_t)p * d + i] = (double)Xs[(size_t)p * d + i] - (double)xref[i];
}

// Re-whitening after a factor change in BF16 mode: z = Lq^{-1}(x - x_ref) for every chain in FP32, the
// precision of the states (Lq is BF16, exact in FP32), by blocked forward substitution with a lookahead of
// one block. One CTA per G chains keeps their right-hand sides in shared memory. Per 64-column block k (its
// unknowns already solved): all threads first update the next block's 64 rows by block k; then warps 0 .. G-1
// stage nothing new but solve the next block's diagonal system (warp g: chain g, the 64-step chain on lane
// shuffles, the diagonal factor staged in shared memory) while the other warps update every row below it by
// block k (G dot products of length 64 per row, the factor's row segment read as eight 16-byte loads, two
// rows per iteration). Finally z and q = |z|^2 / (2 alpha^2) (and log pi = -q for the reference target).
// Dynamic shared memory: rewhiten32_smem(d, G) bytes.
constexpr int RW_G = 4, RW_THREADS = 512;

__host__ __device__ inline size_t rewhiten32_smem(int d, int g) {
    return sizeof(float) * ((size_t)g * d + 2 * 64 * 65 + 2 * 64 + 2 * 64 * 4);
}

// rows [r0, r1) of the G right-hand sides -= L[rows][k0 .. k0 + 64) y, y in shared memory as 64 float4
// (column c: the G chains' values, zero past G); the threads t0, t0 + nt, ... each take four rows per
// iteration, so one broadcast 16-byte load of y feeds 16 fused multiply-adds. Every CTA reads the same factor
// rows, so each starts at its own rotation of the row quads.
__device__ __forceinline__ void rw_update_rows(const uint16_t* __restrict__ Lq, int ldk, int d, int k0, int r0, int r1,
                                               int G, const float4* __restrict__ y, float* __restrict__ rw, int t,
                                               int nt) {
    const int nq = (r1 - r0 + 3) / 4;
    const int rot = nq > 0 ? (int)((blockIdx.x * 97u) % (unsigned)nq) : 0;
    for (int qq = t; qq < nq; qq += nt) {
        const int q = qq + rot < nq ? qq + rot : qq + rot - nq;
        const int i0 = r0 + 4 * q;
        const uint4* lr[4];
#pragma unroll
        for (int r = 0; r < 4; ++r)
            lr[r] = reinterpret_cast<const uint4*>(Lq + (size_t)min(i0 + r, r1 - 1) * ldk + k0);
        float4 acc[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) acc[r] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 2
        for (int c8 = 0; c8 < 8; ++c8) {
            uint4 u[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) u[r] = lr[r][c8];
#pragma unroll
            for (int h = 0; h < 4; ++h) {
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const float4 yc = y[c8 * 8 + 2 * h + e];
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        const uint32_t w = h == 0 ? u[r].x : h == 1 ? u[r].y : h == 2 ? u[r].z : u[r].w;
                        const float l = __uint_as_float(e ? (w & 0xFFFF0000u) : (w << 16));
                        acc[r].x = fmaf(l, yc.x, acc[r].x);
                        acc[r].y = fmaf(l, yc.y, acc[r].y);
                        acc[r].z = fmaf(l, yc.z, acc[r].z);
                        acc[r].w = fmaf(l, yc.w, acc[r].w);
                    }
                }
            }
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int i = i0 + r;
            if (i < r1) {
                const float a[4] = {acc[r].x, acc[r].y, acc[r].z, acc[r].w};
#pragma unroll
                for (int g = 0; g < RW_G; ++g)
                    if (g < G) rw[(size_t)g * d + i] -= a[g];
            }
        }
    }
}

__global__ void __launch_bounds__(RW_THREADS) rewhiten32_kernel(int d, int P, int G, const uint16_t* __restrict__ Lq,
                                                                int ldk, const float* __restrict__ X,
                                                                const float* __restrict__ xref, float* __restrict__ Zs,
                                                                double* __restrict__ qout, double inv_infl2,
                                                                double* __restrict__ lp_ref) {
    extern __shared__ float4 rw_smem4[];
    float* yb = reinterpret_cast<float*>(rw_smem4);   // 2 x 64 x 4: a block's solution ([column][chain]), 16-byte aligned
    float* rdiag = yb + 2 * 64 * 4;                   // 2 x 64: reciprocals of the diagonal blocks' diagonals
    float* Ld = rdiag + 2 * 64;                       // 2 x 64 x 65: diagonal blocks (two buffers)
    float* rw = Ld + 2 * 64 * 65;                     // G x d: right-hand sides, overwritten by z
    __shared__ double sh[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int p0 = blockIdx.x * G, ng = min(G, P - p0);
    const int nblk = (d + 63) / 64;
    for (int g = 0; g < ng; ++g)
        for (int i = tid; i < d; i += RW_THREADS) rw[(size_t)g * d + i] = X[(size_t)(p0 + g) * d + i] - xref[i];
    // diagonal block kb into buffer kb & 1 (all threads)
    auto stage = [&](int kb) {
        const int k0 = kb * 64, nb = min(64, d - k0);
        float* L = Ld + (kb & 1) * 64 * 65;
        for (int e = tid; e < nb * nb; e += RW_THREADS) {
            const int r = e / nb, cc = e - r * nb;
            L[r * 65 + cc] = (cc <= r) ? bf16_bits_to_f32(Lq[(size_t)(k0 + r) * ldk + k0 + cc]) : 0.f;
        }
    };
    // warp g < ng: solve block kb's unknowns of chain g (rows already updated by every earlier block)
    auto solve = [&](int kb) {
        const int k0 = kb * 64, nb = min(64, d - k0);
        const float* L = Ld + (kb & 1) * 64 * 65;
        const float* rd = rdiag + (kb & 1) * 64;
        float* y = yb + (kb & 1) * 64 * 4;
        float* rg = rw + (size_t)warp * d + k0;
        float v0 = lane < nb ? rg[lane] : 0.f, v1 = lane + 32 < nb ? rg[lane + 32] : 0.f;
        for (int j = 0; j < nb; ++j) {
            const float vj = __shfl_sync(0xffffffffu, j < 32 ? v0 : v1, j & 31);
            const float yj = vj * rd[j];
            if (lane > j && lane < nb) v0 = fmaf(-L[lane * 65 + j], yj, v0);
            if (lane + 32 > j && lane + 32 < nb) v1 = fmaf(-L[(lane + 32) * 65 + j], yj, v1);
            if (lane == (j & 31)) {
                if (j < 32) v0 = yj;
                else v1 = yj;
            }
        }
        if (lane < nb) rg[lane] = v0;
        if (lane + 32 < nb) rg[lane + 32] = v1;
        y[lane * 4 + warp] = lane < nb ? v0 : 0.f;   // zero past a short last block
        y[(lane + 32) * 4 + warp] = lane + 32 < nb ? v1 : 0.f;
    };
    stage(0);
    __syncthreads();
    if (tid < min(64, d)) rdiag[tid] = 1.0f / Ld[tid * 65 + tid];
    for (int e = tid; e < 2 * 64 * 4; e += RW_THREADS) yb[e] = 0.f;   // columns of chains past G stay zero
    __syncthreads();
    if (warp < ng) solve(0);
    __syncthreads();
    for (int kb = 0; kb < nblk; ++kb) {
        const int k0 = kb * 64, k1 = k0 + 64;
        const float4* y = reinterpret_cast<const float4*>(yb + (kb & 1) * 64 * 4);
        if (k1 >= d) break;
        const int n1 = min(64, d - k1);
        // the next block's rows by block k, and its diagonal factor staged
        rw_update_rows(Lq, ldk, d, k0, k1, k1 + n1, ng, y, rw, tid, RW_THREADS);
        stage(kb + 1);
        __syncthreads();
        if (tid < n1) rdiag[((kb + 1) & 1) * 64 + tid] = 1.0f / Ld[((kb + 1) & 1) * 64 * 65 + tid * 65 + tid];
        __syncthreads();
        if (warp < ng) {
            solve(kb + 1);   // the next block's unknowns ...
        } else {             // ... while the other warps update the rows below it by block k
            rw_update_rows(Lq, ldk, d, k0, k1 + n1, d, ng, y, rw, tid - 32 * ng, RW_THREADS - 32 * ng);
        }
        __syncthreads();
    }
    for (int g = 0; g < ng; ++g) {
        double acc = 0.0;
        for (int i = tid; i < d; i += RW_THREADS) {
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

// z = work (rounded to T), q = |z|^2 / (2 alpha^2) from the stored z; lp = -q for the reference target.
template <typename T>
__global__ void __launch_bounds__(256) set_z_kernel(int d, const double* __restrict__ work, T* __restrict__ Zs,
                                                    double* __restrict__ qout, double inv_infl2,
                                                    double* __restrict__ lp_ref) {
    __shared__ double sh[32];
    int p = blockIdx.x;
    double acc = 0.0;
    for (int i = threadIdx.x; i < d; i += blockDim.x) {
        T v = (T)work[(size_t)p * d + i];
        if (Zs) Zs[(size_t)p * d + i] = v;
        acc += (double)v * (double)v;
    }
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) {
        double qq = 0.5 * acc * inv_infl2;
        if (qout) qout[p] = qq;
        if (lp_ref) lp_ref[p] = -qq;
    }
}

__global__ void set_scalars_kernel(Ctl* ctl, double beta, double rho, double ba, double inv_infl2) {
    ctl->beta = beta;
    ctl->rho = rho;
    ctl->ba = ba;
    ctl->inv_infl2 = inv_infl2;
    ctl->acc_block = 0ull;
    ctl->s_cur = 0;
}

template <typename A, typename B>
__global__ void convert_kernel(size_t n, const A* __restrict__ in, B* __restrict__ out) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = (B)in[i];
}

// v <- its BF16 rounding (round to nearest even), kept in FP64.
__global__ void round_bf16_kernel(size_t n, double* __restrict__ v) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        v[i] = round_bf16(v[i]);
}

// Row-major d_y x d FP64 matrix -> BF16 bits (round to nearest even), ldk columns, zero padded.
__global__ void to_bf16_rows_kernel(int rows, int d, const double* __restrict__ in, uint16_t* __restrict__ out, int ldk) {
    int i = blockIdx.y;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < ldk; j += gridDim.x * blockDim.x) {
        double v = (j < d) ? round_bf16(in[(size_t)i * d + j]) : 0.0;
        out[(size_t)i * ldk + j] = bf16_bits_of_rounded(v);
    }
}

}  // namespace
}  // namespace diam
