// da_kernels.cuh -- kernels of the delayed-acceptance surrogate (two-stage Metropolis-Hastings of
// Christen & Fox, 2005; not in the paper): an MLP d -> h1 -> h2 -> 1 with GELU, BF16 weights and FP32
// accumulation. The two hidden layers are tcgen05 GEMMs (tc_gemm.cu, TC_GELU epilogue); these kernels are
// the glue: input normalisation, the output layer, the stage-1 screen with survivor compaction, the
// stage-2 exact test, the ring buffer of training pairs, and the training step (loss gradient, column
// reductions, transposes, Adam).
#pragma once
#include "step.cuh"

namespace diam {
namespace {

enum : uint32_t { TAG_MINIBATCH = 5 };

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float z) {
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

// U[r][i] = bf16((x_ri - shift_i) * scale_i), zero padding to ldk (rows of a state buffer)
template <typename T>
__global__ void mlp_input_kernel(int d, const T* __restrict__ Xs, const float* __restrict__ shift,
                                 const float* __restrict__ scale, uint16_t* __restrict__ U, int ldk) {
    const int r = blockIdx.x;
    for (int i = blockIdx.y * blockDim.x + threadIdx.x; i < ldk; i += gridDim.y * blockDim.x) {
        float v = 0.f;
        if (i < d) v = ((float)Xs[(size_t)r * d + i] - shift[i]) * scale[i];
        U[(size_t)r * ldk + i] = f32_to_bf16_bits(v);
    }
}

// s_r = mu + sigma (w3 . H2_r + b3), one thread per row
// musig: the output scaling (mu, sigma) of the current training, in device memory so that a captured
// interval graph sees every retraining
__global__ void mlp_out_kernel(int rows, int h2, const uint16_t* __restrict__ H2, const float* __restrict__ w3,
                               const float* __restrict__ b3, const double* __restrict__ musig, double* __restrict__ s_out) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    float acc = 0.f;
    for (int o = 0; o < h2; ++o) acc += w3[o] * bf16_bits_to_f32(H2[(size_t)r * h2 + o]);
    s_out[r] = musig[0] + musig[1] * (double)(acc + b3[0]);
}


// Stage 1 for every chain (one block, P <= 1024 threads): q(x*) from the proposal's partial sums, then
// with the surrogate active: s(x*) = the exact O(d) terms + the network's value of the linear-map terms,
// log a1 = s(x*) - s(x) + q(x*) - q(x), pass iff log u1 < log a1 (tag 3); inactive: every chain passes. The passing chains are compacted in chain order into idx[0..count).
__global__ void stage1_kernel(int P, int nchunk, Key key, const Ctl* ctl, int active, const double* __restrict__ qpart,
                              const double* __restrict__ lpart_, double inv_infl2, const double* __restrict__ q,
                              double* __restrict__ s_prop,
                              const double* __restrict__ s_cur, double* __restrict__ qsave, int* __restrict__ idx,
                              int8_t* __restrict__ accf, double* __restrict__ lp_nan_trace, DaCounters* cnt,
                              TraceDev tr) {
    __shared__ int wsum[32];
    const int p = threadIdx.x;
    const int64_t t = ctl->t_cur;
    int pass = 0;
    if (p < P) {
        double qs = 0.0;
        for (int c = 0; c < nchunk; ++c) qs += qpart[(size_t)c * P + p];
        const double qpp = 0.5 * qs * inv_infl2;
        qsave[p] = qpp;
        if (active) {
            // s(x*) = exact O(d) terms of log pi + the network's estimate of the linear-map terms
            double lo = 0.0;
            for (int c = 0; c < nchunk; ++c) lo += lpart_[(size_t)c * P + p];
            s_prop[p] += lo;
            const double loga1 = s_prop[p] - s_cur[p] + qpp - q[p];
            const double u1 = uniform53(key, t, (uint32_t)p, TAG_UDA);
            pass = isfinite(loga1) && (log(u1) < loga1);
        } else {
            pass = 1;
        }
        accf[p] = 0;
        if (!pass && t < tr.steps) {
            size_t k = (size_t)t * P + p;
            tr.lp[k] = lp_nan_trace ? lp_nan_trace[0] : NAN;   // log pi(x*) not evaluated
            tr.q[k] = qpp;
            tr.qc[k] = q[p];
            tr.loga[k] = -INFINITY;
            tr.acc[k] = 0;
        }
    }
    // exclusive prefix of pass over the block (chain order), warp ballots then warp totals
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned bal = __ballot_sync(0xffffffffu, pass);
    const int before = __popc(bal & ((1u << lane) - 1u));
    if (lane == 0) wsum[w] = __popc(bal);
    __syncthreads();
    int off = 0;
    for (int k = 0; k < w; ++k) off += wsum[k];
    if (pass) idx[off + before] = p;
    if (threadIdx.x == blockDim.x - 1) {
        int total = off + before + pass;
        cnt->count = total;
        if (active) {
            cnt->tested += (unsigned long long)P;
            cnt->passed += (unsigned long long)total;
        }
        cnt->exact += (unsigned long long)total;
    }
}

// rows idx[k] of the BF16 target operand planes -> rows k of the compact planes (k < count)
__global__ void gather_rows_kernel(const DaCounters* cnt, const int* __restrict__ idx, const uint16_t* __restrict__ hi,
                                   const uint16_t* __restrict__ lo, uint16_t* __restrict__ chi,
                                   uint16_t* __restrict__ clo, int ldk) {
    const int k = blockIdx.x;
    if (k >= cnt->count) return;
    const int p = idx[k];
    const uint4* sh = reinterpret_cast<const uint4*>(hi + (size_t)p * ldk);
    const uint4* sl = reinterpret_cast<const uint4*>(lo + (size_t)p * ldk);
    uint4* dh = reinterpret_cast<uint4*>(chi + (size_t)k * ldk);
    uint4* dl = reinterpret_cast<uint4*>(clo + (size_t)k * ldk);
    for (int j = threadIdx.x; j < ldk / 8; j += blockDim.x) {
        dh[j] = sh[j];
        dl[j] = sl[j];
    }
}

// Stage 2 (one block per survivor k): log pi(x*) from the split-K partial products of the compact rows,
// log a2 = log pi(x*) - log pi(x) - s(x*) + s(x), accept iff log u < log a2 (tag 1); the evaluated pair
// (x*, log pi(x*)) goes to the ring buffer.
__global__ void __launch_bounds__(256) finish_da_kernel(int P, int dy, int nsplit, const float* __restrict__ ws,
                                                         const float* __restrict__ y32, float inv2s2, int tanh_mode,
                                                         int nchunk, Key key,
                                                         const double* __restrict__ lpart,
                                                         const double* __restrict__ qsave, const int* __restrict__ idx,
                                                         const DaCounters* cnt, int active, const double* __restrict__ s_prop,
                                                         double* s_cur, double* lp, double* q, int8_t* accf, Ctl* ctl,
                                                         TraceDev tr, const uint16_t* __restrict__ chi,
                                                         uint16_t* __restrict__ ring_x, float* __restrict__ ring_lp,
                                                         long long ring_cap, int ldk,
                                                         const double* __restrict__ lmap_in = nullptr) {
    __shared__ float shf[32];
    const int k = blockIdx.x;
    if (k >= cnt->count) return;
    const int p = idx[k];
    const int64_t t = ctl->t_cur;
    const size_t plane = (size_t)P * dy;
    double acc;
    if (lmap_in) {   // the map terms already computed for every chain (map carried through the proposal)
        acc = lmap_in[p];
    } else {
        float af = 0.f;   // the linear-map terms in FP32, as in the plain exact test
        for (int m = threadIdx.x; m < dy; m += blockDim.x) {
            float u = 0.f;
            for (int s = 0; s < nsplit; ++s) u += ws[s * plane + (size_t)k * dy + m];
            if (tanh_mode) {
                const float r = y32[m] - tanhf(u);
                af -= r * r * inv2s2;
            } else {
                af -= 0.5f * u * u;
            }
        }
        acc = (double)block_sum(af, shf);
    }
    const double lmap = acc;   // the linear-map part of log pi(x*): what the network learns
    for (int c = 0; c < nchunk; ++c) acc += lpart[(size_t)c * P + p];
    const long long slot = (cnt->head + k) % ring_cap;
    // chi: the survivors' rows in compacted order, or (lmap_in given) every proposal's row in chain order
    const uint4* src = reinterpret_cast<const uint4*>(chi + (size_t)(lmap_in ? p : k) * ldk);
    uint4* dst = reinterpret_cast<uint4*>(ring_x + (size_t)slot * ldk);
    for (int j = threadIdx.x; j < ldk / 8; j += blockDim.x) dst[j] = src[j];
    if (threadIdx.x == 0) {
        ring_lp[slot] = (float)lmap;
        const double lpp = acc, qpp = qsave[p];
        // stage 2 (Christen & Fox): log pi(x*) - log pi(x) - s(x*) + s(x); with stage 1 off this is the plain
        // Metropolis-Hastings ratio of Algorithm 1, log pi(x*) - log pi(x) + q(x*) - q(x)
        const double loga = active ? (lpp - lp[p] - s_prop[p] + s_cur[p]) : (lpp - lp[p] + qpp - q[p]);
        const bool finite = isfinite(lpp);
        const double u = uniform53(key, t, (uint32_t)p, TAG_U);
        const int a = finite && (log(u) < loga);
        if (t < tr.steps) {
            size_t kk = (size_t)t * P + p;
            tr.lp[kk] = lpp; tr.q[kk] = qpp; tr.qc[kk] = q[p]; tr.loga[kk] = loga; tr.acc[kk] = (int8_t)a;
        }
        if (a) {
            lp[p] = lpp;
            q[p] = qpp;
            if (active) s_cur[p] = s_prop[p];
            atomicAdd(&ctl->acc_block, 1ull);
        }
        if (!finite) atomicAdd(&ctl->nonfinite, 1ull);
        accf[p] = (int8_t)a;
    }
}

__global__ void add_kernel(int n, const double* __restrict__ a, double* __restrict__ b) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] += a[i];
}



// ---------------------------------------------------------------------------------------------------- training
// Training slot j (of the non-held-out slots, those with slot % 10 != 9) -> ring slot.
__device__ __forceinline__ long long train_slot(long long j) { return (j / 9) * 10 + (j % 9); }

__host__ __device__ inline long long n_train_slots(long long filled) {
    return 9 * (filled / 10) + (filled % 10 < 9 ? filled % 10 : 9);
}

// Minibatch row b of Adam step a: a Philox-chosen training slot (tag 5), normalised and rounded to BF16;
// target t_b = (log pi - mu) / sigma. held_out = 1: rows b of the held-out slots instead (slot 10 j + 9).
// a_dev (optional): the draw's counter read from device memory instead of a (a training step replayed as a graph).
__global__ void gather_batch_kernel(Key key, long long a, int held_out, long long first, const uint16_t* __restrict__ ring_x,
                                    const float* __restrict__ ring_lp, const DaCounters* cnt, int d, int ldk,
                                    const float* __restrict__ shift, const float* __restrict__ scale, double mu,
                                    double sigma, uint16_t* __restrict__ Xb, float* __restrict__ tb,
                                    float* __restrict__ raw_lp, const long long* __restrict__ a_dev = nullptr) {
    const int b = blockIdx.x;
    if (a_dev) a = a_dev[0];
    const long long filled = cnt->filled;
    long long slot;
    if (held_out) {
        slot = 10 * (first + b) + 9;
        if (slot >= filled) slot = 9 % (filled > 0 ? filled : 1);
    } else {
        const long long ntr = n_train_slots(filled);
        const double u = uniform53(key, a, (uint32_t)b, TAG_MINIBATCH);
        long long j = (long long)(u * (double)ntr);
        if (j >= ntr) j = ntr - 1;
        if (j < 0) j = 0;
        slot = train_slot(j);
    }
    for (int i = threadIdx.x; i < ldk; i += blockDim.x) {
        float v = 0.f;
        if (i < d) v = (bf16_bits_to_f32(ring_x[(size_t)slot * ldk + i]) - shift[i]) * scale[i];
        Xb[(size_t)b * ldk + i] = f32_to_bf16_bits(v);
    }
    if (threadIdx.x == 0) {
        const float lpv = ring_lp[slot];
        tb[b] = (float)(((double)lpv - mu) / sigma);
        if (raw_lp) raw_lp[b] = lpv;
    }
}

// Output layer and loss gradient, one warp per sample: out = w3 . H2 + b3, r = out - t,
// loss += r^2 / (2B), ds = r / B, dZ2 = ds w3 * GELU'(Z2) (FP32 and BF16, both layouts).
__global__ void loss_grad_kernel(int B, int h2, const uint16_t* __restrict__ H2, const float* __restrict__ Z2,
                                 const float* __restrict__ w3, const float* __restrict__ b3, const float* __restrict__ tb,
                                 float* __restrict__ ds, float* __restrict__ dZ2f, uint16_t* __restrict__ dZ2,
                                 uint16_t* __restrict__ dZ2T, double* __restrict__ loss_parts) {
    const int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (b >= B) return;
    float acc = 0.f;
    for (int o = lane; o < h2; o += 32) acc += w3[o] * bf16_bits_to_f32(H2[(size_t)b * h2 + o]);
    acc = warp_sum(acc);
    const float r = acc + b3[0] - tb[b];
    const float dsb = r / (float)B;
    if (lane == 0) {
        ds[b] = dsb;
        loss_parts[b] = 0.5 * (double)r * (double)r / (double)B;
    }
    for (int o = lane; o < h2; o += 32) {
        const float g = dsb * w3[o] * gelu_grad_f(Z2[(size_t)b * h2 + o]);
        dZ2f[(size_t)b * h2 + o] = g;
        const uint16_t gb = f32_to_bf16_bits(g);
        dZ2[(size_t)b * h2 + o] = gb;
        dZ2T[(size_t)o * B + b] = gb;
    }
}

// dZ1 = dH1 * GELU'(Z1): FP32 (for the bias gradient) and BF16 transposed (for dW1)
__global__ void dz1_kernel(int B, int h1, const float* __restrict__ dH1, const float* __restrict__ Z1,
                           float* __restrict__ dZ1f, uint16_t* __restrict__ dZ1T) {
    const size_t n = (size_t)B * h1;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const int b = (int)(e / h1), i = (int)(e % h1);
        const float g = dH1[e] * gelu_grad_f(Z1[e]);
        dZ1f[e] = g;
        dZ1T[(size_t)i * B + b] = f32_to_bf16_bits(g);
    }
}

// Column sums out[c] = sum_b M[b][c] * (wrow ? wrow[b] : 1), c < cols, FP32, in two passes of fixed order.
// Pass 1: grid (ceil(cols / 32), COLSUM_CHUNKS), block 32 x 8: chunk y of the rows, warp w takes its rows
// w, w + 8, ... (lane = column, so every row is read coalesced); the 8 warp sums in warp order go to
// part[y cols + c]. Pass 2 adds the chunks' sums in chunk order.
constexpr int COLSUM_CHUNKS = 16;

template <typename MT>
__global__ void __launch_bounds__(256) colsum_part_kernel(int B, int cols, const MT* __restrict__ M,
                                                          const float* __restrict__ wrow, float* __restrict__ part) {
    __shared__ float red[8][33];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, c = blockIdx.x * 32 + lane, y = blockIdx.y;
    const int b0 = (int)((long long)B * y / gridDim.y), b1 = (int)((long long)B * (y + 1) / gridDim.y);
    float acc = 0.f;
    if (c < cols) {
        for (int b = b0 + w; b < b1; b += 8) {
            float v;
            if constexpr (sizeof(MT) == 2) v = bf16_bits_to_f32(M[(size_t)b * cols + c]);
            else v = M[(size_t)b * cols + c];
            acc += wrow ? v * wrow[b] : v;
        }
    }
    red[w][lane] = acc;
    __syncthreads();
    if (w == 0 && c < cols) {
        float s = 0.f;
#pragma unroll
        for (int k = 0; k < 8; ++k) s += red[k][lane];
        part[(size_t)y * cols + c] = s;
    }
}

__global__ void colsum_final_kernel(int cols, int chunks, const float* __restrict__ part, float* __restrict__ out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cols) return;
    float s = 0.f;
    for (int y = 0; y < chunks; ++y) s += part[(size_t)y * cols + c];
    out[c] = s;
}

// One Adam step (Kingma & Ba) on a parameter tensor of rows x cols with FP32 master weights; the gradient
// is g[r*cols + c] or, if g_t, g[c*ldg + r]. Writes the BF16 copies (row-major with ldq columns and/or
// transposed with ldqt columns) when given.
// c12, t_dev (optional, a training step replayed as a graph): the bias corrections of step s = t_dev[0] - t_dev[1] of
// the training at c12[2 s], c12[2 s + 1] instead of c1, c2.
__global__ void adam_kernel(int rows, int cols, float* __restrict__ th, const float* __restrict__ g, int g_t, int ldg,
                            float* __restrict__ m, float* __restrict__ v, float lr, float b1, float b2, float eps,
                            float c1, float c2, uint16_t* __restrict__ q, int ldq, uint16_t* __restrict__ qt, int ldqt,
                            const float* __restrict__ c12 = nullptr, const long long* __restrict__ t_dev = nullptr) {
    if (c12) {
        const long long st = t_dev[0] - t_dev[1];
        c1 = c12[2 * st];
        c2 = c12[2 * st + 1];
    }
    const size_t n = (size_t)rows * cols;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(e / cols), c = (int)(e % cols);
        const float gv = g_t ? g[(size_t)c * ldg + r] : g[e];
        const float mv = b1 * m[e] + (1.f - b1) * gv;
        const float vv = b2 * v[e] + (1.f - b2) * gv * gv;
        m[e] = mv;
        v[e] = vv;
        const float mh = mv / c1, vh = vv / c2;
        const float w = th[e] - lr * mh / (sqrtf(vh) + eps);
        th[e] = w;
        if (q) q[(size_t)r * ldq + c] = f32_to_bf16_bits(w);
        if (qt) qt[(size_t)c * ldqt + r] = f32_to_bf16_bits(w);
    }
}

// BF16 copies of FP32 weights (row-major with ldq columns and/or transposed)
__global__ void quant_weights_kernel(int rows, int cols, const float* __restrict__ th, uint16_t* __restrict__ q, int ldq,
                                     uint16_t* __restrict__ qt, int ldqt) {
    const size_t n = (size_t)rows * cols;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(e / cols), c = (int)(e % cols);
        const uint16_t h = f32_to_bf16_bits(th[e]);
        if (q) q[(size_t)r * ldq + c] = h;
        if (qt) qt[(size_t)c * ldqt + r] = h;
    }
}

// out[c*ldo + r] = in[r*ldi + c] (BF16), zero for rows <= r < ldo
__global__ void transpose_bf16_kernel(const uint16_t* __restrict__ in, int ldi, int rows, int cols,
                                      uint16_t* __restrict__ out, int ldo) {
    __shared__ uint16_t tile[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        int r = r0 + k, c = c0 + threadIdx.x;
        tile[k][threadIdx.x] = (r < rows && c < cols) ? in[(size_t)r * ldi + c] : (uint16_t)0;
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        int c = c0 + k, r = r0 + threadIdx.x;
        if (c < cols && r < ldo) out[(size_t)c * ldo + r] = tile[threadIdx.x][k];
    }
}

// Statistics of the ring's training slots' log pi (mu, var) and the feature scales 1/sqrt(C_ii).
__global__ void ring_lp_stats_kernel(const float* __restrict__ ring_lp, const DaCounters* cnt, double* out) {
    __shared__ double sh[32];
    const long long ntr = n_train_slots(cnt->filled);
    double s1 = 0.0, s2 = 0.0;
    for (long long j = threadIdx.x; j < ntr; j += blockDim.x) {
        const double v = ring_lp[train_slot(j)];
        s1 += v;
        s2 += v * v;
    }
    s1 = block_sum(s1, sh);
    s2 = block_sum(s2, sh);
    if (threadIdx.x == 0) {
        out[0] = s1;
        out[1] = s2;
        out[2] = (double)ntr;
    }
}

__global__ void feature_scale_kernel(int d, const double* __restrict__ M2, double inv_n, float* __restrict__ scale) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d) return;
    const double var = M2[(size_t)i * d + i] * inv_n;
    scale[i] = var > 0.0 ? (float)(1.0 / sqrt(var)) : 1.0f;
}

// squared error (nats) of the surrogate on rows of a batch: (mu + sigma out_b - lp_b)^2, summed in FP64
__global__ void sq_err_kernel(int rows, const double* __restrict__ s, const float* __restrict__ raw_lp,
                              double* __restrict__ out) {
    __shared__ double sh[32];
    double acc = 0.0;
    for (int r = threadIdx.x; r < rows; r += blockDim.x) {
        const double e = s[r] - (double)raw_lp[r];
        acc += e * e;
    }
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) out[0] += acc;
}

// The graph-replayed training step's counter: the next step.
__global__ void step_count_kernel(long long* t_dev) { t_dev[0] += 1; }

}  // namespace
}  // namespace diam
