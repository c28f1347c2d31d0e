// ops.cu -- op-level C entry points (include/diam_ops.h) over the sampler's kernels.
#include "../../include/diam_ops.h"
#include "linalg.h"
#include "step.cuh"
#include "tc_gemm.h"

using namespace diam;

namespace ops_detail {
__global__ void scale_to_dev_kernel(double* dst, double v) { *dst = v; }

// One small device block per device for the op-level status words and scale (never freed; 32 bytes).
struct OpScratch {
    int status;
    int info;
    double scale;
};
// Thread 0 spins until *flag == expected or limit SM clock cycles have passed; the outcome goes to *status.
__global__ void wait_flag_kernel(const volatile int* flag, int expected, long long limit, int* status) {
    const long long t0 = clock64();
    int st = DEV_OK;
    while (*flag != expected) {
        if (clock64() - t0 > limit) {
            st = DEV_TIMEOUT;
            break;
        }
    }
    *status = st;
}
}  // namespace ops_detail
using namespace ops_detail;

static OpScratch* op_scratch() {
    static OpScratch* per_dev[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    if (!per_dev[dev]) {
        OpScratch* p = nullptr;
        if (cudaMalloc(&p, sizeof(OpScratch)) != cudaSuccess) return nullptr;
        cudaMemset(p, 0, sizeof(OpScratch));
        per_dev[dev] = p;
    }
    return per_dev[dev];
}

extern "C" {

diam_status diam_op_normals(uint64_t seed, uint32_t problem_id, int64_t t0, int32_t n_steps, int32_t P, int32_t d,
                            int32_t ld, int32_t kind, void* out, void* stream) {
    if (!out || n_steps < 0 || P <= 0 || d <= 0 || ld < d || ld % 4 || kind < 0 || kind > 2) return DIAM_EINVAL;
    if (n_steps == 0) return DIAM_OK;
    cudaStream_t st = (cudaStream_t)stream;
    Key key = make_key(seed, problem_id);
    dim3 g((unsigned)((int64_t)n_steps * P), std::max(1, std::min(64, (ld / 4 + 127) / 128)));
    if (kind == 0) { gen_w_kernel<float><<<g, 128, 0, st>>>(key, t0, P, d, ld, (float*)out); count_launch(); }
    else if (kind == 1) { gen_w_kernel<double><<<g, 128, 0, st>>>(key, t0, P, d, ld, (double*)out); count_launch(); }
    else { gen_w_kernel<uint16_t><<<g, 128, 0, st>>>(key, t0, P, d, ld, (uint16_t*)out); count_launch(); }
    return cudaGetLastError() == cudaSuccess ? DIAM_OK : DIAM_ECUDA;
}

diam_status diam_op_wait_flag(const int32_t* flag, int32_t expected, int64_t limit_cycles, void* stream) {
    if (!flag || limit_cycles < 0 || limit_cycles > (1ll << 33)) return DIAM_EINVAL;
    OpScratch* sc = op_scratch();
    if (!sc) return DIAM_ECUDA;
    cudaStream_t st = (cudaStream_t)stream;
    { wait_flag_kernel<<<1, 1, 0, st>>>(flag, expected, (long long)limit_cycles, &sc->status); count_launch(); }
    if (cudaGetLastError() != cudaSuccess) return DIAM_ECUDA;
    int status = 0;
    if (cudaMemcpyAsync(&status, &sc->status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return DIAM_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return DIAM_ECUDA;
    return status == DEV_TIMEOUT ? DIAM_ETIMEOUT : DIAM_OK;
}

diam_status diam_op_cholesky_f64(int32_t n, double* A, int32_t lda, int32_t* info_host, void* stream) {
    if (!A || n <= 0 || lda < n || !info_host) return DIAM_EINVAL;
    OpScratch* sc = op_scratch();
    if (!sc) return DIAM_ECUDA;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(&sc->info, 0, sizeof(int), st) != cudaSuccess) return DIAM_ECUDA;
    if (cholesky_f64(A, n, lda, &sc->info, st) != cudaSuccess) return DIAM_ECUDA;
    if (cudaMemcpyAsync(info_host, &sc->info, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return DIAM_ECUDA;
    return cudaStreamSynchronize(st) == cudaSuccess ? DIAM_OK : DIAM_ECUDA;
}

// Workspace of the tensor-core (Ozaki-split) updates for one op call, freed on scope exit.
struct OzScope {
    OzakiWs ws;
    bool ok = true;
    // rows: the factor's order; rows2 > 0: also the workspace of a triangular solve with rows2 right-hand sides
    OzScope(int rows, int rows2) {
        ws.cap_rows = rows;
        ws.cap2 = rows2;
        ws.capP = rows2 > 0 ? ozaki_panel_rows(rows) : 0;
        ok = cudaMalloc(&ws.SL, ozaki_sl_bytes(rows)) == cudaSuccess &&
             cudaMalloc(&ws.ex, ozaki_ex_bytes(rows)) == cudaSuccess &&
             (rows2 == 0 || (cudaMalloc(&ws.SL2, ozaki_sl_bytes(rows2)) == cudaSuccess &&
                             cudaMalloc(&ws.ex2, ozaki_ex_bytes(rows2)) == cudaSuccess &&
                             cudaMalloc(&ws.SLP, sizeof(uint16_t) * (size_t)std::max<int64_t>(1, ws.capP) * 448) == cudaSuccess &&
                             cudaMalloc(&ws.exP, sizeof(int) * (size_t)std::max<int64_t>(1, ws.capP)) == cudaSuccess));
    }
    ~OzScope() {
        ozaki_ws_release(ws);
        cudaFree(ws.SL);
        cudaFree(ws.ex);
        cudaFree(ws.SL2);
        cudaFree(ws.ex2);
        cudaFree(ws.SLP);
        cudaFree(ws.exP);
    }
};

diam_status diam_op_cholesky_f64_tc(int32_t n, double* A, int32_t lda, int32_t* info_host, void* stream) {
    if (!A || n <= 0 || lda < n || !info_host) return DIAM_EINVAL;
    OpScratch* sc = op_scratch();
    if (!sc) return DIAM_ECUDA;
    cudaStream_t st = (cudaStream_t)stream;
    OzScope oz(n, 0);
    if (!oz.ok) return DIAM_ENOMEM;
    diam_status r = DIAM_OK;
    if (cudaMemsetAsync(&sc->info, 0, sizeof(int), st) != cudaSuccess ||
        cudaMemsetAsync(&sc->status, 0, sizeof(int), st) != cudaSuccess ||
        cholesky_f64(A, n, lda, &sc->info, st, &oz.ws, &sc->status) != cudaSuccess)
        r = DIAM_ECUDA;
    int status = 0;
    if (r == DIAM_OK && (cudaMemcpyAsync(info_host, &sc->info, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                         cudaMemcpyAsync(&status, &sc->status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess))
        r = DIAM_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) r = DIAM_ECUDA;
    if (r == DIAM_OK && status == DEV_TIMEOUT) r = DIAM_ETIMEOUT;
    return r;
}

diam_status diam_op_trsm_lower_f64(int32_t n, int32_t nrows, const double* L, int32_t ldl, double* B, int32_t ldb,
                                   void* stream) {
    if (!L || !B || n <= 0 || nrows < 0 || ldl < n || ldb < n) return DIAM_EINVAL;
    return trsm_lower_f64(L, ldl, n, B, ldb, nrows, (cudaStream_t)stream) == cudaSuccess ? DIAM_OK : DIAM_ECUDA;
}

diam_status diam_op_trsm_lower_f64_tc(int32_t n, int32_t nrows, const double* L, int32_t ldl, double* B, int32_t ldb,
                                      void* stream) {
    if (!L || !B || n <= 0 || nrows < 0 || ldl < n || ldb < n) return DIAM_EINVAL;
    if (nrows == 0) return DIAM_OK;
    OpScratch* sc = op_scratch();
    if (!sc) return DIAM_ECUDA;
    cudaStream_t st = (cudaStream_t)stream;
    OzScope oz(n, nrows);
    if (!oz.ok) return DIAM_ENOMEM;
    diam_status r = DIAM_OK;
    int status = 0;
    if (cudaMemsetAsync(&sc->status, 0, sizeof(int), st) != cudaSuccess ||
        trsm_lower_f64(L, ldl, n, B, ldb, nrows, st, &oz.ws, &sc->status) != cudaSuccess ||
        cudaMemcpyAsync(&status, &sc->status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        r = DIAM_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) r = DIAM_ECUDA;
    if (r == DIAM_OK && status == DEV_TIMEOUT) r = DIAM_ETIMEOUT;
    return r;
}

diam_status diam_op_gemm_bf16_tile(int32_t M, int32_t N, int32_t K, const uint16_t* A, int32_t lda,
                                   const uint16_t* B, const uint16_t* B2, int32_t ldb, int32_t a_lower, float scale,
                                   float* D, int32_t ldd, int32_t bn, void* stream) {
    if (bn != 32 && bn != 64 && bn != 128 && bn != 256) return DIAM_EINVAL;
    if (!A || !B || !D || M <= 0 || N <= 0 || K <= 0 || K % 64 || lda % 64 || ldb % 64 || K > lda || K > ldb ||
        ldd < M)
        return DIAM_EINVAL;
    if (((uintptr_t)A | (uintptr_t)B | (uintptr_t)B2) & 15) return DIAM_EINVAL;
    OpScratch* sc = op_scratch();
    if (!sc) return DIAM_ECUDA;
    cudaStream_t st = (cudaStream_t)stream;
    cudaMemsetAsync(&sc->status, 0, sizeof(int), st);
    { scale_to_dev_kernel<<<1, 1, 0, st>>>(&sc->scale, (double)scale); count_launch(); }
    TcEpi epi{};
    epi.mode = TC_STORE;
    epi.D = D;
    epi.ldd = ldd;
    epi.scale_dev = &sc->scale;
    if (tc_gemm_bf16(M, N, K, A, lda, B, B2, ldb, a_lower, epi, &sc->status, st, bn) != cudaSuccess) return DIAM_ECUDA;
    int status = 0;
    if (cudaMemcpyAsync(&status, &sc->status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return DIAM_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return DIAM_ECUDA;
    return status == DEV_TIMEOUT ? DIAM_ETIMEOUT : DIAM_OK;
}

diam_status diam_op_gemm_bf16(int32_t M, int32_t N, int32_t K, const uint16_t* A, int32_t lda, const uint16_t* B,
                              const uint16_t* B2, int32_t ldb, int32_t a_lower, float scale, float* D, int32_t ldd,
                              void* stream) {
    return diam_op_gemm_bf16_tile(M, N, K, A, lda, B, B2, ldb, a_lower, scale, D, ldd, 128, stream);
}

}  // extern "C"
