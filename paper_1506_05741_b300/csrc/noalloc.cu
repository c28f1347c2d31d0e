// noalloc.cu -- diam_op_gemm_bf16_noalloc: the tensor-core GEMM of diam_op_gemm_bf16 for callers that
// cannot allocate device memory.
//
// Who needs it: code that must not call cudaMalloc at all -- for example a host runtime whose device
// memory is owned by its own pool and forbids outside allocations, or code on a latency-critical path that
// cannot afford the device-wide synchronisation cudaMalloc and cudaFree may cause. diam_op_gemm_bf16
// allocates a small per-device scratch block on its first call; this variant never allocates.
//
// Scratch: one file-scope device array (kScratchBytes, 16 MiB, per GPU that loads the library, held until
// the process exits) holds the FP32 split-K partial products, the status word and the scale. In host code
// the array's name is only a host-side stand-in; the device address is fetched with cudaGetSymbolAddress
// once per device, with that device current, on the first call made on that device. Make that first call
// outside any stream capture.
//
// Every call shares the array and the array keeps the previous call's contents: the partials are fully
// overwritten by each call and the status word is cleared at the start of each call. Calls whose work
// overlaps on the GPU (different streams, or different host threads on the same device) race on the
// array and must be serialised by the caller.
#include <algorithm>
#include <mutex>

#include "../../include/diam_ops.h"
#include "common.cuh"
#include "tc_gemm.h"

using namespace diam;

namespace noalloc_detail {

constexpr size_t kScratchBytes = 16u << 20;   // 16 MiB
constexpr size_t kHeadBytes = 256;            // status word and scale at the start
constexpr size_t kPartialFloats = (kScratchBytes - kHeadBytes) / sizeof(float);
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

struct Head {
    int status;
    int pad;
    double scale_one;
};

__global__ void prep_kernel(Head* h) {
    h->status = 0;
    h->scale_one = 1.0;
}

constexpr int kMaxSplits = 4;
struct SplitRows {
    int m0[kMaxSplits];   // split s wrote rows m >= m0[s] of its plane (a lower-triangular A: rows above get nothing)
};

// D[n*ldd + m] = scale * sum_s part[s][n][m] over the splits that wrote row m, summed in a fixed order
__global__ void reduce_kernel(int M, int N, int S, const float* __restrict__ part, SplitRows rows, float scale,
                              float* __restrict__ D, int ldd) {
    const size_t plane = (size_t)M * N;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < plane; idx += (size_t)gridDim.x * blockDim.x) {
        const size_t n = idx / M, m = idx % M;
        float acc = 0.f;
        for (int s = 0; s < S; ++s)
            if ((int)m >= rows.m0[s]) acc += part[s * plane + idx];
        D[n * ldd + m] = scale * acc;
    }
}

// Device address of g_scratch on the current device (set up on the first call on that device).
static unsigned char* scratch_address() {
    static std::mutex mu;
    static unsigned char* addr[kMaxDevices] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
    std::lock_guard<std::mutex> g(mu);
    if (!addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess) return nullptr;
        addr[dev] = (unsigned char*)p;
    }
    return addr[dev];
}

}  // namespace noalloc_detail

extern "C" diam_status diam_op_gemm_bf16_noalloc(int32_t M, int32_t N, int32_t K, const uint16_t* A, int32_t lda,
                                                 const uint16_t* B, const uint16_t* B2, int32_t ldb, int32_t a_lower,
                                                 float scale, float* D, int32_t ldd, void* stream) {
    using namespace noalloc_detail;
    if (!A || !B || !D || M <= 0 || N <= 0 || K <= 0 || K % 64 || lda % 64 || ldb % 64 || K > lda || K > ldb ||
        ldd < M)
        return DIAM_EINVAL;
    if (((uintptr_t)A | (uintptr_t)B | (uintptr_t)B2) & 15) return DIAM_EINVAL;
    const size_t plane = (size_t)M * N;
    if (plane > kPartialFloats) return DIAM_EINVAL;   // M * N beyond the fixed scratch (about 4.2 M floats)
    unsigned char* base = scratch_address();
    if (!base) return DIAM_ECUDA;
    cudaStream_t st = (cudaStream_t)stream;
    Head* head = (Head*)base;
    float* part = (float*)(base + kHeadBytes);
    // as many K splits (of whole 64-wide blocks) as the scratch holds, at most kMaxSplits
    const int kblocks = K / 64;
    int S = (int)std::min<size_t>(std::min<size_t>(kMaxSplits, (size_t)kblocks), kPartialFloats / plane);
    const int per = (kblocks + S - 1) / S;
    { prep_kernel<<<1, 1, 0, st>>>(head); count_launch(); }
    int used = 0;
    SplitRows rows{};
    for (int s = 0; s < S; ++s) {
        const int kb0 = s * per, kb1 = std::min(kblocks, kb0 + per);
        if (kb0 >= kb1) break;
        // split s reads K columns [64 kb0, 64 kb1) through offset operands. With a lower-triangular A (zero
        // strict upper part), rows m < 64 kb0 get nothing from these columns and the rows from 64 kb0 on form a
        // lower-triangular block again in the split's own frame: the split covers those rows only, with the
        // triangular K skip, and the reduction leaves its plane's upper rows out
        const int m0 = a_lower ? 64 * kb0 : 0;
        if (m0 >= M) break;
        TcEpi epi{};
        epi.mode = TC_STORE;
        epi.D = part + (size_t)used * plane + m0;
        epi.ldd = M;
        epi.scale_dev = &head->scale_one;
        if (tc_gemm_bf16(M - m0, N, (kb1 - kb0) * 64, A + (size_t)m0 * lda + (size_t)kb0 * 64, lda, B + (size_t)kb0 * 64,
                         B2 ? B2 + (size_t)kb0 * 64 : nullptr, ldb, a_lower ? 1 : 0, epi, &head->status, st) != cudaSuccess)
            return DIAM_ECUDA;
        rows.m0[used] = m0;
        ++used;
    }
    { reduce_kernel<<<(unsigned)std::min<size_t>(148 * 16, (plane + 255) / 256), 256, 0, st>>>(M, N, used, part, rows, scale, D, ldd); count_launch(); }
    if (cudaGetLastError() != cudaSuccess) return DIAM_ECUDA;
    int status = 0;
    if (cudaMemcpyAsync(&status, &head->status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return DIAM_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return DIAM_ECUDA;
    return status == DEV_TIMEOUT ? DIAM_ETIMEOUT : DIAM_OK;
}
