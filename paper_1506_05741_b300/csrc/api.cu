// api.cu -- the C ABI of include/diam.h: one sampler context, its device buffers and the host-side
// schedule of Algorithm 1 (arXiv 1506.05741) over P concurrent chains with one pooled factor.
//
// Per step (all chains at once): propose (eq. (diamnl), with the z recursion for the proposal density),
// the target's linear map when it has one (a GEMM with a reducing epilogue), then accept / select /
// record. Per interval of n_lag steps: fold the recorded samples into the pooled FP64 moments (eq.
// (sampmean), (sampcov), as a pairwise centred update), apply Algorithm 1's beta rule, and when due
// factor C_n by FP64 Cholesky; the factor is used from interval k + 1 + refresh_delay on, when the
// whitened states z are recomputed by a triangular solve. The noise products of an interval are one
// batched triangular GEMM (Algorithm 1, "Batch update").
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/diam.h"
#include "gemm_f64.cuh"
#include "linalg.h"
#include "step.cuh"
#include "rec.cuh"
#include "rewhiten.h"
#include "tc_gemm.h"

using namespace diam;

namespace diam {
static std::atomic<unsigned long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1ull, std::memory_order_relaxed); }
}  // namespace diam

namespace {

constexpr int kThreads = 256;
constexpr int TSPLIT_MAX = 8;   // split planes of the target product's K

struct Pending {
    double* L = nullptr;
    double* mean = nullptr;
    int64_t block = -1;
};

}  // namespace

struct DaState;

struct diam_ctx {
    diam_config cfg{};
    DaState* da = nullptr;   // delayed-acceptance surrogate (diam_da_enable)
    int kind = 0, d = 0, P = 0, nl = 0, dy = 0, ldk = 0;
    bool bf = false;
    int dev = 0;
    cudaStream_t st = nullptr;
    bool own_stream = false;
    cudaStream_t side = nullptr;                 // overlaps the interval's noise product with the re-solve
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // pinned staging of large host <-> device copies (two halves, allocated on the first large copy)
    char* stage = nullptr;
    cudaEvent_t stage_ev[2] = {nullptr, nullptr};
    bool stage_failed = false;
    // the refresh's factorisation and the re-solve of z, captured once (fixed buffers) and replayed
    struct Captured {
        cudaGraphExec_t exec = nullptr;
        unsigned long long launches = 0;
    } chol_graph, trsm_graph;
    // refreshes beside the following intervals (BF16 mode, graphs, refresh_delay >= 1): the factorisation of
    // interval k's C_n runs on a stream and workspaces of its own while the next intervals step, and is
    // resolved at the end of interval k + min(delay, 2); with delay >= 2 two of them can be in flight
    struct AsyncRefresh {
        cudaStream_t rs = nullptr;
        cudaEvent_t fork = nullptr, start = nullptr, done = nullptr;   // start / done: timed
        OzakiWs oz;
        double *Cr = nullptr, *M2s = nullptr;   // its matrix; the moments it was built from (for retries)
        int* info = nullptr;                    // its failing pivot + 1, then its own status word (device, 2 ints):
                                                // a device-side timeout in it is reported when it is resolved
        Captured graph;
        bool active = false;
        int64_t blk = 0, n = 0;
        double eps = 0;
    } ar[2];
    int n_ar = 0;   // slots in use (0: refreshes run between the intervals)
    std::string err;
    bool bad = false;
    diam_logpi_fn fn = nullptr;
    void* user = nullptr;
    // interval-end hook (diam_set_interval_hook) and the moments at the last synchronisation (increments)
    diam_interval_fn hook = nullptr;
    void* hook_user = nullptr;
    bool in_hook = false;
    double *snap_mean = nullptr, *snap_M2 = nullptr;
    int64_t snap_n = 0;
    double sigma = 0, ban_a = 0, ban_b = 0, ban_c = 0;
    Key key{};

    // host mirrors of the schedule
    int64_t t = 0, n = 0, acc_refresh = 0, acc_all = 0, refreshes = 0, notspd = 0, chol_attempts = 0;
    uint64_t nonfinite = 0;
    double beta = 0;
    int64_t xi_block = -1, begun_block = -1;
    std::vector<Pending> pend;

    std::vector<void*> allocs;
    Ctl* ctl = nullptr;
    // chain state (T = double in FP64 mode, float in BF16 mode)
    void *X = nullptr, *Z = nullptr, *Xp = nullptr, *Zp = nullptr, *xref = nullptr, *cenT = nullptr, *Xi = nullptr;
    double *lp = nullptr, *q = nullptr, *qp = nullptr, *lpo = nullptr, *lpp = nullptr, *partial = nullptr;
    double *xref64 = nullptr, *L = nullptr, *Lq64 = nullptr, *mean = nullptr, *M2 = nullptr, *cen64 = nullptr;
    double *colpart = nullptr, *svec = nullptr, *delta = nullptr, *Cw = nullptr, *work = nullptr;
    uint16_t *Lq16 = nullptr, *op_hi = nullptr, *op_lo = nullptr, *op_lo2 = nullptr, *histT = nullptr;
    double *qpart = nullptr, *lpart = nullptr, *s16 = nullptr;   // per-chunk proposal sums; BF16 record sums
    int8_t* accf = nullptr;                                      // per-chain decision of the current step
    float* ws = nullptr;                                         // split-K partial target products (BF16 mode)
    int nchunk = 1, tsplit = 1;
    int bn_target = 128, bn_xi = 128;        // tile widths picked by the autotuner (BF16 mode)
    OzakiWs oz;                              // BF16 mode: the refresh's trailing updates on the tensor cores
    // CUDA graph of one interval's n_lag steps (captured once; embeds buffer pointers and the DA switch)
    cudaGraphExec_t graph = nullptr;
    const void* graph_bsum = nullptr;
    int graph_da = -1;
    unsigned long long graph_launches = 0;   // kernel launches inside one replay
    void *W = nullptr, *hist = nullptr;
    int ldw = 0, ldh = 0, nparts = 0;
    // target
    double *inv_lam = nullptr, *Gm = nullptr, *y = nullptr;
    double *tw_ilam = nullptr, *tw_c = nullptr, *ubuf = nullptr;   // twisted target: 1 / lambda_j, c_j; u = G x (FP64)
    float *inv_lam32 = nullptr, *y32 = nullptr;   // FP32 copies for the BF16-mode kernels
    float* psum = nullptr;   // per-tile sums of the interval's records (BF16 mode fold): 2 x tiles x d
    // the linear map carried through the proposal (BF16 mode, linear-map targets): M = A Lq as BF16 hi + lo,
    // A x of the states and of the proposals, A x_ref, the interval's products M W (scaled by beta alpha)
    bool rec = false, ax_dirty = true;
    uint16_t *Lt16 = nullptr, *ALh = nullptr, *ALl = nullptr;
    uint16_t *Lq16lo = nullptr, *Lt16lo = nullptr;   // the TF32 factor's second BF16 term (prec DIAM_FP32)
    bool tf32 = false;                              // prec DIAM_FP32: the factor quantised to TF32
    float *ALf = nullptr, *AXi = nullptr, *Ax = nullptr, *Axp = nullptr, *axref = nullptr;
    double* lmap = nullptr;
    uint16_t* Gq16 = nullptr;
    TargetDev tg{};
    // trace and interval sums
    TraceDev tr{};
    void* bsum = nullptr;   // per-interval, per-chain sums of x: FP64 (FP32 in BF16 mode)
    void* bm2 = nullptr;    // and of x^2 (FP64 mode) / the scatter about the interval mean (BF16 mode)
    double* lpsum = nullptr;
    int64_t bcap = 0;
    double* psrf_ws = nullptr;   // 2 x P x d: per-chain means and variances of a PSRF window
    // phase profiler (cfg.profile): event pairs recorded on the stream, read back at synchronisation points
    struct Evt {
        cudaEvent_t a, b;
        int phase;
    };
    std::vector<Evt> evts;
    size_t evt_used = 0;
    int64_t prof_cnt[DIAM_N_PHASES] = {};
    double prof_ms[DIAM_N_PHASES] = {};
};

enum : int { PH_NOISE = 0, PH_XI = 1, PH_PROPOSE = 2, PH_TARGET = 3, PH_ACCEPT = 4, PH_FOLD = 5, PH_REFRESH = 6,
             PH_REWHITEN = 7, PH_SCREEN = 8, PH_TRAIN = 9, PH_STEP = 10, PH_SYRK = 11 };

// Start timing a phase; returns the event slot (or -1 when profiling is off).
static int ph_begin(diam_ctx* c, int phase) {
    if (!c->cfg.profile) return -1;
    if (c->evt_used == c->evts.size()) {
        diam_ctx::Evt e{};
        if (cudaEventCreate(&e.a) != cudaSuccess || cudaEventCreate(&e.b) != cudaSuccess) return -1;
        c->evts.push_back(e);
    }
    int i = (int)c->evt_used++;
    c->evts[i].phase = phase;
    cudaEventRecord(c->evts[i].a, c->st);
    return i;
}

static void ph_end(diam_ctx* c, int i) {
    if (i >= 0) cudaEventRecord(c->evts[i].b, c->st);
}

// Accumulate the recorded pairs (the stream must be synchronised).
static void prof_flush(diam_ctx* c) {
    for (size_t i = 0; i < c->evt_used; ++i) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, c->evts[i].a, c->evts[i].b) == cudaSuccess) {
            c->prof_ms[c->evts[i].phase] += ms;
            c->prof_cnt[c->evts[i].phase] += 1;
        }
    }
    c->evt_used = 0;
}

// ------------------------------------------------------------------------------------------------ helpers
#define CK(expr)                                                                  \
    do {                                                                          \
        cudaError_t e_ = (expr);                                                  \
        if (e_ != cudaSuccess) return fail(c, DIAM_ECUDA, #expr, cudaGetErrorString(e_)); \
    } while (0)

#define CKS(expr)                        \
    do {                                 \
        diam_status s_ = (expr);         \
        if (s_ != DIAM_OK) return s_;    \
    } while (0)

static diam_status fail(diam_ctx* c, diam_status s, const char* what, const char* why = nullptr) {
    if (c) {
        c->err = std::string(what) + (why ? std::string(": ") + why : std::string());
        if (s != DIAM_ENOTSPD && s != DIAM_EINVAL) c->bad = true;
    }
    return s;
}

// Host <-> device copies ordered on the context's stream (which does not synchronise with the legacy default
// stream). A host-to-device copy from pageable memory is staged before the call returns; a device-to-host
// copy is waited for.
// Host <-> device copies on the context's stream. Copies of at least one stage half go through a pinned
// staging buffer of two halves, so the DMA of one chunk overlaps the host copy of the next (a copy from or
// to pageable memory runs at a fraction of the link's rate); smaller ones, or all of them if the pinned
// buffer cannot be had, are plain copies. h2d returns once the caller's buffer has been read.
constexpr size_t kStageHalf = (size_t)4 << 20;

static bool ensure_stage(diam_ctx* c) {
    if (c->stage) return true;
    if (c->stage_failed) return false;
    void* p = nullptr;
    if (cudaHostAlloc(&p, 2 * kStageHalf, cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        c->stage_failed = true;
        return false;
    }
    if (cudaEventCreateWithFlags(&c->stage_ev[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->stage_ev[1], cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        for (cudaEvent_t& e : c->stage_ev)
            if (e) cudaEventDestroy(e), e = nullptr;
        cudaFreeHost(p);
        c->stage_failed = true;
        return false;
    }
    c->stage = (char*)p;
    return true;
}

static cudaError_t h2d(diam_ctx* c, void* dst, const void* src, size_t n) {
    if (n < kStageHalf || !ensure_stage(c)) return cudaMemcpyAsync(dst, src, n, cudaMemcpyHostToDevice, c->st);
    char* d = (char*)dst;
    const char* s = (const char*)src;
    for (size_t i = 0, o = 0; o < n; ++i, o += kStageHalf) {
        const int b = (int)(i & 1);
        const size_t l = std::min(kStageHalf, n - o);
        cudaError_t e = cudaEventSynchronize(c->stage_ev[b]);   // the last copy out of this half has finished
        if (e != cudaSuccess) return e;
        memcpy(c->stage + b * kStageHalf, s + o, l);
        if ((e = cudaMemcpyAsync(d + o, c->stage + b * kStageHalf, l, cudaMemcpyHostToDevice, c->st)) != cudaSuccess ||
            (e = cudaEventRecord(c->stage_ev[b], c->st)) != cudaSuccess)
            return e;
    }
    return cudaSuccess;
}

static cudaError_t d2h(diam_ctx* c, void* dst, const void* src, size_t n) {
    if (n < kStageHalf || !ensure_stage(c)) {
        cudaError_t e = cudaMemcpyAsync(dst, src, n, cudaMemcpyDeviceToHost, c->st);
        return e == cudaSuccess ? cudaStreamSynchronize(c->st) : e;
    }
    char* d = (char*)dst;
    const char* s = (const char*)src;
    const size_t chunks = (n + kStageHalf - 1) / kStageHalf;
    cudaError_t e = cudaSuccess;
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) e = cudaEventSynchronize(c->stage_ev[b]);   // earlier uploads
    for (size_t i = 0; i <= chunks && e == cudaSuccess; ++i) {
        if (i < chunks) {   // chunk i into half i % 2 (chunk i - 2, its last contents, was copied out already)
            const size_t o = i * kStageHalf, l = std::min(kStageHalf, n - o);
            e = cudaMemcpyAsync(c->stage + (i & 1) * kStageHalf, s + o, l, cudaMemcpyDeviceToHost, c->st);
            if (e == cudaSuccess) e = cudaEventRecord(c->stage_ev[i & 1], c->st);
        }
        if (i > 0 && e == cudaSuccess) {   // chunk i - 1 has landed: out of the stage while chunk i is in flight
            const size_t o = (i - 1) * kStageHalf, l = std::min(kStageHalf, n - o);
            e = cudaEventSynchronize(c->stage_ev[(i - 1) & 1]);
            if (e == cudaSuccess) memcpy(d + o, c->stage + ((i - 1) & 1) * kStageHalf, l);
        }
    }
    return e;
}

template <typename P_>
static diam_status dalloc(diam_ctx* c, P_** p, size_t bytes) {
    void* v = nullptr;
    if (bytes == 0) bytes = 16;
    if (cudaMalloc(&v, bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(c, DIAM_ENOMEM, "cudaMalloc", "out of device memory");
    }
    c->allocs.push_back(v);
    if (cudaMemsetAsync(v, 0, bytes, c->st) != cudaSuccess) return fail(c, DIAM_ECUDA, "cudaMemset");
    *p = (P_*)v;
    return DIAM_OK;
}

static inline unsigned blocks_for(size_t n, int th = kThreads) { return (unsigned)((n + th - 1) / th); }
// Weight 1 / alpha^2 of the proposal-density quadratic q in the test; 0 for the random-walk proposal of eq. (rw),
// whose density is symmetric (q drops out of log a).
static inline double inv_infl2(const diam_ctx* c) {
    return c->cfg.proposal == DIAM_PROP_RW ? 0.0 : 1.0 / (c->cfg.infl * c->cfg.infl);
}
static inline bool is_rw(const diam_ctx* c) { return c->cfg.proposal == DIAM_PROP_RW; }

static diam_status check_usable(diam_ctx* c) {
    if (!c) return DIAM_ESTATE;
    if (c->bad) return DIAM_ESTATE;
    if (cudaSetDevice(c->dev) != cudaSuccess) return fail(c, DIAM_ECUDA, "cudaSetDevice");
    return DIAM_OK;
}

static diam_status sync_and_check(diam_ctx* c) {
    CK(cudaStreamSynchronize(c->st));
    int stt = 0;
    CK(d2h(c, &stt, &c->ctl->status, sizeof(int)));
    if (stt == DEV_TIMEOUT) return fail(c, DIAM_ETIMEOUT, "device", "a bounded wait inside a kernel expired");
    if (stt != 0) return fail(c, DIAM_ECUDA, "device", "kernel reported a bad argument");
    return DIAM_OK;
}

// ------------------------------------------------------------------------------------------------ pieces
template <typename T>
static diam_status linear_target(diam_ctx* c, const T* src) {
    // the target's linear map over all P chains, reduced to one partial per (m-tile, chain)
    if (c->kind != TK_DENSE && c->kind != TK_TANH) return DIAM_OK;
    if (!c->bf) {
        EpiTargetReduce epi{c->partial, c->y, 1.0 / (2.0 * c->sigma * c->sigma), c->kind == TK_TANH};
        CK((gemm_f64<true, true>(c->dy, c->P, c->d, c->Gm, c->d, (const double*)src, c->d, TileRange{0, 0}, epi, c->st)));
    } else {
        TcEpi epi{};
        epi.mode = TC_TARGET;
        epi.partial = c->partial;
        epi.y = c->y;
        epi.inv2s2 = 1.0 / (2.0 * c->sigma * c->sigma);
        epi.tanh_mode = c->kind == TK_TANH;
        CK(tc_gemm_bf16(c->dy, c->P, c->ldk, c->Gq16, c->ldk, c->op_hi, c->op_lo, c->ldk, 0, epi, &c->ctl->status, c->st));
    }
    return DIAM_OK;
}

// log pi of every chain of a state buffer (T), into out (P doubles)
template <typename T>
static diam_status eval_lp(diam_ctx* c, const T* src, double* out) {
    const int d = c->d, P = c->P;
    if (c->kind == TK_REF) {
        { diff_kernel<T><<<dim3(blocks_for(d), P), kThreads, 0, c->st>>>(d, src, (const T*)c->xref, c->work); count_launch(); }
        CK(trsm_lower_f64(c->Lq64, d, d, c->work, d, P, c->st, c->bf ? &c->oz : nullptr, &c->ctl->status));
        { set_z_kernel<T><<<P, kThreads, 0, c->st>>>(d, c->work, (T*)nullptr, nullptr, inv_infl2(c), out); count_launch(); }
        return DIAM_OK;
    }
    if (c->kind == TK_CALLBACK) {
        diam_status s = c->fn(c->user, src, d, P, c->cfg.prec, out, (void*)c->st);
        if (s != DIAM_OK) return fail(c, DIAM_ETARGET, "target callback");
        return DIAM_OK;
    }
    if (c->kind == TK_TWIST) {   // u = G x (every chain) in FP64, then the twisted terms in FP64. The twist's
                                 // coefficients (up to 1 / (sqrt(d) lambda)) amplify any error in u, and the
                                 // twisted targets of Sec. 3.1 are test targets of modest d: in BF16 mode the FP32
                                 // states are widened and multiplied by the BF16-rounded map in FP64
        const double* xs = (const double*)src;
        if (c->bf) {
            const size_t n = (size_t)P * d;
            { convert_kernel<T, double><<<(unsigned)std::min<size_t>(148 * 8, blocks_for(n)), kThreads, 0, c->st>>>(n, src, c->work); count_launch(); }
            xs = c->work;
        }
        EpiStore epi{c->ubuf, c->dy, 1.0, nullptr, 0.0};
        CK((gemm_f64<true, true>(c->dy, P, d, c->Gm, d, xs, d, TileRange{0, 0}, epi, c->st)));
        { twisted_lp_kernel<double><<<P, kThreads, 0, c->st>>>(c->dy, c->ubuf, c->dy, c->tw_ilam, c->tw_c, out); count_launch(); }
        CK(cudaGetLastError());
        return DIAM_OK;
    }
    { od_terms_kernel<T><<<P, kThreads, 0, c->st>>>(d, src, c->lpo, c->tg, c->bf ? c->op_hi : nullptr,
                                                  c->bf ? c->op_lo : nullptr, c->ldk); count_launch(); }
    CKS(linear_target<T>(c, src));
    int np = (c->kind == TK_DENSE || c->kind == TK_TANH) ? c->nparts : 0;
    { sum_lp_kernel<<<blocks_for(P), kThreads, 0, c->st>>>(P, c->lpo, c->partial, np, nullptr, out); count_launch(); }
    CK(cudaGetLastError());
    return DIAM_OK;
}

#include "da_host.cuh"

// z = Lq^{-1}(x - x_ref) and q for every chain (after a factor change); lp = -q for the reference target.
// BF16 mode: chains per CTA of the FP32 re-whitening (its right-hand sides in shared memory).
static int rewhiten32_group(int d) {
    for (int g = RW_G; g > 1; g /= 2)
        if (rewhiten32_smem(d, g) <= 220 * 1024) return g;
    return 1;
}

template <typename T>
static diam_status rewhiten(diam_ctx* c) {
    const int d = c->d, P = c->P;
    int e0 = ph_begin(c, PH_REWHITEN);
    if (c->bf && !c->tf32 && rewhiten_tc_fits(d, c->ldk)) {   // FP32 forward substitution, panel updates on the tensor cores
        CK(rewhiten_tc(d, P, c->Lq16, c->ldk, (const float*)c->X, (const float*)c->xref, (float*)c->Z, c->q, inv_infl2(c),
                       c->kind == TK_REF ? c->lp : nullptr, &c->ctl->status, c->st));
        ph_end(c, e0);
        return DIAM_OK;
    }
    if (c->bf && !c->tf32 && rewhiten32_smem(d, 1) <= 220 * 1024) {   // FP32 forward substitution (q to about 1e-6 of the FP64 solve)
        const int G = rewhiten32_group(d);
        { rewhiten32_kernel<<<(P + G - 1) / G, RW_THREADS, rewhiten32_smem(d, G), c->st>>>(
              d, P, G, c->Lq16, c->ldk, (const float*)c->X, (const float*)c->xref, (float*)c->Z, c->q, inv_infl2(c),
              c->kind == TK_REF ? c->lp : nullptr); count_launch(); }
        CK(cudaGetLastError());
        ph_end(c, e0);
        return DIAM_OK;
    }
    auto body = [&]() -> cudaError_t {
        { diff_kernel<T><<<dim3(blocks_for(d), P), kThreads, 0, c->st>>>(d, (const T*)c->X, (const T*)c->xref, c->work); count_launch(); }
        cudaError_t e = trsm_lower_f64(c->Lq64, d, d, c->work, d, P, c->st, c->bf ? &c->oz : nullptr, &c->ctl->status);
        if (e != cudaSuccess) return e;
        { set_z_kernel<T><<<P, kThreads, 0, c->st>>>(d, c->work, (T*)c->Z, c->q, inv_infl2(c),
                                                    c->kind == TK_REF ? c->lp : nullptr); count_launch(); }
        return cudaGetLastError();
    };
    if (c->bf && c->cfg.graphs && !c->cfg.profile && c->oz.hi) {   // after a first eager re-solve
        CKS(run_captured(c, c->trsm_graph, body));
    } else {
        CK(body());
    }
    ph_end(c, e0);
    return DIAM_OK;
}

static void set_xref_from(diam_ctx* c, const double* src_dev) {
    if (c->bf) {
        { convert_kernel<double, float><<<blocks_for(c->d), kThreads, 0, c->st>>>(c->d, src_dev, (float*)c->xref); count_launch(); }
        { convert_kernel<float, double><<<blocks_for(c->d), kThreads, 0, c->st>>>(c->d, (const float*)c->xref, c->xref64); count_launch(); }
    } else {
        cudaMemcpyAsync(c->xref, src_dev, sizeof(double) * c->d, cudaMemcpyDeviceToDevice, c->st);
        cudaMemcpyAsync(c->xref64, src_dev, sizeof(double) * c->d, cudaMemcpyDeviceToDevice, c->st);
    }
}

// Lq from the FP64 master L: the same matrix in FP64 mode, rounded to BF16 (kept as FP64 values and as
// BF16 bits) in BF16 mode.
static diam_status quantise(diam_ctx* c) {
    if (c->bf) {
        { quantise_factor_kernel<<<dim3(blocks_for(c->ldk), c->d), kThreads, 0, c->st>>>(c->d, c->L, c->d, c->Lq64, c->Lq16,
                                                                                         c->ldk, c->Lq16lo); count_launch(); }
        CK(cudaGetLastError());
    }
    return DIAM_OK;
}

// M = A Lq for a new factor (FP32 on the tensor cores: A Lq[m][j] = sum_k A[m][k] Lq[k][j] through Lq's
// transpose), kept as BF16 hi + lo; and A x_ref for the current x_ref.
static diam_status rec_factor(diam_ctx* c) {
    if (!c->rec) return DIAM_OK;
    const int ldk = c->ldk;
    { transpose_bf16_kernel<<<dim3(ldk / 32, ldk / 32), dim3(32, 8), 0, c->st>>>(c->Lq16, ldk, c->d, ldk, c->Lt16, ldk); count_launch(); }
    TcEpi epi{};
    epi.mode = TC_STORE;
    epi.D = c->ALf;
    epi.ldd = ldk;
    if (c->tf32) {   // Lq = hi + lo (TF32): both terms' products, the lo one as a second K pass
        { transpose_bf16_kernel<<<dim3(ldk / 32, ldk / 32), dim3(32, 8), 0, c->st>>>(c->Lq16lo, ldk, c->d, ldk, c->Lt16lo, ldk); count_launch(); }
        CK(tc_gemm_bf16_a2(c->d, c->dy, ldk, c->Lt16, c->Lt16lo, ldk, c->Gq16, ldk, 0, epi, &c->ctl->status, c->st, 256));
    } else {
        CK(tc_gemm_bf16(c->d, c->dy, ldk, c->Lt16, ldk, c->Gq16, nullptr, ldk, 0, epi, &c->ctl->status, c->st, 256));
    }
    { split_hi_lo_kernel<<<dim3(blocks_for(ldk), c->dy), kThreads, 0, c->st>>>(c->dy, ldk, ldk, c->ALf, c->ALh, c->ALl); count_launch(); }
    CK(cudaGetLastError());
    return DIAM_OK;
}

static diam_status rec_xref(diam_ctx* c) {
    if (!c->rec) return DIAM_OK;
    { axref_kernel<<<c->dy, kThreads, 0, c->st>>>(c->d, c->ldk, c->Gq16, (const float*)c->xref, c->axref); count_launch(); }
    CK(cudaGetLastError());
    return DIAM_OK;
}

// A x of the current states at an interval start: x split into three BF16 terms (hi + lo + lo2 = x exactly), the
// products of A (BF16) with them accumulated in FP32 (two passes: hi + lo, then lo2, added). Every step's map
// A x* = rho (A x) + ... carries this value through the interval, so its error stays in the chain's map terms.
static diam_status rec_ax(diam_ctx* c) {
    if (!c->rec) return DIAM_OK;
    { od_terms_kernel<float><<<c->P, kThreads, 0, c->st>>>(c->d, (const float*)c->X, c->lpo, c->tg, c->op_hi, c->op_lo,
                                                          c->ldk, c->op_lo2); count_launch(); }
    TcEpi epi{};
    epi.mode = TC_STORE;
    epi.D = c->Ax;
    epi.ldd = c->dy;
    // BN = 256: the persistent product, whose chunked accumulation keeps the tensor cores' truncation bias off A x
    CK(tc_gemm_bf16(c->dy, c->P, c->ldk, c->Gq16, c->ldk, c->op_hi, c->op_lo, c->ldk, 0, epi, &c->ctl->status, c->st, 256));
    epi.D = c->ws;
    CK(tc_gemm_bf16(c->dy, c->P, c->ldk, c->Gq16, c->ldk, c->op_lo2, nullptr, c->ldk, 0, epi, &c->ctl->status, c->st, 256));
    const size_t n = (size_t)c->P * c->dy;
    { add_f32_kernel<<<(unsigned)std::min<size_t>(148 * 8, blocks_for(n)), kThreads, 0, c->st>>>(n, c->Ax, c->ws); count_launch(); }
    CK(cudaGetLastError());
    c->ax_dirty = false;
    return DIAM_OK;
}

template <typename T>
static diam_status prepare_block(diam_ctx* c, int64_t blk, cudaStream_t st);

template <typename T>
static diam_status block_begin(diam_ctx* c, int64_t blk) {
    for (auto& pd : c->pend) {
        if (pd.block != blk) continue;
        CK(cudaMemcpyAsync(c->L, pd.L, sizeof(double) * c->d * c->d, cudaMemcpyDeviceToDevice, c->st));
        CKS(quantise(c));
        if (c->cfg.xref_mode == 1 && !is_rw(c)) set_xref_from(c, pd.mean);   // the random walk keeps x_ref = 0
        CKS(rec_factor(c));
        CKS(rec_xref(c));
        // the interval's noise and noise product need only the new quantised factor, z's re-solve needs the
        // states: with the side stream they run side by side (the steps wait for both)
        const bool overlap = c->side && !c->cfg.profile && c->xi_block != blk;
        if (overlap) {
            CK(cudaEventRecord(c->ev_fork, c->st));
            CK(cudaStreamWaitEvent(c->side, c->ev_fork, 0));
            CKS(prepare_block<T>(c, blk, c->side));
            CK(cudaEventRecord(c->ev_join, c->side));
        }
        CKS(rewhiten<T>(c));
        if (overlap) CK(cudaStreamWaitEvent(c->st, c->ev_join, 0));
        pd.block = -1;
    }
    return DIAM_OK;
}

// W for the n_lag steps of interval blk and their noise products xi = beta alpha Lq W (one GEMM), on
// stream st (the context's stream, or the side stream that overlaps them with the re-solve of z).
template <typename T>
static diam_status prepare_block(diam_ctx* c, int64_t blk, cudaStream_t st) {
    const int d = c->d, P = c->P, nl = c->nl;
    const int64_t rows = (int64_t)nl * P;
    // an eighth of the row's four-entry groups per thread block pass: each thread draws eight times
    dim3 g((unsigned)rows, std::max(1u, std::min(64u, blocks_for(c->ldw / 32, 128))));
    if (c->bf) {
        int e0 = ph_begin(c, PH_NOISE);
        { gen_w_kernel<uint16_t><<<g, 128, 0, st>>>(c->key, blk * nl, P, d, c->ldw, (uint16_t*)c->W); count_launch(); }
        ph_end(c, e0);
        int e1 = ph_begin(c, PH_XI);
        TcEpi epi{};
        epi.mode = TC_STORE;
        epi.D = (float*)c->Xi;
        epi.ldd = d;
        epi.scale_dev = &c->ctl->ba;
        if (c->tf32)   // the TF32 factor as hi + lo: the lo term's products as a second K pass
            CK(tc_gemm_bf16_a2(d, (int)rows, c->ldk, c->Lq16, c->Lq16lo, c->ldk, (const uint16_t*)c->W, c->ldw, 1, epi,
                               &c->ctl->status, st, 256));
        else
            CK(tc_gemm_bf16(d, (int)rows, c->ldk, c->Lq16, c->ldk, (const uint16_t*)c->W, nullptr, c->ldw, 1, epi,
                            &c->ctl->status, st, c->bn_xi));
        if (c->rec) {   // the map of every step's noise product: beta alpha (A Lq) W, in one GEMM
            TcEpi em{};
            em.mode = TC_STORE;
            em.D = c->AXi;
            em.ldd = c->dy;
            em.scale_dev = &c->ctl->ba;
            CK(tc_gemm_bf16_a2(c->dy, (int)rows, c->ldk, c->ALh, c->ALl, c->ldk, (const uint16_t*)c->W, c->ldw, 0, em,
                               &c->ctl->status, st, 256));
        }
        ph_end(c, e1);
    } else {
        int e0 = ph_begin(c, PH_NOISE);
        { gen_w_kernel<double><<<g, 128, 0, st>>>(c->key, blk * nl, P, d, c->ldw, (double*)c->W); count_launch(); }
        ph_end(c, e0);
        int e1 = ph_begin(c, PH_XI);
        EpiStore epi{(double*)c->Xi, d, 1.0, &c->ctl->ba, 0.0};
        CK((gemm_f64<true, true>(d, (int)rows, d, c->Lq64, d, (const double*)c->W, c->ldw, TileRange{1, 0}, epi, st)));
        ph_end(c, e1);
    }
    c->xi_block = blk;
    return DIAM_OK;
}

static size_t bsum_elt(const diam_ctx* c) { return c->bf ? sizeof(float) : sizeof(double); }

// Grow the per-interval, per-chain sums to hold interval blk (outside any graph capture).
static diam_status ensure_bsum(diam_ctx* c, int64_t blk) {
    if (!c->cfg.keep_block_sums || blk < c->bcap) return DIAM_OK;
    const int P = c->P, d = c->d;
    int64_t ncap = std::max<int64_t>(2 * c->bcap, blk + 16);
    void *nb = nullptr, *nq = nullptr;
    double* nlp = nullptr;
    CKS(dalloc(c, (char**)&nb, bsum_elt(c) * (size_t)ncap * P * d));
    CKS(dalloc(c, (char**)&nq, bsum_elt(c) * (size_t)ncap * P * d));
    CKS(dalloc(c, &nlp, sizeof(double) * (size_t)ncap * P));
    if (c->bcap) {
        CK(cudaMemcpyAsync(nb, c->bsum, bsum_elt(c) * (size_t)c->bcap * P * d, cudaMemcpyDeviceToDevice, c->st));
        CK(cudaMemcpyAsync(nq, c->bm2, bsum_elt(c) * (size_t)c->bcap * P * d, cudaMemcpyDeviceToDevice, c->st));
        CK(cudaMemcpyAsync(nlp, c->lpsum, sizeof(double) * (size_t)c->bcap * P, cudaMemcpyDeviceToDevice, c->st));
    }
    c->bsum = nb;
    c->bm2 = nq;
    c->lpsum = nlp;
    c->bcap = ncap;
    return DIAM_OK;
}

// The whole step in one launch (step_rec_kernel): BF16 mode, the target's map carried through the proposal or a
// target of O(d) terms only (the diagonal Gaussian; the banana in the 16-byte layout, where one thread holds both
// coordinates of its head), no surrogate screen in force, for d, d_y <= 8192.
static bool fused_step_fits(const diam_ctx* c) {
    const bool vec = (c->d % 4) == 0 && (c->ldw % 4) == 0 && (c->ldh % 4) == 0 && (c->ldk % 4) == 0;
    const bool od = c->kind == TK_DIAG || (c->kind == TK_BANANA && vec && c->d >= 2);
    return c->bf && (c->rec || od) && (!c->da || !c->da->active) && c->d <= 4 * 8 * FUSED_THREADS &&
           c->dy <= 4 * 8 * FUSED_THREADS;
}

template <int NV, int NM, bool VEC, bool STAGE>
static void launch_fused_step(diam_ctx* c, bool setup) {
    DaState* a = c->da;
    const bool keep = c->cfg.keep_block_sums != 0;
    const size_t smem = STAGE ? sizeof(float) * 3 * (size_t)c->d : 0;
    if (setup) {   // outside any capture: the staged rows may take all 48 KB of dynamic shared memory
        if (STAGE) allow_max_dynamic_smem((const void*)step_rec_kernel<NV, NM, VEC, STAGE>);
        return;
    }
    step_rec_kernel<NV, NM, VEC, STAGE><<<c->P, FUSED_THREADS, smem, c->st>>>(
        c->d, c->P, c->nl, c->dy, c->ctl, c->key, c->tg, inv_infl2(c), (float*)c->X, (float*)c->Z,
        (const float*)c->Xi, (const uint16_t*)c->W, c->ldw, (const float*)c->xref, c->Ax,
        c->axref, c->AXi, c->y32, (float)(1.0 / (2.0 * c->sigma * c->sigma)), c->kind == TK_TANH, c->lp, c->q,
        c->accf, c->tr, (float*)c->hist, c->ldh, nullptr, keep ? c->lpsum : nullptr,
        a ? a->cnt : nullptr, a ? a->ring_x : nullptr, a ? a->ring_lp : nullptr, a ? (long long)a->cfg.ring : 1,
        c->ldk);
    count_launch();
}

template <int NV, bool VEC, bool STAGE>
static void fused_step_nm(diam_ctx* c, bool setup) {
    const int nm = (c->dy + 4 * FUSED_THREADS - 1) / (4 * FUSED_THREADS);
    if (nm <= 1) launch_fused_step<NV, 1, VEC, STAGE>(c, setup);
    else if (nm <= 2) launch_fused_step<NV, 2, VEC, STAGE>(c, setup);
    else if (nm <= 4) launch_fused_step<NV, 4, VEC, STAGE>(c, setup);
    else launch_fused_step<NV, 8, VEC, STAGE>(c, setup);
}

template <bool VEC, bool STAGE>
static void fused_step_nv(diam_ctx* c, bool setup) {
    const int nv = (c->d + 4 * FUSED_THREADS - 1) / (4 * FUSED_THREADS);
    if (nv <= 1) fused_step_nm<1, VEC, STAGE>(c, setup);
    else if (nv <= 2) fused_step_nm<2, VEC, STAGE>(c, setup);
    else if (nv <= 4) fused_step_nm<4, VEC, STAGE>(c, setup);
    else if (!STAGE) fused_step_nm<8, VEC, false>(c, setup);
}

// A whole interval of every chain in one launch (interval_rec_kernel): the fused step's conditions, the
// 16-byte layout, and x, z, A x of one chain in shared memory.
constexpr int kIntervalSmemMax = 128 * 1024;

static bool interval_kernel_fits(const diam_ctx* c) {
    const bool vec = (c->d % 4) == 0 && (c->dy % 4) == 0 && (c->ldw % 4) == 0 && (c->ldh % 4) == 0 && (c->ldk % 4) == 0;
    return fused_step_fits(c) && vec && sizeof(float) * (2 * (size_t)c->d + 2 * (size_t)c->dy) <= kIntervalSmemMax;
}

template <int NV, int NM>
static void launch_interval(diam_ctx* c, int ns, bool setup) {
    DaState* a = c->da;
    const bool keep = c->cfg.keep_block_sums != 0;
    const size_t smem = sizeof(float) * (2 * (size_t)c->d + 2 * (size_t)c->dy);
    if (setup) {   // outside any capture (the limit is the kernel's, shared with contexts of other sizes)
        allow_max_dynamic_smem((const void*)interval_rec_kernel<NV, NM>);
        return;
    }
    interval_rec_kernel<NV, NM><<<c->P, FUSED_THREADS, smem, c->st>>>(
        c->d, c->P, c->nl, c->dy, ns, c->ctl, c->key, c->tg, inv_infl2(c), (float*)c->X, (float*)c->Z,
        (const float*)c->Xi, (const uint16_t*)c->W, c->ldw, (const float*)c->xref, c->Ax, c->axref, c->AXi, c->y32,
        (float)(1.0 / (2.0 * c->sigma * c->sigma)), c->kind == TK_TANH, c->lp, c->q, c->accf, c->tr, (float*)c->hist,
        c->ldh, keep ? c->lpsum : nullptr, a ? a->cnt : nullptr, a ? a->ring_x : nullptr, a ? a->ring_lp : nullptr,
        a ? (long long)a->cfg.ring : 1, c->ldk, (c->d % 4) == 0 && (c->dy % 4) == 0 && (c->ldw % 8) == 0);
    count_launch();
}

template <int NV>
static void interval_nm(diam_ctx* c, int ns, bool setup) {
    const int nm = (c->dy + 4 * FUSED_THREADS - 1) / (4 * FUSED_THREADS);
    if (nm <= 1) launch_interval<NV, 1>(c, ns, setup);
    else if (nm <= 2) launch_interval<NV, 2>(c, ns, setup);
    else if (nm <= 4) launch_interval<NV, 4>(c, ns, setup);
    else launch_interval<NV, 8>(c, ns, setup);
}

// ns steps of every chain, from the current step, all inside one interval (setup: prepare the kernel only).
static diam_status interval_steps(diam_ctx* c, int ns, bool setup = false) {
    const int nv = (c->d + 4 * FUSED_THREADS - 1) / (4 * FUSED_THREADS);
    if (nv <= 1) interval_nm<1>(c, ns, setup);
    else if (nv <= 2) interval_nm<2>(c, ns, setup);
    else if (nv <= 4) interval_nm<4>(c, ns, setup);
    else interval_nm<8>(c, ns, setup);
    CK(cudaGetLastError());
    return DIAM_OK;
}

// setup: only prepare the kernel this context will launch (at init, outside any graph capture).
static diam_status fused_step(diam_ctx* c, bool setup = false) {
    const bool vec = (c->d % 4) == 0 && (c->dy % 4) == 0 && (c->ldw % 4) == 0 && (c->ldh % 4) == 0 && (c->ldk % 4) == 0;
    // the chain's x, z, xi rows staged by bulk copies while they fit the default 48 KB of dynamic shared memory
    const bool stage = vec && (size_t)c->d * 12 <= 48 * 1024;
    if (stage) fused_step_nv<true, true>(c, setup);
    else if (vec) fused_step_nv<true, false>(c, setup);
    else fused_step_nv<false, false>(c, setup);
    CK(cudaGetLastError());
    return DIAM_OK;
}

// One step of every chain. The kernels read the step (global t, in-interval s) from the context's device
// scalars and the last one advances it, so the same launch sequence can be captured once as a graph.
template <typename T>
static diam_status do_step(diam_ctx* c) {
    const int d = c->d, P = c->P;
    if (fused_step_fits(c)) {
        int e = ph_begin(c, PH_STEP);
        CKS(fused_step(c));
        ph_end(c, e);
        return DIAM_OK;
    }
    const T* Xi = (const T*)c->Xi;
    constexpr bool BF = std::is_same<T, float>::value;
    const dim3 grid2(P, c->nchunk);
    int e0 = ph_begin(c, PH_PROPOSE);
    if constexpr (BF) {
        const uint16_t* Ws = (const uint16_t*)c->W;
        const bool planes = !c->rec || c->da;   // x* as BF16 hi + lo for a per-step target product or the ring
        { propose_kernel<T, uint16_t><<<grid2, kThreads, 0, c->st>>>(d, P, (const T*)c->X, (const T*)c->Z, Xi, Ws, c->ldw,
                                                               (const T*)c->xref, (T*)c->Xp, (T*)c->Zp, c->qpart, c->lpart,
                                                               c->ctl, c->tg, planes ? c->op_hi : nullptr,
                                                               planes ? c->op_lo : nullptr, c->ldk); count_launch(); }
    } else {
        const T* Ws = (const T*)c->W;
        { propose_kernel<T, T><<<grid2, kThreads, 0, c->st>>>(d, P, (const T*)c->X, (const T*)c->Z, Xi, Ws, c->ldw,
                                                        (const T*)c->xref, (T*)c->Xp, (T*)c->Zp, c->qpart, c->lpart,
                                                        c->ctl, c->tg, nullptr, nullptr, c->ldk); count_launch(); }
    }
    CK(cudaGetLastError());
    ph_end(c, e0);
    int e1 = ph_begin(c, PH_TARGET);
    const double iw = inv_infl2(c);
    if (c->kind == TK_REF || c->kind == TK_CALLBACK || c->kind == TK_TWIST) {
        CKS(eval_lp<T>(c, (const T*)c->Xp, c->lpp));
        { finish_kernel<<<blocks_for(P), kThreads, 0, c->st>>>(P, c->nchunk, c->key, c->qpart, c->lpart, nullptr, 0, c->lpp,
                                                            iw, c->lp, c->q, c->accf, c->ctl, c->tr); count_launch(); }
    } else if (c->kind == TK_DENSE || c->kind == TK_TANH) {
        const double inv2s2 = 1.0 / (2.0 * c->sigma * c->sigma);
        if constexpr (BF) {
          if (c->da) {
            CKS(da_step(c));
          } else if (c->rec) {
            { rec_map_kernel<<<P, kThreads, 0, c->st>>>(P, c->dy, c->ctl, c->Ax, c->axref, c->AXi, c->Axp, c->y32,
                                                       (float)inv2s2, c->kind == TK_TANH, c->lmap); count_launch(); }
            { finish_kernel<<<blocks_for(P), kThreads, 0, c->st>>>(P, c->nchunk, c->key, c->qpart, c->lpart, c->lmap, 1,
                                                                nullptr, iw, c->lp, c->q, c->accf, c->ctl, c->tr); count_launch(); }
          } else {
            TcEpi epi{};
            epi.mode = TC_STORE;
            epi.D = c->ws;
            epi.ldd = c->dy;
            epi.split_stride = (size_t)P * c->dy;
            int used = 1;
            CK(tc_gemm_bf16_splitk(c->dy, P, c->ldk, c->Gq16, c->ldk, c->op_hi, c->op_lo, c->ldk, c->tsplit, epi,
                                   &c->ctl->status, c->st, &used, c->bn_target));
            { finish_linear_kernel<<<P, kThreads, 0, c->st>>>(P, c->dy, used, c->ws, c->y32, (float)inv2s2, c->kind == TK_TANH,
                                                            c->nchunk, c->key, c->qpart, c->lpart, iw, c->lp, c->q,
                                                            c->accf, c->ctl, c->tr); count_launch(); }
          }
        } else {
            EpiTargetReduce epi{c->partial, c->y, inv2s2, c->kind == TK_TANH};
            CK((gemm_f64<true, true>(c->dy, P, d, c->Gm, d, (const double*)c->Xp, d, TileRange{0, 0}, epi, c->st)));
            { finish_kernel<<<blocks_for(P), kThreads, 0, c->st>>>(P, c->nchunk, c->key, c->qpart, c->lpart, c->partial,
                                                                c->nparts, nullptr, iw, c->lp, c->q, c->accf, c->ctl,
                                                                c->tr); count_launch(); }
        }
    } else {
        { finish_kernel<<<blocks_for(P), kThreads, 0, c->st>>>(P, c->nchunk, c->key, c->qpart, c->lpart, nullptr, 0, nullptr,
                                                            iw, c->lp, c->q, c->accf, c->ctl, c->tr); count_launch(); }
    }
    CK(cudaGetLastError());
    ph_end(c, e1);
    int e2 = ph_begin(c, PH_ACCEPT);
    void* bs = (c->cfg.keep_block_sums && !BF) ? c->bsum : nullptr;   // BF16 mode: formed in the fold
    double* ls = c->cfg.keep_block_sums ? c->lpsum : nullptr;
    // the select kernel also copies A x* for accepted chains (carried map), moves the surrogate's ring head
    // past this step's pairs and, in its last block, the step counters
    DaCounters* dac = c->da ? c->da->cnt : nullptr;
    const long long rcap = c->da ? (long long)c->da->cfg.ring : 1;
    if constexpr (BF) {
        { select_kernel<T, float><<<grid2, kThreads, 0, c->st>>>(d, P, c->nl, c->ctl, c->accf, (T*)c->X, (T*)c->Z, (const T*)c->Xp,
                                                                (const T*)c->Zp, (float*)c->hist, c->ldh, (const T*)c->cenT,
                                                                (float*)bs, nullptr, ls, c->lp, c->rec ? c->Ax : nullptr, c->Axp,
                                                                c->dy, dac, rcap); count_launch(); }
    } else {
        { select_kernel<T, double><<<grid2, kThreads, 0, c->st>>>(d, P, c->nl, c->ctl, c->accf, (T*)c->X, (T*)c->Z, (const T*)c->Xp,
                                                                 (const T*)c->Zp, (double*)c->hist, c->ldh, (const T*)c->cenT,
                                                                 (double*)bs, bs ? (double*)c->bm2 : nullptr, ls, c->lp, nullptr,
                                                                 nullptr, 0, dac,
                                                                 rcap); count_launch(); }
    }
    CK(cudaGetLastError());
    ph_end(c, e2);
    return DIAM_OK;
}

// The fold's pass over the interval's FP32 records (BF16 mode): the 16-byte form where the sizes allow it.
static diam_status fold_records(diam_ctx* c, int s0, uint16_t* HT, int ldt, int ntile, float* xs, float* xq) {
    const int d = c->d, P = c->P, nl = c->nl, npb = (P + 31) / 32;
    float* pb = HT ? c->psum + (size_t)ntile * d : nullptr;
    float* ps = HT ? c->psum : nullptr;
    if (d % 4 == 0 && c->ldh % 4 == 0 && P % 8 == 0) {
        { fold_records4_kernel<<<dim3((d + 127) / 128, npb), 256, 0, c->st>>>((const float*)c->hist, c->ldh, P, nl, s0, d,
                                                                           (const float*)c->cenT, HT, ldt, ps, pb, xs, xq); count_launch(); }
    } else {
        { fold_records_kernel<<<dim3((d + 31) / 32, npb), dim3(32, 8), 0, c->st>>>((const float*)c->hist, c->ldh, P, nl, s0, d,
                                                                                (const float*)c->cenT, HT, ldt, ps, pb, xs, xq); count_launch(); }
    }
    CK(cudaGetLastError());
    return DIAM_OK;
}

// Fold the samples of interval blk (those past the burn-in) into the pooled moments.
template <typename T>
static diam_status fold_block(diam_ctx* c, int64_t blk) {
    const int d = c->d, P = c->P, nl = c->nl;
    int64_t tstart = blk * nl;
    int64_t s0 = std::max<int64_t>(0, std::min<int64_t>(nl, c->cfg.burnin - tstart));
    int64_t rows = (nl - s0) * P;
    constexpr bool BF = std::is_same<T, float>::value;
    // BF16 mode: the per-chain interval sums of x come from the records (in the fold's pass over them)
    float* xs = (BF && c->cfg.keep_block_sums) ? (float*)c->bsum + (size_t)blk * P * d : nullptr;
    float* xq = xs ? (float*)c->bm2 + (size_t)blk * P * d : nullptr;
    const int npb = (P + 31) / 32;
    if (rows <= 0) {
        if (xs) CKS(fold_records(c, nl, nullptr, 0, 0, xs, xq));
        return DIAM_OK;
    }
    double nb = (double)rows;
    int R = (int)std::min<int64_t>(64, rows);
    int e0 = ph_begin(c, PH_FOLD);
    if constexpr (BF) {
        // samples as the K index: one pass over the interval's FP32 records writes their BF16 transpose
        // (d x rows, K-contiguous), the per-tile sums of the records and of their BF16 values (the totals give
        // the centring terms, the interval mean from the FP32 records, and s16 for the lower-triangle SYRK on
        // the tensor cores, whose epilogue does the FP64 fold) and the per-chain interval sums
        const int ldt = ((int)rows + 63) / 64 * 64, ntile = (int)(nl - s0) * npb;
        CKS(fold_records(c, (int)s0, c->histT, ldt, ntile, xs, xq));
        if (ldt > rows)   // the K padding of the SYRK operand
            CK(cudaMemset2DAsync(c->histT + rows, sizeof(uint16_t) * ldt, 0, sizeof(uint16_t) * (ldt - rows), d, c->st));
        { fold_sums_kernel<<<(d + 31) / 32, kThreads, 0, c->st>>>(d, ntile, c->psum, c->psum + (size_t)ntile * d, c->cen64,
                                                                c->mean, 1.0 / nb, c->svec, c->delta, c->s16); count_launch(); }
    } else {
        const double* H = (const double*)c->hist + (size_t)s0 * P * c->ldh;
        { colsum_partial_kernel<double><<<dim3(blocks_for(d), R), kThreads, 0, c->st>>>(H, c->ldh, (int)rows, d, c->colpart); count_launch(); }
        { fold_prep_kernel<<<blocks_for(d), kThreads, 0, c->st>>>(d, R, c->colpart, c->cen64, c->mean, 1.0 / nb, c->svec,
                                                                c->delta); count_launch(); }
    }
    double w = (double)c->n * nb / ((double)c->n + nb);
    if constexpr (BF) {
        const int ldt = ((int)rows + 63) / 64 * 64;
        TcEpi epi{};
        epi.mode = TC_FOLD;
        epi.M2 = c->M2;
        epi.ldm = d;
        epi.s = c->s16;   // G - s16 s16^T / nb: the scatter of exactly the values the SYRK multiplies
        epi.delta = c->delta;
        epi.inb = 1.0 / nb;
        epi.w = w;
        ph_end(c, e0);   // the SYRK itself timed on its own (one tensor-core launch)
        const int e1 = ph_begin(c, PH_SYRK);
        CK(tc_gemm_bf16(d, d, ldt, c->histT, ldt, c->histT, nullptr, ldt, 0, epi, &c->ctl->status, c->st, 256));
        ph_end(c, e1);
        e0 = ph_begin(c, PH_FOLD);
    } else {
        const double* H = (const double*)c->hist + (size_t)s0 * P * c->ldh;
        EpiFold epi{c->M2, d, c->svec, c->delta, 1.0 / nb, w};
        CK((gemm_f64<false, false>(d, d, (int)rows, H, c->ldh, H, c->ldh, TileRange{0, 1}, epi, c->st)));
    }
    { mean_update_kernel<T><<<blocks_for(d), kThreads, 0, c->st>>>(d, nb / ((double)c->n + nb), c->delta, c->mean,
                                                                 c->cen64, (T*)c->cenT); count_launch(); }
    CK(cudaGetLastError());
    ph_end(c, e0);
    c->n += rows;
    return DIAM_OK;
}

// Replay of a captured launch sequence (captured on first use, on the context's stream, with the work it
// forks onto other streams joined back); the library's launch counter counts the kernels of every replay.
template <typename F>
static diam_status run_captured(diam_ctx* c, diam_ctx::Captured& g, F body, cudaStream_t st = nullptr) {
    if (!st) st = c->st;
    if (!g.exec) {
        cudaGraph_t gr = nullptr;
        const unsigned long long l0 = g_launches.load();
        CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        cudaError_t eb = body();
        cudaError_t e = cudaStreamEndCapture(st, &gr);
        if (eb != cudaSuccess || e != cudaSuccess) {
            if (gr) cudaGraphDestroy(gr);
            return fail(c, DIAM_ECUDA, "graph capture", cudaGetErrorString(eb != cudaSuccess ? eb : e));
        }
        cudaError_t ei = cudaGraphInstantiate(&g.exec, gr, 0);
        cudaGraphDestroy(gr);
        CK(ei);
        g.launches = g_launches.load() - l0;
        g_launches.fetch_sub(g.launches);
    }
    CK(cudaGraphLaunch(g.exec, st));
    g_launches.fetch_add(g.launches);
    return DIAM_OK;
}

// Cholesky refresh at the end of interval blk (skip / jitter rule, retries with a larger jitter).
static diam_status refresh(diam_ctx* c, int64_t blk) {
    const int d = c->d;
    int e0 = ph_begin(c, PH_REFRESH);
    double inv_n = 1.0 / (double)c->n;
    // the first attempt loads by max(eps_jitter, eps_jitter_min) (relative); the caller's floor
    double eps = std::max(c->cfg.eps_jitter, c->cfg.eps_jitter_min);
    bool ok = false;
    for (int attempt = 0; attempt < 4 && !ok; ++attempt) {
        // C_n + eps diag(C_n): every variance loaded by the same relative amount (the skip / jitter rule)
        { build_c_kernel<<<dim3(blocks_for(d), d), kThreads, 0, c->st>>>(d, c->M2, d, inv_n, eps, c->Cw); count_launch(); }
        CK(cudaMemsetAsync(&c->ctl->chol_info, 0, sizeof(int), c->st));
        // after a first eager factorisation, replayed as a captured graph (profiled too: the phase's events
        // lie outside the capture)
        if (c->bf && c->cfg.graphs && c->oz.hi) {
            CKS(run_captured(c, c->chol_graph, [&]() {
                return cholesky_f64(c->Cw, d, d, &c->ctl->chol_info, c->st, &c->oz, &c->ctl->status);
            }));
        } else {
            CK(cholesky_f64(c->Cw, d, d, &c->ctl->chol_info, c->st, c->bf ? &c->oz : nullptr, &c->ctl->status));
        }
        CKS(sync_and_check(c));
        int info = 0;
        CK(d2h(c, &info, &c->ctl->chol_info, sizeof(int)));
        ok = (info == 0);
        eps *= 100.0;
        c->chol_attempts++;
    }
    ph_end(c, e0);
    if (!ok) {
        c->notspd++;
        c->err = "refresh skipped: C_n + jitter not positive definite (previous factor kept)";
        return DIAM_OK;
    }
    Pending& pd = c->pend[(size_t)(blk % (int64_t)c->pend.size())];
    CK(cudaMemcpyAsync(pd.L, c->Cw, sizeof(double) * d * d, cudaMemcpyDeviceToDevice, c->st));
    CK(cudaMemcpyAsync(pd.mean, c->mean, sizeof(double) * d, cudaMemcpyDeviceToDevice, c->st));
    pd.block = blk + 1 + c->cfg.refresh_delay;
    c->refreshes++;
    return DIAM_OK;
}

// The refresh of interval blk beside the following intervals (its factor is due at interval blk + 1 + delay):
// C_n with the first jitter built and the moments kept on the context's stream, then the factorisation, on
// the slot's stream with its own workspaces, into pending slot blk. refresh_finish_due resolves it.
static bool refresh_async_ok(const diam_ctx* c) {
    return c->bf && c->cfg.graphs && !c->cfg.profile && c->cfg.refresh_delay >= 1 && c->n_ar > 0;
}

static diam_status refresh_launch(diam_ctx* c, int64_t blk) {
    const int d = c->d;
    diam_ctx::AsyncRefresh& r = c->ar[blk % c->n_ar];
    if (r.active) return fail(c, DIAM_ESTATE, "refresh", "slot still in flight");
    const double eps = std::max(c->cfg.eps_jitter, c->cfg.eps_jitter_min);
    { build_c_kernel<<<dim3(blocks_for(d), d), kThreads, 0, c->st>>>(d, c->M2, d, 1.0 / (double)c->n, eps, r.Cr); count_launch(); }
    CK(cudaMemcpyAsync(r.M2s, c->M2, sizeof(double) * d * d, cudaMemcpyDeviceToDevice, c->st));
    Pending& pd = c->pend[(size_t)(blk % (int64_t)c->pend.size())];
    CK(cudaMemcpyAsync(pd.mean, c->mean, sizeof(double) * d, cudaMemcpyDeviceToDevice, c->st));
    CK(cudaMemsetAsync(r.info, 0, 2 * sizeof(int), c->st));
    CK(cudaEventRecord(r.fork, c->st));
    CK(cudaStreamWaitEvent(r.rs, r.fork, 0));
    CK(cudaEventRecord(r.start, r.rs));
    auto body = [&]() { return cholesky_f64(r.Cr, d, d, r.info, r.rs, &r.oz, r.info + 1); };
    if (r.oz.hi) {   // after a first eager factorisation (which creates the workspace's streams)
        CKS(run_captured(c, r.graph, body, r.rs));
    } else {
        CK(body());
    }
    CK(cudaMemcpyAsync(pd.L, r.Cr, sizeof(double) * d * d, cudaMemcpyDeviceToDevice, r.rs));
    CK(cudaEventRecord(r.done, r.rs));
    r.active = true;
    r.blk = blk;
    r.n = c->n;
    r.eps = eps;
    return DIAM_OK;
}

// Wait for a refresh in flight and apply the refresh rule's outcome: its pending factor, or the retries
// with a larger jitter (from the kept moments, in order on the context's stream), or the skip.
static diam_status refresh_finish_slot(diam_ctx* c, diam_ctx::AsyncRefresh& r) {
    if (!r.active) return DIAM_OK;
    r.active = false;
    const int d = c->d;
    CK(cudaStreamWaitEvent(c->st, r.done, 0));   // later work on the stream is ordered after it
    CK(cudaEventSynchronize(r.done));
    CKS(sync_and_check(c));
    float ms = 0.f;   // its device time beside the intervals, in the refresh phase's accumulators
    if (cudaEventElapsedTime(&ms, r.start, r.done) == cudaSuccess) {
        c->prof_ms[PH_REFRESH] += ms;
        c->prof_cnt[PH_REFRESH] += 1;
    }
    int iv[2] = {0, 0};
    CK(d2h(c, iv, r.info, sizeof(iv)));
    if (iv[1] == DEV_TIMEOUT) return fail(c, DIAM_ETIMEOUT, "refresh", "a bounded wait inside the factorisation expired");
    if (iv[1] != 0) return fail(c, DIAM_ECUDA, "refresh", "a factorisation kernel reported a bad argument");
    int info = iv[0];
    c->chol_attempts++;
    Pending& pd = c->pend[(size_t)(r.blk % (int64_t)c->pend.size())];
    bool ok = info == 0;
    double eps = r.eps * 100.0;
    for (int attempt = 1; attempt < 4 && !ok; ++attempt) {
        { build_c_kernel<<<dim3(blocks_for(d), d), kThreads, 0, c->st>>>(d, r.M2s, d, 1.0 / (double)r.n, eps, r.Cr); count_launch(); }
        CK(cudaMemsetAsync(r.info, 0, sizeof(int), c->st));
        CK(cholesky_f64(r.Cr, d, d, r.info, c->st, &c->oz, &c->ctl->status));
        CKS(sync_and_check(c));
        CK(d2h(c, &info, r.info, sizeof(int)));
        ok = info == 0;
        eps *= 100.0;
        c->chol_attempts++;
        if (ok) CK(cudaMemcpyAsync(pd.L, r.Cr, sizeof(double) * d * d, cudaMemcpyDeviceToDevice, c->st));
    }
    if (!ok) {
        c->notspd++;
        c->err = "refresh skipped: C_n + jitter not positive definite (previous factor kept)";
        return DIAM_OK;
    }
    pd.block = r.blk + 1 + c->cfg.refresh_delay;
    c->refreshes++;
    return DIAM_OK;
}

// Resolve the refreshes in flight built at or before interval last (all of them: last < 0), oldest first.
static diam_status refresh_finish_due(diam_ctx* c, int64_t last) {
    for (;;) {
        diam_ctx::AsyncRefresh* o = nullptr;
        for (int i = 0; i < c->n_ar; ++i)
            if (c->ar[i].active && (last < 0 || c->ar[i].blk <= last) && (!o || c->ar[i].blk < o->blk)) o = &c->ar[i];
        if (!o) return DIAM_OK;
        CKS(refresh_finish_slot(c, *o));
    }
}

static diam_status refresh_finish(diam_ctx* c) { return refresh_finish_due(c, -1); }

static void push_scalars(diam_ctx* c) {
    // the random walk of eq. (rw) moves from x itself: rho = 1 (with x_ref = 0, x* = x + xi exactly)
    double rho = is_rw(c) ? 1.0 : std::sqrt(1.0 - c->beta * c->beta);
    { set_scalars_kernel<<<1, 1, 0, c->st>>>(c->ctl, c->beta, rho, c->beta * c->cfg.infl, inv_infl2(c)); count_launch(); }
}

template <typename T>
static diam_status block_end(diam_ctx* c, int64_t blk) {
    CKS(fold_block<T>(c, blk));
    CKS(sync_and_check(c));
    prof_flush(c);
    unsigned long long acc = 0, nonf = 0;
    CK(d2h(c, &acc, &c->ctl->acc_block, sizeof(acc)));
    CK(d2h(c, &nonf, &c->ctl->nonfinite, sizeof(nonf)));
    c->acc_all += (int64_t)acc;
    c->nonfinite = nonf;
    if (c->hook) {   // the synchronisation point: the interval's samples are in the moments, the refresh is next
        c->in_hook = true;
        const diam_status hs = c->hook(c->hook_user, c, blk);
        c->in_hook = false;
        if (c->bad) return DIAM_ESTATE;
        if (hs != DIAM_OK) return fail(c, hs == DIAM_ENOTSPD ? DIAM_ETARGET : hs, "interval hook", "returned an error");
    }
    const diam_config& g = c->cfg;
    if (g.adapt_beta) {  // Algorithm 1: raise beta above the window, lower it below
        double ahat = (double)acc / ((double)c->P * c->nl);
        if (ahat > g.acc_hi) c->beta *= g.beta_factor;
        else if (ahat < g.acc_lo) c->beta /= g.beta_factor;
        if (c->beta < g.beta_min) c->beta = g.beta_min;
        if (c->beta > g.beta_max) c->beta = g.beta_max;
    }
    if ((blk + 1) * (int64_t)c->nl > g.burnin) c->acc_refresh += (int64_t)acc;
    // the refreshes in flight whose factors may be due at the next interval: built at or before
    // blk - min(delay, 2) (at most two run beside the intervals)
    CKS(refresh_finish_due(c, blk - std::max(1, c->n_ar)));
    if (c->acc_refresh >= g.min_samples_refresh && c->n > 0) {
        if (refresh_async_ok(c)) CKS(refresh_launch(c, blk));
        else CKS(refresh(c, blk));
    }
    push_scalars(c);
    CK(cudaGetLastError());
    if (c->da) CKS(da_after_interval(c));
    return DIAM_OK;
}

// Replay the captured graph of one interval's steps (capturing it first if needed).
template <typename T>
static diam_status interval_graph(diam_ctx* c) {
    const int da_sig = c->da ? (c->da->active ? 1 : 0) : -1;
    if (c->graph && (c->graph_bsum != (const void*)c->bsum || c->graph_da != da_sig)) {
        cudaGraphExecDestroy(c->graph);
        c->graph = nullptr;
    }
    if (!c->graph) {
        cudaGraph_t g = nullptr;
        const unsigned long long l0 = g_launches.load();
        CK(cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal));
        diam_status s = DIAM_OK;
        for (int k = 0; k < c->nl && s == DIAM_OK; ++k) s = do_step<T>(c);
        cudaError_t e = cudaStreamEndCapture(c->st, &g);
        if (s != DIAM_OK) {
            if (g) cudaGraphDestroy(g);
            return s;
        }
        CK(e);
        cudaError_t ei = cudaGraphInstantiate(&c->graph, g, 0);
        cudaGraphDestroy(g);
        CK(ei);
        c->graph_bsum = c->bsum;
        c->graph_da = da_sig;
        c->graph_launches = g_launches.load() - l0;
        g_launches.fetch_sub(c->graph_launches);   // counted when they run, below
    }
    CK(cudaGraphLaunch(c->graph, c->st));
    g_launches.fetch_add(c->graph_launches);
    return DIAM_OK;
}

template <typename T>
static diam_status run_steps(diam_ctx* c, int64_t n_steps) {
    { set_step_kernel<<<1, 1, 0, c->st>>>(c->ctl, (long long)c->t, (int)(c->t % c->nl)); count_launch(); }
    while (n_steps > 0) {
        int64_t blk = c->t / c->nl;
        int s = (int)(c->t % c->nl);
        if (s == 0 && c->begun_block != blk) {
            CKS(block_begin<T>(c, blk));
            { centre_kernel<T><<<blocks_for(c->d), kThreads, 0, c->st>>>(c->d, c->P, (const T*)c->X, (T*)c->cenT, c->cen64); count_launch(); }
            c->begun_block = blk;
            c->ax_dirty = true;   // A x recomputed exactly at every interval start
        }
        if (c->rec && c->ax_dirty) CKS(rec_ax(c));
        if (c->xi_block != blk) CKS(prepare_block<T>(c, blk, c->st));
        CKS(ensure_bsum(c, blk));
        const bool whole = s == 0 && n_steps >= c->nl && c->cfg.graphs && c->kind != TK_CALLBACK && !c->cfg.profile;
        if (s == 0 && n_steps >= c->nl && c->cfg.graphs && interval_kernel_fits(c)) {
            int e = ph_begin(c, PH_STEP);
            CKS(interval_steps(c, c->nl));
            ph_end(c, e);
            c->t += c->nl;
            n_steps -= c->nl;
        } else if (whole) {
            CKS(interval_graph<T>(c));
            c->t += c->nl;
            n_steps -= c->nl;
        } else {
            CKS(do_step<T>(c));
            c->t++;
            n_steps--;
        }
        if (c->t % c->nl == 0) CKS(block_end<T>(c, blk));
    }
    return DIAM_OK;
}

// ------------------------------------------------------------------------------------------------ init
// Tile widths of the tensor-core products this context launches, timed on its own buffers (the outputs
// written here are scratch: the split-K planes and the noise-product buffer, both rewritten before use).
static diam_status autotune(diam_ctx* c) {
    if (c->ws) {
        TcEpi epi{};
        epi.mode = TC_STORE;
        epi.D = c->ws;
        epi.ldd = c->dy;
        epi.split_stride = (size_t)c->P * c->dy;
        // tile width and split of K together: each split count gets its best width, the fastest pair wins
        float best = 1e30f;
        for (int sp = 1; sp <= TSPLIT_MAX && sp <= 2 * c->ldk / 64; sp *= 2) {
            float ms = 1e30f;
            const int bn = tc_autotune(c->dy, c->P, c->ldk, c->Gq16, c->ldk, c->op_hi, c->op_lo, c->ldk, sp, 0, epi,
                                       &c->ctl->status, c->st, &ms);
            if (ms < best) {
                best = ms;
                c->bn_target = bn;
                c->tsplit = sp;
            }
        }
    }
    TcEpi ex{};
    ex.mode = TC_STORE;
    ex.D = (float*)c->Xi;
    ex.ldd = c->d;
    ex.scale_dev = &c->ctl->ba;
    c->bn_xi = tc_autotune(c->d, c->nl * c->P, c->ldk, c->Lq16, c->ldk, (const uint16_t*)c->W, nullptr, c->ldw, 1, 1, ex,
                           &c->ctl->status, c->st, nullptr);
    return sync_and_check(c);
}

template <typename T>
static diam_status init_state(diam_ctx* c, const double* x0, const double* C0, const double* xref0) {
    const int d = c->d, P = c->P;
    double* tmp = nullptr;
    CKS(dalloc(c, &tmp, sizeof(double) * (size_t)std::max(P * d, d * d)));
    if (x0) {
        CK(cudaMemcpyAsync(tmp, x0, sizeof(double) * (size_t)P * d, cudaMemcpyHostToDevice, c->st));
        { convert_kernel<double, T><<<blocks_for((size_t)P * d), kThreads, 0, c->st>>>((size_t)P * d, tmp, (T*)c->X); count_launch(); }
    }
    // A_0: Cholesky factor of C0, or the identity (Algorithm 1)
    if (C0) {
        CK(cudaMemcpyAsync(c->L, C0, sizeof(double) * d * d, cudaMemcpyHostToDevice, c->st));
        CK(cudaMemsetAsync(&c->ctl->chol_info, 0, sizeof(int), c->st));
        CK(cholesky_f64(c->L, d, d, &c->ctl->chol_info, c->st, c->bf ? &c->oz : nullptr, &c->ctl->status));
        CKS(sync_and_check(c));
        int info = 0;
        CK(d2h(c, &info, &c->ctl->chol_info, sizeof(int)));
        if (info) return fail(c, DIAM_EINVAL, "diam_init", "C0 is not positive definite");
    } else {
        std::vector<double> I((size_t)d * d, 0.0);
        for (int i = 0; i < d; ++i) I[(size_t)i * d + i] = 1.0;
        CK(h2d(c, c->L, I.data(), sizeof(double) * d * d));
    }
    CKS(quantise(c));
    if (xref0 && !is_rw(c)) {   // the random walk keeps x_ref = 0 (unused by its proposal)
        CK(cudaMemcpyAsync(tmp, xref0, sizeof(double) * d, cudaMemcpyHostToDevice, c->st));
        set_xref_from(c, tmp);
    }
    CKS(rec_factor(c));
    CKS(rec_xref(c));
    push_scalars(c);
    CKS(rewhiten<T>(c));
    if (c->kind != TK_REF) CKS(eval_lp<T>(c, (const T*)c->X, c->lp));
    CKS(sync_and_check(c));
    if (c->bf) CKS(autotune(c));
    return DIAM_OK;
}

static diam_status alloc_all(diam_ctx* c) {
    const int d = c->d, P = c->P, nl = c->nl;
    const size_t ts = c->bf ? sizeof(float) : sizeof(double);
    const size_t Pd = (size_t)P * d, rows = (size_t)nl * P;
    CKS(dalloc(c, &c->ctl, sizeof(Ctl)));
    CKS(dalloc(c, &c->X, ts * Pd));
    CKS(dalloc(c, &c->Z, ts * Pd));
    CKS(dalloc(c, &c->Xp, ts * Pd));
    CKS(dalloc(c, &c->Zp, ts * Pd));
    CKS(dalloc(c, &c->xref, ts * d));
    CKS(dalloc(c, &c->cenT, ts * d));
    CKS(dalloc(c, &c->Xi, ts * rows * d));
    for (double** p : {&c->lp, &c->q, &c->qp, &c->lpo, &c->lpp}) CKS(dalloc(c, p, sizeof(double) * P));
    c->nparts = c->bf ? (c->dy + 127) / 128 : (c->dy + 63) / 64;  // m-tiles of the target product
    CKS(dalloc(c, &c->partial, sizeof(double) * (size_t)c->nparts * P));
    c->nchunk = (d + CHUNK - 1) / CHUNK;
    CKS(dalloc(c, &c->qpart, sizeof(double) * (size_t)c->nchunk * P));
    CKS(dalloc(c, &c->lpart, sizeof(double) * (size_t)c->nchunk * P));
    CKS(dalloc(c, &c->accf, (size_t)P));
    CKS(dalloc(c, &c->s16, sizeof(double) * d));
    if (c->bf && c->dy > 0 && (c->kind == TK_DENSE || c->kind == TK_TANH)) {
        // split of the target product's K (the autotuner picks it with the tile width): room for 8 planes
        int tiles = ((c->dy + 127) / 128) * ((P + 127) / 128);
        c->tsplit = std::max(1, std::min(8, 148 / std::max(tiles, 1)));
        c->tsplit = std::min(c->tsplit, c->ldk / 64);
        CKS(dalloc(c, &c->ws, sizeof(float) * (size_t)TSPLIT_MAX * P * c->dy));
    }
    for (double** p : {&c->xref64, &c->mean, &c->cen64, &c->svec, &c->delta}) CKS(dalloc(c, p, sizeof(double) * d));
    CKS(dalloc(c, &c->colpart, sizeof(double) * 64 * d));
    CKS(dalloc(c, &c->L, sizeof(double) * d * d));
    CKS(dalloc(c, &c->M2, sizeof(double) * d * d));
    CKS(dalloc(c, &c->Cw, sizeof(double) * d * d));
    CKS(dalloc(c, &c->work, sizeof(double) * Pd));
    c->pend.resize((size_t)c->cfg.refresh_delay + 1);
    for (auto& pd : c->pend) {
        CKS(dalloc(c, &pd.L, sizeof(double) * d * d));
        CKS(dalloc(c, &pd.mean, sizeof(double) * d));
    }
    if (c->bf) {
        CKS(dalloc(c, &c->oz.SL, ozaki_sl_bytes(d)));
        CKS(dalloc(c, &c->oz.ex, ozaki_ex_bytes(d)));
        c->oz.cap_rows = d;
        CKS(dalloc(c, &c->oz.SL2, ozaki_sl_bytes(P)));
        CKS(dalloc(c, &c->oz.ex2, ozaki_ex_bytes(P)));
        c->oz.cap2 = P;
        c->oz.capP = ozaki_panel_rows(d);
        CKS(dalloc(c, &c->oz.SLP, sizeof(uint16_t) * (size_t)std::max<int64_t>(1, c->oz.capP) * 448));
        CKS(dalloc(c, &c->oz.exP, sizeof(int) * (size_t)std::max<int64_t>(1, c->oz.capP)));
        if (c->cfg.refresh_delay >= 1 && c->cfg.graphs) {   // refreshes beside the following intervals
            c->n_ar = c->cfg.refresh_delay >= 2 ? 2 : 1;
            for (int i = 0; i < c->n_ar; ++i) {
                diam_ctx::AsyncRefresh& r = c->ar[i];
                CKS(dalloc(c, &r.Cr, sizeof(double) * d * d));
                CKS(dalloc(c, &r.M2s, sizeof(double) * d * d));
                CKS(dalloc(c, &r.info, 2 * sizeof(int)));
                CKS(dalloc(c, &r.oz.SL, ozaki_sl_bytes(d)));
                CKS(dalloc(c, &r.oz.ex, ozaki_ex_bytes(d)));
                r.oz.cap_rows = d;
                r.oz.lo_high = true;   // ahead of the intervals' work: the chain waits on these updates
                CK(cudaStreamCreateWithFlags(&r.rs, cudaStreamNonBlocking));
                CK(cudaEventCreateWithFlags(&r.fork, cudaEventDisableTiming));
                CK(cudaEventCreate(&r.start));
                CK(cudaEventCreate(&r.done));
            }
        }
        CKS(dalloc(c, &c->Lq64, sizeof(double) * d * d));
        CKS(dalloc(c, &c->Lq16, sizeof(uint16_t) * (size_t)d * c->ldk));
        if (c->tf32) CKS(dalloc(c, &c->Lq16lo, sizeof(uint16_t) * (size_t)d * c->ldk));
        CKS(dalloc(c, &c->op_hi, sizeof(uint16_t) * (size_t)P * c->ldk));
        CKS(dalloc(c, &c->op_lo, sizeof(uint16_t) * (size_t)P * c->ldk));
        CKS(dalloc(c, &c->op_lo2, sizeof(uint16_t) * (size_t)P * c->ldk));
        c->ldw = c->ldk;
        c->ldh = d;
        CKS(dalloc(c, &c->W, sizeof(uint16_t) * rows * c->ldw));
        CKS(dalloc(c, &c->hist, sizeof(float) * rows * c->ldh));
        CKS(dalloc(c, &c->histT, sizeof(uint16_t) * (size_t)d * ((rows + 63) / 64 * 64)));
        // the fold's tile sums: one per (step, 32-chain block)
        CKS(dalloc(c, &c->psum, sizeof(float) * 2 * (size_t)d * ((size_t)nl * ((P + 31) / 32))));
        if ((c->kind == TK_TANH || c->kind == TK_DENSE) && c->cfg.carry_map) {
            c->rec = true;
            const size_t dy = (size_t)std::max(c->dy, 1);
            CKS(dalloc(c, &c->Lt16, sizeof(uint16_t) * (size_t)c->ldk * c->ldk));
            if (c->tf32) CKS(dalloc(c, &c->Lt16lo, sizeof(uint16_t) * (size_t)c->ldk * c->ldk));
            CKS(dalloc(c, &c->ALf, sizeof(float) * dy * c->ldk));
            CK(cudaMemsetAsync(c->ALf, 0, sizeof(float) * dy * c->ldk, c->st));   // padding columns stay zero
            CKS(dalloc(c, &c->ALh, sizeof(uint16_t) * dy * c->ldk));
            CKS(dalloc(c, &c->ALl, sizeof(uint16_t) * dy * c->ldk));
            CKS(dalloc(c, &c->AXi, sizeof(float) * rows * dy));
            CKS(dalloc(c, &c->Ax, sizeof(float) * (size_t)P * dy));
            CKS(dalloc(c, &c->Axp, sizeof(float) * (size_t)P * dy));
            CKS(dalloc(c, &c->axref, sizeof(float) * dy));
            CKS(dalloc(c, &c->lmap, sizeof(double) * (size_t)P));
        }
    } else {
        c->Lq64 = c->L;
        c->ldw = (d + 3) / 4 * 4;
        c->ldh = d;
        CKS(dalloc(c, &c->W, sizeof(double) * rows * c->ldw));
        CKS(dalloc(c, &c->hist, sizeof(double) * rows * c->ldh));
    }
    if (c->cfg.trace_steps > 0) {
        size_t nt = (size_t)c->cfg.trace_steps * P;
        CKS(dalloc(c, &c->tr.lp, sizeof(double) * nt));
        CKS(dalloc(c, &c->tr.q, sizeof(double) * nt));
        CKS(dalloc(c, &c->tr.qc, sizeof(double) * nt));
        CKS(dalloc(c, &c->tr.loga, sizeof(double) * nt));
        CKS(dalloc(c, &c->tr.acc, nt));
        c->tr.steps = c->cfg.trace_steps;
    }
    return DIAM_OK;
}

static diam_status upload_target(diam_ctx* c, const diam_target* tg) {
    const int d = c->d, dy = c->dy;
    c->tg.kind = c->kind;
    c->tg.d_y = dy;
    c->tg.ban_a = tg->ban_a;
    c->tg.ban_b = tg->ban_b;
    c->tg.ban_c = tg->ban_c;
    std::vector<double> il((size_t)d, 0.0);
    if (c->kind == TK_DIAG || c->kind == TK_TANH || c->kind == TK_BANANA) {
        if (!tg->lam) return fail(c, DIAM_EINVAL, "diam_init", "target needs lam");
        for (int i = 0; i < d; ++i) {
            if (c->kind == TK_BANANA && i < 2) continue;
            if (!(tg->lam[i] > 0)) return fail(c, DIAM_EINVAL, "diam_init", "lam must be positive");
            il[i] = 1.0 / tg->lam[i];
        }
    }
    CKS(dalloc(c, &c->inv_lam, sizeof(double) * d));
    CK(h2d(c, c->inv_lam, il.data(), sizeof(double) * d));
    c->tg.inv_lam = c->inv_lam;
    {
        std::vector<float> il32(il.begin(), il.end());
        CKS(dalloc(c, &c->inv_lam32, sizeof(float) * d));
        CK(h2d(c, c->inv_lam32, il32.data(), sizeof(float) * d));
        c->tg.inv_lam32 = c->inv_lam32;
    }
    if (c->kind == TK_TWIST) {
        if (!tg->G || !tg->lam || !tg->y || dy <= 0) return fail(c, DIAM_EINVAL, "diam_init", "twisted target needs G, lam, y");
        std::vector<double> ilam((size_t)dy);
        for (int j = 0; j < dy; ++j) {
            if (!(tg->lam[j] > 0)) return fail(c, DIAM_EINVAL, "diam_init", "lam must be positive");
            ilam[j] = 1.0 / tg->lam[j];
        }
        CKS(dalloc(c, &c->tw_ilam, sizeof(double) * dy));
        CKS(dalloc(c, &c->tw_c, sizeof(double) * dy));
        CK(h2d(c, c->tw_ilam, ilam.data(), sizeof(double) * dy));
        CK(h2d(c, c->tw_c, tg->y, sizeof(double) * dy));
        CKS(dalloc(c, &c->Gm, sizeof(double) * (size_t)dy * d));
        CK(h2d(c, c->Gm, tg->G, sizeof(double) * (size_t)dy * d));
        if (c->bf) {   // BF16 mode: the map rounded to BF16 (the mixed method's map), its product taken in FP64
            const size_t n = (size_t)dy * d;
            { round_bf16_kernel<<<(unsigned)std::min<size_t>(148 * 8, blocks_for(n)), kThreads, 0, c->st>>>(n, c->Gm); count_launch(); }
            CK(cudaGetLastError());
        }
        CKS(dalloc(c, &c->ubuf, sizeof(double) * (size_t)c->P * dy));
    }
    if (c->kind == TK_DENSE || c->kind == TK_TANH) {
        const double* M = c->kind == TK_DENSE ? tg->G : tg->A;
        if (!M || dy <= 0) return fail(c, DIAM_EINVAL, "diam_init", "target needs its matrix and d_y");
        if (c->kind == TK_TANH && (!tg->y || !(tg->sigma > 0)))
            return fail(c, DIAM_EINVAL, "diam_init", "tanh target needs y and sigma > 0");
        CKS(dalloc(c, &c->Gm, sizeof(double) * (size_t)dy * d));
        CK(h2d(c, c->Gm, M, sizeof(double) * (size_t)dy * d));
        if (c->bf) {
            CKS(dalloc(c, &c->Gq16, sizeof(uint16_t) * (size_t)dy * c->ldk));
            { to_bf16_rows_kernel<<<dim3(blocks_for(c->ldk), dy), kThreads, 0, c->st>>>(dy, d, c->Gm, c->Gq16, c->ldk); count_launch(); }
            CK(cudaGetLastError());
        }
        CKS(dalloc(c, &c->y, sizeof(double) * std::max(dy, 1)));
        CKS(dalloc(c, &c->y32, sizeof(float) * std::max(dy, 1)));
        if (tg->y) {
            CK(h2d(c, c->y, tg->y, sizeof(double) * dy));
            std::vector<float> y32(tg->y, tg->y + dy);
            CK(h2d(c, c->y32, y32.data(), sizeof(float) * dy));
        }
    }
    CK(cudaStreamSynchronize(c->st));   // the staged host copies are complete before the host arrays go
    return DIAM_OK;
}

// ------------------------------------------------------------------------------------------------ ABI
extern "C" {

const char* diam_status_string(diam_status s) {
    switch (s) {
        case DIAM_OK: return "ok";
        case DIAM_EINVAL: return "invalid argument";
        case DIAM_ENOMEM: return "out of device memory";
        case DIAM_ECUDA: return "CUDA error";
        case DIAM_ENOTSPD: return "covariance not positive definite";
        case DIAM_ETIMEOUT: return "device wait timed out";
        case DIAM_ETARGET: return "target callback failed";
        case DIAM_ESTATE: return "context in error state";
    }
    return "unknown";
}

const char* diam_last_error(const diam_ctx* c) { return c ? c->err.c_str() : "null context"; }

uint64_t diam_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

diam_status diam_config_default(diam_config* cfg, int32_t d, int32_t P) {
    if (!cfg || d <= 0 || P <= 0) return DIAM_EINVAL;
    memset(cfg, 0, sizeof(*cfg));
    cfg->d = d;
    cfg->P = P;
    cfg->n_lag = 100;
    cfg->M = 10;
    cfg->beta0 = std::min(2.4 / std::sqrt((double)d), 0.5);
    cfg->infl = 1.0;
    cfg->adapt_beta = 1;
    cfg->xref_mode = 1;
    cfg->acc_lo = 0.3;
    cfg->acc_hi = 0.5;
    cfg->beta_factor = 1.1;
    cfg->beta_min = 1e-4;
    cfg->beta_max = 0.999;
    cfg->eps_jitter = 1e-10;
    cfg->min_samples_refresh = -1;
    cfg->burnin = 0;
    cfg->refresh_delay = 0;
    cfg->prec = DIAM_FP64;
    cfg->graphs = 1;
    cfg->proposal = DIAM_PROP_DIAM;
    cfg->carry_map = 1;
    cfg->eps_jitter_min = 0.0;
    return DIAM_OK;
}

diam_status diam_init(const diam_config* cfg, const diam_target* tg, const double* x0, const double* C0,
                      const double* xref0, void* stream, diam_ctx** out) {
    if (!cfg || !tg || !out) return DIAM_EINVAL;
    *out = nullptr;
    // an error that an earlier, failed call left in this thread's CUDA error state (a rejected launch or argument;
    // not a sticky device fault, which every call below would report again) is not this context's
    (void)cudaGetLastError();
    if (cfg->d <= 0 || cfg->P <= 0 || cfg->n_lag <= 0 || !(cfg->infl > 0) || !(cfg->beta0 > 0 && cfg->beta0 < 1) ||
        cfg->refresh_delay < 0 || cfg->refresh_delay > 8 || (cfg->prec != DIAM_FP64 && cfg->prec != DIAM_BF16 && cfg->prec != DIAM_FP32) ||
        tg->kind < 0 || tg->kind > DIAM_T_TWISTED || (tg->kind == DIAM_T_CALLBACK && !tg->fn) ||
        (int64_t)cfg->n_lag * cfg->P > (1 << 24) || cfg->trace_steps < 0 ||
        (cfg->proposal != DIAM_PROP_DIAM && cfg->proposal != DIAM_PROP_RW) ||
        (cfg->proposal == DIAM_PROP_RW && tg->kind == DIAM_T_REF_GAUSS) || !(cfg->eps_jitter_min >= 0))
        return DIAM_EINVAL;
    diam_ctx* c = new diam_ctx();
    c->cfg = *cfg;
    if (c->cfg.min_samples_refresh < 0) c->cfg.min_samples_refresh = cfg->d + 1;
    c->kind = tg->kind;
    c->d = cfg->d;
    c->P = cfg->P;
    c->nl = cfg->n_lag;
    c->dy = (tg->kind == DIAM_T_DENSE_GAUSS || tg->kind == DIAM_T_TANH_REG || tg->kind == DIAM_T_TWISTED) ? tg->d_y : 0;
    c->ldk = (cfg->d + 63) / 64 * 64;
    c->bf = cfg->prec != DIAM_FP64;   // the mixed modes: BF16, or BF16 with the factor quantised to TF32
    c->tf32 = cfg->prec == DIAM_FP32;
    c->fn = tg->fn;
    c->user = tg->user;
    c->sigma = tg->sigma;
    c->beta = cfg->beta0;
    c->key = make_key(cfg->seed, cfg->problem_id);
    cudaGetDevice(&c->dev);
    if (stream) {
        c->st = (cudaStream_t)stream;
    } else {
        if (cudaStreamCreateWithFlags(&c->st, cudaStreamNonBlocking) != cudaSuccess) {
            delete c;
            return DIAM_ECUDA;
        }
        c->own_stream = true;
    }
    if (cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess) {
        diam_destroy(c);
        return DIAM_ECUDA;
    }
    diam_status s = alloc_all(c);
    if (s == DIAM_OK && fused_step_fits(c)) s = fused_step(c, true);
    if (s == DIAM_OK && interval_kernel_fits(c)) s = interval_steps(c, 0, true);
    if (s == DIAM_OK && c->bf && rewhiten_tc_fits(c->d, c->ldk) && rewhiten_tc_setup(c->d) != cudaSuccess)
        s = fail(c, DIAM_ECUDA, "cudaFuncSetAttribute");
    if (s == DIAM_OK && c->bf && rewhiten32_smem(c->d, 1) <= 220 * 1024 &&
        allow_max_dynamic_smem((const void*)rewhiten32_kernel) != cudaSuccess)
        s = fail(c, DIAM_ECUDA, "cudaFuncSetAttribute");
    if (s == DIAM_OK) s = upload_target(c, tg);
    if (s == DIAM_OK) s = c->bf ? init_state<float>(c, x0, C0, xref0) : init_state<double>(c, x0, C0, xref0);
    if (s != DIAM_OK) {
        diam_destroy(c);
        return s;
    }
    *out = c;
    return DIAM_OK;
}

diam_status diam_run_batch(diam_ctx* c, int64_t n_steps) {
    CKS(check_usable(c));
    if (c->in_hook) return fail(c, DIAM_EINVAL, "diam_run_batch", "called from the interval hook");
    if (n_steps < 0) return fail(c, DIAM_EINVAL, "diam_run_batch", "n_steps < 0");
    return c->bf ? run_steps<float>(c, n_steps) : run_steps<double>(c, n_steps);
}

__global__ void merge_moments_kernel(int d, double* M2, const double* extM2, const double* delta, double w) {
    int i = blockIdx.y;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j <= i; j += gridDim.x * blockDim.x)
        M2[(size_t)i * d + j] += extM2[(size_t)i * d + j] + delta[i] * delta[j] * w;
}

__global__ void merge_mean_kernel(int d, double* mean, const double* extm, double* delta, double frac) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d) return;
    double dl = extm[i] - mean[i];
    delta[i] = dl;
    mean[i] += dl * frac;
}

// The increment since the last synchronisation: mi = (n m - n0 m0) / ni, delta = m0 - mi (the pairwise
// update of Chan, Golub and LeVeque, M2 = M2_0 + M2_i + delta delta^T n0 ni / n, run backwards).
__global__ void increment_mean_kernel(int d, const double* mean, const double* m0, double n, double n0, double* mi,
                                      double* delta) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d) return;
    const double v = (n * mean[i] - n0 * m0[i]) / (n - n0);
    mi[i] = v;
    delta[i] = m0[i] - v;
}

// out (d x d, full) = M2 - M2_0 - delta delta^T w, from the lower triangles of M2 and M2_0
__global__ void increment_m2_kernel(int d, const double* M2, const double* M20, const double* delta, double w,
                                    double* out) {
    const int r = blockIdx.y;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < d; c += gridDim.x * blockDim.x) {
        const size_t k = (size_t)max(r, c) * d + min(r, c);
        out[(size_t)r * d + c] = M2[k] - M20[k] - delta[r] * delta[c] * w;
    }
}

// The moments as they stand become the reference of the next increment.
static diam_status take_snapshot(diam_ctx* c) {
    const int d = c->d;
    if (!c->snap_mean) {
        CKS(dalloc(c, &c->snap_mean, sizeof(double) * d));
        CKS(dalloc(c, &c->snap_M2, sizeof(double) * d * d));
    }
    CK(cudaMemcpyAsync(c->snap_mean, c->mean, sizeof(double) * d, cudaMemcpyDeviceToDevice, c->st));
    CK(cudaMemcpyAsync(c->snap_M2, c->M2, sizeof(double) * d * d, cudaMemcpyDeviceToDevice, c->st));
    c->snap_n = c->n;
    return DIAM_OK;
}

diam_status diam_set_interval_hook(diam_ctx* c, diam_interval_fn fn, void* user) {
    CKS(check_usable(c));
    if (c->in_hook) return fail(c, DIAM_EINVAL, "diam_set_interval_hook", "inside the hook");
    c->hook = fn;
    c->hook_user = user;
    return DIAM_OK;
}

diam_status diam_flush(diam_ctx* c) {
    CKS(check_usable(c));
    CKS(refresh_finish(c));
    return sync_and_check(c);
}

diam_status diam_sync_moments(diam_ctx* c, const double* ext_mean, const double* ext_M2, int64_t ext_n) {
    CKS(check_usable(c));
    if (ext_n < 0 || (ext_n > 0 && (!ext_mean || !ext_M2))) return fail(c, DIAM_EINVAL, "diam_sync_moments");
    if (ext_n > 0) {
        const int d = c->d;
        double* em = c->svec;  // interval scratch is free between intervals only: use the refresh buffers
        CKS(sync_and_check(c));
        CK(h2d(c, c->Cw, ext_M2, sizeof(double) * d * d));
        CK(h2d(c, c->work, ext_mean, sizeof(double) * d));
        double nn = (double)c->n, ne = (double)ext_n;
        { merge_mean_kernel<<<blocks_for(d), kThreads, 0, c->st>>>(d, c->mean, c->work, em, ne / (nn + ne)); count_launch(); }
        { merge_moments_kernel<<<dim3(blocks_for(d), d), kThreads, 0, c->st>>>(d, c->M2, c->Cw, em, nn * ne / (nn + ne)); count_launch(); }
        CK(cudaGetLastError());
        c->n += ext_n;
    }
    CKS(take_snapshot(c));
    return sync_and_check(c);
}

static diam_status read_moments(diam_ctx* c, double* mean, double* M, int64_t* n, bool as_cov) {
    CKS(check_usable(c));
    CKS(sync_and_check(c));
    const int d = c->d;
    if (mean) CK(d2h(c, mean, c->mean, sizeof(double) * d));
    if (M) {   // scaled and mirrored on the device (the refresh's scratch matrix), then one copy
        const double s = (as_cov && c->n > 0) ? 1.0 / (double)c->n : 1.0;
        { symmetrize_kernel<<<dim3((d + 31) / 32, (d + 31) / 32), dim3(32, 8), 0, c->st>>>(d, c->M2, s, c->Cw); count_launch(); }
        CK(cudaGetLastError());
        CK(d2h(c, M, c->Cw, sizeof(double) * d * d));
    }
    if (n) *n = c->n;
    return DIAM_OK;
}

diam_status diam_get_moments(diam_ctx* c, double* mean, double* cov, int64_t* n) {
    return read_moments(c, mean, cov, n, true);
}

diam_status diam_export_moments(diam_ctx* c, double* mean, double* M2, int64_t* n) {
    return read_moments(c, mean, M2, n, false);
}

diam_status diam_export_increment(diam_ctx* c, double* mean, double* M2, int64_t* n) {
    CKS(check_usable(c));
    if (!c->snap_mean || c->snap_n == 0) return read_moments(c, mean, M2, n, false);   // everything is new
    CKS(sync_and_check(c));
    const int d = c->d;
    const int64_t ni = c->n - c->snap_n;
    if (ni <= 0) {
        if (mean) memset(mean, 0, sizeof(double) * d);
        if (M2) memset(M2, 0, sizeof(double) * d * d);
        if (n) *n = 0;
        return DIAM_OK;
    }
    // the fold's scratch vectors are free between intervals
    const double nn = (double)c->n, n0 = (double)c->snap_n;
    { increment_mean_kernel<<<blocks_for(d), kThreads, 0, c->st>>>(d, c->mean, c->snap_mean, nn, n0, c->svec, c->delta); count_launch(); }
    if (M2) {
        { increment_m2_kernel<<<dim3(blocks_for(d), d), kThreads, 0, c->st>>>(d, c->M2, c->snap_M2, c->delta,
                                                                               n0 * (double)ni / nn, c->Cw); count_launch(); }
    }
    CK(cudaGetLastError());
    if (mean) CK(d2h(c, mean, c->svec, sizeof(double) * d));
    if (M2) CK(d2h(c, M2, c->Cw, sizeof(double) * d * d));
    if (n) *n = ni;
    return DIAM_OK;
}

diam_status diam_get_state(diam_ctx* c, double* x, double* lp, diam_stats* stats) {
    CKS(check_usable(c));
    CKS(sync_and_check(c));
    // with stats, the refreshes in flight are resolved first (they count, and their factors are kept, as in
    // order); the states and log pi do not depend on them (those refreshes use workspaces of their own and
    // are resolved, with the same outcome, at the interval their factor is due), so reading only x or lp
    // leaves them running beside the next intervals
    if (stats) CKS(refresh_finish(c));
    const size_t Pd = (size_t)c->P * c->d;
    if (x) {
        if (c->bf) {
            { convert_kernel<float, double><<<blocks_for(Pd), kThreads, 0, c->st>>>(Pd, (const float*)c->X, c->work); count_launch(); }
            CK(cudaStreamSynchronize(c->st));
            CK(d2h(c, x, c->work, sizeof(double) * Pd));
        } else {
            CK(d2h(c, x, c->X, sizeof(double) * Pd));
        }
    }
    if (lp) CK(d2h(c, lp, c->lp, sizeof(double) * c->P));
    if (stats) {
        unsigned long long acc = 0, nonf = 0;
        CK(d2h(c, &acc, &c->ctl->acc_block, sizeof(acc)));
        CK(d2h(c, &nonf, &c->ctl->nonfinite, sizeof(nonf)));
        stats->steps = c->t;
        stats->n = c->n;
        stats->accepted = c->acc_all + (c->t % c->nl ? (int64_t)acc : 0);
        stats->refreshes = c->refreshes;
        stats->notspd = c->notspd;
        stats->nonfinite = (int64_t)nonf;
        stats->beta = c->beta;
        stats->chol_attempts = c->chol_attempts;
    }
    return DIAM_OK;
}

diam_status diam_get_factor(diam_ctx* c, double* L, double* Lq, double* xref, double* beta) {
    CKS(check_usable(c));
    CKS(sync_and_check(c));
    const int d = c->d;
    if (L) CK(d2h(c, L, c->L, sizeof(double) * d * d));
    if (Lq) CK(d2h(c, Lq, c->Lq64, sizeof(double) * d * d));
    if (xref) CK(d2h(c, xref, c->xref64, sizeof(double) * d));
    if (beta) *beta = c->beta;
    return DIAM_OK;
}

diam_status diam_get_trace(diam_ctx* c, double* lp_prop, double* q_prop, double* q_cur, double* loga, int8_t* acc,
                           int64_t n_steps) {
    CKS(check_usable(c));
    CKS(sync_and_check(c));
    int64_t T = std::min<int64_t>(std::min<int64_t>(c->t, c->tr.steps), n_steps);
    size_t nt = (size_t)std::max<int64_t>(T, 0) * c->P;
    if (nt == 0) return DIAM_OK;
    if (lp_prop) CK(d2h(c, lp_prop, c->tr.lp, nt * 8));
    if (q_prop) CK(d2h(c, q_prop, c->tr.q, nt * 8));
    if (q_cur) CK(d2h(c, q_cur, c->tr.qc, nt * 8));
    if (loga) CK(d2h(c, loga, c->tr.loga, nt * 8));
    if (acc) CK(d2h(c, acc, c->tr.acc, nt));
    return DIAM_OK;
}

diam_status diam_get_block_sums(diam_ctx* c, double* xsum, double* lpsum, int64_t* n_blocks) {
    CKS(check_usable(c));
    if (!n_blocks) return fail(c, DIAM_EINVAL, "diam_get_block_sums");
    CKS(sync_and_check(c));
    // BF16 mode forms an interval's sums when the interval completes (FP64 mode: step by step)
    const int64_t have = c->bf ? c->t / c->nl : (c->t + c->nl - 1) / c->nl;
    int64_t nb = std::min<int64_t>(*n_blocks, std::min<int64_t>(c->bcap, have));
    if (!c->cfg.keep_block_sums) nb = 0;
    if (nb > 0) {
        const size_t n = (size_t)nb * c->P * c->d;
        if (xsum && !c->bf) CK(d2h(c, xsum, c->bsum, sizeof(double) * n));
        if (xsum && c->bf) {   // FP32 sums, widened on the host
            std::vector<float> tmp(n);
            CK(d2h(c, tmp.data(), c->bsum, sizeof(float) * n));
            for (size_t k = 0; k < n; ++k) xsum[k] = (double)tmp[k];
        }
        if (lpsum) CK(d2h(c, lpsum, c->lpsum, sizeof(double) * (size_t)nb * c->P));
    }
    *n_blocks = nb;
    return DIAM_OK;
}

diam_status diam_get_psrf(diam_ctx* c, int64_t first_block, int64_t n_blocks, double* psrf) {
    CKS(check_usable(c));
    CKS(sync_and_check(c));
    const int64_t have = std::min<int64_t>(c->bcap, c->t / c->nl);   // completed intervals
    if (!psrf || !c->cfg.keep_block_sums || c->P < 2 || first_block < 0 || n_blocks < 1 || first_block + n_blocks > have)
        return fail(c, DIAM_EINVAL, "diam_get_psrf", "needs keep_block_sums, P >= 2 and completed intervals");
    const int d = c->d, P = c->P;
    if (!c->psrf_ws) CKS(dalloc(c, &c->psrf_ws, sizeof(double) * 2 * (size_t)P * d + sizeof(double) * d));
    double* cm = c->psrf_ws;
    double* cv = cm + (size_t)P * d;
    double* out = cv + (size_t)P * d;
    const dim3 g((d + 255) / 256, P);
    if (c->bf) {
        { psrf_chain_kernel<float><<<g, 256, 0, c->st>>>(d, P, c->nl, (long long)first_block, (int)n_blocks, (const float*)c->bsum,
                                                      (const float*)c->bm2, 0, cm, cv); count_launch(); }
    } else {
        { psrf_chain_kernel<double><<<g, 256, 0, c->st>>>(d, P, c->nl, (long long)first_block, (int)n_blocks, (const double*)c->bsum,
                                                       (const double*)c->bm2, 1, cm, cv); count_launch(); }
    }
    { psrf_final_kernel<<<(d + 255) / 256, 256, 0, c->st>>>(d, P, (double)n_blocks * c->nl, cm, cv, out); count_launch(); }
    CK(cudaGetLastError());
    CK(d2h(c, psrf, out, sizeof(double) * d));
    return DIAM_OK;
}

// ---- checkpoint: a flat list of (device buffer, bytes) plus the host schedule
struct HostState {
    int64_t t, n, acc_refresh, acc_all, refreshes, notspd, xi_block, begun_block, chol_attempts;
    double beta;
    int64_t pend_block[9];
    int64_t bcap;
};

static std::vector<std::pair<void*, size_t>> state_buffers(diam_ctx* c) {
    const size_t ts = c->bf ? 4 : 8, Pd = (size_t)c->P * c->d, d = (size_t)c->d;
    std::vector<std::pair<void*, size_t>> v = {
        {c->ctl, sizeof(Ctl)}, {c->X, ts * Pd},        {c->Z, ts * Pd},        {c->lp, 8 * (size_t)c->P},
        {c->q, 8 * (size_t)c->P}, {c->xref, ts * d},   {c->xref64, 8 * d},     {c->cenT, ts * d},
        {c->cen64, 8 * d},     {c->L, 8 * d * d},      {c->mean, 8 * d},       {c->M2, 8 * d * d}};
    for (auto& pd : c->pend) {
        v.push_back({pd.L, 8 * d * d});
        v.push_back({pd.mean, 8 * d});
    }
    if (c->tr.steps) {
        size_t nt = (size_t)c->tr.steps * c->P;
        v.push_back({c->tr.lp, nt * 8});
        v.push_back({c->tr.q, nt * 8});
        v.push_back({c->tr.qc, nt * 8});
        v.push_back({c->tr.loga, nt * 8});
        v.push_back({c->tr.acc, nt});
    }
    if (c->bcap) {
        v.push_back({c->bsum, bsum_elt(c) * (size_t)c->bcap * Pd});
        v.push_back({c->bm2, bsum_elt(c) * (size_t)c->bcap * Pd});
        v.push_back({c->lpsum, 8 * (size_t)c->bcap * c->P});
    }
    return v;
}

diam_status diam_save(diam_ctx* c, void* buf, size_t* size) {
    CKS(check_usable(c));
    if (c->in_hook) return fail(c, DIAM_EINVAL, "diam_save", "called from the interval hook");
    if (!size) return fail(c, DIAM_EINVAL, "diam_save");
    CKS(sync_and_check(c));
    CKS(refresh_finish(c));   // the refresh in flight counts (and its factor is saved) as in order
    auto bufs = state_buffers(c);
    size_t total = sizeof(HostState);
    for (auto& b : bufs) total += b.second;
    if (!buf) {
        *size = total;
        return DIAM_OK;
    }
    if (*size < total) return fail(c, DIAM_EINVAL, "diam_save", "buffer too small");
    HostState hs{};
    hs.t = c->t; hs.n = c->n; hs.acc_refresh = c->acc_refresh; hs.acc_all = c->acc_all;
    hs.refreshes = c->refreshes; hs.notspd = c->notspd; hs.xi_block = -1; hs.begun_block = c->begun_block;
    hs.beta = c->beta; hs.bcap = c->bcap; hs.chol_attempts = c->chol_attempts;
    for (size_t i = 0; i < c->pend.size(); ++i) hs.pend_block[i] = c->pend[i].block;
    char* o = (char*)buf;
    memcpy(o, &hs, sizeof(hs));
    o += sizeof(hs);
    for (auto& b : bufs) {
        CK(d2h(c, o, b.first, b.second));
        o += b.second;
    }
    *size = total;
    return DIAM_OK;
}

diam_status diam_load(diam_ctx* c, const void* buf, size_t size) {
    CKS(check_usable(c));
    if (c->in_hook) return fail(c, DIAM_EINVAL, "diam_load", "called from the interval hook");
    if (!buf || size < sizeof(HostState)) return fail(c, DIAM_EINVAL, "diam_load");
    HostState hs;
    memcpy(&hs, buf, sizeof(hs));
    CKS(sync_and_check(c));
    CKS(refresh_finish(c));   // nothing may still write the pending factors
    if (hs.bcap > c->bcap) {  // grow the interval-sum store to the saved capacity
        void* nb = nullptr;
        double* nlp = nullptr;
        void* nq = nullptr;
        CKS(dalloc(c, (char**)&nb, bsum_elt(c) * (size_t)hs.bcap * c->P * c->d));
        CKS(dalloc(c, (char**)&nq, bsum_elt(c) * (size_t)hs.bcap * c->P * c->d));
        CKS(dalloc(c, &nlp, sizeof(double) * (size_t)hs.bcap * c->P));
        c->bsum = nb;
        c->bm2 = nq;
        c->lpsum = nlp;
        c->bcap = hs.bcap;
    }
    if (hs.bcap != c->bcap) return fail(c, DIAM_EINVAL, "diam_load", "checkpoint does not match this context");
    auto bufs = state_buffers(c);
    size_t total = sizeof(HostState);
    for (auto& b : bufs) total += b.second;
    if (total != size) return fail(c, DIAM_EINVAL, "diam_load", "checkpoint does not match this context");
    const char* in = (const char*)buf + sizeof(hs);
    for (auto& b : bufs) {
        CK(h2d(c, b.first, in, b.second));
        in += b.second;
    }
    c->t = hs.t; c->n = hs.n; c->acc_refresh = hs.acc_refresh; c->acc_all = hs.acc_all;
    c->refreshes = hs.refreshes; c->notspd = hs.notspd; c->begun_block = hs.begun_block; c->beta = hs.beta;
    c->chol_attempts = hs.chol_attempts;
    for (size_t i = 0; i < c->pend.size(); ++i) c->pend[i].block = hs.pend_block[i];
    c->xi_block = -1;  // noise products are regenerated from the counter-based streams
    c->snap_n = 0;     // the next increment counts from here: every loaded sample is new
    if (c->graph) {
        cudaGraphExecDestroy(c->graph);
        c->graph = nullptr;
    }
    CKS(quantise(c));
    CKS(rec_factor(c));
    CKS(rec_xref(c));
    c->ax_dirty = true;
    return sync_and_check(c);
}

diam_status diam_get_profile(diam_ctx* c, int64_t* counts, double* ms, int32_t reset) {
    CKS(check_usable(c));
    CKS(sync_and_check(c));
    prof_flush(c);
    for (int i = 0; i < DIAM_N_PHASES; ++i) {
        if (counts) counts[i] = c->prof_cnt[i];
        if (ms) ms[i] = c->prof_ms[i];
        if (reset) {
            c->prof_cnt[i] = 0;
            c->prof_ms[i] = 0.0;
        }
    }
    return DIAM_OK;
}

diam_status diam_da_config_default(diam_da_config* g) {
    if (!g) return DIAM_EINVAL;
    memset(g, 0, sizeof(*g));
    g->h1 = 512;
    g->h2 = 512;
    g->retrain_every = 20;
    g->ring = 200000;
    g->train_steps = 200;
    g->batch = 1024;
    g->first_train_min = 20000;
    g->lr = 1e-3;
    g->beta1 = 0.9;
    g->beta2 = 0.999;
    g->adam_eps = 1e-8;
    g->rmse_bound = 0.5;
    g->seed = 12345;
    return DIAM_OK;
}

diam_status diam_da_enable(diam_ctx* c, const diam_da_config* g, const double* W1, const double* b1, const double* W2,
                           const double* b2, const double* w3, const double* b3) {
    CKS(check_usable(c));
    if (!g || !W1 || !b1 || !W2 || !b2 || !w3 || !b3) return fail(c, DIAM_EINVAL, "diam_da_enable");
    if (!c->bf || (c->kind != TK_DENSE && c->kind != TK_TANH) || c->P > 1024 || c->da || is_rw(c))
        return fail(c, DIAM_EINVAL, "diam_da_enable",
                    "needs BF16 mode, a linear-map target, the DIAM proposal, P <= 1024, once");
    if (g->h1 <= 0 || g->h2 <= 0 || g->h1 % 128 || g->h2 % 128 || g->batch <= 0 || g->batch % 128 || g->ring < 100 ||
        g->train_steps < 0 || g->retrain_every <= 0)
        return fail(c, DIAM_EINVAL, "diam_da_enable", "bad surrogate configuration");
    return da_alloc(c, g, W1, b1, W2, b2, w3, b3);
}

diam_status diam_da_train(diam_ctx* c, double* rmse) {
    CKS(check_usable(c));
    if (!c->da) return fail(c, DIAM_EINVAL, "diam_da_train", "delayed acceptance not enabled");
    return da_train_now(c, rmse);
}

diam_status diam_da_get_stats(diam_ctx* c, diam_da_stats* s) {
    CKS(check_usable(c));
    if (!c->da || !s) return fail(c, DIAM_EINVAL, "diam_da_get_stats");
    CKS(sync_and_check(c));
    DaCounters hc{};
    CK(d2h(c, &hc, c->da->cnt, sizeof(hc)));
    s->trainings = c->da->trainings;
    s->stage1_tested = (int64_t)hc.tested;
    s->stage1_passed = (int64_t)hc.passed;
    s->exact_evals = (int64_t)hc.exact;
    s->ring_filled = hc.filled;
    s->last_rmse = c->da->last_rmse;
    s->active = c->da->active ? 1 : 0;
    s->pad = 0;
    return DIAM_OK;
}

diam_status diam_da_adam_step(diam_ctx* c, const double* gW1, const double* gb1, const double* gW2, const double* gb2,
                              const double* gw3, const double* gb3) {
    CKS(check_usable(c));
    if (!c->da || !gW1 || !gb1 || !gW2 || !gb2 || !gw3 || !gb3) return fail(c, DIAM_EINVAL, "diam_da_adam_step");
    DaState* a = c->da;
    const int d = c->d, h1 = a->h1, h2 = a->h2;
    CKS(sync_and_check(c));
    // the gradient buffers in the layouts the training writes: dW1 as [d][h1], dW2 as [h1][h2]
    std::vector<float> t((size_t)c->ldk * h1, 0.f);
    for (int i = 0; i < h1; ++i)
        for (int k = 0; k < d; ++k) t[(size_t)k * h1 + i] = (float)gW1[(size_t)i * d + k];
    CK(h2d(c, a->gW1T, t.data(), sizeof(float) * t.size()));
    t.assign((size_t)h1 * h2, 0.f);
    for (int o = 0; o < h2; ++o)
        for (int i = 0; i < h1; ++i) t[(size_t)i * h2 + o] = (float)gW2[(size_t)o * h1 + i];
    CK(h2d(c, a->gW2T, t.data(), sizeof(float) * t.size()));
    auto up = [&](float* dst, const double* src, size_t n) -> diam_status {
        std::vector<float> v(src, src + n);
        CK(h2d(c, dst, v.data(), sizeof(float) * n));
        return DIAM_OK;
    };
    CKS(up(a->gb1, gb1, h1)); CKS(up(a->gb2, gb2, h2)); CKS(up(a->gw3, gw3, h2)); CKS(up(a->gb3, gb3, 1));
    da_adam(c);
    CK(cudaGetLastError());
    return sync_and_check(c);
}

diam_status diam_da_get_weights(diam_ctx* c, double* W1, double* b1, double* W2, double* b2, double* w3, double* b3) {
    CKS(check_usable(c));
    if (!c->da) return fail(c, DIAM_EINVAL, "diam_da_get_weights");
    CKS(sync_and_check(c));
    DaState* a = c->da;
    auto down = [&](double* dst, const float* src, size_t n) -> diam_status {
        if (!dst) return DIAM_OK;
        std::vector<float> t(n);
        CK(d2h(c, t.data(), src, sizeof(float) * n));
        for (size_t i = 0; i < n; ++i) dst[i] = t[i];
        return DIAM_OK;
    };
    CKS(down(W1, a->W1, (size_t)a->h1 * c->d)); CKS(down(b1, a->b1, a->h1)); CKS(down(W2, a->W2, (size_t)a->h2 * a->h1));
    CKS(down(b2, a->b2, a->h2)); CKS(down(w3, a->w3, a->h2)); CKS(down(b3, a->b3, 1));
    return DIAM_OK;
}

diam_status diam_da_grad(diam_ctx* c, int32_t B, const double* U, const double* t, double* loss, double* gW1,
                         double* gb1, double* gW2, double* gb2, double* gw3, double* gb3) {
    CKS(check_usable(c));
    if (!c->da || !U || !t || B <= 0 || B % 128 || B > c->da->B) return fail(c, DIAM_EINVAL, "diam_da_grad");
    DaState* a = c->da;
    const int d = c->d, ldk = c->ldk, h1 = a->h1, h2 = a->h2;
    std::vector<uint16_t> xb((size_t)B * ldk, 0);
    for (int b = 0; b < B; ++b)
        for (int i = 0; i < d; ++i) {
            float f = (float)round_bf16(U[(size_t)b * d + i]);
            uint32_t bits;
            memcpy(&bits, &f, 4);
            xb[(size_t)b * ldk + i] = (uint16_t)(bits >> 16);
        }
    std::vector<float> tf(t, t + B);
    CK(h2d(c, a->Xb, xb.data(), sizeof(uint16_t) * xb.size()));
    CK(h2d(c, a->tb, tf.data(), sizeof(float) * B));
    const int saveB = a->B;
    a->B = B;
    diam_status s = da_backward(c);
    a->B = saveB;
    CKS(s);
    CKS(sync_and_check(c));
    std::vector<double> lpart(B);
    CK(d2h(c, lpart.data(), a->loss_parts, sizeof(double) * B));
    if (loss) {
        double L = 0.0;
        for (double v : lpart) L += v;
        *loss = L;
    }
    std::vector<float> g;
    if (gW1) {
        g.resize((size_t)ldk * h1);
        CK(d2h(c, g.data(), a->gW1T, sizeof(float) * g.size()));
        for (int i = 0; i < h1; ++i)
            for (int k = 0; k < d; ++k) gW1[(size_t)i * d + k] = g[(size_t)k * h1 + i];
    }
    if (gW2) {
        g.resize((size_t)h1 * h2);
        CK(d2h(c, g.data(), a->gW2T, sizeof(float) * g.size()));
        for (int o = 0; o < h2; ++o)
            for (int i = 0; i < h1; ++i) gW2[(size_t)o * h1 + i] = g[(size_t)i * h2 + o];
    }
    auto down = [&](double* dst, const float* src, size_t n) -> diam_status {
        if (!dst) return DIAM_OK;
        std::vector<float> tt(n);
        CK(d2h(c, tt.data(), src, sizeof(float) * n));
        for (size_t i = 0; i < n; ++i) dst[i] = tt[i];
        return DIAM_OK;
    };
    CKS(down(gb1, a->gb1, h1)); CKS(down(gb2, a->gb2, h2)); CKS(down(gw3, a->gw3, h2)); CKS(down(gb3, a->gb3, 1));
    return DIAM_OK;
}

void diam_destroy(diam_ctx* c) {
    if (!c || c->in_hook) return;
    cudaSetDevice(c->dev);
    for (auto& r : c->ar)
        if (r.rs) cudaStreamSynchronize(r.rs);   // a refresh still in flight
    if (c->st) cudaStreamSynchronize(c->st);
    for (auto& e : c->evts) {
        cudaEventDestroy(e.a);
        cudaEventDestroy(e.b);
    }
    if (c->graph) cudaGraphExecDestroy(c->graph);
    if (c->chol_graph.exec) cudaGraphExecDestroy(c->chol_graph.exec);
    if (c->trsm_graph.exec) cudaGraphExecDestroy(c->trsm_graph.exec);
    ozaki_ws_release(c->oz);
    for (auto& r : c->ar) {
        if (r.graph.exec) cudaGraphExecDestroy(r.graph.exec);
        ozaki_ws_release(r.oz);
    }
    for (void* p : c->allocs) cudaFree(p);
    if (c->side) {
        cudaStreamSynchronize(c->side);
        cudaStreamDestroy(c->side);
    }
    if (c->stage) {
        for (cudaEvent_t e : c->stage_ev) cudaEventSynchronize(e), cudaEventDestroy(e);
        cudaFreeHost(c->stage);
    }
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    for (auto& r : c->ar) {
        if (r.rs) cudaStreamDestroy(r.rs);
        for (cudaEvent_t e : {r.fork, r.start, r.done})
            if (e) cudaEventDestroy(e);
    }
    if (c->own_stream && c->st) cudaStreamDestroy(c->st);
    delete c->da;
    delete c;
}

}  // extern "C"
