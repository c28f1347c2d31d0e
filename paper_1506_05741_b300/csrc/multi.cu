// multi.cu -- many independent DIAM problems driven together (include/diam.h, diam_multi_*).
//
// Each problem is an ordinary sampler context on a stream of its own. A run gives every problem a host
// thread that calls diam_run_batch on it; whole intervals replay that problem's captured graph, and the
// per-interval host work (beta rule, refresh decision, Cholesky) of one problem overlaps the GPU work of
// the others. Problems share nothing, so the result of each equals its run alone.
#include <cuda_runtime.h>

#include <algorithm>
#include <thread>
#include <vector>

#include "../../include/diam.h"

struct diam_multi {
    std::vector<diam_ctx*> ctx;
    std::vector<cudaStream_t> streams;
    int dev = 0;
};

extern "C" {

diam_status diam_multi_init(int32_t n, const diam_config* cfgs, const diam_target* targets, const double* const* x0,
                            const double* const* C0, diam_multi** out) {
    if (n <= 0 || !cfgs || !targets || !out) return DIAM_EINVAL;
    *out = nullptr;
    diam_multi* m = new diam_multi();
    cudaGetDevice(&m->dev);
    for (int j = 0; j < n; ++j) {
        cudaStream_t s = nullptr;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
            diam_multi_destroy(m);
            return DIAM_ECUDA;
        }
        m->streams.push_back(s);
        diam_ctx* c = nullptr;
        diam_status st = diam_init(&cfgs[j], &targets[j], x0 ? x0[j] : nullptr, C0 ? C0[j] : nullptr, nullptr, (void*)s, &c);
        if (st != DIAM_OK) {
            diam_multi_destroy(m);
            return st;
        }
        m->ctx.push_back(c);
    }
    *out = m;
    return DIAM_OK;
}

diam_status diam_multi_run(diam_multi* m, int64_t n_steps) {
    if (!m || n_steps < 0) return DIAM_EINVAL;
    const size_t n = m->ctx.size();
    std::vector<diam_status> st(n, DIAM_OK);
    std::vector<std::thread> th;
    th.reserve(n);
    for (size_t j = 0; j < n; ++j)
        th.emplace_back([m, j, n_steps, &st] {
            cudaSetDevice(m->dev);
            st[j] = diam_run_batch(m->ctx[j], n_steps);
        });
    for (auto& t : th) t.join();
    for (diam_status s : st)
        if (s != DIAM_OK) return s;
    return DIAM_OK;
}

diam_ctx* diam_multi_context(diam_multi* m, int32_t j) {
    if (!m || j < 0 || (size_t)j >= m->ctx.size()) return nullptr;
    return m->ctx[(size_t)j];
}

void diam_multi_destroy(diam_multi* m) {
    if (!m) return;
    cudaSetDevice(m->dev);
    for (diam_ctx* c : m->ctx) diam_destroy(c);
    for (cudaStream_t s : m->streams) cudaStreamDestroy(s);
    delete m;
}

}  // extern "C"
