// da_host.cuh -- host side of the delayed-acceptance surrogate (included by api.cu, after the context and
// its helpers). Two-stage Metropolis-Hastings (Christen & Fox, 2005) with an MLP surrogate of log pi; the
// paper has no surrogate. Per step: surrogate of every proposal (two tcgen05 GEMMs with the GELU epilogue
// and an output dot product), stage-1 screen with survivor compaction, exact target only for the
// survivors (split-K GEMM with a device-side row count), stage-2 test. Per training: Adam steps on
// minibatches from the ring of exactly evaluated pairs, then the held-out RMSE decides whether stage 1 runs.
#pragma once
#include "da_kernels.cuh"

struct DaState {
    diam_da_config cfg{};
    int h1 = 0, h2 = 0, B = 0;
    bool active = false;
    int64_t trainings = 0, adam_t = 0, intervals = 0;
    double last_rmse = NAN, mu = 0.0, sigma = 1.0;
    // FP32 master weights, Adam moments, BF16 copies
    float *W1 = nullptr, *b1 = nullptr, *W2 = nullptr, *b2 = nullptr, *w3 = nullptr, *b3 = nullptr;
    float *mW1, *vW1, *mb1, *vb1, *mW2, *vW2, *mb2, *vb2, *mw3, *vw3, *mb3, *vb3;
    uint16_t *W1q = nullptr, *W2q = nullptr, *W2Tq = nullptr;
    float *shift = nullptr, *scale = nullptr;
    // per step
    uint16_t *U = nullptr, *H1 = nullptr, *H2 = nullptr, *Chi = nullptr, *Clo = nullptr;
    double *s_prop = nullptr, *s_cur = nullptr, *qsave = nullptr;
    int* idx = nullptr;
    DaCounters* cnt = nullptr;
    // ring of exactly evaluated pairs
    uint16_t* ring_x = nullptr;
    float* ring_lp = nullptr;
    // training
    uint16_t *Xb, *XbT, *H1b, *H2b, *H1T, *dZ2, *dZ2T, *dZ1T;
    float *tb, *raw_lp, *Z1, *Z2, *ds, *dZ2f, *dH1, *dZ1f, *gW1T, *gW2T, *gb1, *gb2, *gw3, *gb3;
    float* cs_part;   // COLSUM_CHUNKS x max(h1, h2): the column sums' partial sums
    double *loss_parts, *sbatch, *stats;
    double* musig;   // device copy of (mu, sigma)
    // a training's steps replayed as one captured step: the step counter (current, first) and the Adam bias
    // corrections of every step of the training, computed on the host as the eager steps compute them
    long long* tdev = nullptr;
    float* c12 = nullptr;
    Key key{};
};

static diam_status da_forward(diam_ctx* c, int rows, const uint16_t* U, uint16_t* H1, uint16_t* H2, float* Z1, float* Z2,
                              double* s_out) {
    DaState* a = c->da;
    TcEpi e1{};
    e1.mode = TC_GELU;
    e1.Hout = H1;
    e1.ldo = a->h1;
    e1.Zout = Z1;
    e1.ldz = a->h1;
    e1.bias = a->b1;
    // the network's products are small (a few hundred by a minibatch): 32-column tiles give four times the CTAs
    CK(tc_gemm_bf16(a->h1, rows, c->ldk, a->W1q, c->ldk, U, nullptr, c->ldk, 0, e1, &c->ctl->status, c->st, 32));
    TcEpi e2{};
    e2.mode = TC_GELU;
    e2.Hout = H2;
    e2.ldo = a->h2;
    e2.Zout = Z2;
    e2.ldz = a->h2;
    e2.bias = a->b2;
    CK(tc_gemm_bf16(a->h2, rows, a->h1, a->W2q, a->h1, H1, nullptr, a->h1, 0, e2, &c->ctl->status, c->st, 32));
    if (s_out) {
        { mlp_out_kernel<<<blocks_for(rows), kThreads, 0, c->st>>>(rows, a->h2, H2, a->w3, a->b3, a->musig, s_out); count_launch(); }
    }
    CK(cudaGetLastError());
    return DIAM_OK;
}

// s(x) of every chain's current state (after a training changed the surrogate)
static diam_status da_refresh_s_cur(diam_ctx* c) {
    DaState* a = c->da;
    { mlp_input_kernel<float><<<dim3(c->P, 4), kThreads, 0, c->st>>>(c->d, (const float*)c->X, a->shift, a->scale, a->U, c->ldk); count_launch(); }
    CKS(da_forward(c, c->P, a->U, a->H1, a->H2, nullptr, nullptr, a->s_cur));
    // plus the exact O(d) terms of the current states
    { od_terms_kernel<float><<<c->P, kThreads, 0, c->st>>>(c->d, (const float*)c->X, c->lpo, c->tg, nullptr, nullptr, c->ldk); count_launch(); }
    { add_kernel<<<blocks_for(c->P), kThreads, 0, c->st>>>(c->P, c->lpo, a->s_cur); count_launch(); }
    CK(cudaGetLastError());
    return DIAM_OK;
}

// Forward + backward on the minibatch in a->Xb / a->tb (B rows): gradients into a->g*, loss parts.
// out = the column sums of the B x cols matrix M (rows weighted by wrow when given), two fixed-order passes
template <typename MT>
static void da_colsum(diam_ctx* c, int B, int cols, const MT* M, const float* wrow, float* out) {
    DaState* a = c->da;
    { colsum_part_kernel<MT><<<dim3((cols + 31) / 32, COLSUM_CHUNKS), 256, 0, c->st>>>(B, cols, M, wrow, a->cs_part); count_launch(); }
    { colsum_final_kernel<<<blocks_for(cols), kThreads, 0, c->st>>>(cols, COLSUM_CHUNKS, a->cs_part, out); count_launch(); }
}

static diam_status da_backward(diam_ctx* c) {
    DaState* a = c->da;
    const int B = a->B, h1 = a->h1, h2 = a->h2;
    CKS(da_forward(c, B, a->Xb, a->H1b, a->H2b, a->Z1, a->Z2, nullptr));
    { loss_grad_kernel<<<(B + 7) / 8, 256, 0, c->st>>>(B, h2, a->H2b, a->Z2, a->w3, a->b3, a->tb, a->ds, a->dZ2f, a->dZ2, a->dZ2T,
                                                     a->loss_parts); count_launch(); }
    da_colsum<uint16_t>(c, B, h2, a->H2b, a->ds, a->gw3);
    da_colsum<float>(c, B, 1, a->ds, nullptr, a->gb3);
    da_colsum<float>(c, B, h2, a->dZ2f, nullptr, a->gb2);
    // dW2 (as [h1][h2]) = sum_b H1[b][i] dZ2[b][o]
    { transpose_bf16_kernel<<<dim3((h1 + 31) / 32, (B + 31) / 32), dim3(32, 8), 0, c->st>>>(a->H1b, h1, B, h1, a->H1T, B); count_launch(); }
    TcEpi ew{};
    ew.mode = TC_STORE;
    ew.D = a->gW2T;
    ew.ldd = h2;
    CK(tc_gemm_bf16(h2, h1, B, a->dZ2T, B, a->H1T, nullptr, B, 0, ew, &c->ctl->status, c->st, 32));
    // dH1 = dZ2 W2, then dZ1 = dH1 * GELU'(Z1)
    TcEpi eh{};
    eh.mode = TC_STORE;
    eh.D = a->dH1;
    eh.ldd = h1;
    CK(tc_gemm_bf16(h1, B, h2, a->W2Tq, h2, a->dZ2, nullptr, h2, 0, eh, &c->ctl->status, c->st, 32));
    { dz1_kernel<<<blocks_for((size_t)B * h1), kThreads, 0, c->st>>>(B, h1, a->dH1, a->Z1, a->dZ1f, a->dZ1T); count_launch(); }
    da_colsum<float>(c, B, h1, a->dZ1f, nullptr, a->gb1);
    // dW1 (as [d][h1]) = sum_b U[b][k] dZ1[b][i]
    { transpose_bf16_kernel<<<dim3((c->ldk + 31) / 32, (B + 31) / 32), dim3(32, 8), 0, c->st>>>(a->Xb, c->ldk, B, c->ldk, a->XbT, B); count_launch(); }
    TcEpi e1{};
    e1.mode = TC_STORE;
    e1.D = a->gW1T;
    e1.ldd = h1;
    CK(tc_gemm_bf16(h1, c->ldk, B, a->dZ1T, B, a->XbT, nullptr, B, 0, e1, &c->ctl->status, c->st));
    CK(cudaGetLastError());
    return DIAM_OK;
}

// graph: the bias corrections and the step are read from a->c12 / a->tdev (a step captured for replay); the caller
// advances a->adam_t by the replays.
static void da_adam(diam_ctx* c, bool graph = false) {
    DaState* a = c->da;
    const diam_da_config& g = a->cfg;
    if (!graph) a->adam_t++;
    const float c1 = graph ? 0.f : (float)(1.0 - std::pow(g.beta1, (double)a->adam_t));
    const float c2 = graph ? 0.f : (float)(1.0 - std::pow(g.beta2, (double)a->adam_t));
    const float* c12 = graph ? a->c12 : nullptr;
    const long long* tdev = graph ? a->tdev : nullptr;
    const float lr = (float)g.lr, b1 = (float)g.beta1, b2 = (float)g.beta2, ep = (float)g.adam_eps;
    const int h1 = a->h1, h2 = a->h2, d = c->d;
    auto launch = [&](int rows, int cols, float* th, const float* gr, int gt, int ldg, float* m, float* v, uint16_t* q, int ldq,
                      uint16_t* qt, int ldqt) {
        unsigned nb = std::min<unsigned>(148 * 8, blocks_for((size_t)rows * cols));
        { adam_kernel<<<nb, kThreads, 0, c->st>>>(rows, cols, th, gr, gt, ldg, m, v, lr, b1, b2, ep, c1, c2, q, ldq, qt, ldqt,
                                                  c12, tdev); count_launch(); }
    };
    launch(h1, d, a->W1, a->gW1T, 1, h1, a->mW1, a->vW1, a->W1q, c->ldk, nullptr, 0);
    launch(1, h1, a->b1, a->gb1, 0, 0, a->mb1, a->vb1, nullptr, 0, nullptr, 0);
    launch(h2, h1, a->W2, a->gW2T, 1, h2, a->mW2, a->vW2, a->W2q, h1, a->W2Tq, h2);
    launch(1, h2, a->b2, a->gb2, 0, 0, a->mb2, a->vb2, nullptr, 0, nullptr, 0);
    launch(1, h2, a->w3, a->gw3, 0, 0, a->mw3, a->vw3, nullptr, 0, nullptr, 0);
    launch(1, 1, a->b3, a->gb3, 0, 0, a->mb3, a->vb3, nullptr, 0, nullptr, 0);
}

// The training's steps as one captured step replayed train_steps times (the same kernels and arguments as the
// eager steps; the minibatch counter and the bias corrections come from device memory). *done false if the
// context's stream cannot be captured: nothing was launched, and the caller runs the steps one by one.
static diam_status da_train_graph(diam_ctx* c, bool* done) {
    *done = false;
    DaState* a = c->da;
    const diam_da_config& g = a->cfg;
    const int steps = g.train_steps;
    if (steps <= 0) {
        *done = true;
        return DIAM_OK;
    }
    std::vector<float> cc(2 * (size_t)steps);
    for (int s = 0; s < steps; ++s) {   // step s of the training is Adam step adam_t + s + 1
        cc[2 * s] = (float)(1.0 - std::pow(g.beta1, (double)(a->adam_t + s + 1)));
        cc[2 * s + 1] = (float)(1.0 - std::pow(g.beta2, (double)(a->adam_t + s + 1)));
    }
    const long long t0[2] = {a->adam_t, a->adam_t};
    if (cudaMemcpyAsync(a->c12, cc.data(), sizeof(float) * cc.size(), cudaMemcpyHostToDevice, c->st) != cudaSuccess ||
        cudaMemcpyAsync(a->tdev, t0, sizeof(t0), cudaMemcpyHostToDevice, c->st) != cudaSuccess ||
        cudaStreamSynchronize(c->st) != cudaSuccess) {
        cudaGetLastError();
        return DIAM_OK;
    }
    cudaGraph_t gr = nullptr;
    const unsigned long long l0 = g_launches.load();
    if (cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return DIAM_OK;
    }
    { gather_batch_kernel<<<a->B, kThreads, 0, c->st>>>(a->key, 0, 0, 0, a->ring_x, a->ring_lp, a->cnt, c->d, c->ldk, a->shift,
                                                      a->scale, a->mu, a->sigma, a->Xb, a->tb, nullptr, a->tdev); count_launch(); }
    const diam_status bs = da_backward(c);
    da_adam(c, true);
    { step_count_kernel<<<1, 1, 0, c->st>>>(a->tdev); count_launch(); }
    const cudaError_t ec = cudaStreamEndCapture(c->st, &gr);
    const unsigned long long per = g_launches.load() - l0;
    g_launches.fetch_sub(per);
    cudaGraphExec_t ex = nullptr;
    if (bs != DIAM_OK || ec != cudaSuccess || cudaGraphInstantiate(&ex, gr, 0) != cudaSuccess) {
        if (gr) cudaGraphDestroy(gr);
        cudaGetLastError();
        return DIAM_OK;
    }
    cudaGraphDestroy(gr);
    *done = true;   // from here on the training is this graph's, whether its launches succeed or not
    cudaError_t el = cudaSuccess;
    int s = 0;
    for (; s < steps && el == cudaSuccess; ++s) el = cudaGraphLaunch(ex, c->st);
    cudaGraphExecDestroy(ex);
    g_launches.fetch_add(per * (unsigned long long)s);
    a->adam_t += s;
    if (el != cudaSuccess) return fail(c, DIAM_ECUDA, "diam_da_train", cudaGetErrorString(el));
    return DIAM_OK;
}

static diam_status da_train_now(diam_ctx* c, double* rmse_out) {
    DaState* a = c->da;
    int e0 = ph_begin(c, PH_TRAIN);
    CKS(sync_and_check(c));
    DaCounters hc{};
    CK(d2h(c, &hc, a->cnt, sizeof(hc)));
    if (hc.filled < 20) return fail(c, DIAM_EINVAL, "diam_da_train", "ring buffer holds too few pairs");
    // normalisation frozen for this surrogate: shift = x_ref, scale = 1/sqrt(C_ii), targets (lp - mu)/sigma
    CK(cudaMemcpyAsync(a->shift, c->xref, sizeof(float) * c->d, cudaMemcpyDeviceToDevice, c->st));
    if (c->n > 0) {
        { feature_scale_kernel<<<blocks_for(c->d), kThreads, 0, c->st>>>(c->d, c->M2, 1.0 / (double)c->n, a->scale); count_launch(); }
    }
    { ring_lp_stats_kernel<<<1, 1024, 0, c->st>>>(a->ring_lp, a->cnt, a->stats); count_launch(); }
    double st3[3] = {0, 0, 0};
    CK(cudaMemcpyAsync(st3, a->stats, sizeof(st3), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    const double ntr = std::max(1.0, st3[2]);
    a->mu = st3[0] / ntr;
    a->sigma = std::sqrt(std::max(1e-30, st3[1] / ntr - a->mu * a->mu));
    const double ms[2] = {a->mu, a->sigma};
    CK(cudaMemcpyAsync(a->musig, ms, sizeof(ms), cudaMemcpyHostToDevice, c->st));
    bool graphed = false;
    CKS(da_train_graph(c, &graphed));
    if (!graphed) {   // the steps one by one (a stream that cannot be captured)
        for (int s = 0; s < a->cfg.train_steps; ++s) {
            { gather_batch_kernel<<<a->B, kThreads, 0, c->st>>>(a->key, a->adam_t, 0, 0, a->ring_x, a->ring_lp, a->cnt, c->d,
                                                              c->ldk, a->shift, a->scale, a->mu, a->sigma, a->Xb, a->tb,
                                                              nullptr); count_launch(); }
            CKS(da_backward(c));
            da_adam(c);
        }
    }
    // held-out RMSE (slots 10 j + 9), in minibatch-sized chunks, at most 8 chunks
    CK(cudaMemsetAsync(a->stats, 0, sizeof(double), c->st));
    const long long nho = hc.filled / 10;
    long long used = 0;
    for (long long first = 0; first < nho && first < 8LL * a->B; first += a->B) {
        const int rows = (int)std::min<long long>(a->B, nho - first);
        { gather_batch_kernel<<<rows, kThreads, 0, c->st>>>(a->key, 0, 1, first, a->ring_x, a->ring_lp, a->cnt, c->d, c->ldk,
                                                          a->shift, a->scale, a->mu, a->sigma, a->Xb, a->tb, a->raw_lp); count_launch(); }
        CKS(da_forward(c, rows, a->Xb, a->H1b, a->H2b, nullptr, nullptr, a->sbatch));
        { sq_err_kernel<<<1, kThreads, 0, c->st>>>(rows, a->sbatch, a->raw_lp, a->stats); count_launch(); }
        used += rows;
    }
    double se = 0.0;
    CK(cudaMemcpyAsync(&se, a->stats, sizeof(double), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    a->last_rmse = used > 0 ? std::sqrt(se / (double)used) : NAN;
    a->active = used > 0 && a->last_rmse <= a->cfg.rmse_bound;
    a->trainings++;
    CKS(da_refresh_s_cur(c));
    ph_end(c, e0);
    if (rmse_out) *rmse_out = a->last_rmse;
    return sync_and_check(c);
}

// Per-step DA path (BF16 mode, linear-map target): screen, compact, exact test for the survivors. The
// network estimates the linear-map part of log pi only; the O(d) terms enter the surrogate exactly.
static diam_status da_step(diam_ctx* c) {
    DaState* a = c->da;
    const int P = c->P;
    int e0 = ph_begin(c, PH_SCREEN);
    if (a->active) {
        { mlp_input_kernel<float><<<dim3(P, 4), kThreads, 0, c->st>>>(c->d, (const float*)c->Xp, a->shift, a->scale, a->U, c->ldk); count_launch(); }
        CKS(da_forward(c, P, a->U, a->H1, a->H2, nullptr, nullptr, a->s_prop));
    }
    const int nthr = (P + 31) / 32 * 32;
    { stage1_kernel<<<1, nthr, 0, c->st>>>(P, c->nchunk, c->key, c->ctl, a->active ? 1 : 0, c->qpart, c->lpart, inv_infl2(c), c->q, a->s_prop,
                                         a->s_cur, a->qsave, a->idx, c->accf, nullptr, a->cnt, c->tr); count_launch(); }
    // stage 1 off: every chain passes in chain order, so the exact test reads the proposals' rows in place
    const uint16_t* bh = c->op_hi;
    const uint16_t* bl = c->op_lo;
    if (a->active && !c->rec) {
        { gather_rows_kernel<<<P, kThreads, 0, c->st>>>(a->cnt, a->idx, c->op_hi, c->op_lo, a->Chi, a->Clo, c->ldk); count_launch(); }
        bh = a->Chi;
        bl = a->Clo;
    }
    CK(cudaGetLastError());
    ph_end(c, e0);
    int e1 = ph_begin(c, PH_TARGET);
    const float inv2s2 = (float)(1.0 / (2.0 * c->sigma * c->sigma));
    if (c->rec) {   // the map carried through the proposal: every chain's map terms at O(d_y) cost
        { rec_map_kernel<<<P, kThreads, 0, c->st>>>(P, c->dy, c->ctl, c->Ax, c->axref, c->AXi, c->Axp, c->y32, inv2s2,
                                                   c->kind == TK_TANH, c->lmap); count_launch(); }
        { finish_da_kernel<<<P, kThreads, 0, c->st>>>(P, c->dy, 0, nullptr, c->y32, inv2s2, c->kind == TK_TANH, c->nchunk,
                                                    c->key, c->lpart, a->qsave, a->idx, a->cnt, a->active ? 1 : 0, a->s_prop,
                                                    a->s_cur, c->lp, c->q, c->accf, c->ctl, c->tr, c->op_hi, a->ring_x,
                                                    a->ring_lp, (long long)a->cfg.ring, c->ldk, c->lmap); count_launch(); }
    } else {
        TcEpi epi{};
        epi.mode = TC_STORE;
        epi.D = c->ws;
        epi.ldd = c->dy;
        epi.split_stride = (size_t)P * c->dy;
        epi.n_dev = &a->cnt->count;
        int used = 1;
        CK(tc_gemm_bf16_splitk(c->dy, P, c->ldk, c->Gq16, c->ldk, bh, bl, c->ldk, c->tsplit, epi, &c->ctl->status,
                               c->st, &used, c->bn_target));
        { finish_da_kernel<<<P, kThreads, 0, c->st>>>(P, c->dy, used, c->ws, c->y32, inv2s2, c->kind == TK_TANH, c->nchunk,
                                                    c->key, c->lpart, a->qsave, a->idx, a->cnt, a->active ? 1 : 0, a->s_prop,
                                                    a->s_cur, c->lp, c->q, c->accf, c->ctl, c->tr, bh, a->ring_x,
                                                    a->ring_lp, (long long)a->cfg.ring, c->ldk); count_launch(); }
    }
    CK(cudaGetLastError());
    ph_end(c, e1);
    return DIAM_OK;
}

// Training schedule, at every interval end (after the interval's synchronisation).
static diam_status da_after_interval(diam_ctx* c) {
    DaState* a = c->da;
    a->intervals++;
    const int64_t period = (int64_t)std::max(1, c->cfg.M) * std::max(1, a->cfg.retrain_every);
    if (a->trainings == 0) {   // the first training waits for enough pairs: the ring's count, read back
        DaCounters hc{};
        CK(d2h(c, &hc, a->cnt, sizeof(hc)));
        if (hc.filled >= a->cfg.first_train_min) CKS(da_train_now(c, nullptr));
    } else if (a->intervals % period == 0) {   // later ones on the interval count alone: no read, no host wait
        CKS(da_train_now(c, nullptr));
    }
    return DIAM_OK;
}

static diam_status da_alloc(diam_ctx* c, const diam_da_config* g, const double* W1, const double* b1, const double* W2,
                            const double* b2, const double* w3, const double* b3) {
    DaState* a = new DaState();
    c->da = a;
    a->cfg = *g;
    a->h1 = g->h1;
    a->h2 = g->h2;
    a->B = g->batch;
    a->key = make_key(g->seed, c->cfg.problem_id);
    const int d = c->d, ldk = c->ldk, P = c->P, h1 = a->h1, h2 = a->h2, B = a->B;
    auto F = [&](float** p, size_t n) { return dalloc(c, p, sizeof(float) * n); };
    auto H = [&](uint16_t** p, size_t n) { return dalloc(c, p, sizeof(uint16_t) * n); };
    auto D = [&](double** p, size_t n) { return dalloc(c, p, sizeof(double) * n); };
    CKS(F(&a->W1, (size_t)h1 * d)); CKS(F(&a->b1, h1)); CKS(F(&a->W2, (size_t)h2 * h1)); CKS(F(&a->b2, h2));
    CKS(F(&a->w3, h2)); CKS(F(&a->b3, 1));
    for (float** p : {&a->mW1, &a->vW1}) CKS(F(p, (size_t)h1 * d));
    for (float** p : {&a->mb1, &a->vb1}) CKS(F(p, h1));
    for (float** p : {&a->mW2, &a->vW2}) CKS(F(p, (size_t)h2 * h1));
    for (float** p : {&a->mb2, &a->vb2, &a->mw3, &a->vw3}) CKS(F(p, h2));
    for (float** p : {&a->mb3, &a->vb3}) CKS(F(p, 1));
    CKS(H(&a->W1q, (size_t)h1 * ldk)); CKS(H(&a->W2q, (size_t)h2 * h1)); CKS(H(&a->W2Tq, (size_t)h1 * h2));
    CKS(F(&a->shift, d)); CKS(F(&a->scale, d));
    CKS(H(&a->U, (size_t)P * ldk)); CKS(H(&a->H1, (size_t)P * h1)); CKS(H(&a->H2, (size_t)P * h2));
    CKS(H(&a->Chi, (size_t)P * ldk)); CKS(H(&a->Clo, (size_t)P * ldk));
    CKS(D(&a->s_prop, P)); CKS(D(&a->s_cur, P)); CKS(D(&a->qsave, P));
    CKS(dalloc(c, &a->idx, sizeof(int) * P));
    CKS(dalloc(c, &a->cnt, sizeof(DaCounters)));
    CKS(H(&a->ring_x, (size_t)g->ring * ldk)); CKS(F(&a->ring_lp, g->ring));
    CKS(H(&a->Xb, (size_t)B * ldk)); CKS(H(&a->XbT, (size_t)ldk * B)); CKS(H(&a->H1b, (size_t)B * h1)); CKS(H(&a->H2b, (size_t)B * h2));
    CKS(H(&a->H1T, (size_t)h1 * B)); CKS(H(&a->dZ2, (size_t)B * h2)); CKS(H(&a->dZ2T, (size_t)h2 * B)); CKS(H(&a->dZ1T, (size_t)h1 * B));
    CKS(F(&a->tb, B)); CKS(F(&a->raw_lp, B)); CKS(F(&a->Z1, (size_t)B * h1)); CKS(F(&a->Z2, (size_t)B * h2)); CKS(F(&a->ds, B));
    CKS(F(&a->dZ2f, (size_t)B * h2)); CKS(F(&a->dH1, (size_t)B * h1)); CKS(F(&a->dZ1f, (size_t)B * h1));
    CKS(F(&a->gW1T, (size_t)ldk * h1)); CKS(F(&a->gW2T, (size_t)h1 * h2)); CKS(F(&a->gb1, h1)); CKS(F(&a->gb2, h2));
    CKS(F(&a->gw3, h2)); CKS(F(&a->gb3, 1)); CKS(F(&a->cs_part, (size_t)COLSUM_CHUNKS * std::max(h1, h2)));
    CKS(D(&a->loss_parts, B)); CKS(D(&a->sbatch, B)); CKS(D(&a->stats, 4)); CKS(D(&a->musig, 2));
    CKS(dalloc(c, &a->tdev, 2 * sizeof(long long)));
    CKS(F(&a->c12, 2 * (size_t)std::max(1, g->train_steps)));
    {
        const double ms[2] = {a->mu, a->sigma};
        CK(cudaMemcpyAsync(a->musig, ms, sizeof(ms), cudaMemcpyHostToDevice, c->st));
        CK(cudaStreamSynchronize(c->st));
    }
    // initial weights (FP64 host -> FP32 masters -> BF16 copies); unit feature scales until the first training
    std::vector<float> tmp;
    auto up = [&](float* dst, const double* src, size_t n) -> diam_status {
        tmp.assign(src, src + n);
        CK(h2d(c, dst, tmp.data(), sizeof(float) * n));
        return DIAM_OK;
    };
    CKS(up(a->W1, W1, (size_t)h1 * d)); CKS(up(a->b1, b1, h1)); CKS(up(a->W2, W2, (size_t)h2 * h1));
    CKS(up(a->b2, b2, h2)); CKS(up(a->w3, w3, h2)); CKS(up(a->b3, b3, 1));
    std::vector<float> ones((size_t)d, 1.0f);
    CK(h2d(c, a->scale, ones.data(), sizeof(float) * d));
    { quant_weights_kernel<<<std::min<unsigned>(148 * 8, blocks_for((size_t)h1 * d)), kThreads, 0, c->st>>>(h1, d, a->W1, a->W1q, ldk, nullptr, 0); count_launch(); }
    { quant_weights_kernel<<<std::min<unsigned>(148 * 8, blocks_for((size_t)h2 * h1)), kThreads, 0, c->st>>>(h2, h1, a->W2, a->W2q, h1, a->W2Tq, h2); count_launch(); }
    CK(cudaGetLastError());
    if (g->screen_from_start) {   // stage 1 from now on with the given network, unit scalings (shift 0, scale 1)
        a->active = true;
        CKS(da_refresh_s_cur(c));
    }
    return sync_and_check(c);
}
