/*
 * diam.h -- C ABI of the B300 (sm_103a) DIAM sampler: dimension-independent adaptive Metropolis over P
 * concurrent chains (Chen, Law, Ltaief, Keyes: "Accelerated dimension-independent adaptive Metropolis",
 * arXiv 1506.05741).
 *
 * What one call computes, in the paper's terms:
 *   - the proposal of eq. (diam) / eq. (diamnl):  x* = x_ref + sqrt(1 - beta^2)(x_n - x_ref) + beta*alpha*A_n W_n,
 *     W_n ~ N(0, Id), for all P chains at once; the n_lag noise products of one interval are one batched
 *     triangular product (Algorithm 1, "Batch update");
 *   - the Metropolis-Hastings test of eq. (accept), written as in Algorithm 1:
 *     log a = log pi(x*) + q(x*) - log pi(x_n) - q(x_n),  q(v) = |A_n^{-1}(v - x_ref)|^2 / (2 alpha^2);
 *   - every n_lag steps: the beta rule of Algorithm 1, the moments of eq. (sampmean) / eq. (sampcov) pooled
 *     over all chains (Sec. 2.4.1), and A_n = Cholesky(C_n).
 *
 * Conventions (every entry point):
 *   - Host pointers are owned by the caller and only read/written during the call. Target arrays are
 *     copied to the device by diam_init; the caller may free them afterwards.
 *   - The context owns all of its device memory. Calls on one context must not overlap in time (one host
 *     thread at a time); distinct contexts are independent.
 *   - Matrices are row-major. Chain states are chain-major: chain p's d-vector is contiguous (P x d).
 *   - No C++ exception crosses this boundary. Every call returns a diam_status; on failure
 *     diam_last_error(ctx) holds a one-line reason. DIAM_ENOTSPD is not fatal (the previous factor is
 *     kept); every other non-zero status leaves the context in DIAM_ESTATE until destroyed.
 *   - diam_run_batch enqueues its work on the context's stream and synchronises with the host once per
 *     interval of n_lag steps (to read the acceptance count that drives the beta rule and the refresh
 *     decision). Device-side errors (a bounded wait that expired) are reported by that synchronisation
 *     or by the next call that synchronises.
 */
#ifndef DIAM_H
#define DIAM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DIAM_ABI_VERSION 1

#if defined(__GNUC__)
#define DIAM_API __attribute__((visibility("default")))
#else
#define DIAM_API
#endif

typedef enum {
    DIAM_OK = 0,
    DIAM_EINVAL = 1,     /* bad argument (sizes, null pointers, unsupported combination) */
    DIAM_ENOMEM = 2,     /* device allocation failed */
    DIAM_ECUDA = 3,      /* a CUDA runtime / driver call failed */
    DIAM_ENOTSPD = 4,    /* refresh skipped: C_n + jitter was not positive definite; old factor kept */
    DIAM_ETIMEOUT = 5,   /* a bounded device-side wait expired; the kernel returned without its result */
    DIAM_ETARGET = 6,    /* the user log-density callback failed */
    DIAM_ESTATE = 7      /* the context is in an error state or was not initialised */
} diam_status;

/* Arithmetic of the chain update. FP64: every step in FP64 (the plain form).
 * BF16: the factor A_n, the noise W and the target's linear map are rounded once (to nearest even) to
 * BF16 and those same rounded values define both the proposal and its density; the products run on the
 * tensor cores with FP32 accumulation, chain states are FP32, and the Cholesky refresh and the moment
 * accumulation stay in FP64.
 * FP32: the BF16 mode with the factor A_n rounded to TF32 instead (11 significant bits: a TF32-representable
 * factor, exactly the sum of two BF16 values, whose products take a second tensor-core pass); W and the map stay
 * BF16. The re-solve of z after a factor change is the FP64-accurate triangular solve. */
typedef enum { DIAM_FP64 = 0, DIAM_FP32 = 1, DIAM_BF16 = 2 } diam_prec;

/* Synthetic targets (log pi up to a constant, eq. (bayes)).
 *  DIAG_GAUSS : -sum_i x_i^2 / (2 lam_i)
 *  DENSE_GAUSS: -|G x|^2 / 2, G is d_y x d
 *  TANH_REG   : -sum_i x_i^2 / (2 lam_i) - sum_k (y_k - tanh((A x)_k))^2 / (2 sigma^2), A is d_y x d
 *  BANANA     : -x1^2/(2a) - (x2 + b x1^2 - c)^2 / 2 - sum_{i>=3} x_i^2 / (2 lam_i)
 *  REF_GAUSS  : the current reference Gaussian N(x_ref, alpha^2 A_n A_n^T), evaluated from x by a
 *               triangular solve; every proposal is accepted (a test target, Sec. 2.3.2)
 *  CALLBACK   : user function on device memory (see diam_logpi_fn)
 *  TWISTED    : -sum_j (u_j + c_j u_{j-1}^2)^2 / (2 lam_j), u = G x (G is d_y x d, lam and c = y hold d_y
 *               entries, c_0 unused): the twisted Gaussians pi_5, pi_6 of Sec. 3.1 (G = V^T, lam the eigenvalues
 *               of pi_1's covariance, c the twist coefficients), a unit-Jacobian transform of N(0, diag(lam)) */
typedef enum {
    DIAM_T_DIAG_GAUSS = 0,
    DIAM_T_DENSE_GAUSS = 1,
    DIAM_T_TANH_REG = 2,
    DIAM_T_BANANA = 3,
    DIAM_T_REF_GAUSS = 4,
    DIAM_T_CALLBACK = 5,
    DIAM_T_TWISTED = 6
} diam_target_kind;

/* User log-density: X is P x d on the device (FP64 when prec = FP64, FP32 when prec = BF16), lp_out is
 * P doubles on the device, stream is the cudaStream_t the call must use (work on it is ordered with the
 * sampler's; the call may synchronise that stream: callback targets never run inside a captured graph, but it
 * must not synchronise the whole device). A non-finite value rejects that proposal and is counted in
 * diam_stats.nonfinite. Return DIAM_OK, or DIAM_ETARGET to stop diam_run_batch (the context is then left in
 * DIAM_ESTATE). */
typedef diam_status (*diam_logpi_fn)(void* user, const void* X, int32_t d, int32_t P, int32_t prec,
                                     double* lp_out, void* stream);

typedef struct {
    int32_t kind;           /* diam_target_kind */
    int32_t d_y;            /* rows of G or A */
    const double* lam;      /* d (host): lambda_i (d_y for TWISTED); unused for DENSE_GAUSS / REF_GAUSS / CALLBACK */
    const double* G;        /* d_y x d (host), DENSE_GAUSS and TWISTED */
    const double* A;        /* d_y x d (host), TANH_REG */
    const double* y;        /* d_y (host): TANH_REG observations; TWISTED twist coefficients */
    double sigma;           /* TANH_REG noise std */
    double ban_a, ban_b, ban_c;
    diam_logpi_fn fn;       /* CALLBACK */
    void* user;
} diam_target;

typedef struct {
    int32_t d, P;           /* dimension, number of concurrent chains */
    int32_t n_lag;          /* steps between factor refreshes (Algorithm 1) */
    int32_t M;              /* intervals per batch between synchronisations (Sec. 2.4.1) */
    double beta0;           /* initial beta; Algorithm 1 uses min(2.4/sqrt(d), 0.5) */
    double infl;            /* inflation alpha of eq. (diamnl); 1 = eq. (diam) */
    int32_t adapt_beta;     /* 1: Algorithm 1's beta rule, pooled over chains */
    int32_t xref_mode;      /* 0: x_ref = 0 (or xref0); 1: x_ref = running mean, set at each refresh */
    double acc_lo, acc_hi;  /* acceptance window; Sec. 3.2 uses [0.3, 0.5] for DIAM */
    double beta_factor;     /* multiplicative beta change (the paper leaves it open; default 1.1) */
    double beta_min, beta_max;
    double eps_jitter;      /* refresh factors chol(C_n + eps diag(C_n)), eps = max(eps_jitter, eps_jitter_min) at
                               the first attempt, x100 per retry (3 retries) */
    int64_t min_samples_refresh;  /* refresh only after this many accepted moves (< 0: d + 1) */
    int64_t burnin;         /* n_0: steps kept out of the moments (footnote to Algorithm 1) */
    int32_t refresh_delay;  /* the factor built at the end of interval k is used from interval k+1+delay;
                               with delay >= 1, BF16 mode and graphs on, its Cholesky runs on streams of
                               its own beside the following intervals' steps (at most two factorisations
                               in flight) and is resolved, retries included, before its factor is due */
    int32_t prec;           /* diam_prec */
    uint64_t seed;          /* Philox4x32-10 key */
    uint32_t problem_id;    /* mixed into the key; distinct problems draw distinct streams */
    int32_t trace_steps;    /* keep a per-step, per-chain trace for the first trace_steps steps (0: off) */
    int32_t keep_block_sums;/* 1: keep per-interval, per-chain sums of x, of x^2 (as the scatter about the
                               interval mean in BF16 mode) and of log pi (for ESS and the PSRF) */
    int32_t profile;        /* 1: time every phase with CUDA events on the context's stream (diam_get_profile) */
    int32_t graphs;         /* 1 (default): each whole interval's n_lag steps run as one launch (BF16 mode with a
                               linear-map target and no surrogate screen in force: one block walks each chain
                               through the interval) or replay one captured CUDA graph; 0: launches step by
                               step (the same results, bit for bit) */
    int32_t proposal;       /* diam_proposal: DIAM_PROP_DIAM (default) or DIAM_PROP_RW */
    int32_t carry_map;      /* BF16 mode, linear-map targets: 1 (default) carries A x through the proposal (the
                               map of an interval's noise is one product at the interval start, O(d_y) per step);
                               0 evaluates A x* for every proposal (a tensor-core product per step) */
    double eps_jitter_min;  /* floor of the refresh rule's first jitter (0: none). The library's default is 0;
                               BF16-mode callers set it (the tests and the benchmark use 1e-4: the BF16 records' rounding in C_n defeats smaller loadings) */
    int32_t reserved[2];
} diam_config;

/* Proposal of the chain update (config field proposal).
 * DIAM: x* = x_ref + sqrt(1 - beta^2)(x - x_ref) + beta alpha A_n W (eq. (diam), (diamnl)), with the quadratic q of
 *       the reference Gaussian in the test. With A_n fixed (no refresh) and x_ref = 0 this is the
 *       preconditioned Crank-Nicolson proposal of eq. (pcn) (Sec. 2.3.2).
 * RW:   x* = x + beta alpha A_n W (eq. (rw), Sec. 2.3.1), a symmetric proposal: log a = log pi(x*) - log pi(x)
 *       (q = 0). x_ref is not used. With the factor refreshed from the pooled moments this is the adaptive
 *       Metropolis sampler of Sec. 2.3.3 (eq. (sampcov), (sampmean)). FP64 and BF16 modes; not with delayed
 *       acceptance. */
typedef enum { DIAM_PROP_DIAM = 0, DIAM_PROP_RW = 1 } diam_proposal;

typedef struct {
    int64_t steps;          /* steps done by every chain */
    int64_t n;              /* samples in the moments (P per step after burn-in, plus imported ones) */
    int64_t accepted;       /* accepted moves, all chains */
    int64_t refreshes;      /* factors built */
    int64_t notspd;         /* refreshes skipped because C_n was not positive definite */
    int64_t nonfinite;      /* proposals whose log-density was not finite (always rejected) */
    double beta;            /* beta in effect */
    int64_t chol_attempts;  /* Cholesky factorisations run by refreshes (retries included) */
} diam_stats;

typedef struct diam_ctx diam_ctx;

/* Fill cfg with the defaults above for dimension d and P chains. */
DIAM_API diam_status diam_config_default(diam_config* cfg, int32_t d, int32_t P);

/* Create a sampler on the current CUDA device. x0 (P x d, host) may be NULL (all chains start at 0).
 * C0 (d x d, host) is the covariance whose Cholesky factor is A_0 (NULL: A_0 = Id, Algorithm 1). xref0
 * (d, host) is the initial x_ref (NULL: 0). stream is a cudaStream_t (NULL: the context creates its own). */
DIAM_API diam_status diam_init(const diam_config* cfg, const diam_target* target, const double* x0, const double* C0,
                      const double* xref0, void* stream, diam_ctx** out);

/* Advance every chain n_steps steps (any n_steps >= 0; refreshes happen at multiples of n_lag). */
DIAM_API diam_status diam_run_batch(diam_ctx* ctx, int64_t n_steps);

/* Wait for the work the context runs beside its stream (a refresh factorisation in flight, see
 * refresh_delay) and apply its outcome; afterwards the context's stream is ordered after that work.
 * State queries and checkpoints do this themselves. Synchronises. */
DIAM_API diam_status diam_flush(diam_ctx* ctx);

/* Synchronisation point of Sec. 2.4.1 (eq. (mom2g), (mom1g)). With the pooled reading used here the
 * local moments already are the global ones; this call merges moments exported by other samplers (other
 * processes, other GPUs) into them: ext_mean (d), ext_M2 (d x d, the centred sum
 * sum_i (x_i - ext_mean)(x_i - ext_mean)^T) and ext_n samples. ext_* may be NULL / 0 (no import). Every call
 * marks a synchronisation: diam_export_increment counts from the moments as they stand after it.
 * Synchronises the stream. */
DIAM_API diam_status diam_sync_moments(diam_ctx* ctx, const double* ext_mean, const double* ext_M2, int64_t ext_n);

/* The moments of the samples this context folded since its last diam_sync_moments (since diam_init if there
 * was none; after diam_load every sample the context holds counts as new), in the mergeable form of diam_export_moments: mean (d), M2 (d x d centred sum)
 * and n (0: no new samples; mean and M2 are then zero). This is what a sampler adds to a pool of samplers
 * between two synchronisations: each member exports its increment, imports every other member's with
 * diam_sync_moments, and all members then hold the moments of every member's samples, each counted once
 * (eq. (mom2g), (mom1g) with sample counts as weights). Computed from the current and the last synchronised
 * moments (the pairwise update of Chan, Golub and LeVeque run backwards, FP64). Synchronises. */
DIAM_API diam_status diam_export_increment(diam_ctx* ctx, double* mean, double* M2, int64_t* n);

/* Interval-end hook: fn(user, ctx, interval) is called by diam_run_batch on the calling host thread at the end
 * of every interval of n_lag steps, after the interval's samples are folded into the moments and before the
 * beta rule and the refresh that uses those moments: the synchronisation point of Sec. 2.4.1 for a pool of
 * samplers (processes, GPUs) sharing one factor. Inside the hook the caller may use diam_export_increment,
 * diam_export_moments, diam_get_moments, diam_sync_moments and the other getters on ctx (each synchronises);
 * diam_run_batch, diam_save, diam_load and diam_destroy on ctx return DIAM_EINVAL there. A status other than
 * DIAM_OK from fn stops diam_run_batch, which returns that status (DIAM_ETARGET for DIAM_ENOTSPD) with the
 * context left in DIAM_ESTATE. fn = NULL removes the hook. */
typedef diam_status (*diam_interval_fn)(void* user, diam_ctx* ctx, int64_t interval);
DIAM_API diam_status diam_set_interval_hook(diam_ctx* ctx, diam_interval_fn fn, void* user);

/* Pooled moments of eq. (sampmean), (sampcov): mean (d), cov (d x d, may be NULL), n. Synchronises. */
DIAM_API diam_status diam_get_moments(diam_ctx* ctx, double* mean, double* cov, int64_t* n);

/* The same moments in mergeable form: mean (d), M2 (d x d centred sum), n. Synchronises. */
DIAM_API diam_status diam_export_moments(diam_ctx* ctx, double* mean, double* M2, int64_t* n);

/* Chain states (P x d) and log pi (P); any output may be NULL. Synchronises the context's stream. With stats,
 * the Cholesky refreshes still running beside the intervals (refresh_delay >= 1) are waited for and counted;
 * x and lp alone are read without waiting for them. */
DIAM_API diam_status diam_get_state(diam_ctx* ctx, double* x, double* lp, diam_stats* stats);

/* Factor in effect: L (d x d, FP64 master, lower), Lq (the rounded factor actually used; equals L for
 * FP64), x_ref (d), beta. Any output may be NULL. Synchronises. */
DIAM_API diam_status diam_get_factor(diam_ctx* ctx, double* L, double* Lq, double* xref, double* beta);

/* Per-step trace for the first min(steps, trace_steps) steps, each (steps x P): log pi(x*), q(x*), q(x_n),
 * log a, accepted flag. n_steps is the number of rows the caller's buffers hold. Synchronises. */
DIAM_API diam_status diam_get_trace(diam_ctx* ctx, double* lp_prop, double* q_prop, double* q_cur, double* loga,
                           int8_t* acc, int64_t n_steps);

/* Per-interval, per-chain sums (needs keep_block_sums): xsum (n_blocks x P x d), lpsum (n_blocks x P).
 * *n_blocks is the capacity on input and the count on output: in FP64 mode every interval begun (the
 * current one partial), in BF16 mode the completed intervals (their x sums are formed from the interval's
 * records when it completes). Synchronises. */
DIAM_API diam_status diam_get_block_sums(diam_ctx* ctx, double* xsum, double* lpsum, int64_t* n_blocks);

/* Potential scale reduction factor sqrt(R_i) of Sec. 2.4.2 (eq. (winco), (btwco), (psrf)) for every
 * coordinate i, over the completed intervals first_block .. first_block + n_blocks - 1: each chain's mean
 * and variance (1/n normalisation of eq. (sampcov), n = n_blocks n_lag samples per chain) from its interval
 * sums, then the between-chain variance B_i and the mean within-chain variance W_i across the P chains.
 * psrf (host, d entries) receives sqrt(R_i). Needs keep_block_sums and P >= 2; computed on the device in
 * FP64 from the interval sums (FP32 sums in BF16 mode). DIAM_EINVAL if the window is not available.
 * Synchronises. */
DIAM_API diam_status diam_get_psrf(diam_ctx* ctx, int64_t first_block, int64_t n_blocks, double* psrf);

/* Checkpoint: the full sampler state (chains, factor, moments, beta, counters, pending factors). Philox
 * is counter-based, so save + load + run N reproduces run N bit for bit. diam_save with buf = NULL
 * returns the size in *size. diam_load expects a context created with the same diam_config. */
DIAM_API diam_status diam_save(diam_ctx* ctx, void* buf, size_t* size);
DIAM_API diam_status diam_load(diam_ctx* ctx, const void* buf, size_t size);

/* ---------------------------------------------------------------------------------------------------
 * Delayed acceptance with a learned surrogate (not in the paper; two-stage Metropolis-Hastings of
 * Christen & Fox, 2005). The surrogate s(x) ~ log pi(x) is the target's exact O(d) terms plus a small MLP
 * (d -> h1 -> h2 -> 1, GELU, BF16 weights, FP32 accumulation on the tensor cores) that learns the
 * linear-map terms (the expensive part). It screens every proposal first:
 *   stage 1: accept with probability min(1, exp(s(x*) - s(x) + q(x*) - q(x)))       (uniform tag 3)
 *   stage 2: for the survivors only, log pi(x*) is evaluated and the move is accepted with probability
 *            min(1, exp(log pi(x*) - log pi(x) - s(x*) + s(x)))                     (uniform tag 1)
 * so the chain still targets pi exactly. The network is trained on the GPU (own forward, backward and
 * Adam kernels) on a ring buffer of exactly evaluated pairs (x*, log pi(x*)) from the chains; after each
 * training its RMSE on held-out pairs decides whether stage 1 is used; when it exceeds rmse_bound (or
 * before the first training) every proposal goes straight to the exact test (plain DIAM). Needs
 * prec = BF16 and P <= 1024. */
typedef struct {
    int32_t h1, h2;             /* hidden widths (multiples of 128) */
    int32_t retrain_every;      /* trainings every retrain_every synchronisations (of M intervals) */
    int32_t ring;               /* ring-buffer capacity in pairs */
    int32_t train_steps;        /* Adam steps per training */
    int32_t batch;              /* minibatch size (multiple of 128) */
    int32_t first_train_min;    /* pairs needed before the first training (at an interval end) */
    int32_t screen_from_start;  /* 1: stage 1 runs from diam_da_enable on, with the given weights and unit input
                                   and output scaling (s = the O(d) terms + the network's output), until a training
                                   decides otherwise; 0 (default): only after a training within rmse_bound */
    double lr, beta1, beta2, adam_eps;
    double rmse_bound;          /* held-out RMSE (nats) above which stage 1 is switched off */
    uint64_t seed;              /* minibatch selection stream */
} diam_da_config;

typedef struct {
    int64_t trainings;          /* trainings done */
    int64_t stage1_tested;      /* proposals screened by the surrogate */
    int64_t stage1_passed;      /* of those, passed to the exact test */
    int64_t exact_evals;        /* exact log-density evaluations (all proposals when stage 1 is off) */
    int64_t ring_filled;        /* pairs in the ring */
    double last_rmse;           /* held-out RMSE of the last training (nats) */
    int32_t active;             /* 1: stage 1 in use */
    int32_t pad;
} diam_da_stats;

/* Defaults: h1 = h2 = 512, retrain_every = 20, ring = 200000, train_steps = 200, batch = 1024,
 * first_train_min = 20000, lr = 1e-3, beta1 = 0.9, beta2 = 0.999, adam_eps = 1e-8, rmse_bound = 0.5. */
DIAM_API diam_status diam_da_config_default(diam_da_config* cfg);

/* Enable delayed acceptance with initial weights (host, FP64, row-major): W1 (h1 x d), b1 (h1),
 * W2 (h2 x h1), b2 (h2), w3 (h2), b3 (1). */
DIAM_API diam_status diam_da_enable(diam_ctx* ctx, const diam_da_config* cfg, const double* W1, const double* b1,
                                    const double* W2, const double* b2, const double* w3, const double* b3);

/* Train now (whatever the schedule) on the ring buffer; returns the held-out RMSE in *rmse. Synchronises. */
DIAM_API diam_status diam_da_train(diam_ctx* ctx, double* rmse);

DIAM_API diam_status diam_da_get_stats(diam_ctx* ctx, diam_da_stats* stats);

/* One forward + backward pass of the network on a given batch (B rows, multiple of 128; U already
 * normalised, B x d, FP64 host, rounded to BF16 on upload; targets t in network units), without updating
 * anything: the loss mean((out - t)^2)/2 and its gradients (FP64 host, same shapes as diam_da_enable's
 * weights). For checking the training kernels. Synchronises. */
DIAM_API diam_status diam_da_grad(diam_ctx* ctx, int32_t B, const double* U, const double* t, double* loss,
                                  double* gW1, double* gb1, double* gW2, double* gb2, double* gw3, double* gb3);

/* One Adam step (Kingma & Ba 2015: bias-corrected first and second moments, the configured lr, beta1, beta2,
 * adam_eps; the step count continues the context's) on the FP32 master weights with the given gradients (FP64
 * host, rounded to FP32 on upload; same shapes as diam_da_enable's weights), through the kernel the training
 * uses; the BF16 copies the network runs on are rewritten. For checking the training's update. Synchronises. */
DIAM_API diam_status diam_da_adam_step(diam_ctx* ctx, const double* gW1, const double* gb1, const double* gW2,
                                       const double* gb2, const double* gw3, const double* gb3);

/* Current weights (FP32 masters, widened), same shapes as diam_da_enable's. Synchronises. */
DIAM_API diam_status diam_da_get_weights(diam_ctx* ctx, double* W1, double* b1, double* W2, double* b2, double* w3,
                                         double* b3);

/* ---------------------------------------------------------------------------------------------------
 * Many independent samplers run together (uneven dimensions, separate targets): the batched form of the
 * sampler. Problem j has its own configuration, target and start state, its own context and its own
 * stream. diam_multi_run advances every problem by n_steps steps; one host thread per problem drives its
 * context (whole intervals run as one launch or replay that problem's captured interval graph), so the problems' kernels
 * interleave on the GPU. x0 and C0 may be NULL or hold NULL entries (per-problem defaults). */
typedef struct diam_multi diam_multi;
DIAM_API diam_status diam_multi_init(int32_t n, const diam_config* cfgs, const diam_target* targets,
                                     const double* const* x0, const double* const* C0, diam_multi** out);
DIAM_API diam_status diam_multi_run(diam_multi* m, int64_t n_steps);
/* The context of problem j (owned by m; use it with the single-sampler getters). */
DIAM_API diam_ctx* diam_multi_context(diam_multi* m, int32_t j);
DIAM_API void diam_multi_destroy(diam_multi* m);

/* Phase timings collected while cfg.profile = 1: for each phase, the number of timed launches of its
 * kernels and their summed device time in milliseconds (CUDA events on the context's stream). Phases:
 * 0 noise draw, 1 noise product (batched triangular GEMM), 2 propose, 3 target (linear map + reduction),
 * 4 accept / select / record, 5 moment fold (column sums + SYRK), 6 Cholesky refresh (with its
 * retries), 7 re-whitening solve after a factor change, 8 surrogate screening (stage 1), 9 surrogate
 * training, 10 the fused steps (propose + map + test + record in one launch per step, or one launch per whole
 * interval; BF16 mode with the map carried through the proposal and no surrogate screen in force; phases
 * 2-4 then stay empty), 11 the fold's SYRK alone (BF16 mode: one tensor-core launch; phase 5 keeps the rest of
 * the fold).
 * counts and ms hold DIAM_N_PHASES entries each. A refresh factorised beside the next interval (refresh_delay
 * >= 1) is timed on its own stream whether or not cfg.profile is set, and counted in phase 6.
 * reset = 1 clears the accumulators after reading. Synchronises. */
#define DIAM_N_PHASES 12
DIAM_API diam_status diam_get_profile(diam_ctx* ctx, int64_t* counts, double* ms, int32_t reset);

DIAM_API void diam_destroy(diam_ctx* ctx);
DIAM_API const char* diam_last_error(const diam_ctx* ctx);
DIAM_API const char* diam_status_string(diam_status s);

/* Number of CUDA kernel launches this library has made in the calling process (all contexts and op-level
 * entry points), for accounting what ran on the GPU. */
DIAM_API uint64_t diam_kernel_launches(void);

#ifdef __cplusplus
}
#endif
#endif /* DIAM_H */
