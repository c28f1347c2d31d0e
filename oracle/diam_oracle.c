/*
 * diam_oracle.c -- plain, slow FP64 CPU oracle for the DIAM hot path.
 *
 * TEST INFRASTRUCTURE. Only the tests, the smoke check and the benchmark's CPU-baseline leg load this
 * file's library. The sampling library (the CUDA path) never links, calls or includes it, and this file
 * includes nothing of the CUDA path.
 *
 * Paper: "Accelerated dimension-independent adaptive Metropolis" (arXiv 1506.05741).
 * Every routine cites the passage it follows. The sampler is Algorithm 1 with the proposal of eq. (diam) /
 * eq. (diamnl) (Sec. 2.3.4), the MH acceptance of eq. (accept) (Sec. 2.2), the moments of eq. (sampcov) /
 * eq. (sampmean) (Sec. 2.3.3) pooled over the P concurrent chains of Sec. 2.4.1.
 *
 * Readings where the paper is silent (listed in full in the design notes):
 *  - one proposal factor shared by all chains, built from the moments pooled over every chain;
 *  - the proposal-density quadratic uses (x - x_ref) (Algorithm 1 prints A_n^{-1} x, which is the same
 *    thing when x_ref = 0);
 *  - random numbers: Philox4x32-10 (Salmon et al., SC'11) with a fixed counter layout; Gaussian draws by
 *    the Box-Muller transform computed in IEEE FP32 with series for log / sin / cos written out below, so
 *    that the CUDA path can reproduce each draw bit for bit;
 *  - the refresh is skipped until enough moves were accepted, and the Cholesky factor is taken of
 *    C + eps diag(C), retrying with a larger eps.
 *
 * Everything else is the plain definition: forward substitution for the quadratic, a textbook
 * Cholesky-Banachiewicz factorisation, sums over samples for the moments.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_EXPORT __attribute__((visibility("default")))

/* ------------------------------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw: "Parallel random numbers: as easy as 1, 2, 3", SC'11).  */
/* Ten rounds; each round multiplies two words by fixed odd constants, and the key is bumped by the    */
/* Weyl increments between rounds.                                                                     */
/* ------------------------------------------------------------------------------------------------ */
ORC_EXPORT void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Stream layout (not in the paper, which draws with LAPACK LARNV): key = (seed low word, seed high word
 * xor problem_id * 0x9E3779B9); counter = (j, step low word, chain, tag | step high word << 8). */
enum { ORC_TAG_W = 0, ORC_TAG_U = 1, ORC_TAG_X0 = 2, ORC_TAG_UDA = 3 };

ORC_EXPORT void orc_key(uint64_t seed, uint32_t problem_id, uint32_t key[2]) {
    key[0] = (uint32_t)seed;
    key[1] = (uint32_t)(seed >> 32) ^ (uint32_t)(problem_id * 0x9E3779B9u);
}

static void orc_draw(uint64_t seed, uint32_t pid, uint32_t j, int64_t t, uint32_t p, uint32_t tag, uint32_t out[4]) {
    uint32_t key[2], ctr[4];
    orc_key(seed, pid, key);
    ctr[0] = j;
    ctr[1] = (uint32_t)t;
    ctr[2] = p;
    ctr[3] = tag | ((uint32_t)((uint64_t)t >> 32) << 8);
    orc_philox4x32_10(ctr, key, out);
}

/* ------------------------------------------------------------------------------------------------ */
/* Box-Muller in IEEE FP32 (Box & Muller 1958). ln and sin/cos are written out from their series so   */
/* the result is fixed by IEEE arithmetic alone: ln m = 2 atanh(s), s = (m-1)/(m+1), m in [1/sqrt2,   */
/* sqrt2]; sin/cos by Taylor series on [0, pi/4] with quadrant symmetry. Built with -ffp-contract=off, */
/* every fused multiply-add below is an explicit fmaf.                                                 */
/* ------------------------------------------------------------------------------------------------ */
static const float F_1_3 = 0x1.555556p-2f, F_1_5 = 0x1.99999ap-3f, F_1_7 = 0x1.24924ap-3f, F_1_9 = 0x1.c71c72p-4f;
static const float F_LN2 = 0x1.62e430p-1f, F_SQRT2 = 0x1.6a09e6p+0f, F_PI_2 = 0x1.921fb6p+0f;
static const float F_S3 = 0x1.555556p-3f, F_S5 = 0x1.111112p-7f, F_S7 = 0x1.a01a02p-13f, F_S9 = 0x1.71de3ap-19f;
static const float F_C4 = 0x1.555556p-5f, F_C6 = 0x1.6c16c2p-10f, F_C8 = 0x1.a01a02p-16f, F_C10 = 0x1.27e4fcp-22f;

/* ln(u1), u1 = ((a >> 8) + 1) * 2^-24 in [2^-24, 1]. */
ORC_EXPORT float orc_ln_u24(uint32_t a) {
    uint32_t k = (a >> 8) + 1u;               /* 1 .. 2^24 */
    int e = 31 - __builtin_clz(k);            /* k = 2^e * m, m in [1, 2) */
    float m = ldexpf((float)k, -e);           /* exact */
    if (m > F_SQRT2) { m = m * 0.5f; e += 1; }
    float s = (m - 1.0f) / (m + 1.0f);
    float w = s * s;
    float poly = F_1_9;
    poly = fmaf(poly, w, F_1_7);
    poly = fmaf(poly, w, F_1_5);
    poly = fmaf(poly, w, F_1_3);
    poly = fmaf(poly, w, 1.0f);
    float lnm = (2.0f * s) * poly;
    return fmaf((float)(e - 24), F_LN2, lnm);
}

/* (cos, sin) of 2*pi*u2 with u2 = (b >> 8) * 2^-24: quadrant from the top two bits, the rest a fraction. */
ORC_EXPORT void orc_cossin_u24(uint32_t b, float* c_out, float* s_out) {
    uint32_t q = b >> 30;
    uint32_t f = (b >> 8) & 0x3FFFFFu;        /* r = f * 2^-22 in [0, 1) */
    int swap = f > (1u << 21);
    uint32_t fw = swap ? ((1u << 22) - f) : f;
    float phi = ((float)fw * 0x1p-22f) * F_PI_2;    /* in [0, pi/4] */
    float p2 = phi * phi;
    float ts = F_S9;
    ts = fmaf(ts, p2, -F_S7);
    ts = fmaf(ts, p2, F_S5);
    ts = fmaf(ts, p2, -F_S3);
    ts = fmaf(ts, p2, 1.0f);
    float sphi = phi * ts;
    float tc = -F_C10;
    tc = fmaf(tc, p2, F_C8);
    tc = fmaf(tc, p2, -F_C6);
    tc = fmaf(tc, p2, F_C4);
    tc = fmaf(tc, p2, -0.5f);
    tc = fmaf(tc, p2, 1.0f);
    float s = swap ? tc : sphi;               /* sin(pi r / 2) */
    float c = swap ? sphi : tc;               /* cos(pi r / 2) */
    float co, si;
    switch (q) {
        case 0: co = c; si = s; break;
        case 1: co = -s; si = c; break;
        case 2: co = -c; si = -s; break;
        default: co = s; si = -c; break;
    }
    *c_out = co;
    *s_out = si;
}

ORC_EXPORT void orc_boxmuller(uint32_t a, uint32_t b, float* n0, float* n1) {
    float r = sqrtf(-2.0f * orc_ln_u24(a));
    float c, s;
    orc_cossin_u24(b, &c, &s);
    *n0 = r * c;
    *n1 = r * s;
}

/* W_n for chain p at step t (Algorithm 1's W ~ N(0, Id)): Philox call j gives components 4j .. 4j+3. */
ORC_EXPORT void orc_normals(uint64_t seed, uint32_t pid, int64_t t, uint32_t p, int d, float* w) {
    for (int j = 0; 4 * j < d; ++j) {
        uint32_t r[4];
        float n[4];
        orc_draw(seed, pid, (uint32_t)j, t, p, ORC_TAG_W, r);
        orc_boxmuller(r[0], r[1], &n[0], &n[1]);
        orc_boxmuller(r[2], r[3], &n[2], &n[3]);
        for (int k = 0; k < 4 && 4 * j + k < d; ++k) w[4 * j + k] = n[k];
    }
}

/* u ~ Uniform(0, 1] for the accept test of Algorithm 1: 53 bits, u = (u53 + 1) 2^-53. */
ORC_EXPORT double orc_uniform(uint64_t seed, uint32_t pid, uint32_t tag, int64_t t, uint32_t p) {
    uint32_t r[4];
    orc_draw(seed, pid, 0u, t, p, tag, r);
    uint64_t u53 = ((uint64_t)(r[0] >> 11) << 32) | (uint64_t)r[1];
    return (double)(u53 + 1u) * 0x1p-53;
}

/* ------------------------------------------------------------------------------------------------ */
/* Quantisation of the factor and the noise (mixed precision): round to nearest, ties to even.        */
/* ------------------------------------------------------------------------------------------------ */
ORC_EXPORT double orc_round_bf16(double v) {
    uint64_t bits;
    memcpy(&bits, &v, 8);
    if (((bits >> 52) & 0x7FF) == 0x7FF) return v;            /* inf / nan */
    uint64_t lsb = (bits >> 45) & 1u;
    bits += ((uint64_t)1 << 44) - 1u + lsb;
    bits &= ~(((uint64_t)1 << 45) - 1u);
    double r;
    memcpy(&r, &bits, 8);
    return r;
}

ORC_EXPORT double orc_round_f32(double v) { return (double)(float)v; }

/* TF32: 10 explicit significand bits (FP32's exponent range), round to nearest, ties to even, from FP64. */
ORC_EXPORT double orc_round_tf32(double v) {
    uint64_t bits;
    memcpy(&bits, &v, 8);
    if (((bits >> 52) & 0x7FF) == 0x7FF) return v;            /* inf / nan */
    uint64_t lsb = (bits >> 42) & 1u;
    bits += ((uint64_t)1 << 41) - 1u + lsb;
    bits &= ~(((uint64_t)1 << 42) - 1u);
    double r;
    memcpy(&r, &bits, 8);
    return r;
}

/* The proposal factor's quantisation by precision mode: 0 FP64 (none), 1 TF32, 2 BF16. */
static double orc_round_factor(int prec, double v) {
    return prec == 2 ? orc_round_bf16(v) : prec == 1 ? orc_round_tf32(v) : v;
}

/* ------------------------------------------------------------------------------------------------ */
/* Dense linear algebra, written as the textbook definitions.                                        */
/* ------------------------------------------------------------------------------------------------ */

/* Cholesky-Banachiewicz: C = L L^T, L lower, row-major n x n (upper part set to 0). Returns 0 on
 * success, -1 if a pivot is not positive (C not positive definite). Algorithm 1: "Update A_n =
 * Cholesky(C_n)". */
ORC_EXPORT int orc_cholesky(int n, const double* C, double* L) {
    memset(L, 0, sizeof(double) * (size_t)n * n);
    for (int i = 0; i < n; ++i) {
        for (int j = 0; j <= i; ++j) {
            double s = C[(size_t)i * n + j];
            for (int k = 0; k < j; ++k) s -= L[(size_t)i * n + k] * L[(size_t)j * n + k];
            if (i == j) {
                if (!(s > 0.0)) return -1;
                L[(size_t)i * n + i] = sqrt(s);
            } else {
                L[(size_t)i * n + j] = s / L[(size_t)j * n + j];
            }
        }
    }
    return 0;
}

/* Forward substitution y = L^{-1} b (L lower, row-major). */
ORC_EXPORT void orc_forward_sub(int n, const double* L, const double* b, double* y) {
    for (int i = 0; i < n; ++i) {
        double s = b[i];
        for (int k = 0; k < i; ++k) s -= L[(size_t)i * n + k] * y[k];
        y[i] = s / L[(size_t)i * n + i];
    }
}

/* ------------------------------------------------------------------------------------------------ */
/* Targets: log pi up to an additive constant (eq. (bayes), Sec. 2.1).                               */
/* ------------------------------------------------------------------------------------------------ */
enum { ORC_T_DIAG = 0, ORC_T_DENSE = 1, ORC_T_TANH = 2, ORC_T_BANANA = 3, ORC_T_REF = 4, ORC_T_TWIST = 6 };

typedef struct {
    int32_t kind;
    int32_t d;
    int32_t d_y;
    int32_t pad_;
    const double* lam;     /* d: prior / diagonal variances lambda_i */
    const double* G;       /* d_y x d row-major: dense Gaussian, log pi = -|G x|^2 / 2; the map u = G x of the
                              twisted target */
    const double* A;       /* d_y x d row-major: forward map of the tanh regression */
    const double* y;       /* d_y observations (tanh regression); twist coefficients c_j (twisted target) */
    double sigma;          /* observation noise std */
    double ban_a, ban_b, ban_c;  /* banana: -x1^2/(2a) - (x2 + b x1^2 - c)^2 / 2 */
} orc_target;

typedef struct {
    int32_t d, P, n_lag, M;
    double beta0, infl;
    int32_t adapt_beta, xref_mode;
    double acc_lo, acc_hi, beta_factor, beta_min, beta_max;
    double eps_jitter;
    int64_t min_samples_refresh;
    int32_t refresh_delay, prec;        /* prec: 0 = FP64; 2 = BF16-quantised factor, noise and maps; 1 = the
                                           same with the factor quantised to TF32 instead */
    uint64_t seed;
    uint32_t problem_id;
    int32_t threads;
    int64_t trace_steps;                /* per-step trace kept for the first trace_steps steps */
    int32_t record_traj;                /* keep every post-step state x_{n+1} */
    uint32_t chain0;                    /* chain p draws the Philox streams of chain chain0 + p (a sample of a
                                           larger run's chains; chains are independent while beta is fixed
                                           and no refresh happens) */
    int64_t burnin;                     /* n_0 of Algorithm 1's footnote: steps before any moment is kept */
    int32_t proposal;                   /* 0: DIAM, eq. (diam) / (diamnl); 1: random walk, eq. (rw) (Sec. 2.3.1):
                                           x* = x + beta infl A_n W, a symmetric move, so q drops out of the test;
                                           adaptive Metropolis (Sec. 2.3.3) when A_n is refreshed */
    int32_t pad2_;
    double eps_jitter_min;              /* floor of the first jitter of the refresh rule */
    int32_t moments_mode;               /* 0: one factor from the moments pooled over all chains;
                                           1: the per-chain factors of Sec. 2.4.1 (refresh_delay 0) */
    int32_t pad3_;
} orc_config;

typedef struct {
    orc_config cfg;
    orc_target tgt;
    double *lam, *G, *A, *y;            /* owned copies; G, A quantised to BF16 when prec != FP64 */
    /* chain state */
    double *x, *lp;                     /* P x d, P */
    double beta;
    int64_t t;                          /* steps done */
    /* proposal factor in effect: A_n of eq. (diam) and x_ref */
    double *L, *Lq, *xref;
    /* pending factors (refresh delay) */
    int npend;
    double **pendL, **pendX;
    int64_t *pend_block;
    /* moments (eq. sampcov, sampmean) as plain sums over all post-step samples of all chains */
    int64_t n;
    double *sum, *S;                    /* d, d x d */
    int64_t acc_block, acc_total;       /* accepted moves in this block / counted for the refresh rule */
    int64_t acc_all;                    /* every accepted move, burn-in included */
    int64_t refreshes, notspd, chol_attempts;
    /* trace */
    double *tr_lp, *tr_q, *tr_qc, *tr_loga;
    int8_t *tr_acc;
    double *traj;
    double *blk_beta;
    int64_t nblk_rec;
    double *scratch;                    /* threads x (4 d) */
    /* per-chain factors (Sec. 2.4.1): chain p proposes with its own factor A_n^p, x_ref^p and beta^p, refreshed every interval from
     * its local view of the global moments, eq. (mom2pg), (mom1pg), (cov2pg): the raw sums of the batches merged
     * so far (every chain's samples, eq. (mom2g), (mom1g)) plus chain p's own samples of the current batch */
    double *Lp, *Lqp, *xrefp, *betap;   /* P x d x d, P x d x d, P x d, P */
    int64_t *accp;                      /* accepted moves of each chain in the current interval */
    double *Sloc, *sumloc;              /* P x d x d, P x d: sums of x x^T and x over the current batch */
    int64_t nloc;                       /* samples of each chain in the current batch */
    double *Sglob, *sumglob;            /* d x d, d: the same sums over the merged batches */
    int64_t nglob;
} orc_sampler;

static double orc_logpi(const orc_sampler* s, const double* x, double* work) {
    const orc_target* T = &s->tgt;
    int d = T->d;
    double lp = 0.0;
    switch (T->kind) {
        case ORC_T_DIAG:
            for (int i = 0; i < d; ++i) lp -= 0.5 * x[i] * x[i] / s->lam[i];
            return lp;
        case ORC_T_DENSE:
            for (int k = 0; k < T->d_y; ++k) {
                double g = 0.0;
                for (int i = 0; i < d; ++i) g += s->G[(size_t)k * d + i] * x[i];
                lp -= 0.5 * g * g;
            }
            return lp;
        case ORC_T_TANH: {
            for (int i = 0; i < d; ++i) lp -= 0.5 * x[i] * x[i] / s->lam[i];
            double inv2s2 = 1.0 / (2.0 * T->sigma * T->sigma);
            for (int k = 0; k < T->d_y; ++k) {
                double a = 0.0;
                for (int i = 0; i < d; ++i) a += s->A[(size_t)k * d + i] * x[i];
                double r = s->y[k] - tanh(a);
                lp -= r * r * inv2s2;
            }
            return lp;
        }
        case ORC_T_BANANA: {
            double x1 = x[0], x2 = d > 1 ? x[1] : 0.0;
            double v = x2 + T->ban_b * x1 * x1 - T->ban_c;
            lp = -x1 * x1 / (2.0 * T->ban_a) - 0.5 * v * v;
            for (int i = 2; i < d; ++i) lp -= 0.5 * x[i] * x[i] / s->lam[i];
            return lp;
        }
        case ORC_T_TWIST: {
            /* the twisted Gaussians of Sec. 3.1 (pi_5, pi_6): u = G x (G = V^T), the twist
             * phi(u)_j = u_j + c_j u_{j-1}^2 (c_0 = 0; a unit Jacobian), and phi(u) ~ N(0, diag(lambda)) */
            double prev = 0.0;
            for (int k = 0; k < T->d_y; ++k) {
                double u = 0.0;
                for (int i = 0; i < d; ++i) u += s->G[(size_t)k * d + i] * x[i];
                double ph = k > 0 ? u + s->y[k] * prev * prev : u;
                lp -= 0.5 * ph * ph / s->lam[k];
                prev = u;
            }
            return lp;
        }
        case ORC_T_REF: {
            /* the current reference Gaussian N(x_ref, infl^2 Lq Lq^T): a target for which every proposal
             * of eq. (diamnl) is accepted (Sec. 2.3.2: the pCN move preserves N(0, A A^T)). */
            double* dv = work;
            double* z = work + d;
            for (int i = 0; i < d; ++i) dv[i] = x[i] - s->xref[i];
            orc_forward_sub(d, s->Lq, dv, z);
            for (int i = 0; i < d; ++i) lp -= 0.5 * z[i] * z[i];
            return lp / (s->cfg.infl * s->cfg.infl);
        }
    }
    return NAN;
}

ORC_EXPORT double orc_target_logpi(const orc_target* T, const double* x) {
    /* standalone evaluation for tests (no reference Gaussian) */
    orc_sampler s;
    memset(&s, 0, sizeof(s));
    s.tgt = *T;
    s.lam = (double*)T->lam;
    s.G = (double*)T->G;
    s.A = (double*)T->A;
    s.y = (double*)T->y;
    return orc_logpi(&s, x, NULL);
}

/* q(v) = |Lq^{-1}(v - x_ref)|^2 / (2 infl^2): minus the log density of the reference Gaussian that the
 * proposal preserves (Algorithm 1's weighted quadratic, with the x_ref shift of eq. (diam)). */
static double orc_quad(const orc_sampler* s, const double* Lq, const double* xref, const double* v, double* work) {
    int d = s->cfg.d;
    double* dv = work;
    double* z = work + d;
    for (int i = 0; i < d; ++i) dv[i] = v[i] - xref[i];
    orc_forward_sub(d, Lq, dv, z);
    double q = 0.0;
    for (int i = 0; i < d; ++i) q += z[i] * z[i];
    return 0.5 * q / (s->cfg.infl * s->cfg.infl);
}

static void orc_set_quantised_factor(orc_sampler* s) {
    int d = s->cfg.d;
    size_t nn = (size_t)d * d;
    for (size_t i = 0; i < nn; ++i) s->Lq[i] = orc_round_factor(s->cfg.prec, s->L[i]);
}

static void orc_set_xref(orc_sampler* s, const double* m) {
    for (int i = 0; i < s->cfg.d; ++i) s->xref[i] = s->cfg.prec != 0 ? orc_round_f32(m[i]) : m[i];
}

static void orc_recompute_lp(orc_sampler* s) {
    int d = s->cfg.d, P = s->cfg.P;
    for (int p = 0; p < P; ++p) s->lp[p] = orc_logpi(s, s->x + (size_t)p * d, s->scratch);
}

ORC_EXPORT orc_sampler* orc_new(const orc_config* cfg, const orc_target* tgt, const double* x0,
                                const double* C0, const double* xref0) {
    orc_sampler* s = (orc_sampler*)calloc(1, sizeof(orc_sampler));
    s->cfg = *cfg;
    s->tgt = *tgt;
    int d = cfg->d, P = cfg->P, dy = tgt->d_y;
    size_t nn = (size_t)d * d;
    const int nlam = tgt->kind == ORC_T_TWIST ? dy : d;   /* the twisted target's variances are per row of G */
    s->lam = (double*)calloc((size_t)(nlam > d ? nlam : d), sizeof(double));
    if (tgt->lam) memcpy(s->lam, tgt->lam, sizeof(double) * nlam);
    if (tgt->G) {
        s->G = (double*)malloc(sizeof(double) * (size_t)dy * d);
        for (size_t i = 0; i < (size_t)dy * d; ++i) s->G[i] = cfg->prec != 0 ? orc_round_bf16(tgt->G[i]) : tgt->G[i];
    }
    if (tgt->A) {
        s->A = (double*)malloc(sizeof(double) * (size_t)dy * d);
        for (size_t i = 0; i < (size_t)dy * d; ++i) s->A[i] = cfg->prec != 0 ? orc_round_bf16(tgt->A[i]) : tgt->A[i];
    }
    if (tgt->y) {
        s->y = (double*)malloc(sizeof(double) * (size_t)dy);
        memcpy(s->y, tgt->y, sizeof(double) * dy);
    }
    s->x = (double*)calloc((size_t)P * d, sizeof(double));
    if (x0) memcpy(s->x, x0, sizeof(double) * (size_t)P * d);
    s->lp = (double*)calloc((size_t)P, sizeof(double));
    s->L = (double*)calloc(nn, sizeof(double));
    s->Lq = (double*)calloc(nn, sizeof(double));
    s->xref = (double*)calloc((size_t)d, sizeof(double));
    s->sum = (double*)calloc((size_t)d, sizeof(double));
    s->S = (double*)calloc(nn, sizeof(double));
    int nthr = cfg->threads > 0 ? cfg->threads : 1;
    s->scratch = (double*)calloc((size_t)nthr * 4 * d + 4 * (size_t)d, sizeof(double));
    /* Algorithm 1: A_0 = Id unless an initial covariance is given; x_ref = 0 unless given. */
    if (C0) {
        if (orc_cholesky(d, C0, s->L) != 0) { free(s); return NULL; }
    } else {
        for (int i = 0; i < d; ++i) s->L[(size_t)i * d + i] = 1.0;
    }
    orc_set_quantised_factor(s);
    if (xref0) orc_set_xref(s, xref0);
    s->beta = cfg->beta0;
    if (cfg->moments_mode == 1) {   /* R2: every chain starts from A_0 and x_ref of the pooled start */
        size_t pd = (size_t)P * d;
        s->Lp = (double*)malloc(sizeof(double) * pd * d);
        s->Lqp = (double*)malloc(sizeof(double) * pd * d);
        s->xrefp = (double*)malloc(sizeof(double) * pd);
        s->betap = (double*)malloc(sizeof(double) * P);
        s->accp = (int64_t*)calloc((size_t)P, sizeof(int64_t));
        s->Sloc = (double*)calloc(pd * d, sizeof(double));
        s->sumloc = (double*)calloc(pd, sizeof(double));
        s->Sglob = (double*)calloc(nn, sizeof(double));
        s->sumglob = (double*)calloc((size_t)d, sizeof(double));
        for (int p = 0; p < P; ++p) {
            memcpy(s->Lp + (size_t)p * nn, s->L, sizeof(double) * nn);
            memcpy(s->Lqp + (size_t)p * nn, s->Lq, sizeof(double) * nn);
            memcpy(s->xrefp + (size_t)p * d, s->xref, sizeof(double) * d);
            s->betap[p] = cfg->beta0;
        }
    }
    s->npend = cfg->refresh_delay + 1;
    s->pendL = (double**)calloc((size_t)s->npend, sizeof(double*));
    s->pendX = (double**)calloc((size_t)s->npend, sizeof(double*));
    s->pend_block = (int64_t*)calloc((size_t)s->npend, sizeof(int64_t));
    for (int i = 0; i < s->npend; ++i) s->pend_block[i] = -1;
    if (cfg->trace_steps > 0) {
        size_t nt = (size_t)cfg->trace_steps * P;
        s->tr_lp = (double*)calloc(nt, sizeof(double));
        s->tr_q = (double*)calloc(nt, sizeof(double));
        s->tr_qc = (double*)calloc(nt, sizeof(double));
        s->tr_loga = (double*)calloc(nt, sizeof(double));
        s->tr_acc = (int8_t*)calloc(nt, 1);
    }
    orc_recompute_lp(s);
    return s;
}

ORC_EXPORT void orc_free(orc_sampler* s) {
    if (!s) return;
    free(s->lam); free(s->G); free(s->A); free(s->y);
    free(s->x); free(s->lp); free(s->L); free(s->Lq); free(s->xref); free(s->sum); free(s->S);
    for (int i = 0; i < s->npend; ++i) { free(s->pendL[i]); free(s->pendX[i]); }
    free(s->pendL); free(s->pendX); free(s->pend_block);
    free(s->tr_lp); free(s->tr_q); free(s->tr_qc); free(s->tr_loga); free(s->tr_acc);
    free(s->traj); free(s->blk_beta); free(s->scratch);
    free(s->Lp); free(s->Lqp); free(s->xrefp); free(s->betap); free(s->accp);
    free(s->Sloc); free(s->sumloc); free(s->Sglob); free(s->sumglob);
    free(s);
}

/* End of an interval of n_lag steps (Algorithm 1, "if n = k n_lag"): beta update from the acceptance
 * ratio, moments, Cholesky of C_n; the new factor takes effect refresh_delay + 1 blocks later. */
/* Factor of C + eps diag(C) with the refresh rule's retries (eps x100, four attempts in all): 0 on success. */
static int orc_jittered_cholesky(orc_sampler* s, const double* C, double* L) {
    const orc_config* c = &s->cfg;
    int d = c->d;
    size_t nn = (size_t)d * d;
    double eps = c->eps_jitter > c->eps_jitter_min ? c->eps_jitter : c->eps_jitter_min;
    int ok = -1;
    double* Cj = (double*)malloc(sizeof(double) * nn);
    for (int attempt = 0; attempt < 4 && ok != 0; ++attempt) {
        memcpy(Cj, C, sizeof(double) * nn);
        for (int i = 0; i < d; ++i) Cj[(size_t)i * d + i] *= 1.0 + eps;
        ok = orc_cholesky(d, Cj, L);
        eps *= 100.0;
        s->chol_attempts++;
    }
    free(Cj);
    return ok;
}

/* Interval end with per-chain factors (Sec. 2.4.1): each chain's beta rule on its own acceptance; each chain's factor from
 * its local view of the global moments, C^{p,glob} = S^{p,glob} - m^{p,glob} (m^{p,glob})^T, with
 * S^{p,glob} = (sum over the merged batches + chain p's sum over this batch) / (their sample count) -- the
 * weights k M P n_lag and m n_lag of eq. (mom2pg) as counts; after M intervals the batch's samples of every
 * chain are merged into the global sums (eq. (mom2g), (mom1g)). */
static void orc_block_end_r2(orc_sampler* s, int64_t blk) {
    const orc_config* c = &s->cfg;
    int d = c->d, P = c->P;
    size_t nn = (size_t)d * d;
    int64_t acc_blk = 0;
    for (int p = 0; p < P; ++p) {
        acc_blk += s->accp[p];
        if (c->adapt_beta) {
            double ahat = (double)s->accp[p] / (double)c->n_lag;
            double b = s->betap[p];
            if (ahat > c->acc_hi) b *= c->beta_factor;
            else if (ahat < c->acc_lo) b /= c->beta_factor;
            if (b < c->beta_min) b = c->beta_min;
            if (b > c->beta_max) b = c->beta_max;
            s->betap[p] = b;
        }
        s->accp[p] = 0;
    }
    if ((blk + 1) * (int64_t)c->n_lag > c->burnin) s->acc_total += acc_blk;
    s->acc_block = 0;
    const int64_t n = s->nglob + s->nloc;
    if (s->acc_total >= c->min_samples_refresh && n > 0) {
        double* m = (double*)malloc(sizeof(double) * d);
        double* C = (double*)malloc(sizeof(double) * nn);
        double* L = (double*)malloc(sizeof(double) * nn);
        int any = 0;
        for (int p = 0; p < P; ++p) {
            const double* Sl = s->Sloc + (size_t)p * nn;
            const double* sl = s->sumloc + (size_t)p * d;
            for (int i = 0; i < d; ++i) m[i] = (s->sumglob[i] + sl[i]) / (double)n;
            for (int i = 0; i < d; ++i)
                for (int j = 0; j < d; ++j)
                    C[(size_t)i * d + j] = (s->Sglob[(size_t)i * d + j] + Sl[(size_t)i * d + j]) / (double)n - m[i] * m[j];
            if (orc_jittered_cholesky(s, C, L) == 0) {
                double* Lp = s->Lp + (size_t)p * nn;
                double* Lqp = s->Lqp + (size_t)p * nn;
                memcpy(Lp, L, sizeof(double) * nn);
                for (size_t k = 0; k < nn; ++k) Lqp[k] = orc_round_factor(c->prec, L[k]);
                if (c->xref_mode == 1 && c->proposal == 0)
                    for (int i = 0; i < d; ++i) s->xrefp[(size_t)p * d + i] = c->prec != 0 ? orc_round_f32(m[i]) : m[i];
                any = 1;
            } else {
                s->notspd++;
            }
        }
        if (any) s->refreshes++;
        free(m); free(C); free(L);
    }
    if ((blk + 1) % (c->M > 0 ? c->M : 1) == 0) {   /* the batch's samples of every chain join the global sums */
        for (int p = 0; p < P; ++p) {
            for (size_t k = 0; k < nn; ++k) s->Sglob[k] += s->Sloc[(size_t)p * nn + k];
            for (int i = 0; i < d; ++i) s->sumglob[i] += s->sumloc[(size_t)p * d + i];
        }
        s->nglob += (int64_t)P * s->nloc;
        memset(s->Sloc, 0, sizeof(double) * (size_t)P * nn);
        memset(s->sumloc, 0, sizeof(double) * (size_t)P * d);
        s->nloc = 0;
    }
}

static void orc_block_end(orc_sampler* s, int64_t blk) {
    const orc_config* c = &s->cfg;
    int d = c->d;
    size_t nn = (size_t)d * d;
    if (c->moments_mode == 1) {
        orc_block_end_r2(s, blk);
        return;
    }
    /* beta adaptation: raise above the window, lower below it (Algorithm 1; window of Sec. 3.2) */
    if (c->adapt_beta) {
        double ahat = (double)s->acc_block / ((double)c->P * c->n_lag);
        if (ahat > c->acc_hi) s->beta *= c->beta_factor;
        else if (ahat < c->acc_lo) s->beta /= c->beta_factor;
        if (s->beta < c->beta_min) s->beta = c->beta_min;
        if (s->beta > c->beta_max) s->beta = c->beta_max;
    }
    if ((blk + 1) * (int64_t)c->n_lag > c->burnin) s->acc_total += s->acc_block;
    s->acc_block = 0;
    int slot = (int)(blk % s->npend);
    if (s->acc_total >= c->min_samples_refresh && s->n > 0) {
        /* eq. (sampmean), eq. (sampcov): m_n = (1/n) sum x_i, C_n = (1/n) sum x_i x_i^T - m_n m_n^T */
        double* m = (double*)malloc(sizeof(double) * d);
        double* C = (double*)malloc(sizeof(double) * nn);
        double* L = (double*)malloc(sizeof(double) * nn);
        for (int i = 0; i < d; ++i) m[i] = s->sum[i] / (double)s->n;
        for (int i = 0; i < d; ++i)
            for (int j = 0; j < d; ++j) C[(size_t)i * d + j] = s->S[(size_t)i * d + j] / (double)s->n - m[i] * m[j];
        /* skip / jitter rule (the paper is silent on degenerate C_n): factor C_n + eps diag(C_n), i.e. every
         * variance loaded by the same relative amount, retrying with eps x 100 up to three times */
        double eps = c->eps_jitter > c->eps_jitter_min ? c->eps_jitter : c->eps_jitter_min;
        int ok = -1;
        for (int attempt = 0; attempt < 4 && ok != 0; ++attempt) {
            double* Cj = (double*)malloc(sizeof(double) * nn);
            memcpy(Cj, C, sizeof(double) * nn);
            for (int i = 0; i < d; ++i) Cj[(size_t)i * d + i] *= 1.0 + eps;
            ok = orc_cholesky(d, Cj, L);
            free(Cj);
            eps *= 100.0;
            s->chol_attempts++;
        }
        if (ok == 0) {
            free(s->pendL[slot]); free(s->pendX[slot]);
            s->pendL[slot] = L;
            s->pendX[slot] = m;
            s->pend_block[slot] = blk + 1 + c->refresh_delay;
            s->refreshes++;
            L = NULL; m = NULL;
        } else {
            s->notspd++;
        }
        free(L); free(m); free(C);
    }
}

/* Apply a pending factor whose time has come (start of block blk). */
static void orc_block_begin(orc_sampler* s, int64_t blk) {
    for (int i = 0; i < s->npend; ++i) {
        if (s->pend_block[i] == blk && s->pendL[i]) {
            memcpy(s->L, s->pendL[i], sizeof(double) * (size_t)s->cfg.d * s->cfg.d);
            orc_set_quantised_factor(s);
            if (s->cfg.xref_mode == 1 && s->cfg.proposal == 0) orc_set_xref(s, s->pendX[i]);
            free(s->pendL[i]); free(s->pendX[i]);
            s->pendL[i] = NULL; s->pendX[i] = NULL;
            s->pend_block[i] = -1;
            if (s->tgt.kind == ORC_T_REF) orc_recompute_lp(s);  /* the reference target moved */
        }
    }
}

/* One step of every chain: eq. (diamnl) proposal, eq. (accept) test as written in Algorithm 1. */
static void orc_step(orc_sampler* s) {
    const orc_config* c = &s->cfg;
    int d = c->d, P = c->P;
    int64_t t = s->t;
    if (t % c->n_lag == 0) orc_block_begin(s, t / c->n_lag);
    const int rw = c->proposal == 1, r2 = c->moments_mode == 1;
    int8_t* acc = (int8_t*)calloc((size_t)P, 1);
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(c->threads > 0 ? c->threads : 1)
#endif
    for (int p = 0; p < P; ++p) {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double* work = s->scratch + (size_t)tid * 4 * d;
        double* xp = work + 2 * d;
        double* Wd = work + 3 * d;
        /* the proposal's factor, x_ref and beta: the pooled ones or chain p's own (Sec. 2.4.1) */
        const double* Lq = r2 ? s->Lqp + (size_t)p * d * d : s->Lq;
        const double* xref = r2 ? s->xrefp + (size_t)p * d : s->xref;
        const double beta = r2 ? s->betap[p] : s->beta;
        const double rho = sqrt(1.0 - beta * beta), ba = beta * c->infl;
        float* Wf = (float*)malloc(sizeof(float) * d);
        orc_normals(c->seed, c->problem_id, t, c->chain0 + (uint32_t)p, d, Wf);
        for (int i = 0; i < d; ++i) Wd[i] = c->prec != 0 ? orc_round_bf16((double)Wf[i]) : (double)Wf[i];
        free(Wf);
        const double* x = s->x + (size_t)p * d;
        /* DIAM: x* = x_ref + sqrt(1 - beta^2)(x_n - x_ref) + beta * infl * A_n W_n;  RW: x* = x_n + beta * infl * A_n W_n */
        for (int i = 0; i < d; ++i) {
            double xi = 0.0;
            for (int k = 0; k <= i; ++k) xi += Lq[(size_t)i * d + k] * Wd[k];
            xp[i] = rw ? x[i] + ba * xi : xref[i] + rho * (x[i] - xref[i]) + ba * xi;
        }
        double lpp = orc_logpi(s, xp, work);
        /* q: minus the log density of the Gaussian the DIAM move preserves; the random walk's density is
         * symmetric and cancels (eq. (rw)) */
        double qp = rw ? 0.0 : orc_quad(s, Lq, xref, xp, work);
        double qc = rw ? 0.0 : orc_quad(s, Lq, xref, x, work);
        double loga = lpp + qp - (s->lp[p] + qc);
        double u = orc_uniform(c->seed, c->problem_id, ORC_TAG_U, t, c->chain0 + (uint32_t)p);
        int a = log(u) < loga;
        if (t < c->trace_steps) {
            size_t k = (size_t)t * P + p;
            s->tr_lp[k] = lpp; s->tr_q[k] = qp; s->tr_qc[k] = qc; s->tr_loga[k] = loga; s->tr_acc[k] = (int8_t)a;
        }
        if (a) {
            memcpy(s->x + (size_t)p * d, xp, sizeof(double) * d);
            s->lp[p] = lpp;
            acc[p] = 1;
        }
    }
    /* moments over the post-step states of all chains, in chain order; the first n_0 steps are burn-in
     * (footnote to Algorithm 1) and enter neither the moments nor the count of accepted moves */
    for (int p = 0; p < P; ++p) {
        const double* x = s->x + (size_t)p * d;
        s->acc_block += acc[p];
        s->acc_all += acc[p];
        if (r2) s->accp[p] += acc[p];
        if (t < c->burnin) continue;
        for (int i = 0; i < d; ++i) {
            s->sum[i] += x[i];
            for (int j = 0; j < d; ++j) s->S[(size_t)i * d + j] += x[i] * x[j];
        }
        s->n += 1;
        if (r2) {   /* chain p's own sums over the current batch */
            double* Sl = s->Sloc + (size_t)p * d * d;
            double* sl = s->sumloc + (size_t)p * d;
            for (int i = 0; i < d; ++i) {
                sl[i] += x[i];
                for (int j = 0; j < d; ++j) Sl[(size_t)i * d + j] += x[i] * x[j];
            }
        }
    }
    if (r2 && t >= c->burnin) s->nloc += 1;
    free(acc);
    if (s->traj) memcpy(s->traj + (size_t)t * P * d, s->x, sizeof(double) * (size_t)P * d);
    s->t = t + 1;
    if (s->t % c->n_lag == 0) {
        int64_t blk = t / c->n_lag;
        if (s->blk_beta && blk < s->nblk_rec) s->blk_beta[blk] = s->beta;
        orc_block_end(s, blk);
    }
}

/* Run n_steps steps; optional trajectory record (n_steps x P x d) of every post-step state. */
ORC_EXPORT int orc_run(orc_sampler* s, int64_t n_steps, int record) {
    if (record) {
        double* traj = (double*)realloc(s->traj, sizeof(double) * (size_t)(s->t + n_steps) * s->cfg.P * s->cfg.d);
        if (!traj) return -1;
        s->traj = traj;
    } else {
        free(s->traj);
        s->traj = NULL;
    }
    int64_t nb = (s->t + n_steps) / s->cfg.n_lag + 1;
    double* bb = (double*)realloc(s->blk_beta, sizeof(double) * (size_t)nb);
    if (!bb) return -1;
    for (int64_t k = s->nblk_rec; k < nb; ++k) bb[k] = 0.0;
    s->blk_beta = bb;
    s->nblk_rec = nb;
    for (int64_t k = 0; k < n_steps; ++k) orc_step(s);
    return 0;
}

/* ---- getters ---- */
ORC_EXPORT int64_t orc_steps(const orc_sampler* s) { return s->t; }
ORC_EXPORT double orc_beta(const orc_sampler* s) { return s->beta; }
ORC_EXPORT void orc_counts(const orc_sampler* s, int64_t* out) {
    out[0] = s->n; out[1] = s->acc_all; out[2] = s->refreshes; out[3] = s->notspd;
    out[4] = s->chol_attempts;
}
ORC_EXPORT void orc_get_state(const orc_sampler* s, double* x, double* lp) {
    memcpy(x, s->x, sizeof(double) * (size_t)s->cfg.P * s->cfg.d);
    memcpy(lp, s->lp, sizeof(double) * (size_t)s->cfg.P);
}
ORC_EXPORT void orc_get_factor(const orc_sampler* s, double* L, double* Lq, double* xref) {
    size_t nn = (size_t)s->cfg.d * s->cfg.d;
    if (L) memcpy(L, s->L, sizeof(double) * nn);
    if (Lq) memcpy(Lq, s->Lq, sizeof(double) * nn);
    if (xref) memcpy(xref, s->xref, sizeof(double) * s->cfg.d);
}
/* Per-chain factors (Sec. 2.4.1): chain p's factor in use, its quantised form and x_ref, and its beta. */
ORC_EXPORT void orc_get_chain_factor(const orc_sampler* s, int p, double* L, double* Lq, double* xref, double* beta) {
    size_t nn = (size_t)s->cfg.d * s->cfg.d;
    if (!s->Lp || p < 0 || p >= s->cfg.P) return;
    if (L) memcpy(L, s->Lp + (size_t)p * nn, sizeof(double) * nn);
    if (Lq) memcpy(Lq, s->Lqp + (size_t)p * nn, sizeof(double) * nn);
    if (xref) memcpy(xref, s->xrefp + (size_t)p * s->cfg.d, sizeof(double) * s->cfg.d);
    if (beta) *beta = s->betap[p];
}

/* mean m_n and covariance C_n of eq. (sampmean) / eq. (sampcov) */
ORC_EXPORT void orc_get_moments(const orc_sampler* s, double* mean, double* cov) {
    int d = s->cfg.d;
    for (int i = 0; i < d; ++i) mean[i] = s->sum[i] / (double)s->n;
    if (cov)
        for (int i = 0; i < d; ++i)
            for (int j = 0; j < d; ++j) cov[(size_t)i * d + j] = s->S[(size_t)i * d + j] / (double)s->n - mean[i] * mean[j];
}
ORC_EXPORT void orc_get_trace(const orc_sampler* s, double* lp, double* q, double* qc, double* loga, int8_t* acc) {
    size_t nt = (size_t)(s->t < s->cfg.trace_steps ? s->t : s->cfg.trace_steps) * s->cfg.P;
    memcpy(lp, s->tr_lp, nt * 8); memcpy(q, s->tr_q, nt * 8); memcpy(qc, s->tr_qc, nt * 8);
    memcpy(loga, s->tr_loga, nt * 8); memcpy(acc, s->tr_acc, nt);
}
ORC_EXPORT void orc_get_traj(const orc_sampler* s, double* traj) {
    memcpy(traj, s->traj, sizeof(double) * (size_t)s->t * s->cfg.P * s->cfg.d);
}
ORC_EXPORT void orc_get_block_beta(const orc_sampler* s, double* b, int64_t n) {
    memcpy(b, s->blk_beta, sizeof(double) * (size_t)(n < s->nblk_rec ? n : s->nblk_rec));
}
