/*
 * CPU oracle for coupled score-weighted Markov chain pool decoding (MCPD).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the bench's CPU-baseline leg may
 * load this library.  It shares no code with the CUDA library: it is a plain, slow restatement of
 * the paper's definitions, written so that a reader can check it against the paper by eye.
 *
 * What it follows (paper sections):
 *   - Section "Knill's Method": posterior pi(z|y), naive ranking R_i, pruning to the active set A.
 *   - Section "Score-Weighted Update Gibbs Sampler": a_j, s_i, gamma = 100 n_a, tau_w, w_i.
 *   - Single-site map Phi_i(x,u) = 1{u <= p_i(1|x_-i)} (Preliminaries) and Algorithms 1-3.
 *   - H_r and H_{k:l} (Section "Coupled Estimator and Fixed-Budget GPU Execution").
 *   - Algorithm 4: fixed horizon B, slot refill, N_p(B), N*_p(B), slot mean A_p(B), theta_CT.
 *   - The meeting cap of the experiments (Appendix, setup of the estimator lengths): a pair that
 *     has not met when its clock reaches the cap stops there and keeps H_{k:l} with every inner
 *     sum cut at the cap, the finite-cap approximation of the uncapped estimator.
 * Every random number is a Philox4x32-10 block (Salmon, Moraes, Dror, Shaw, SC'11) with the key
 * (seed low, seed high) and the counter (block index, replication, global slot id,
 * tag << 24 | instance), tags 0 (step words), 1 (initial state) and 2 (a uniform's low word), so
 * that any implementation keyed the same way draws the same stream.  Everything is IEEE double; build with -ffp-contract=off so that no multiply-add is fused.
 *
 * Parity status: pinned (see tests/test_oracle_pins.py) except where a function says otherwise.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_ENOMEM (-2)
#define ORC_ESTEP_LIMIT (-3)
#define ORC_EFAITHFUL (-4)

#define SCAN_SCORE 0
#define SCAN_UNIFORM 1
#define SCAN_SYSTEMATIC 2
#define SCAN_CUSTOM 3

#define TWO32 4294967296.0

/* ------------------------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al., SC'11): 10 rounds of the 4x32 Philox S-box, Weyl key schedule. */
void orc_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Counter layout of the written spec: (time word, replication, global slot, tag<<24 | instance). */
static void draw_block(uint64_t seed, uint32_t instance, uint32_t tag, uint32_t c0, uint32_t rep,
                       uint32_t slot, uint32_t out[4]) {
    uint32_t ctr[4] = {c0, rep, slot, (tag << 24) | (instance & 0xFFFFFFu)};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    orc_philox(ctr, key, out);
}

/* ------------------------------------------------------------------------------------------ */
typedef struct orc_model {
    int32_t n, m, na, deg_max, scan;
    int32_t *active;   /* [na] original index of active clone a, ascending */
    int32_t *label;    /* [n]  active label of an original clone, -1 if pruned */
    int32_t *ptr;      /* [na+1] pools of active clone a (CSR, ascending pool ids) */
    int32_t *pools;
    int32_t *pptr;     /* [m+1] active members of pool j */
    int32_t *pmem;
    uint8_t *y;        /* [m] observed outcomes */
    int32_t *dA;       /* [m] pool size restricted to the active clones, d_j^A */
    double a_plus, a_minus, lambda;
    double *eta;       /* [n] naive log score */
    double *score;     /* [na] s_i */
    double *w;         /* [na] scan weights */
    uint64_t *V;       /* [na] integer weights, sum n_a * 2^32 */
    uint32_t *prob;    /* [na] alias table */
    uint32_t *alias;
    uint64_t *T;       /* [(deg_max+1)^2] acceptance thresholds, T[np*(deg_max+1)+nn] */
    uint64_t *Tnu;     /* [na] initial-state thresholds, NULL for the all-negative start */
} orc_model;

void orc_model_free(orc_model *M) {
    if (!M) return;
    free(M->active); free(M->label); free(M->ptr); free(M->pools); free(M->pptr); free(M->pmem);
    free(M->y); free(M->dA); free(M->eta); free(M->score); free(M->w); free(M->V);
    free(M->prob); free(M->alias); free(M->T); free(M->Tnu);
    free(M);
}

/* Likelihood ratio terms (Knill's method): Pr(y=1|xi=1) = 1-fn, Pr(y=1|xi=0) = fp.
 * a_j = log Pr(y_j|xi=1) - log Pr(y_j|xi=0); lambda = log(q/(1-q)) split as log q - log(1-q). */
static void likelihood_constants(double fp, double fn, double q, double *a_plus, double *a_minus,
                                 double *lambda) {
    *a_plus = log(1.0 - fn) - log(fp);
    *a_minus = log(fn) - log(1.0 - fp);
    *lambda = log(q) - log(1.0 - q);
}

/* p(1|x_-i) = sigma(lambda + n+ a+ + n- a-) as a 64-bit threshold floor(p * 2^64), clamped to
 * [1, 2^64-1].  The exponent is summed in exactly this order. */
double orc_conditional_prob(const orc_model *M, int32_t np, int32_t nn) {
    double z = (M->lambda + (double)np * M->a_plus) + (double)nn * M->a_minus;
    return 1.0 / (1.0 + exp(-z));
}

static uint64_t prob_to_threshold(double p) {
    uint64_t t;
    if (!(p < 1.0)) t = UINT64_MAX;
    else if (!(p > 0.0)) t = 0;
    else t = (uint64_t)ldexp(p, 64);   /* truncation = floor for a positive value */
    return t;
}

uint64_t orc_threshold(const orc_model *M, int32_t np, int32_t nn) {
    uint64_t t = prob_to_threshold(orc_conditional_prob(M, np, nn));
    return t == 0 ? 1 : t;
}

static int cmp_eta_desc(const void *pa, const void *pb, void *ctx) {
    const double *eta = (const double *)ctx;
    int32_t a = *(const int32_t *)pa, b = *(const int32_t *)pb;
    if (eta[a] > eta[b]) return -1;
    if (eta[a] < eta[b]) return 1;
    return (a > b) - (a < b);
}

/* qsort_r is a GNU extension; a plain insertion sort keeps the oracle portable and obvious. */
static void sort_by_eta(int32_t *idx, int32_t n, const double *eta) {
    for (int32_t i = 1; i < n; ++i) {
        int32_t v = idx[i], j = i - 1;
        while (j >= 0 && cmp_eta_desc(&idx[j], &v, (void *)eta) > 0) { idx[j + 1] = idx[j]; --j; }
        idx[j + 1] = v;
    }
}

/* Integer Vose alias table over columns of mass K = 2^32, FIFO queues in ascending index. */
static void build_alias(int32_t na, const uint64_t *V_in, uint32_t *prob, uint32_t *alias) {
    const uint64_t K = (uint64_t)1 << 32;
    uint64_t *V = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)na);
    int32_t *small = (int32_t *)malloc(sizeof(int32_t) * (size_t)na * 2 + 8);
    int32_t *large = (int32_t *)malloc(sizeof(int32_t) * (size_t)na + 8);
    int32_t sh = 0, st = 0, lh = 0, lt = 0;
    memcpy(V, V_in, sizeof(uint64_t) * (size_t)na);
    for (int32_t i = 0; i < na; ++i) {
        if (V[i] < K) small[st++] = i; else large[lt++] = i;
    }
    for (int32_t i = 0; i < na; ++i) { prob[i] = 0xFFFFFFFFu; alias[i] = (uint32_t)i; }
    while (sh < st && lh < lt) {
        int32_t s = small[sh++];
        int32_t g = large[lh];
        prob[s] = (uint32_t)V[s];
        alias[s] = (uint32_t)g;
        V[g] -= K - V[s];
        if (V[g] < K) { lh++; small[st++] = g; }
    }
    free(V); free(small); free(large);
}

/* Build everything the sampler needs from (design, y, rates, prior).
 * scan: 0 paper score weights, 1 uniform, 2 systematic (uncoupled only), 3 custom weights. */
int orc_model_new(int32_t n, int32_t m, const int32_t *clone_ptr, const int32_t *clone_pools,
                  const uint8_t *y, double fp, double fn, double q, int32_t n_active, int32_t scan,
                  const double *custom_w, const double *init_marginals, orc_model **out) {
    *out = NULL;
    if (n <= 0 || m < 0 || !(fp > 0 && fp < 1) || !(fn > 0 && fn < 1) || !(q > 0 && q < 1))
        return ORC_EINVAL;
    if (scan < 0 || scan > 3 || (scan == SCAN_CUSTOM && !custom_w)) return ORC_EINVAL;
    for (int32_t i = 0; i < n; ++i) {
        if (clone_ptr[i + 1] < clone_ptr[i]) return ORC_EINVAL;
        for (int32_t e = clone_ptr[i]; e < clone_ptr[i + 1]; ++e) {
            if (clone_pools[e] < 0 || clone_pools[e] >= m) return ORC_EINVAL;
            if (e > clone_ptr[i] && clone_pools[e] <= clone_pools[e - 1]) return ORC_EINVAL;
        }
    }
    orc_model *M = (orc_model *)calloc(1, sizeof(orc_model));
    if (!M) return ORC_ENOMEM;
    M->n = n; M->m = m; M->scan = scan;
    likelihood_constants(fp, fn, q, &M->a_plus, &M->a_minus, &M->lambda);
    M->y = (uint8_t *)malloc((size_t)m + 1);
    for (int32_t j = 0; j < m; ++j) M->y[j] = y[j] ? 1 : 0;

    /* Naive ranking (Knill et al.) as a log score: eta_i = log(q/(1-q)) + log R_i, where R_i, the
     * product over the pools of i of Pr(y_j|xi_j=1)/Pr(y_j|xi_j=0), is a+ per positive and a- per
     * negative pool: eta_i = (lambda + n+_i a+) + n-_i a-.  Equal counts give exactly equal
     * scores, so ties are broken by index as the reading of the pruning rule says. */
    M->eta = (double *)malloc(sizeof(double) * (size_t)n);
    for (int32_t i = 0; i < n; ++i) {
        int32_t npos = 0, nneg = 0;
        for (int32_t e = clone_ptr[i]; e < clone_ptr[i + 1]; ++e) {
            if (M->y[clone_pools[e]]) npos++; else nneg++;
        }
        M->eta[i] = (M->lambda + (double)npos * M->a_plus) + (double)nneg * M->a_minus;
    }
    /* Pruning: keep the top n_active clones by eta (ties: lower index), relabel ascending. */
    int32_t na = (n_active <= 0 || n_active >= n) ? n : n_active;
    M->na = na;
    M->label = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    M->active = (int32_t *)malloc(sizeof(int32_t) * (size_t)na);
    {
        int32_t *order = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
        for (int32_t i = 0; i < n; ++i) { order[i] = i; M->label[i] = -1; }
        if (na < n) sort_by_eta(order, n, M->eta);
        for (int32_t r = 0; r < na; ++r) M->label[order[r]] = 0;
        int32_t a = 0;
        for (int32_t i = 0; i < n; ++i) if (M->label[i] == 0) { M->label[i] = a; M->active[a++] = i; }
        free(order);
    }
    /* Active CSR and the pool -> active member lists. */
    M->ptr = (int32_t *)malloc(sizeof(int32_t) * (size_t)(na + 1));
    M->ptr[0] = 0;
    for (int32_t a = 0; a < na; ++a) {
        int32_t i = M->active[a];
        M->ptr[a + 1] = M->ptr[a] + (clone_ptr[i + 1] - clone_ptr[i]);
    }
    int32_t nnz = M->ptr[na];
    M->pools = (int32_t *)malloc(sizeof(int32_t) * (size_t)nnz + 4);
    M->deg_max = 0;
    for (int32_t a = 0; a < na; ++a) {
        int32_t i = M->active[a];
        int32_t d = clone_ptr[i + 1] - clone_ptr[i];
        if (d > M->deg_max) M->deg_max = d;
        for (int32_t e = 0; e < d; ++e) M->pools[M->ptr[a] + e] = clone_pools[clone_ptr[i] + e];
    }
    M->dA = (int32_t *)calloc((size_t)m + 1, sizeof(int32_t));
    for (int32_t e = 0; e < nnz; ++e) M->dA[M->pools[e]]++;
    M->pptr = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m + 1));
    M->pptr[0] = 0;
    for (int32_t j = 0; j < m; ++j) M->pptr[j + 1] = M->pptr[j] + M->dA[j];
    M->pmem = (int32_t *)malloc(sizeof(int32_t) * (size_t)nnz + 4);
    {
        int32_t *fill = (int32_t *)calloc((size_t)m + 1, sizeof(int32_t));
        for (int32_t a = 0; a < na; ++a)
            for (int32_t e = M->ptr[a]; e < M->ptr[a + 1]; ++e) {
                int32_t j = M->pools[e];
                M->pmem[M->pptr[j] + fill[j]++] = a;
            }
        free(fill);
    }
    /* Score weights: s_i = sum_{j: A_ji = 1} d_j^A a_j; tau_w = log(100 n_a) / (s_max - s_min);
     * w_i = 0.5 softmax(tau_w s)_i + 0.5 / n_a, the softmax shifted by s_max. */
    M->score = (double *)malloc(sizeof(double) * (size_t)na);
    M->w = (double *)malloc(sizeof(double) * (size_t)na);
    for (int32_t a = 0; a < na; ++a) {
        double s = 0.0;
        for (int32_t e = M->ptr[a]; e < M->ptr[a + 1]; ++e) {
            int32_t j = M->pools[e];
            s = s + (double)M->dA[j] * (M->y[j] ? M->a_plus : M->a_minus);
        }
        M->score[a] = s;
    }
    if (scan == SCAN_SCORE) {
        double smax = M->score[0], smin = M->score[0];
        for (int32_t a = 1; a < na; ++a) {
            if (M->score[a] > smax) smax = M->score[a];
            if (M->score[a] < smin) smin = M->score[a];
        }
        double gamma = 100.0 * (double)na;
        double tau = (smax > smin) ? log(gamma) / (smax - smin) : 0.0;
        double E = 0.0;
        for (int32_t a = 0; a < na; ++a) { M->w[a] = exp(tau * (M->score[a] - smax)); E = E + M->w[a]; }
        for (int32_t a = 0; a < na; ++a) M->w[a] = 0.5 * (M->w[a] / E) + 0.5 / (double)na;
    } else if (scan == SCAN_CUSTOM) {
        double E = 0.0;
        for (int32_t a = 0; a < na; ++a) {
            if (!(custom_w[a] > 0.0) || !isfinite(custom_w[a])) { orc_model_free(M); return ORC_EINVAL; }
            E = E + custom_w[a];
        }
        for (int32_t a = 0; a < na; ++a) M->w[a] = custom_w[a] / E;
    } else {
        for (int32_t a = 0; a < na; ++a) M->w[a] = 1.0 / (double)na;
    }
    /* Integer weights V_i summing to n_a 2^32 and the alias table. */
    M->V = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)na);
    M->prob = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)na);
    M->alias = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)na);
    if (scan == SCAN_UNIFORM || scan == SCAN_SYSTEMATIC) {
        for (int32_t a = 0; a < na; ++a) M->V[a] = (uint64_t)1 << 32;
    } else {
        double Kall = (double)na * TWO32;
        uint64_t total = 0;
        for (int32_t a = 0; a < na; ++a) {
            uint64_t v = (uint64_t)floor(M->w[a] * Kall);
            M->V[a] = v < 1 ? 1 : v;
            total += M->V[a];
        }
        int64_t deficit = (int64_t)(((uint64_t)na << 32) - total);
        int32_t big = 0;
        for (int32_t a = 1; a < na; ++a) if (M->V[a] > M->V[big]) big = a;
        M->V[big] = (uint64_t)((int64_t)M->V[big] + deficit);
        for (int32_t a = 0; a < na; ++a)
            if (M->V[a] < ((uint64_t)1 << 30)) { orc_model_free(M); return ORC_EINVAL; }
    }
    build_alias(na, M->V, M->prob, M->alias);
    /* Acceptance thresholds for every (n+, n-) pair a site can see. */
    int32_t side = M->deg_max + 1;
    M->T = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)side * (size_t)side);
    for (int32_t np = 0; np < side; ++np)
        for (int32_t nn = 0; nn < side; ++nn) M->T[np * side + nn] = orc_threshold(M, np, nn);
    if (init_marginals) {
        M->Tnu = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)na);
        for (int32_t a = 0; a < na; ++a) {
            double v = init_marginals[a];
            if (!(v >= 0.0 && v <= 1.0)) { orc_model_free(M); return ORC_EINVAL; }
            M->Tnu[a] = prob_to_threshold(v);
        }
    }
    *out = M;
    return ORC_OK;
}

/* ------------------------------------------------------------------------------------------ */
/* Accessors for tests. */
void orc_model_dims(const orc_model *M, int32_t out[4]) {
    out[0] = M->na; out[1] = M->m; out[2] = M->deg_max; out[3] = M->ptr[M->na];
}
void orc_model_constants(const orc_model *M, double out[3]) {
    out[0] = M->a_plus; out[1] = M->a_minus; out[2] = M->lambda;
}
void orc_model_tables(const orc_model *M, double *eta, int32_t *active, double *score, double *w,
                      uint64_t *V, uint32_t *prob, uint32_t *alias, uint64_t *T) {
    int32_t side = M->deg_max + 1;
    if (eta) memcpy(eta, M->eta, sizeof(double) * (size_t)M->n);
    if (active) memcpy(active, M->active, sizeof(int32_t) * (size_t)M->na);
    if (score) memcpy(score, M->score, sizeof(double) * (size_t)M->na);
    if (w) memcpy(w, M->w, sizeof(double) * (size_t)M->na);
    if (V) memcpy(V, M->V, sizeof(uint64_t) * (size_t)M->na);
    if (prob) memcpy(prob, M->prob, sizeof(uint32_t) * (size_t)M->na);
    if (alias) memcpy(alias, M->alias, sizeof(uint32_t) * (size_t)M->na);
    if (T) memcpy(T, M->T, sizeof(uint64_t) * (size_t)side * (size_t)side);
}

/* Full conditional of active clone i at state x (x_i itself is ignored): with c_j^{-i} the number
 * of other positive active clones in pool j, n+ (n-) counts the pools of i with c_j^{-i} = 0 and
 * y_j = 1 (y_j = 0).  Pools that hold another positive are positive either way and cancel from
 * pi(x^{i<-1}) / pi(x^{i<-0}). */
void orc_conditional_counts(const orc_model *M, const uint8_t *x, int32_t i, int32_t *np,
                            int32_t *nn) {
    int32_t p = 0, q = 0;
    for (int32_t e = M->ptr[i]; e < M->ptr[i + 1]; ++e) {
        int32_t j = M->pools[e];
        int32_t others = 0;
        for (int32_t u = M->pptr[j]; u < M->pptr[j + 1]; ++u)
            if (M->pmem[u] != i) others += x[M->pmem[u]];
        if (others == 0) { if (M->y[j]) p++; else q++; }
    }
    *np = p; *nn = q;
}

/* Site drawn by one 32-bit word: column = floor(w n_a / 2^32), coin = the low 32 bits of w n_a;
 * the column keeps itself when coin < prob[column], else it yields its alias. */
int32_t orc_select_site(const orc_model *M, uint32_t w) {
    uint64_t prod = (uint64_t)w * (uint64_t)(uint32_t)M->na;
    uint32_t col = (uint32_t)(prod >> 32);
    uint32_t coin = (uint32_t)prod;
    return coin < M->prob[col] ? (int32_t)col : (int32_t)M->alias[col];
}

/* Phi_i(x, u): x_i <- 1{U < T(n+, n-)} with U the 64-bit uniform; returns the new bit. */
int32_t orc_phi(const orc_model *M, uint8_t *x, int32_t i, uint64_t U) {
    int32_t np, nn;
    orc_conditional_counts(M, x, i, &np, &nn);
    x[i] = U < M->T[np * (M->deg_max + 1) + nn] ? 1 : 0;
    return x[i];
}

/* ------------------------------------------------------------------------------------------ */
typedef struct orc_run {
    int64_t k, ell;          /* averaging window k:l (coupled) */
    int64_t burn, length;    /* b and T (uncoupled: estimate averages X_b .. X_{b+T-1}) */
    int64_t horizon;         /* B, progress units per slot */
    int64_t step_limit;      /* safety limit on one replication's time index */
    uint64_t seed;
    int64_t slot_offset;
    int32_t instance;
    int32_t coupled;         /* 1: Algorithms 3 and 4; 0: Algorithm 1 / 2 per replication */
    int32_t pad;
    int64_t meeting_cap;     /* > 0 (coupled, >= max(l, L, 1)): stop an unmet pair at t = cap */
    int64_t lag;             /* L >= 1 of the lagged pair (0 reads as 1) */
} orc_run;

/* Draw (I_t, U_t) for time t of replication rep in slot `slot`. */
static void step_draw(const orc_model *M, const orc_run *R, uint32_t slot, uint32_t rep, int64_t t,
                      int32_t *site, uint64_t *U) {
    uint32_t b[4], lo[4];
    draw_block(R->seed, (uint32_t)R->instance, 0, (uint32_t)(t >> 1), rep, slot, b);
    uint32_t ws = (t & 1) ? b[2] : b[0];
    uint32_t wu = (t & 1) ? b[3] : b[1];
    draw_block(R->seed, (uint32_t)R->instance, 2, (uint32_t)t, rep, slot, lo);
    *U = ((uint64_t)wu << 32) | (uint64_t)lo[0];
    *site = (M->scan == SCAN_SYSTEMATIC) ? (int32_t)(t % M->na) : orc_select_site(M, ws);
}

/* Z_0 ~ nu: all-negative by default, else independent Bernoulli(nu_i) through 64-bit draws. */
static void initial_state(const orc_model *M, const orc_run *R, uint32_t slot, uint32_t rep,
                          uint8_t *z) {
    for (int32_t a = 0; a < M->na; ++a) {
        z[a] = 0;
        if (M->Tnu) {
            uint32_t b[4];
            draw_block(R->seed, (uint32_t)R->instance, 1, (uint32_t)(a >> 1), rep, slot, b);
            uint64_t u = (a & 1) ? (((uint64_t)b[2] << 32) | b[3]) : (((uint64_t)b[0] << 32) | b[1]);
            z[a] = u < M->Tnu[a] ? 1 : 0;
        }
    }
}

typedef struct rep_result {
    int64_t C, tau, draws;
    int32_t status;
    int32_t capped;          /* stopped at the meeting cap before meeting (tau = 0) */
} rep_result;

/* Weight of X_t and of Y_t in G = L H_{k:l} once the sums over r and j are swapped: the number of
 * window indices r in k..l with r <= t and r = t (mod lag), i.e. of j >= 0 with
 * k <= t - j lag <= min(l, t).  For lag 1 it is min(max(t - k + 1, 0), L). */
static int64_t lag_weight(int64_t k, int64_t ell, int64_t lag, int64_t t) {
    if (t < k) return 0;
    int64_t hi = t < ell ? t : ell;
    int64_t jmax = (t - k) / lag;                     /* t - j lag >= k */
    int64_t jmin = (t - hi + lag - 1) / lag;          /* t - j lag <= hi (ceiling) */
    return jmax >= jmin ? jmax - jmin + 1 : 0;
}

/* One coupled replication with lag L >= 1 (Algorithm 3 and the lag coupling of the supplement for
 * L = 1; for L > 1 the lag-L coupling of Jacob, O'Leary and Atchade (2020) that the paper's
 * time-averaged estimator is taken from).  X_0 = Y_0 = Z_0; the pre-lag updates
 * X_{t+1} = Phi_{I_t}(X_t, U_t), t = 0..L-1, move X alone; for t >= L the common (I_t, U_t) give
 * X_{t+1} = Phi_{I_t}(X_t, U_t) and Y_{t+1-L} = Phi_{I_t}(Y_{t-L}, U_t).  The meeting time is
 * tau = inf{t >= L : X_t = Y_{t-L}}, and the replication runs until t >= l and the pair has met,
 * or, with a meeting cap c, until t = c if the pair has not met by then (C = c, tau reported 0).
 * The estimator G_j = L_w H_{k:l}(h_j), L_w = l - k + 1, is accumulated in one of two ways:
 *   literal = 1: store the paths and evaluate H_r = X_r + sum_{j>=1} (X_{r+jL} - Y_{r+(j-1)L}) for
 *                each r in k..l, over the terms with r + jL <= C (the others vanish by
 *                faithfulness, since C >= tau; a capped pair keeps exactly these terms);
 *   literal = 0: the same double sum with the order of summation swapped, accumulated as the
 *                paths are produced: G_j = sum_{t=0}^{C} w(t) X_t[j] - sum_{u=0}^{C-L} w(u) Y_u[j]
 *                with w = lag_weight (X_t enters H_r for the r = t - jL, j >= 0, in the window;
 *                Y_u for the r = u - (j-1)L, j >= 1).
 * trajX / trajY (optional, literal mode or tests) receive X_0..X_C and Y_0..Y_{C-L}; sites the
 * drawn I_0..I_{C-1}. */
static rep_result coupled_replication(const orc_model *M, const orc_run *R, uint32_t slot,
                                      uint32_t rep, int64_t *G, int literal, uint8_t *trajX,
                                      uint8_t *trajY, int32_t *sites, int64_t traj_cap) {
    const int32_t na = M->na;
    const int64_t k = R->k, ell = R->ell;
    const int64_t lag = R->lag > 0 ? R->lag : 1;
    rep_result res = {0, 0, 0, ORC_OK, 0};
    uint8_t *X = (uint8_t *)malloc((size_t)na), *Y = (uint8_t *)malloc((size_t)na);
    initial_state(M, R, slot, rep, X);
    memcpy(Y, X, (size_t)na);                                  /* X_0 = Y_0 = Z_0 */
    for (int32_t a = 0; a < na; ++a) G[a] = 0;
    int store = literal || trajX;
    int64_t cap = traj_cap;
    uint8_t *PX = trajX, *PY = trajY;
    uint8_t *ownX = NULL, *ownY = NULL;
    if (literal && !trajX) {
        cap = (R->step_limit > 0 ? R->step_limit : 1000000) + 1;
        ownX = PX = (uint8_t *)malloc((size_t)cap * (size_t)na);
        ownY = PY = (uint8_t *)malloc((size_t)cap * (size_t)na);
    }
#define KEEP_X(tt) do { if (store && (tt) < cap) memcpy(PX + (size_t)(tt) * na, X, (size_t)na); } while (0)
#define KEEP_Y(tt) do { if (store && (tt) < cap) memcpy(PY + (size_t)(tt) * na, Y, (size_t)na); } while (0)
    KEEP_X(0);
    KEEP_Y(0);
    /* X_0 and Y_0 enter with the same weight and are equal: G starts at 0. */
    int32_t I;
    uint64_t U;
    int64_t t = 0;
    for (; t < lag; ++t) {                                     /* pre-lag: X alone */
        step_draw(M, R, slot, rep, t, &I, &U);
        if (sites && t < cap) sites[t] = I;
        orc_phi(M, X, I, U);
        res.draws += 1;
        KEEP_X(t + 1);
        if (!literal) {
            int64_t wx = lag_weight(k, ell, lag, t + 1);
            for (int32_t a = 0; a < na; ++a) G[a] += wx * (int64_t)X[a];
        }
    }
    int met = memcmp(X, Y, (size_t)na) == 0;                     /* X_L = Y_0 ? */
    res.tau = met ? lag : 0;
    while (t < ell || !met) {
        if (R->meeting_cap > 0 && t >= R->meeting_cap) { res.capped = 1; break; }   /* t >= l: unmet */
        if (R->step_limit > 0 && t >= R->step_limit) { res.status = ORC_ESTEP_LIMIT; break; }
        step_draw(M, R, slot, rep, t, &I, &U);
        if (sites && t < cap) sites[t] = I;
        /* X_{t+1} = Phi_{I_t}(X_t, U_t) and Y_{t+1-L} = Phi_{I_t}(Y_{t-L}, U_t), common (I_t, U_t). */
        orc_phi(M, X, I, U);
        orc_phi(M, Y, I, U);
        t += 1;
        res.draws += 1;
        KEEP_X(t);
        KEEP_Y(t - lag);
        int eq = memcmp(X, Y, (size_t)na) == 0;                  /* X_t = Y_{t-L} ? */
        if (met && !eq) res.status = ORC_EFAITHFUL;              /* Theorem 1(d) violated */
        if (!met && eq) res.tau = t;
        met = eq;
        if (!literal) {
            int64_t wx = lag_weight(k, ell, lag, t), wy = lag_weight(k, ell, lag, t - lag);
            for (int32_t a = 0; a < na; ++a) G[a] += wx * (int64_t)X[a] - wy * (int64_t)Y[a];
        }
    }
    res.C = t;                                     /* C = max(l, tau), or the cap if capped */
    if (literal && res.status == ORC_OK) {
        int64_t C = res.C;
        if (C >= cap) res.status = ORC_EINVAL;
        else {
            for (int64_t r = k; r <= ell; ++r) {
                for (int32_t a = 0; a < na; ++a) {
                    int64_t h = PX[(size_t)r * na + a];
                    for (int64_t j = 1; r + j * lag <= C; ++j)
                        h += (int64_t)PX[(size_t)(r + j * lag) * na + a] -
                             (int64_t)PY[(size_t)(r + (j - 1) * lag) * na + a];
                    G[a] += h;
                }
            }
        }
    }
#undef KEEP_X
#undef KEEP_Y
    free(ownX); free(ownY);
    free(X); free(Y);
    return res;
}

/* One uncoupled chain (Algorithms 1 and 2): X_0 ~ nu, X_{t+1} = Phi_{I_t}(X_t, U_t) for
 * t = 0..b+T-2, G_j = sum_{t=b}^{b+T-1} X_t[j]; cost C = b + T - 1 draws.
 * trajX (optional, tests) receives X_0..X_C and sites the drawn I_0..I_{C-1}, up to traj_cap. */
static rep_result uncoupled_replication(const orc_model *M, const orc_run *R, uint32_t slot,
                                        uint32_t rep, int64_t *G, uint8_t *trajX, int32_t *sites,
                                        int64_t traj_cap) {
    const int32_t na = M->na;
    const int64_t b = R->burn, T = R->length;
    rep_result res = {0, 0, 0, ORC_OK, 0};
    uint8_t *X = (uint8_t *)malloc((size_t)na);
    initial_state(M, R, slot, rep, X);
    if (trajX && traj_cap > 0) memcpy(trajX, X, (size_t)na);
    for (int32_t a = 0; a < na; ++a) G[a] = (b == 0) ? X[a] : 0;
    for (int64_t t = 0; t <= b + T - 2; ++t) {
        int32_t I;
        uint64_t U;
        step_draw(M, R, slot, rep, t, &I, &U);
        if (sites && t < traj_cap) sites[t] = I;
        orc_phi(M, X, I, U);
        res.draws += 1;
        if (trajX && t + 1 < traj_cap) memcpy(trajX + (size_t)(t + 1) * na, X, (size_t)na);
        if (t + 1 >= b && t + 1 <= b + T - 1)
            for (int32_t a = 0; a < na; ++a) G[a] += X[a];
    }
    res.C = b + T - 1;
    free(X);
    return res;
}

/* Number of N*_p buckets: every retained replication costs at least max(l, L) (coupled) or
 * b + T - 1 (uncoupled) progress units, so 1 <= N*_p <= max(1, B / that). */
int64_t orc_num_buckets(const orc_run *R) {
    int64_t lag = R->lag > 1 ? R->lag : 1;
    int64_t unit = R->coupled ? (R->ell > lag ? R->ell : lag) : (R->burn + R->length - 1);
    if (unit < 1) unit = 1;
    int64_t nb = R->horizon / unit;
    return nb < 1 ? 1 : nb;
}

typedef struct slot_out {
    int32_t nstar, reps_started;
    int64_t S_retained;
} slot_out;

/* Algorithm 4 for one logical slot: replications are run in sequence; replication r is started
 * while S_p(r-1) < B; those with S_p(r) <= B are retained; if none is (N_p(B) = 0) the first
 * replication, which completed beyond B, is retained alone.  Gp receives the sum of the retained
 * replications' G vectors, i.e. L N*_p A_p(B). */
static int32_t run_slot(const orc_model *M, const orc_run *R, int64_t p, int64_t *Gp, int64_t *Gr,
                        slot_out *so, int64_t stats[7]) {
    const int32_t na = M->na;
    uint32_t slot = (uint32_t)(R->slot_offset + p);
    int64_t S = 0, N = 0;
    int32_t status = ORC_OK;
    for (int32_t a = 0; a < na; ++a) Gp[a] = 0;
    so->reps_started = 0;
    so->S_retained = 0;
    for (uint32_t r = 0;; ++r) {
        rep_result rr = R->coupled ? coupled_replication(M, R, slot, r, Gr, 0, NULL, NULL, NULL, 0)
                                   : uncoupled_replication(M, R, slot, r, Gr, NULL, NULL, 0);
        so->reps_started++;
        stats[0] += rr.draws;
        stats[1] += 1;
        if (rr.status != ORC_OK) { status = rr.status; if (rr.status == ORC_ESTEP_LIMIT) stats[4]++; break; }
        if (rr.tau > stats[2]) stats[2] = rr.tau;
        stats[3] += rr.tau;
        stats[6] += rr.capped;
        S += rr.C;                                               /* S_p(r) */
        if (S <= R->horizon) {
            N += 1;
            for (int32_t a = 0; a < na; ++a) Gp[a] += Gr[a];
            so->S_retained += rr.C;
        } else {
            if (N == 0) {                                        /* zero-completion correction */
                N = 1;
                for (int32_t a = 0; a < na; ++a) Gp[a] += Gr[a];
                so->S_retained += rr.C;
                stats[5]++;
            }
            break;
        }
        if (!(S < R->horizon)) break;                            /* refill only while S_p(r) < B */
    }
    so->nstar = (int32_t)N;
    return status;
}

typedef struct job {
    const orc_model *M;
    const orc_run *R;
    int64_t p0, p1, nb, p_base;
    int64_t *S1;                 /* [nb][na] */
    unsigned __int128 *S2;       /* [nb][na] */
    int64_t *count;              /* [nb] */
    int32_t *slot_nstar;
    int64_t *slot_S;
    int32_t *slot_reps;
    int64_t *slot_G;
    int64_t stats[7];
    int32_t status;
} job;

static void *job_main(void *arg) {
    job *J = (job *)arg;
    const int32_t na = J->M->na;
    int64_t *Gp = (int64_t *)malloc(sizeof(int64_t) * (size_t)na);
    int64_t *Gr = (int64_t *)malloc(sizeof(int64_t) * (size_t)na);
    for (int64_t p = J->p0; p < J->p1; ++p) {
        slot_out so;
        int32_t st = run_slot(J->M, J->R, p, Gp, Gr, &so, J->stats);
        if (st != ORC_OK && J->status == ORC_OK) J->status = st;
        int64_t local = p - J->p_base;
        if (J->slot_nstar) J->slot_nstar[local] = so.nstar;
        if (J->slot_S) J->slot_S[local] = so.S_retained;
        if (J->slot_reps) J->slot_reps[local] = so.reps_started;
        if (J->slot_G) memcpy(J->slot_G + (size_t)local * na, Gp, sizeof(int64_t) * (size_t)na);
        if (st != ORC_OK) continue;
        int64_t bkt = so.nstar - 1;
        if (bkt < 0 || bkt >= J->nb) { J->status = ORC_EINVAL; continue; }
        J->count[bkt] += 1;
        for (int32_t a = 0; a < na; ++a) {
            J->S1[(size_t)bkt * na + a] += Gp[a];
            J->S2[(size_t)bkt * na + a] += (unsigned __int128)((__int128)Gp[a] * (__int128)Gp[a]);
        }
    }
    free(Gp); free(Gr);
    return NULL;
}

/* Run slots [p_begin, p_end) with `threads` worker threads and sum them into the N*_p buckets:
 * S1[n-1][j] = sum_{p: N*_p = n} G_pj and S2[n-1][j] = sum G_pj^2 as 128-bit (lo, hi) words.
 * stats: [draws, replications started, max tau, sum tau, step-limit hits, zero-completion slots,
 *         replications stopped at the meeting cap].
 * Per-slot outputs are optional (NULL to skip). */
int orc_run_slots(const orc_model *M, const orc_run *R, int64_t p_begin, int64_t p_end,
                  int32_t threads, int64_t *S1, uint64_t *S2_lo, uint64_t *S2_hi, int64_t *count,
                  int32_t *slot_nstar, int64_t *slot_S, int32_t *slot_reps, int64_t *slot_G,
                  int64_t stats[7]) {
    if (R->coupled && (R->k < 0 || R->k > R->ell)) return ORC_EINVAL;
    if (R->coupled && (R->lag < 0 || R->lag > (int64_t)1 << 20)) return ORC_EINVAL;
    if (R->coupled && R->meeting_cap != 0 &&
        (R->meeting_cap < R->ell || R->meeting_cap < (R->lag > 1 ? R->lag : 1))) return ORC_EINVAL;
    if (!R->coupled && (R->burn < 0 || R->length < 1 || R->burn + R->length < 2)) return ORC_EINVAL;
    if (R->horizon < 0 || p_end < p_begin) return ORC_EINVAL;
    const int32_t na = M->na;
    const int64_t nb = orc_num_buckets(R);
    if (threads < 1) threads = 1;
    int64_t P = p_end - p_begin;
    if (threads > P && P > 0) threads = (int32_t)P;
    job *jobs = (job *)calloc((size_t)threads, sizeof(job));
    pthread_t *tid = (pthread_t *)calloc((size_t)threads, sizeof(pthread_t));
    for (int32_t w = 0; w < threads; ++w) {
        job *J = &jobs[w];
        J->M = M; J->R = R; J->nb = nb; J->p_base = p_begin;
        J->p0 = p_begin + P * w / threads;
        J->p1 = p_begin + P * (w + 1) / threads;
        J->S1 = (int64_t *)calloc((size_t)nb * na, sizeof(int64_t));
        J->S2 = (unsigned __int128 *)calloc((size_t)nb * na, sizeof(unsigned __int128));
        J->count = (int64_t *)calloc((size_t)nb, sizeof(int64_t));
        J->slot_nstar = slot_nstar; J->slot_S = slot_S; J->slot_reps = slot_reps; J->slot_G = slot_G;
        if (threads == 1) job_main(J); else pthread_create(&tid[w], NULL, job_main, J);
    }
    int32_t status = ORC_OK;
    for (int32_t s = 0; s < 7; ++s) stats[s] = 0;
    for (int64_t e = 0; e < nb * na; ++e) { S1[e] = 0; S2_lo[e] = 0; S2_hi[e] = 0; }
    for (int64_t b = 0; b < nb; ++b) count[b] = 0;
    for (int32_t w = 0; w < threads; ++w) {
        job *J = &jobs[w];
        if (threads > 1) pthread_join(tid[w], NULL);
        for (int64_t e = 0; e < nb * na; ++e) {
            S1[e] += J->S1[e];
            unsigned __int128 acc = ((unsigned __int128)S2_hi[e] << 64) | S2_lo[e];
            acc += J->S2[e];
            S2_lo[e] = (uint64_t)acc;
            S2_hi[e] = (uint64_t)(acc >> 64);
        }
        for (int64_t b = 0; b < nb; ++b) count[b] += J->count[b];
        stats[0] += J->stats[0]; stats[1] += J->stats[1];
        if (J->stats[2] > stats[2]) stats[2] = J->stats[2];
        stats[3] += J->stats[3]; stats[4] += J->stats[4]; stats[5] += J->stats[5];
        stats[6] += J->stats[6];
        if (J->status != ORC_OK && status == ORC_OK) status = J->status;
        free(J->S1); free(J->S2); free(J->count);
    }
    free(jobs); free(tid);
    return status;
}

/* The swapped-sum weight of X_t and Y_t (tests). */
int64_t orc_lag_weight(int64_t k, int64_t ell, int64_t lag, int64_t t) { return lag_weight(k, ell, lag, t); }

/* One replication with its paths, for tests of the coupling and of the estimator identity. */
int orc_replication(const orc_model *M, const orc_run *R, int64_t p, int32_t rep, int32_t literal,
                    int64_t *G, int64_t out4[4], uint8_t *trajX, uint8_t *trajY, int32_t *sites,
                    int64_t traj_cap) {
    uint32_t slot = (uint32_t)(R->slot_offset + p);
    rep_result rr;
    if (R->coupled)
        rr = coupled_replication(M, R, slot, (uint32_t)rep, G, literal, trajX, trajY, sites, traj_cap);
    else
        rr = uncoupled_replication(M, R, slot, (uint32_t)rep, G, trajX, sites, traj_cap);
    out4[0] = rr.C; out4[1] = rr.tau; out4[2] = rr.draws; out4[3] = rr.capped;
    return rr.status;
}

/* theta_CT = (1/P) sum_p A_p(B) with A_p = G_p / (L N*_p), computed from the buckets as
 * theta_j = (sum_{n ascending} S1[n][j] / n) / (P L); the standard error treats the P slot means
 * as i.i.d. (Assumption 2):  Q_j = (sum_n S2[n][j] / n^2) / L^2,
 * se_j = sqrt(max(0, (Q_j - (P theta_j) theta_j) / (P (P - 1)))); se = NaN when P < 2. */
void orc_finalize(int32_t na, int64_t nb, const int64_t *S1, const uint64_t *S2_lo,
                  const uint64_t *S2_hi, int64_t P, int64_t L, double *est, double *se) {
    const double dP = (double)P, dL = (double)L;
    for (int32_t a = 0; a < na; ++a) {
        double s1 = 0.0, s2 = 0.0;
        for (int64_t b = 0; b < nb; ++b) {
            double n = (double)(b + 1);
            s1 = s1 + (double)S1[(size_t)b * na + a] / n;
            double sq = (double)S2_hi[(size_t)b * na + a] * 18446744073709551616.0
                        + (double)S2_lo[(size_t)b * na + a];
            s2 = s2 + sq / (n * n);
        }
        double th = s1 / (dP * dL);
        est[a] = th;
        if (P < 2) { se[a] = NAN; continue; }
        double Q = s2 / (dL * dL);
        double var = (Q - (dP * th) * th) / (dP * (dP - 1.0));
        se[a] = var > 0.0 ? sqrt(var) : 0.0;
    }
}
