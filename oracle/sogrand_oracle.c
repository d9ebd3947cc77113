/*
 * sogrand_oracle.c -- plain, sequential, FP64 CPU oracle of SOGRAND decoding
 * and of block-turbo decoding of product codes.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links or calls this
 * file; only the tests, the package smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header or table with the CUDA path.
 *
 * What it follows (arXiv 2310.10737, "Soft-output (SO) GRAND and iterative
 * decoding to outperform LDPCs"):
 *   Sec. III-B     GRAND query loop; membership test H x = 0; even-code
 *                  parity skip (only noise patterns of the parity of y).
 *   Sec. IV        Theorem 1 / Corollary: APP of each list word and of
 *                  "not in the list", geometric approximation with
 *                  phi = (2^k-1)/(2^n-1); per-query likelihood bookkeeping.
 *   Sec. V-B       SISO definitions (L_Ch, L_A, L_APP, L_E) and eq. LLRi.
 *   Sec. VI        block turbo decoding of product codes (steps 0/1/2),
 *                  alpha-scaled extrinsic exchange, early stop.
 * The query order is 1-line ORBGRAND, which the paper only cites.  Readings
 * of the points the paper leaves open (all listed in the design notes):
 *   * cost(z) = sum_{r in z} r + c * |z| over reliability ranks r = 1..n
 *     (ranks by |lambda| ascending, ties by bit index);
 *   * within one cost: Hamming weight ascending, then the ascending rank
 *     vector in lexicographic order;
 *   * c = round-half-up of intercept/slope of the least-squares line through
 *     a_r = round-half-up(256 |lambda|_(r)) (exact integers), clamped to
 *     [0, c_max]; a_r saturates at 2^20 - 1;
 *   * even codes ("reading B"): the search and the remaining mass are
 *     conditioned on the parity class of y, phi_B = (2^k-1)/(2^(n-1)-1);
 *     "reading A" keeps the literal 1 - sum and phi = (2^k-1)/(2^n-1);
 *   * the SISO input is lambda = fl32(L_Ch + L_A) (one FP32 rounding) and all
 *     decisions (hard bits, ranks, c) are taken on that FP32 value;
 *   * the remaining mass 1 - sum_{j<=q_L} p(z^j) is evaluated as what it is,
 *     the mass of the patterns not queried (a positive sum, in log domain),
 *     because subtracting the queried mass from the total loses every digit
 *     once the queried mass dominates.  The paper-literal difference is
 *     also returned as a diagnostic.
 * All probabilities are relative to p(0^n | r) (odds domain): p(z|r)/p(0|r)
 * = prod_{i in z} exp(-|lambda_i|); every formula used is a ratio in which
 * p(0^n|r) cancels.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_NMAX 128

typedef struct {
    int n;
    int k;
    const uint8_t *H; /* (n-k) x n, row-major, entries 0/1 */
    int even;         /* 1: even code, parity skip (Sec. III-B) */
    int reading;      /* 0: reading B (parity class); 1: reading A (literal);
                         2: Forney's approximation (eq. missingterm): reading B's
                         search, the mass outside the list taken as 0 */
    int c_max;        /* clamp of the 1-line parameter */
} oracle_code;

/* ------------------------------------------------------------------ */
/* log-domain helpers                                                  */
/* ------------------------------------------------------------------ */
static double logadd(double a, double b)
{
    if (a == -INFINITY) return b;
    if (b == -INFINITY) return a;
    if (a < b) { double t = a; a = b; b = t; }
    return a + log1p(exp(b - a));
}

/* log sigma(x) = log 1/(1+e^-x) */
static double log_sigmoid(double x)
{
    if (x >= 0) return -log1p(exp(-x));
    return x - log1p(exp(x));
}

/* log(2^a - 1) for integer a >= 1 */
static double log_pow2m1(int a)
{
    return a * log(2.0) + log1p(-ldexp(1.0, -a));
}

/* ------------------------------------------------------------------ */
/* code membership: dense GF(2) matrix-vector product (Sec. III-B)     */
/* ------------------------------------------------------------------ */
static int is_codeword(const oracle_code *code, const uint8_t *x)
{
    int m = code->n - code->k;
    for (int t = 0; t < m; t++) {
        int s = 0;
        const uint8_t *h = code->H + (size_t)t * code->n;
        for (int i = 0; i < code->n; i++) s ^= (h[i] & x[i]);
        if (s) return 0;
    }
    return 1;
}

/* ------------------------------------------------------------------ */
/* 1-line parameter c from the sorted reliabilities (exact integers)   */
/* ------------------------------------------------------------------ */
int oracle_one_line_c(int n, const float *absl_sorted, int c_max)
{
    int64_t sy = 0, sxy = 0;
    const int64_t amax = (1 << 20) - 1;
    for (int r = 1; r <= n; r++) {
        double v = (double)absl_sorted[r - 1];
        int64_t a;
        if (!(v < (double)amax)) a = amax; /* also catches +inf */
        else {
            a = (int64_t)floor(v * 256.0 + 0.5);
            if (a > amax) a = amax;
        }
        sy += a;
        sxy += (int64_t)r * a;
    }
    int64_t sx = (int64_t)n * (n + 1) / 2;
    int64_t sxx = (int64_t)n * (n + 1) * (2 * n + 1) / 6;
    int64_t D = (int64_t)n * sxx - sx * sx;
    int64_t Nb = (int64_t)n * sxy - sx * sy; /* slope numerator */
    if (Nb <= 0) return 0;
    int64_t num = sy * D - Nb * sx; /* intercept/slope = num / (n * Nb) */
    int64_t top = 2 * num + (int64_t)n * Nb;
    if (top < 0) return 0;
    int64_t c = top / (2 * (int64_t)n * Nb);
    if (c > c_max) c = c_max;
    return (int)c;
}

/* ------------------------------------------------------------------ */
/* 1-line ORBGRAND query order                                          */
/* ------------------------------------------------------------------ */
typedef int (*emit_fn)(void *ctx, const int *ranks, int w, int64_t cost);

typedef struct {
    int n;
    int w;
    int64_t cost;
    int ranks[OR_NMAX];
    emit_fn fn;
    void *ctx;
} subset_gen;

/* all w-subsets {r_1 < ... < r_w} of {start..n} with sum m, ascending-lexicographic */
static int gen_rec(subset_gen *g, int depth, int start, int64_t m)
{
    int rem = g->w - depth;
    if (rem == 0) return m == 0 ? g->fn(g->ctx, g->ranks, g->w, g->cost) : 0;
    if (rem == 1) {
        if (m >= start && m <= g->n) {
            g->ranks[depth] = (int)m;
            return g->fn(g->ctx, g->ranks, g->w, g->cost);
        }
        return 0;
    }
    int64_t k = rem - 1;
    for (int v = start; v <= g->n; v++) {
        int64_t rest = m - v;
        int64_t minrest = k * v + k * (k + 1) / 2;
        if (rest < minrest) break;
        int64_t maxrest = k * g->n - k * (k - 1) / 2;
        if (rest > maxrest) continue;
        g->ranks[depth] = v;
        int s = gen_rec(g, depth + 1, v + 1, rest);
        if (s) return s;
    }
    return 0;
}

/* Patterns of one cost level C (weights ascending), restricted to the
 * parity class cls (-1: all weights). */
static int gen_level(subset_gen *g, int c, int cls, int64_t C)
{
    int n = g->n;
    for (int w = 0; w <= n; w++) {
        if (cls >= 0 && (w & 1) != cls) continue;
        int64_t m = C - (int64_t)c * w;
        int64_t mmin = (int64_t)w * (w + 1) / 2;
        if (m < mmin) break;
        int64_t mmax = (int64_t)w * (2 * n - w + 1) / 2;
        if (m > mmax) continue;
        g->w = w;
        g->cost = C;
        int s = gen_rec(g, 0, 1, m);
        if (s) return s;
    }
    return 0;
}

/* Whole query sequence: cost 0, 1, 2, ...  Returns 1 if the callback
 * stopped it, 0 if every pattern of the class was emitted. */
static int gen_all(int n, int c, int cls, emit_fn fn, void *ctx)
{
    subset_gen g;
    g.n = n;
    g.fn = fn;
    g.ctx = ctx;
    int64_t cmax = (int64_t)c * n + (int64_t)n * (n + 1) / 2;
    for (int64_t C = 0; C <= cmax; C++) {
        int s = gen_level(&g, c, cls, C);
        if (s) return s;
    }
    return 0;
}

/* ---- test hook: dump the canonical order ---- */
typedef struct {
    int n;
    int64_t max_q, q;
    uint8_t *ranks_out;
    int32_t *cost_out, *w_out;
} trace_ctx;

static int trace_emit(void *vctx, const int *ranks, int w, int64_t cost)
{
    trace_ctx *t = (trace_ctx *)vctx;
    if (t->ranks_out) {
        uint8_t *row = t->ranks_out + (size_t)t->q * t->n;
        memset(row, 0, (size_t)t->n);
        for (int i = 0; i < w; i++) row[ranks[i] - 1] = 1;
    }
    if (t->cost_out) t->cost_out[t->q] = (int32_t)cost;
    if (t->w_out) t->w_out[t->q] = w;
    t->q++;
    return t->q >= t->max_q;
}

int64_t oracle_trace(int n, int c, int cls, int64_t max_q, uint8_t *ranks_out, int32_t *cost_out, int32_t *w_out)
{
    if (n < 1 || n > OR_NMAX || max_q < 1) return -1;
    trace_ctx t = {n, max_q, 0, ranks_out, cost_out, w_out};
    gen_all(n, c, cls, trace_emit, &t);
    return t.q;
}

/* ------------------------------------------------------------------ */
/* remaining (unqueried) mass                                           */
/* ------------------------------------------------------------------ */
typedef struct {
    const double *absl; /* |lambda| by rank, index r-1 */
    int64_t skip, seen;
    double logsum;
} rest_ctx;

static int rest_emit(void *vctx, const int *ranks, int w, int64_t cost)
{
    (void)cost;
    rest_ctx *r = (rest_ctx *)vctx;
    r->seen++;
    if (r->seen <= r->skip) return 0;
    double lp = 0;
    for (int i = 0; i < w; i++) lp -= r->absl[ranks[i] - 1];
    r->logsum = logadd(r->logsum, lp);
    return 0;
}

/* log of the mass of the patterns of cost level C in class cls that come
 * after the first `skip` patterns of that level */
static double level_rest_log(int n, int c, int cls, const double *absl, int64_t C, int64_t skip)
{
    subset_gen g;
    rest_ctx r = {absl, skip, 0, -INFINITY};
    g.n = n;
    g.fn = rest_emit;
    g.ctx = &r;
    gen_level(&g, c, cls, C);
    return r.logsum;
}

/* Log-domain DP over ranks of the mass of all patterns with cost > Cstar,
 * split by parity: tail[p].  Also returns the mass of all patterns with
 * cost <= Cstar by parity (head[p]).  head[j][p] is the mass of the patterns
 * built from the ranks seen so far with cost exactly j and parity p; a
 * pattern enters the tail the moment adding a rank lifts its cost over
 * Cstar, and from then on every later rank may or may not join it. */
static void tail_dp(int n, int c, const double *absl, int64_t Cstar, double tail[2], double head_tot[2])
{
    int64_t J = Cstar + 1;
    double *h0 = (double *)malloc(sizeof(double) * (size_t)J);
    double *h1 = (double *)malloc(sizeof(double) * (size_t)J);
    for (int64_t j = 0; j < J; j++) h0[j] = h1[j] = -INFINITY;
    h0[0] = 0.0; /* empty pattern: mass 1 (odds domain), parity 0 */
    double o0 = -INFINITY, o1 = -INFINITY;
    for (int r = 1; r <= n; r++) {
        int64_t d = r + (int64_t)c;
        double lt = -absl[r - 1];
        double n0 = logadd(o0, o1 + lt);
        double n1 = logadd(o1, o0 + lt);
        int64_t jlo = Cstar - d + 1;
        if (jlo < 0) jlo = 0;
        for (int64_t j = jlo; j <= Cstar; j++) {
            n0 = logadd(n0, h1[j] + lt);
            n1 = logadd(n1, h0[j] + lt);
        }
        for (int64_t j = Cstar; j >= d; j--) {
            double a0 = h1[j - d] + lt, a1 = h0[j - d] + lt;
            h0[j] = logadd(h0[j], a0);
            h1[j] = logadd(h1[j], a1);
        }
        o0 = n0;
        o1 = n1;
    }
    tail[0] = o0;
    tail[1] = o1;
    head_tot[0] = head_tot[1] = -INFINITY;
    for (int64_t j = 0; j < J; j++) {
        head_tot[0] = logadd(head_tot[0], h0[j]);
        head_tot[1] = logadd(head_tot[1], h1[j]);
    }
    free(h0);
    free(h1);
}

/* ------------------------------------------------------------------ */
/* SOGRAND SISO                                                         */
/* ------------------------------------------------------------------ */
#define OR_LMAX 4096

typedef struct {
    const oracle_code *code;
    int n, c, cls, L;
    int64_t cap;
    double thr, logphi;
    double absl[OR_NMAX]; /* |lambda| by rank */
    int perm[OR_NMAX];    /* rank r-1 -> bit index */
    uint8_t y[OR_NMAX], x[OR_NMAX];
    int64_t q;            /* queries made */
    int64_t cur_C, cur_idx; /* cost level of the last query and its index within that level (1-based) */
    double S;             /* running sum of queried mass (paper's bookkeeping) */
    int nhit;
    uint8_t *hit_word; /* [L][n] codewords found, in query order */
    double *hit_logp;  /* [L] log p(z)/p(0) of their noise patterns */
    int64_t *hit_q;    /* [L] query index at which each was found */
    int stop_thr;
} siso_ctx;

/* log of the remaining mass after the query at (C, idx) */
static double remaining_log(const siso_ctx *s, int64_t C, int64_t idx)
{
    double tail[2], head[2];
    tail_dp(s->n, s->c, s->absl, C, tail, head);
    double rest = level_rest_log(s->n, s->c, s->cls, s->absl, C, idx);
    double r;
    if (s->cls < 0) r = logadd(tail[0], tail[1]);
    else {
        r = tail[s->cls];
        if (s->code->reading == 1) /* reading A: the other class counts too */
            r = logadd(r, logadd(tail[s->cls ^ 1], head[s->cls ^ 1]));
    }
    return logadd(r, rest);
}

static double pmiss_of(const double *logp, int nh, double M)
{
    double D = M;
    for (int l = 0; l < nh; l++) D = logadd(D, logp[l]);
    return M == -INFINITY ? 0.0 : exp(M - D);
}

static int siso_emit(void *vctx, const int *ranks, int w, int64_t cost)
{
    siso_ctx *s = (siso_ctx *)vctx;
    if (cost != s->cur_C) {
        s->cur_C = cost;
        s->cur_idx = 0;
    }
    s->q++;
    s->cur_idx++;
    double lp = 0;
    for (int i = 0; i < w; i++) lp -= s->absl[ranks[i] - 1];
    s->S += exp(lp);
    memcpy(s->x, s->y, (size_t)s->n);
    for (int i = 0; i < w; i++) s->x[s->perm[ranks[i] - 1]] ^= 1;
    if (is_codeword(s->code, s->x)) {
        int h = s->nhit++;
        memcpy(s->hit_word + (size_t)h * s->n, s->x, (size_t)s->n);
        s->hit_logp[h] = lp;
        s->hit_q[h] = s->q;
        if (s->nhit >= s->L) return 1;
        if (s->thr > 0 && s->code->reading != 2) { /* Forney's prediction is always 0: no threshold */
            double M = remaining_log(s, s->cur_C, s->cur_idx) + s->logphi;
            if (pmiss_of(s->hit_logp, s->nhit, M) < s->thr) {
                s->stop_thr = 1;
                return 1;
            }
        }
    }
    return s->q >= s->cap;
}

typedef struct {
    int n_sort;
    int idx;
    float key;
} sort_item;

static int cmp_rank(const void *a, const void *b)
{
    const sort_item *x = (const sort_item *)a, *y = (const sort_item *)b;
    if (x->key < y->key) return -1;
    if (x->key > y->key) return 1;
    return (x->idx > y->idx) - (x->idx < y->idx);
}

/*
 * One SISO decoding (Fig. siso): inputs L_Ch and L_A (NULL = zeros), outputs
 * L_APP, L_E, hard decision, P(not in list), query count, the list, and
 * diagnostics diag[10] = {c, C*, index in level, log R, log R (paper-literal
 * difference), S, log phi, exhausted, parity, thr-stop}.
 * Returns 0, or -1 for a non-finite input (outputs then: L_APP = lambda,
 * L_E = 0, queries = -1).
 */
int oracle_siso(const oracle_code *code, const float *lch, const float *la, int L, int64_t cap, double thr,
                double *lapp, double *lext, uint8_t *hard, double *pmiss, int64_t *queries, int32_t *list_count,
                uint8_t *list_words, double *list_logp, double *list_app, int64_t *list_q, double *diag)
{
    int n = code->n, k = code->k;
    if (n < 2 || n > OR_NMAX || k < 1 || k >= n || L < 1 || L > OR_LMAX || cap < 1) return -2;
    siso_ctx *s = (siso_ctx *)calloc(1, sizeof(siso_ctx));
    float lam[OR_NMAX];
    int finite = 1;
    for (int i = 0; i < n; i++) {
        float a = la ? la[i] : 0.0f;
        lam[i] = lch[i] + a; /* one FP32 rounding; built with -ffp-contract=off */
        if (!isfinite(lam[i])) finite = 0;
    }
    if (!finite) {
        for (int i = 0; i < n; i++) {
            lapp[i] = lam[i];
            lext[i] = 0;
            hard[i] = lam[i] < 0;
        }
        *pmiss = 1;
        *queries = -1;
        if (list_count) *list_count = 0;
        free(s);
        return -1;
    }
    s->hit_word = (uint8_t *)malloc((size_t)L * n);
    s->hit_logp = (double *)malloc(sizeof(double) * (size_t)L);
    s->hit_q = (int64_t *)malloc(sizeof(int64_t) * (size_t)L);
    s->code = code;
    s->n = n;
    s->L = L;
    s->cap = cap;
    s->thr = thr;
    int par = 0;
    for (int i = 0; i < n; i++) {
        s->y[i] = lam[i] < 0.0f; /* lambda = 0 -> bit 0 */
        par ^= s->y[i];
    }
    sort_item it[OR_NMAX];
    for (int i = 0; i < n; i++) {
        it[i].idx = i;
        it[i].key = fabsf(lam[i]);
    }
    qsort(it, (size_t)n, sizeof(sort_item), cmp_rank);
    float absf[OR_NMAX];
    for (int r = 0; r < n; r++) {
        s->perm[r] = it[r].idx;
        absf[r] = it[r].key;
        s->absl[r] = (double)it[r].key;
    }
    s->c = oracle_one_line_c(n, absf, code->c_max);
    s->cls = code->even ? par : -1;
    if (code->even && code->reading != 1) s->logphi = log_pow2m1(k) - log_pow2m1(n - 1);
    else s->logphi = log_pow2m1(k) - log_pow2m1(n);
    s->cur_C = -1;
    int stopped = gen_all(n, s->c, s->cls, siso_emit, s);
    int exhausted = !stopped;

    double logR;
    if (exhausted) {
        if (s->cls >= 0 && code->reading == 1) {
            double tail[2], head[2];
            tail_dp(n, s->c, s->absl, 0, tail, head);
            logR = logadd(tail[s->cls ^ 1], head[s->cls ^ 1]);
        } else logR = -INFINITY;
    } else logR = remaining_log(s, s->cur_C, s->cur_idx);
    if (code->reading == 2) logR = -INFINITY; /* Forney: nothing outside the list */

    /* paper-literal remaining mass: (class total) - S, FP64 */
    double tp = 1, tm = 1;
    for (int r = 0; r < n; r++) {
        double t = exp(-s->absl[r]);
        tp *= 1 + t;
        tm *= 1 - t;
    }
    double total;
    if (s->cls < 0 || code->reading == 1) total = tp;
    else total = s->cls == 0 ? 0.5 * (tp + tm) : 0.5 * (tp - tm);
    double direct = total - s->S;

    double M = logR + s->logphi;
    int nh = s->nhit;
    if (nh == 0) {
        for (int i = 0; i < n; i++) {
            lapp[i] = lam[i];
            lext[i] = 0;
            hard[i] = s->y[i];
        }
        *pmiss = 1;
    } else {
        for (int i = 0; i < n; i++) {
            double l = (double)lam[i];
            double a0 = M + log_sigmoid(l), a1 = M + log_sigmoid(-l);
            for (int h = 0; h < nh; h++) {
                if (s->hit_word[(size_t)h * n + i]) a1 = logadd(a1, s->hit_logp[h]);
                else a0 = logadd(a0, s->hit_logp[h]);
            }
            lapp[i] = a0 - a1;
            lext[i] = lapp[i] - l;
            hard[i] = lapp[i] < 0;
        }
        *pmiss = pmiss_of(s->hit_logp, nh, M);
    }
    *queries = s->q;
    if (list_count) *list_count = nh;
    double D = M;
    for (int h = 0; h < nh; h++) D = logadd(D, s->hit_logp[h]);
    for (int h = 0; h < nh; h++) {
        if (list_words) memcpy(list_words + (size_t)h * n, s->hit_word + (size_t)h * n, (size_t)n);
        if (list_logp) list_logp[h] = s->hit_logp[h];
        if (list_app) list_app[h] = exp(s->hit_logp[h] - D);
        if (list_q) list_q[h] = s->hit_q[h];
    }
    if (diag) {
        diag[0] = s->c;
        diag[1] = (double)s->cur_C;
        diag[2] = (double)s->cur_idx;
        diag[3] = logR;
        diag[4] = direct > 0 ? log(direct) : -INFINITY;
        diag[5] = s->S;
        diag[6] = s->logphi;
        diag[7] = exhausted;
        diag[8] = par;
        diag[9] = s->stop_thr;
    }
    free(s->hit_word);
    free(s->hit_logp);
    free(s->hit_q);
    free(s);
    return 0;
}

/* ------------------------------------------------------------------ */
/* product codes: block turbo decoding (Sec. VI, Fig. turboDec)         */
/* ------------------------------------------------------------------ */
/* Position of bit i of word w of the second set of checks: column w of the
   n_col x n_row frame (product code), or wrapped diagonal w of the n x n
   array (QC-GLDPC: bit i is X[(w + i) mod n][i]). */
static size_t second_pos(int diag, int nr, int w, int i)
{
    return diag ? (size_t)((w + i) % nr) * nr + i : (size_t)i * nr + w;
}

/* every row of the frame is a row-code word and every word of the second set
   (columns, or wrapped diagonals) a column-code word */
static int frame_valid(const oracle_code *row, const oracle_code *col, int diag, const uint8_t *B, uint8_t *tmp)
{
    int nr = row->n, nc = col->n;
    for (int i = 0; i < nc; i++)
        if (!is_codeword(row, B + (size_t)i * nr)) return 0;
    for (int w = 0; w < nr; w++) {
        for (int i = 0; i < nc; i++) tmp[i] = B[second_pos(diag, nr, w, i)];
        if (!is_codeword(col, tmp)) return 0;
    }
    return 1;
}

/*
 * Decode one n x n frame (row-major L_Ch).  L_A starts at 0; each half
 * iteration decodes every row (odd halves) or column (even halves) with the
 * SISO above, stores L_E (as FP32, the state's precision), takes the hard
 * decision of L_APP and stops when every row and column is a codeword;
 * otherwise the next half uses L_A = fl32(alpha * L_E).
 * Outputs: bits (n*n, the last hard decision), half iterations run,
 * status (0 decoded, 1 max iterations, 2 invalid input), total queries and
 * the "parallelized" count (sum over halves of the max per-word queries).
 */
static int product_core(const oracle_code *row, const oracle_code *col, int diag, const float *lch, int L,
                        int64_t cap, double thr, float alpha, int max_iter, uint8_t *bits, int32_t *half_iters,
                        uint8_t *status, int64_t *queries, int64_t *par_queries, double *lapp_trace)
{
    int nr = row->n, nc = col->n;
    size_t nn = (size_t)nr * nc;
    float *LE = (float *)calloc(nn, sizeof(float));
    uint8_t *B = (uint8_t *)calloc(nn, 1);
    float wl[OR_NMAX], wa[OR_NMAX];
    double lapp[OR_NMAX], lext[OR_NMAX], pm;
    uint8_t hd[OR_NMAX], tmp[OR_NMAX];
    int64_t qsum = 0, qpar = 0, q;
    int st = 1, h;
    for (h = 1; h <= 2 * max_iter; h++) {
        int rows = h & 1;
        /* a row half decodes the n_col rows (row code, n_row bits each); a
           column half the n_row columns (column code, n_col bits each) */
        const oracle_code *code = rows ? row : col;
        int nw = rows ? nc : nr, len = code->n;
        int64_t qmax = 0;
        for (int w = 0; w < nw; w++) {
            for (int i = 0; i < len; i++) {
                size_t pos = rows ? (size_t)w * nr + i : second_pos(diag, nr, w, i);
                wl[i] = lch[pos];
                wa[i] = alpha * LE[pos]; /* FP32 product, no contraction */
            }
            int rc = oracle_siso(code, wl, wa, L, cap, thr, lapp, lext, hd, &pm, &q, NULL, NULL, NULL, NULL, NULL,
                                 NULL);
            if (rc != 0) {
                st = 2;
                goto done;
            }
            qsum += q;
            if (q > qmax) qmax = q;
            for (int i = 0; i < len; i++) {
                size_t pos = rows ? (size_t)w * nr + i : second_pos(diag, nr, w, i);
                LE[pos] = (float)lext[i];
                B[pos] = hd[i];
                if (lapp_trace) lapp_trace[(size_t)(h - 1) * nn + pos] = lapp[i];
            }
        }
        qpar += qmax;
        if (frame_valid(row, col, diag, B, tmp)) {
            st = 0;
            break;
        }
    }
done:
    if (h > 2 * max_iter) h = 2 * max_iter;
    memcpy(bits, B, nn);
    *half_iters = h;
    *status = (uint8_t)st;
    *queries = qsum;
    *par_queries = qpar;
    free(LE);
    free(B);
    return 0;
}

/* product of a row code and a column code (an n_col x n_row frame) */
int oracle_product2(const oracle_code *row, const oracle_code *col, const float *lch, int L, int64_t cap,
                    double thr, float alpha, int max_iter, uint8_t *bits, int32_t *half_iters, uint8_t *status,
                    int64_t *queries, int64_t *par_queries)
{
    return product_core(row, col, 0, lch, L, cap, thr, alpha, max_iter, bits, half_iters, status, queries,
                        par_queries, NULL);
}

/* QC-GLDPC of a component code (Sec. VI): rows and wrapped diagonals of an
   n x n array, decoded alternately like the rows and columns of a product
   code, the iteration stopping once every row and diagonal is a codeword */
int oracle_gldpc(const oracle_code *code, const float *lch, int L, int64_t cap, double thr, float alpha,
                 int max_iter, uint8_t *bits, int32_t *half_iters, uint8_t *status, int64_t *queries,
                 int64_t *par_queries)
{
    return product_core(code, code, 1, lch, L, cap, thr, alpha, max_iter, bits, half_iters, status, queries,
                        par_queries, NULL);
}

/* square product code: the same code on rows and columns */
int oracle_product(const oracle_code *code, const float *lch, int L, int64_t cap, double thr, float alpha,
                   int max_iter, uint8_t *bits, int32_t *half_iters, uint8_t *status, int64_t *queries,
                   int64_t *par_queries)
{
    return oracle_product2(code, code, lch, L, cap, thr, alpha, max_iter, bits, half_iters, status, queries,
                           par_queries);
}

/* The product decoder above with the L_APP of every half iteration recorded:
   lapp_trace [2 * max_iter][n_col * n_row], row-major positions, entry h - 1
   holding half h's L_APP (halves the frame did not run are left untouched).
   For pinning the extrinsic exchange between halves. */
int oracle_product_trace(const oracle_code *row, const oracle_code *col, const float *lch, int L, int64_t cap,
                         double thr, float alpha, int max_iter, uint8_t *bits, int32_t *half_iters, uint8_t *status,
                         int64_t *queries, int64_t *par_queries, double *lapp_trace)
{
    return product_core(row, col, 0, lch, L, cap, thr, alpha, max_iter, bits, half_iters, status, queries,
                        par_queries, lapp_trace);
}
