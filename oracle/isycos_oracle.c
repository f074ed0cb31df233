/*
 * isycos_oracle.c -- TEST INFRASTRUCTURE, not part of the product.
 *
 * A plain, slow, single-threaded CPU oracle for the computations of iSYCOS
 * (Ho et al., "A Unified Approach for Multi-Scale Synchronous Correlation Search
 * in Big Time Series", arXiv 2204.09131):
 *
 *   - the window-level KSG mutual information (Sec. 4.2, Eq. KSGmi; Def. 4.2),
 *     with the counting rule of the box-assisted example in Sec. 7.1;
 *   - the normalised score I_w / H_w of Sec. 5.4 (Eq. normalizedMI);
 *   - SYCOS_TD (Sec. 5.1, Algorithm 1) and SYCOS_BU (Sec. 5.2, Algorithm 2) with the
 *     MI-based noise pruning of Sec. 6 (Def. 6.2; Secs. 6.2 and 6.3);
 *   - the iSYCOS selection between them (Sec. 5.3, Algorithm 3) and the chunked search
 *     of the distributed iSYCOS (Sec. 7.3, Algorithm 4).
 *
 * Only the tests, __graft_entry__.smoke() and bench.py's cpu_baseline / reference
 * leg may load or call this file.  It shares no code, header, table or constant
 * generator with the CUDA library: both sides implement the same published
 * definitions independently, and the tests compare them.
 *
 * Arithmetic contract (where the paper is silent; every reading is listed in the
 * design notes of the repository):
 *   - distances are computed in IEEE binary32 exactly as fabsf(a - b) and
 *     fmaxf(|dx|, |dy|) (max-norm, footnote of Sec. 7.1); all decisions that turn
 *     floats into integers (neighbour sets, marginal counts) are taken in binary32;
 *   - the k nearest neighbours of point i are the first k points j != i in the
 *     lexicographic order of (d_ij, j), j the time index inside the window;
 *   - marginal counts are inclusive (<=) and exclude the point itself
 *     (Sec. 7.1: p1 counts p2, p3, p5 but not itself);
 *   - Kraskov's second estimator: per-dimension distances d_x, d_y taken over
 *     the k-neighbour set, psi(n_x) and psi(n_y) without +1, the -1/k term (Eq. KSGmi);
 *   - psi(n) for integer n is -gamma + sum_{t=1}^{n-1} 1/t, evaluated by the forward
 *     recurrence psi(n+1) = psi(n) + 1/n in binary64;
 *   - the canonical score sums use 2^-32 fixed-point images of psi(n) and ln(n) held in
 *     int64, so that the sums are exact and independent of summation order; the
 *     oracle also reports the plain binary64 evaluation of Eq. KSGmi ("exact").
 *
 * Pins: the estimator against the Sec. 7.1 example, hand-worked windows, independent
 * brute forces and closed forms; the searches against hand-traced score tables (layers,
 * partitions, noise skips, rings, acceptance, ties, restarts, one-sided pruning, the
 * late-acceptance history, the chunks of Algorithm 4, the pair-count runtime of
 * Algorithm 3).  Parity unpinned: which partitions Algorithm 3 samples when it samples
 * fewer than all of them (a seeded choice the paper leaves open).
 *
 * Build: gcc -O2 -fno-fast-math -ffp-contract=off -shared -fPIC (no flush-to-zero).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_ENOMEM (-2)
#define ORC_ETRUNC (-5)

/* Euler-Mascheroni constant, psi(1) = -gamma. */
static const double ORC_EULER_GAMMA = 0.57721566490153286060651209008240243;

/* ------------------------------------------------------------------------- */
/* Planted mistakes.  A test switches one of these on to show that the pins   */
/* catch it; every public result is computed with mutation 0 otherwise.       */
/* ------------------------------------------------------------------------- */
enum {
    ORC_MUT_NONE = 0,
    ORC_MUT_DROP_INV_K = 1,      /* drop the -1/k term of Eq. KSGmi                */
    ORC_MUT_STRICT_COUNT = 2,    /* count |x_i - x_j| <  d_x instead of <=         */
    ORC_MUT_COUNT_SELF = 3,      /* let n_x, n_y include the point itself          */
    ORC_MUT_PSI_PLUS_ONE = 4,    /* use psi(n_x + 1) (Kraskov's first estimator)   */
    ORC_MUT_SWAP_NY = 5,         /* count n_y with the x distance                  */
    ORC_MUT_TIE_LATE = 6,        /* break distance ties toward the larger index    */
    ORC_MUT_EUCLID = 7,          /* Euclidean instead of max-norm distance         */
    ORC_MUT_H_SIGN = 8,          /* keep the garbled sign of the entropy formula   */
    ORC_MUT_PSI_M_MINUS = 9,     /* use psi(m - 1) in place of psi(m)              */
    /* the searches' readings */
    ORC_MUT_ACCEPT_GE = 10,      /* Alg. 2 acceptance with >= instead of >         */
    ORC_MUT_TIE_LAST = 11,       /* the last maximum of a ring wins                */
    ORC_MUT_TD_NO_CLAMP = 12,    /* reduce(s_w) = s_w / 2 without the s_min floor  */
    ORC_MUT_TD_DELTA_OVERLAP = 13, /* w_delta = [t_e0, t_e1], one point in w_o too */
    ORC_MUT_NOISE_NO_IO = 14,    /* Def. 6.2 without its I_w > 0 condition         */
    ORC_MUT_BU_SQUARE = 15,      /* evaluate the whole square, not the ring N_r    */
    ORC_MUT_BU_DROP_BOTH = 16,   /* a noisy side drops both sides' neighbours      */
    ORC_MUT_NO_HISTORY = 17,     /* plain hill climbing: accept only if > I_w      */
    ORC_MUT_CHUNK_NO_OVERLAP = 18, /* Alg. 4 chunks [i, i + L) without the s_max lead */
    ORC_MUT_RUNTIME_WINDOWS = 19, /* Alg. 3 runtime = windows scored, not pairs    */
    ORC_MUT_TINY_TEST = 20,      /* noise test on windows of fewer than k+1 points */
    ORC_MUT_RUN_NO_RESET = 21,   /* TD: a window that is not noise keeps the count */
    ORC_MUT_BU_RUN_NO_RESET = 22, /* BU: a step that is not noise keeps the count  */
    ORC_MUT_TD_TAIL = 23,        /* TD: also score (and keep, if correlated) a window
                                    ending at the partition end                     */
    ORC_MUT_SAMPLE_DRAW = 24     /* Alg. 3: sampling draws outputs 0 .. m-1 of the
                                    stream instead of 1 .. m                        */
};
static int g_mutation = ORC_MUT_NONE;

void orc_set_mutation(int32_t mutation) { g_mutation = mutation; }
int32_t orc_get_mutation(void) { return g_mutation; }

/* ------------------------------------------------------------------------- */
/* Digamma and logarithm tables                                              */
/* ------------------------------------------------------------------------- */

/* psi[n] for n = 1 .. n_max (psi[0] = NaN), by the forward recurrence. */
int orc_digamma_table(int32_t n_max, double *psi)
{
    if (n_max < 1 || psi == NULL) return ORC_EINVAL;
    psi[0] = NAN;
    psi[1] = -ORC_EULER_GAMMA;
    for (int32_t n = 1; n < n_max; ++n) psi[n + 1] = psi[n] + 1.0 / (double)n;
    return ORC_OK;
}

/* 2^-32 fixed-point images: psi_fx[n] = round(psi(n) 2^32), log_fx[n] = round(ln(n) 2^32),
 * for n = 1 .. n_max; entry 0 is 0. */
int orc_fixed_tables(int32_t n_max, int64_t *psi_fx, int64_t *log_fx)
{
    if (n_max < 1) return ORC_EINVAL;
    double *psi = (double *)malloc(sizeof(double) * ((size_t)n_max + 1));
    if (!psi) return ORC_ENOMEM;
    orc_digamma_table(n_max, psi);
    if (psi_fx) psi_fx[0] = 0;
    if (log_fx) log_fx[0] = 0;
    for (int32_t n = 1; n <= n_max; ++n) {
        if (psi_fx) psi_fx[n] = llround(ldexp(psi[n], 32));
        if (log_fx) log_fx[n] = llround(ldexp(log((double)n), 32));
    }
    free(psi);
    return ORC_OK;
}

/* Lazily built tables shared by the functions below (single-threaded oracle). */
#define ORC_TABLE_MAX 65537
static double *g_psi = NULL;
static int64_t *g_psi_fx = NULL;
static int64_t *g_log_fx = NULL;

static int orc_tables_ready(void)
{
    if (g_psi) return 1;
    double *psi = (double *)malloc(sizeof(double) * (ORC_TABLE_MAX + 1));
    int64_t *pf = (int64_t *)malloc(sizeof(int64_t) * (ORC_TABLE_MAX + 1));
    int64_t *lf = (int64_t *)malloc(sizeof(int64_t) * (ORC_TABLE_MAX + 1));
    if (!psi || !pf || !lf) { free(psi); free(pf); free(lf); return 0; }
    orc_digamma_table(ORC_TABLE_MAX, psi);
    orc_fixed_tables(ORC_TABLE_MAX, pf, lf);
    g_psi = psi; g_psi_fx = pf; g_log_fx = lf;
    return 1;
}

/* ------------------------------------------------------------------------- */
/* KSG estimator on one window (Sec. 4.2, Eq. KSGmi; Sec. 7.1 example)       */
/* ------------------------------------------------------------------------- */

typedef struct {
    double mi;        /* canonical Eq. KSGmi (fixed-point sums, fixed evaluation order) */
    double h_w;       /* canonical plug-in joint entropy of the window (Sec. 5.4)       */
    double nmi;       /* mi / h_w, 0 when h_w == 0                                     */
    int64_t s_psi;    /* sum_i psi_fx[n_x,i] + psi_fx[n_y,i]                            */
    int64_t s_log;    /* sum_i log_fx[c_i]                                              */
    double mi_exact;  /* Eq. KSGmi evaluated directly in binary64                        */
    double h_exact;   /* ln m - (1/m) sum_i ln c_i evaluated directly in binary64        */
} orc_mi;

static float orc_dist(float xi, float yi, float xj, float yj)
{
    float ax = fabsf(xi - xj);
    float ay = fabsf(yi - yj);
    if (g_mutation == ORC_MUT_EUCLID) return sqrtf(ax * ax + ay * ay);
    return fmaxf(ax, ay);
}

/* (d1, j1) precedes (d2, j2) in the neighbour order. */
static int orc_before(float d1, int64_t j1, float d2, int64_t j2)
{
    if (d1 < d2) return 1;
    if (d1 > d2) return 0;
    if (g_mutation == ORC_MUT_TIE_LATE) return j1 > j2;
    return j1 < j2;
}

/* Counts for one point i of the window {(x_j, y_j)}, j = 0 .. m-1.
 * Estimator 0 (Kraskov's second, Eq. KSGmi): nx, ny = marginal counts (j != i, inclusive)
 * within the per-dimension neighbour distances dxm, dym.
 * Estimator 1 (Kraskov's first): nx, ny = #{j != i : |x_i - x_j| < eps} (strict), the
 * marginal strips both of half-width eps (reported in dxm, dym).
 * c: multiplicity of (x_i, y_i) (includes i); eps: k-th neighbour distance. */
int orc_ksg_point_est(const float *x, const float *y, int64_t m, int32_t k, int32_t est,
                      int64_t i, int32_t *nx, int32_t *ny, int32_t *c, float *eps, float *dxm,
                      float *dym)
{
    if (k < 1 || m < (int64_t)k + 1 || i < 0 || i >= m || (est != 0 && est != 1)) return ORC_EINVAL;
    float *bd = (float *)malloc(sizeof(float) * (size_t)k);
    int64_t *bj = (int64_t *)malloc(sizeof(int64_t) * (size_t)k);
    if (!bd || !bj) { free(bd); free(bj); return ORC_ENOMEM; }

    /* k nearest neighbours: keep the first k of (d_ij, j), j != i, by insertion. */
    int32_t filled = 0;
    for (int64_t j = 0; j < m; ++j) {
        if (j == i) continue;
        float d = orc_dist(x[i], y[i], x[j], y[j]);
        if (filled == k && !orc_before(d, j, bd[k - 1], bj[k - 1])) continue;
        int32_t pos = (filled < k) ? filled++ : k - 1;
        while (pos > 0 && orc_before(d, j, bd[pos - 1], bj[pos - 1])) {
            bd[pos] = bd[pos - 1];
            bj[pos] = bj[pos - 1];
            --pos;
        }
        bd[pos] = d;
        bj[pos] = j;
    }

    /* Per-dimension distances to the k neighbours (Sec. 7.1: "dx and dy"). */
    float dx = 0.0f, dy = 0.0f;
    for (int32_t r = 0; r < k; ++r) {
        float ax = fabsf(x[i] - x[bj[r]]);
        float ay = fabsf(y[i] - y[bj[r]]);
        if (ax > dx) dx = ax;
        if (ay > dy) dy = ay;
    }

    /* Marginal counts: points inside the marginal strips (inclusive), self excluded. */
    int32_t cx = 0, cy = 0, cc = 0;
    if (est == 1) {
        /* Kraskov's first estimator: strips of half-width eps = d to the k-th neighbour,
         * points strictly inside counted. */
        float e = bd[k - 1];
        for (int64_t j = 0; j < m; ++j) {
            if (x[j] == x[i] && y[j] == y[i]) ++cc;
            if (j == i) continue;
            if (fabsf(x[i] - x[j]) < e) ++cx;
            if (fabsf(y[i] - y[j]) < e) ++cy;
        }
        dx = e;
        dy = e;
    }
    for (int64_t j = 0; j < m && est == 0; ++j) {
        float ax = fabsf(x[i] - x[j]);
        float ay = fabsf(y[i] - y[j]);
        if (g_mutation == ORC_MUT_SWAP_NY) ay = ax;
        int self = (j == i);
        if (x[j] == x[i] && y[j] == y[i]) ++cc;
        if (self && g_mutation != ORC_MUT_COUNT_SELF) continue;
        if (g_mutation == ORC_MUT_STRICT_COUNT) {
            if (ax < dx) ++cx;
            if (ay < dy) ++cy;
        } else {
            if (ax <= dx) ++cx;
            if (ay <= dy) ++cy;
        }
    }
    if (nx) *nx = cx;
    if (ny) *ny = cy;
    if (c) *c = cc;
    if (eps) *eps = bd[k - 1];
    if (dxm) *dxm = dx;
    if (dym) *dym = dy;
    free(bd);
    free(bj);
    return ORC_OK;
}

int orc_ksg_point(const float *x, const float *y, int64_t m, int32_t k, int64_t i,
                  int32_t *nx, int32_t *ny, int32_t *c, float *eps, float *dxm, float *dym)
{
    return orc_ksg_point_est(x, y, m, k, 0, i, nx, ny, c, eps, dxm, dym);
}

/* MI of the window {(x_j, y_j)}, j = 0 .. m-1.  Estimator 0 is Eq. KSGmi (Kraskov's second
 * estimator); estimator 1 is Kraskov's first, psi(k) + psi(m) - <psi(n_x + 1) + psi(n_y + 1)>.
 * Per-point arrays may be NULL. */
int orc_ksg_window_est(const float *x, const float *y, int64_t m, int32_t k, int32_t est,
                       int32_t *nx, int32_t *ny, int32_t *c, float *eps, float *dxm, float *dym,
                       orc_mi *out)
{
    if (k < 1 || m < (int64_t)k + 1 || m > ORC_TABLE_MAX - 1 || out == NULL) return ORC_EINVAL;
    if (est != 0 && est != 1) return ORC_EINVAL;
    if (!orc_tables_ready()) return ORC_ENOMEM;
    int64_t s_psi = 0, s_log = 0;
    double sum_psi = 0.0, sum_log = 0.0;
    for (int64_t i = 0; i < m; ++i) {
        int32_t a, b, cc;
        float e, u, v;
        int rc = orc_ksg_point_est(x, y, m, k, est, i, &a, &b, &cc, &e, &u, &v);
        if (rc != ORC_OK) return rc;
        if (nx) nx[i] = a;
        if (ny) ny[i] = b;
        if (c) c[i] = cc;
        if (eps) eps[i] = e;
        if (dxm) dxm[i] = u;
        if (dym) dym[i] = v;
        int32_t ia = a, ib = b;
        if (est == 1 || g_mutation == ORC_MUT_PSI_PLUS_ONE) { ia += 1; ib += 1; }
        s_psi += g_psi_fx[ia] + g_psi_fx[ib];
        s_log += g_log_fx[cc];
        sum_psi += g_psi[ia] + g_psi[ib];
        sum_log += log((double)cc);
    }
    double inv_k = (est == 1 || g_mutation == ORC_MUT_DROP_INV_K) ? 0.0 : 1.0 / (double)k;
    int64_t mm = (g_mutation == ORC_MUT_PSI_M_MINUS) ? m - 1 : m;
    double md = (double)m;

    /* Canonical evaluation order: ((psi(k) - 1/k) + psi(m)) - S_psi / m (estimator 1: the
     * same with 1/k = 0, which leaves psi(k) unchanged). */
    double psi_k = ldexp((double)g_psi_fx[k], -32);
    double psi_m = ldexp((double)g_psi_fx[mm], -32);
    double mean_psi = ldexp((double)s_psi, -32) / md;
    out->mi = ((psi_k - inv_k) + psi_m) - mean_psi;
    double ln_m = ldexp((double)g_log_fx[m], -32);
    out->h_w = ln_m - ldexp((double)s_log, -32) / md;
    if (g_mutation == ORC_MUT_H_SIGN) out->h_w = -out->h_w;
    out->nmi = (out->h_w > 0.0) ? out->mi / out->h_w : 0.0;
    out->s_psi = s_psi;
    out->s_log = s_log;

    /* Direct binary64 form of Eq. KSGmi: psi(k) - 1/k - <psi(n_x) + psi(n_y)> + psi(n). */
    out->mi_exact = g_psi[k] - inv_k - sum_psi / md + g_psi[mm];
    out->h_exact = log(md) - sum_log / md;
    if (g_mutation == ORC_MUT_H_SIGN) out->h_exact = -out->h_exact;
    return ORC_OK;
}

int orc_ksg_window(const float *x, const float *y, int64_t m, int32_t k,
                   int32_t *nx, int32_t *ny, int32_t *c, float *eps, float *dxm, float *dym,
                   orc_mi *out)
{
    return orc_ksg_window_est(x, y, m, k, 0, nx, ny, c, eps, dxm, dym, out);
}

/* ------------------------------------------------------------------------- */
/* Searches (Sec. 5.1 Algorithm 1, Sec. 5.2 Algorithm 2, Sec. 6 pruning)     */
/* ------------------------------------------------------------------------- */

typedef struct {
    int32_t k;           /* KSG neighbours                                            */
    int32_t score_kind;  /* 0: normalised I/H (Sec. 5.4), 1: raw I in nats           */
    double sigma;        /* correlation threshold (Def. 3.5)                          */
    double tau;          /* noise threshold (Def. 6.2)                                */
    int32_t s_min, s_max;
    int32_t delta_td;    /* <= 0: max(k + 1, s_w / 4) per layer                       */
    int32_t delta_bu;    /* <= 0: max(1, s_min / 4)                                   */
    int32_t h;           /* LAHC history length, <= 0: 8                              */
    int32_t t_max_idle;  /* < 0: 3                                                    */
    int32_t p;           /* consecutive noise detections before pruning, <= 0: 3      */
    int32_t pruning;     /* 0 off, 1 on                                               */
    int32_t max_steps;   /* LAHC step cap per climb, <= 0: 10000                      */
    int32_t chunks;      /* Algorithm 4: number of overlapping chunks n_p, <= 1: none   */
    uint64_t seed;
} orc_params;

typedef struct { int64_t t_s, t_e; double score, mi; } orc_window;

/* Score callback: fills *score (the value compared with sigma and tau) and *mi (raw I). */
typedef int (*orc_score_fn)(void *user, int64_t t_s, int64_t t_e, double *score, double *mi);

/* Default scorer over a resident pair of series. */
typedef struct {
    const float *x;
    const float *y;
    int64_t n;
    int32_t k;
    int32_t score_kind;
    int64_t evals;
    int32_t estimator;   /* 0: Kraskov 2 (Eq. KSGmi), 1: Kraskov 1 */
    int32_t pad;
} orc_series_scorer;

int orc_series_score(void *user, int64_t t_s, int64_t t_e, double *score, double *mi)
{
    orc_series_scorer *s = (orc_series_scorer *)user;
    if (t_s < 0 || t_e >= s->n || t_e < t_s) return ORC_EINVAL;
    orc_mi r;
    int rc = orc_ksg_window_est(s->x + t_s, s->y + t_s, t_e - t_s + 1, s->k, s->estimator,
                                NULL, NULL, NULL, NULL, NULL, NULL, &r);
    if (rc != ORC_OK) return rc;
    s->evals++;
    *mi = r.mi;
    *score = (s->score_kind == 1) ? r.mi : r.nmi;
    return ORC_OK;
}

/* Address of orc_series_score, for callers that pass it back as a function pointer. */
void *orc_series_score_addr(void) { return (void *)&orc_series_score; }

typedef struct {
    orc_window *v;
    int64_t n, cap;
} orc_wlist;

static int orc_push(orc_wlist *l, int64_t ts, int64_t te, double score, double mi)
{
    if (l->n == l->cap) {
        int64_t nc = l->cap ? 2 * l->cap : 64;
        orc_window *nv = (orc_window *)realloc(l->v, sizeof(orc_window) * (size_t)nc);
        if (!nv) return ORC_ENOMEM;
        l->v = nv;
        l->cap = nc;
    }
    l->v[l->n].t_s = ts;
    l->v[l->n].t_e = te;
    l->v[l->n].score = score;
    l->v[l->n].mi = mi;
    l->n++;
    return ORC_OK;
}

static int orc_cmp_window(const void *a, const void *b)
{
    const orc_window *u = (const orc_window *)a, *v = (const orc_window *)b;
    return (u->t_s > v->t_s) - (u->t_s < v->t_s);
}

static int orc_emit(orc_wlist *l, orc_window *out, int64_t cap, int64_t *n_out)
{
    qsort(l->v, (size_t)l->n, sizeof(orc_window), orc_cmp_window);
    if (n_out) *n_out = l->n;
    if (l->n > cap) return ORC_ETRUNC;
    if (l->n) memcpy(out, l->v, sizeof(orc_window) * (size_t)l->n);
    return ORC_OK;
}

static int orc_check_params(const orc_params *p, int64_t t_begin, int64_t t_end)
{
    if (!p || p->k < 1 || p->s_min < p->k + 1 || p->s_max < p->s_min) return ORC_EINVAL;
    if (t_begin < 0 || t_end < t_begin) return ORC_EINVAL;
    return ORC_OK;
}

/* Sec. 5.1, Algorithm 1 with the TD noise pruning of Sec. 6.2.
 * The searched range is [t_begin, t_end) (t_end exclusive); windows are inclusive [t_s, t_e]. */
int orc_search_td(orc_score_fn f, void *user, int64_t t_begin, int64_t t_end,
                  const orc_params *p, orc_window *out, int64_t cap, int64_t *n_out,
                  int64_t *n_evals)
{
    int rc = orc_check_params(p, t_begin, t_end);
    if (rc) return rc;
    int pcount = p->p > 0 ? p->p : 3;
    orc_wlist S = {0, 0, 0};
    int64_t evals = 0;
    int64_t s_w = p->s_max;
    for (;;) {
        /* Uncorrelated partitions: maximal ranges of [t_begin, t_end) not covered by S. */
        qsort(S.v, (size_t)S.n, sizeof(orc_window), orc_cmp_window);
        int64_t n_part = 0;
        int64_t *pa = (int64_t *)malloc(sizeof(int64_t) * (size_t)(S.n + 1));
        int64_t *pb = (int64_t *)malloc(sizeof(int64_t) * (size_t)(S.n + 1));
        if (!pa || !pb) { free(pa); free(pb); free(S.v); return ORC_ENOMEM; }
        int64_t cur = t_begin;
        for (int64_t q = 0; q < S.n; ++q) {
            if (S.v[q].t_s > cur) { pa[n_part] = cur; pb[n_part] = S.v[q].t_s - 1; ++n_part; }
            cur = S.v[q].t_e + 1;
        }
        if (cur <= t_end - 1) { pa[n_part] = cur; pb[n_part] = t_end - 1; ++n_part; }

        int64_t delta = p->delta_td > 0 ? p->delta_td : s_w / 4;
        if (p->delta_td <= 0 && delta < p->k + 1) delta = p->k + 1;

        for (int64_t q = 0; q < n_part && rc == ORC_OK; ++q) {
            int64_t a = pa[q], b = pb[q];
            int64_t t = a;
            int shifted = 0;     /* the current window is the previous one moved by delta */
            int noise_run = 0;
            int64_t last_start = a - 1;    /* start of the last window scored (for a mutation) */
            while (t + s_w - 1 <= b) {
                double sc, mi;
                rc = f(user, t, t + s_w - 1, &sc, &mi);
                if (rc) break;
                ++evals;
                last_start = t;
                if (sc >= p->sigma) {
                    rc = orc_push(&S, t, t + s_w - 1, sc, mi);
                    if (rc) break;
                    t = t + s_w;               /* next window starts at t_e + 1 */
                    shifted = 0;
                    noise_run = 0;
                    continue;
                }
                int noise = 0;
                if (p->pruning && shifted) {
                    /* w = w_o (overlap with the previous window) followed by w_delta (new data). */
                    int64_t o_s = t, o_e = t + s_w - delta - 1;
                    int64_t d_s = t + s_w - delta, d_e = t + s_w - 1;
                    if (g_mutation == ORC_MUT_TD_DELTA_OVERLAP) d_s -= 1;
                    if ((o_e - o_s + 1 >= p->k + 1 && d_e - d_s + 1 >= p->k + 1) || g_mutation == ORC_MUT_TINY_TEST) {
                        double so, mo, sd, md;
                        rc = f(user, o_s, o_e, &so, &mo);
                        if (rc) break;
                        rc = f(user, d_s, d_e, &sd, &md);
                        if (rc) break;
                        evals += 2;
                        /* Def. 6.2 with w = w_o, w' = w_delta, w'' = w: requires I_{w_o} > 0. */
                        noise = (so > 0.0 || g_mutation == ORC_MUT_NOISE_NO_IO) && (sd < p->tau) && (sc < so);
                    }
                }
                noise_run = noise ? noise_run + 1 : (g_mutation == ORC_MUT_RUN_NO_RESET ? noise_run : 0);
                if (noise_run >= pcount) {
                    t = t + s_w;               /* skip the rest of the shifting (Sec. 6.2) */
                    noise_run = 0;
                    shifted = 0;
                } else {
                    t = t + delta;
                    shifted = 1;
                }
            }
            if (g_mutation == ORC_MUT_TD_TAIL && rc == ORC_OK && b - s_w + 1 >= a &&
                b - s_w + 1 > last_start) {
                double sc, mi;
                rc = f(user, b - s_w + 1, b, &sc, &mi);
                if (rc == ORC_OK) ++evals;
                if (rc == ORC_OK && sc >= p->sigma) rc = orc_push(&S, b - s_w + 1, b, sc, mi);
            }
        }
        free(pa);
        free(pb);
        if (rc) { free(S.v); return rc; }
        if (s_w <= p->s_min) break;
        s_w = s_w / 2;                         /* reduce(s_w) */
        if (s_w < p->s_min && g_mutation != ORC_MUT_TD_NO_CLAMP) s_w = p->s_min;
    }
    if (n_evals) *n_evals = evals;
    rc = orc_emit(&S, out, cap, n_out);
    free(S.v);
    return rc;
}

/* SplitMix64 (Steele, Lea and Flood 2014): output number n of the stream with state seed. */
uint64_t orc_splitmix64_at(uint64_t seed, uint64_t n)
{
    uint64_t z = seed + n * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Sec. 5.2, Algorithm 2 with the BU noise pruning of Sec. 6.3. */
int orc_search_bu(orc_score_fn f, void *user, int64_t t_begin, int64_t t_end,
                  const orc_params *p, orc_window *out, int64_t cap, int64_t *n_out,
                  int64_t *n_evals)
{
    int rc = orc_check_params(p, t_begin, t_end);
    if (rc) return rc;
    int64_t delta = p->delta_bu > 0 ? p->delta_bu : (p->s_min / 4 > 1 ? p->s_min / 4 : 1);
    int32_t h = p->h > 0 ? p->h : 8;
    int32_t t_max_idle = p->t_max_idle >= 0 ? p->t_max_idle : 3;
    int32_t pcount = p->p > 0 ? p->p : 3;
    int32_t max_steps = p->max_steps > 0 ? p->max_steps : 10000;
    double *L = (double *)malloc(sizeof(double) * (size_t)h);
    if (!L) return ORC_ENOMEM;
    orc_wlist S = {0, 0, 0};
    int64_t evals = 0;
    int64_t last_end = t_begin - 1;
    int64_t c = t_begin;
    uint64_t climb = 0;
    while (c + p->s_min <= t_end && rc == ORC_OK) {
        int64_t ws = c, we = c + p->s_min - 1;
        double Iw, mw;
        rc = f(user, ws, we, &Iw, &mw);
        if (rc) break;
        ++evals;
        for (int32_t q = 0; q < h; ++q) L[q] = Iw;
        int32_t t_idle = 0;
        int32_t noise_run[2] = {0, 0};
        int dropped[2] = {0, 0};           /* 0: leftward, 1: rightward */
        uint64_t step = 0;
        while (t_idle <= t_max_idle && step < (uint64_t)max_steps) {
            int64_t r = t_idle + 1;
            int have_best = 0;
            int64_t bs = 0, be = 0;
            double bsc = 0.0, bmi = 0.0;
            int have_ext[2] = {0, 0};
            double ext_sc[2] = {0.0, 0.0};
            for (int64_t a = -r; a <= r && rc == ORC_OK; ++a) {
                for (int64_t b = -r; b <= r; ++b) {
                    int64_t aa = a < 0 ? -a : a, ab = b < 0 ? -b : b;
                    if ((aa > ab ? aa : ab) != r && g_mutation != ORC_MUT_BU_SQUARE) continue;     /* ring N_r only */
                    if (dropped[0] && a < 0) continue;
                    if (dropped[1] && b > 0) continue;
                    int64_t ts = ws + a * delta, te = we + b * delta;
                    int64_t mm = te - ts + 1;
                    if (mm < p->s_min || mm > p->s_max) continue;
                    if (ts < t_begin || te > t_end - 1 || ts <= last_end) continue;
                    double sc, mi;
                    rc = f(user, ts, te, &sc, &mi);
                    if (rc) break;
                    ++evals;
                    if (!have_best || sc > bsc || (g_mutation == ORC_MUT_TIE_LAST && sc == bsc)) {   /* first maximum wins */
                        have_best = 1; bs = ts; be = te; bsc = sc; bmi = mi;
                    }
                    if (a == -r && b == 0) { have_ext[0] = 1; ext_sc[0] = sc; }
                    if (a == 0 && b == r) { have_ext[1] = 1; ext_sc[1] = sc; }
                }
            }
            if (rc) break;
            if (p->pruning) {
                for (int side = 0; side < 2; ++side) {
                    if (!have_ext[side]) continue;
                    int64_t es = side == 0 ? ws - r * delta : we + 1;
                    int64_t ee = side == 0 ? ws - 1 : we + r * delta;
                    int noise = 0;
                    if (ee - es + 1 >= p->k + 1 || g_mutation == ORC_MUT_TINY_TEST) {
                        double sd, md;
                        rc = f(user, es, ee, &sd, &md);
                        if (rc) break;
                        ++evals;
                        /* Def. 6.2 with w = current window, w' = extension, w'' = neighbour. */
                        noise = (Iw > 0.0 || g_mutation == ORC_MUT_NOISE_NO_IO) && (sd < p->tau) && (ext_sc[side] < Iw);
                    }
                    noise_run[side] = noise ? noise_run[side] + 1
                                            : (g_mutation == ORC_MUT_BU_RUN_NO_RESET ? noise_run[side] : 0);
                    if (noise_run[side] >= pcount) {
                        dropped[side] = 1;
                        if (g_mutation == ORC_MUT_BU_DROP_BOTH) dropped[1 - side] = 1;
                    }
                }
                if (rc) break;
            }
            int32_t v = (int32_t)(orc_splitmix64_at(p->seed, (climb << 32) + step + 1) % (uint64_t)h);
            int better = (bsc > L[v] || bsc > Iw);
            if (g_mutation == ORC_MUT_ACCEPT_GE) better = (bsc >= L[v] || bsc >= Iw);
            if (g_mutation == ORC_MUT_NO_HISTORY) better = bsc > Iw;
            if (have_best && better) {
                ws = bs; we = be; Iw = bsc; mw = bmi;
                t_idle = 0;
            } else {
                t_idle += 1;
            }
            if (Iw > L[v]) L[v] = Iw;
            ++step;
        }
        if (rc) break;
        if (Iw >= p->sigma) {
            rc = orc_push(&S, ws, we, Iw, mw);
            if (rc) break;
            last_end = we;
        }
        c = (we + 1 > c + p->s_min) ? we + 1 : c + p->s_min;
        ++climb;
    }
    free(L);
    if (rc) { free(S.v); return rc; }
    if (n_evals) *n_evals = evals;
    rc = orc_emit(&S, out, cap, n_out);
    free(S.v);
    return rc;
}

/* ------------------------------------------------------------------------- */
/* Chunked search (Sec. 7.3, Algorithm 4)                                     */
/* ------------------------------------------------------------------------- */

/* Algorithm 4 maps the chunks (i - s_max, i + N / n_p), i = 0, N / n_p, 2 N / n_p, ...,
 * of the series to workers and collects the windows each finds.  Reading: N / n_p is the
 * integer quotient L (at least 1), a chunk is the half-open range [i - s_max, i + L)
 * clipped to [t_begin, t_end), the windows are concatenated in chunk order and then
 * sorted stably by t_s; overlapping windows of neighbouring chunks are all kept.
 * alg = 0 runs SYCOS_TD on every chunk, 1 SYCOS_BU. */
typedef struct {
    orc_window w;
    int64_t order;
} orc_ordered;

static int orc_cmp_ordered(const void *a, const void *b)
{
    const orc_ordered *u = (const orc_ordered *)a, *v = (const orc_ordered *)b;
    if (u->w.t_s != v->w.t_s) return (u->w.t_s > v->w.t_s) - (u->w.t_s < v->w.t_s);
    return (u->order > v->order) - (u->order < v->order);
}

int orc_search_chunked(orc_score_fn f, void *user, int64_t t_begin, int64_t t_end,
                       const orc_params *p, int32_t alg, orc_window *out, int64_t cap,
                       int64_t *n_out, int64_t *n_evals)
{
    int rc = orc_check_params(p, t_begin, t_end);
    if (rc) return rc;
    if (alg != 0 && alg != 1) return ORC_EINVAL;
    int64_t N = t_end - t_begin;
    int64_t np = p->chunks > 1 ? p->chunks : 1;
    int64_t L = N / np;
    if (L < 1) L = 1;
    orc_params q = *p;
    q.chunks = 0;
    orc_window *buf = (orc_window *)malloc(sizeof(orc_window) * 65536);
    orc_ordered *all = NULL;
    int64_t n_all = 0, cap_all = 0, evals = 0;
    if (!buf) return ORC_ENOMEM;
    for (int64_t i = 0; i < N && rc == ORC_OK; i += L) {
        int64_t a = t_begin + (i - p->s_max > 0 ? i - p->s_max : 0);
        if (g_mutation == ORC_MUT_CHUNK_NO_OVERLAP) a = t_begin + i;
        int64_t b = t_begin + (i + L < N ? i + L : N);
        int64_t nw = 0, ne = 0;
        rc = (alg == 0 ? orc_search_td : orc_search_bu)(f, user, a, b, &q, buf, 65536, &nw, &ne);
        if (rc) break;
        evals += ne;
        for (int64_t j = 0; j < nw; ++j) {
            if (n_all == cap_all) {
                int64_t nc = cap_all ? 2 * cap_all : 256;
                orc_ordered *na = (orc_ordered *)realloc(all, sizeof(orc_ordered) * (size_t)nc);
                if (!na) { rc = ORC_ENOMEM; break; }
                all = na;
                cap_all = nc;
            }
            all[n_all].w = buf[j];
            all[n_all].order = n_all;
            n_all++;
        }
    }
    free(buf);
    if (rc == ORC_OK) {
        if (n_all > 1) qsort(all, (size_t)n_all, sizeof(orc_ordered), orc_cmp_ordered);
        if (n_out) *n_out = n_all;
        if (n_evals) *n_evals = evals;
        if (n_all > cap) rc = ORC_ETRUNC;
        else
            for (int64_t j = 0; j < n_all; ++j) out[j] = all[j].w;
    }
    free(all);
    return rc;
}

/* ------------------------------------------------------------------------- */
/* iSYCOS selection (Sec. 5.3, Algorithm 3, Eqs. effscore / normalizedeffscore) */
/* ------------------------------------------------------------------------- */

/* Normalised efficiency scores (Eqs. normalizeruntime, normalizedwindows,
 * normalizedeffscore_TD / _BU): t~ = t / (t_TD + t_BU), n~L_TD = nL_TD / (nS_BU + nL_TD),
 * n~S_BU = nS_BU / (nS_BU + nL_TD), nscore = alpha / t~ + (1 - alpha) n~.
 * Readings: when both runtimes are 0 each normalised runtime is 1/2; when both window counts
 * are 0 both normalised counts are 0. */
void orc_nscores(double t_td, double t_bu, double nl_td, double ns_bu, double alpha,
                 double *ns_td_out, double *ns_bu_out)
{
    double tt = t_td + t_bu;
    double rt_td = tt > 0.0 ? t_td / tt : 0.5;
    double rt_bu = tt > 0.0 ? t_bu / tt : 0.5;
    double nn = ns_bu + nl_td;
    double wl_td = nn > 0.0 ? nl_td / nn : 0.0;
    double ws_bu = nn > 0.0 ? ns_bu / nn : 0.0;
    *ns_td_out = alpha * (1.0 / rt_td) + (1.0 - alpha) * wl_td;
    *ns_bu_out = alpha * (1.0 / rt_bu) + (1.0 - alpha) * ws_bu;
}

/* A scorer wrapper that adds up the pair comparisons m (m - 1) of every scored window: the
 * deterministic "runtime" of a search. */
typedef struct {
    orc_score_fn f;
    void *user;
    double cost;
} orc_cost_scorer;

static int orc_cost_score(void *user, int64_t t_s, int64_t t_e, double *score, double *mi)
{
    orc_cost_scorer *c = (orc_cost_scorer *)user;
    double m = (double)(t_e - t_s + 1);
    c->cost += g_mutation == ORC_MUT_RUNTIME_WINDOWS ? 1.0 : m * (m - 1.0);
    return c->f(c->user, t_s, t_e, score, mi);
}

typedef struct {
    int32_t partitions;   /* M, <= 0: 20                                   */
    int32_t samples;      /* m, <= 0: 6 (the paper's experiments sample 6) */
    double alpha;         /* weight of the runtime factor, < 0: 0.5         */
    double rho;           /* small windows: size <= rho * s_max, <= 0: 0.5  */
} orc_select_params;

/* Algorithm 3: sample `samples` of `partitions` equal partitions of [t_begin, t_end), run
 * SYCOS_TD and SYCOS_BU on each, score them (runtime = pair comparisons of the windows each
 * search scores), and run the selected search on the whole range.  *selected = 0 (TD) or 1. */
int orc_search_auto(orc_score_fn f, void *user, int64_t t_begin, int64_t t_end,
                    const orc_params *p, const orc_select_params *sp, orc_window *out,
                    int64_t cap, int64_t *n_out, int64_t *n_evals, int32_t *selected,
                    double *scores)
{
    int rc = orc_check_params(p, t_begin, t_end);
    if (rc) return rc;
    int32_t M = (sp && sp->partitions > 0) ? sp->partitions : 20;
    int32_t ms = (sp && sp->samples > 0) ? sp->samples : 6;
    double alpha = (sp && sp->alpha >= 0.0) ? sp->alpha : 0.5;
    double rho = (sp && sp->rho > 0.0) ? sp->rho : 0.5;
    int64_t N = t_end - t_begin;
    if (ms > M) ms = M;
    int64_t L = N / M;
    int32_t *idx = (int32_t *)malloc(sizeof(int32_t) * (size_t)M);
    if (!idx) return ORC_ENOMEM;
    for (int32_t i = 0; i < M; ++i) idx[i] = i;
    /* Random sampling: partial Fisher-Yates shuffle driven by SplitMix64 outputs of the stream
     * seed ^ 0x5E1EC7 (one draw per sampled partition). */
    for (int32_t i = 0; i < ms; ++i) {
        uint64_t r = orc_splitmix64_at(p->seed ^ 0x5E1EC7ULL,
                                       (uint64_t)i + (g_mutation == ORC_MUT_SAMPLE_DRAW ? 0 : 1));
        int32_t j = i + (int32_t)(r % (uint64_t)(M - i));
        int32_t t = idx[i]; idx[i] = idx[j]; idx[j] = t;
    }
    double t_td = 0.0, t_bu = 0.0, nl_td = 0.0, ns_bu = 0.0;
    int64_t evals = 0;
    orc_window *buf = (orc_window *)malloc(sizeof(orc_window) * 65536);
    if (!buf) { free(idx); return ORC_ENOMEM; }
    for (int32_t i = 0; i < ms && L > 0 && rc == ORC_OK; ++i) {
        int64_t a = t_begin + (int64_t)idx[i] * L, b = a + L;
        for (int alg = 0; alg < 2 && rc == ORC_OK; ++alg) {
            orc_cost_scorer cs = {f, user, 0.0};
            int64_t nw = 0, ne = 0;
            rc = (alg == 0 ? orc_search_td : orc_search_bu)(orc_cost_score, &cs, a, b, p, buf, 65536,
                                                             &nw, &ne);
            if (rc) break;
            evals += ne;
            for (int64_t q = 0; q < nw; ++q) {
                double size = (double)(buf[q].t_e - buf[q].t_s + 1);
                int small = size <= rho * (double)p->s_max;
                if (alg == 0 && !small) nl_td += 1.0;
                if (alg == 1 && small) ns_bu += 1.0;
            }
            if (alg == 0) t_td += cs.cost; else t_bu += cs.cost;
        }
    }
    free(buf);
    free(idx);
    if (rc) return rc;
    t_td /= (double)ms;     /* average runtimes over the m partitions */
    t_bu /= (double)ms;
    double s_td, s_bu;
    orc_nscores(t_td, t_bu, nl_td, ns_bu, alpha, &s_td, &s_bu);
    if (scores) { scores[0] = s_td; scores[1] = s_bu; }
    int32_t sel = s_td > s_bu ? 0 : 1;
    if (selected) *selected = sel;
    int64_t ne = 0;
    /* the selected search over the whole range, in chunks when n_p > 1 (Algorithm 4) */
    if (p->chunks > 1)
        rc = orc_search_chunked(f, user, t_begin, t_end, p, sel, out, cap, n_out, &ne);
    else
        rc = (sel == 0 ? orc_search_td : orc_search_bu)(f, user, t_begin, t_end, p, out, cap, n_out, &ne);
    if (n_evals) *n_evals = evals + ne;
    return rc;
}
