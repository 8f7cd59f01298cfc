/*
 * messi_oracle.c -- plain FP64 CPU reference of the MESSI exact k-NN method.
 *
 * TEST INFRASTRUCTURE ONLY (see messi_oracle.h).  Built with gcc
 * -O2 -fopenmp -ffp-contract=off so every FP64 operation is a separately
 * rounded IEEE operation in the order written here.
 */
#include "messi_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------------------------------------------------------- Sec. 2.2 */

/* The breakpoints are the doubles nearest the N(0,1) quantiles PhiInv(j/c):
 * the real quantile is irrational, so its nearest double is unique and any
 * correct evaluation of the definition gives the same table.  To decide
 * which double is nearest, Phi is evaluated in double-double arithmetic (a
 * value is an unevaluated sum hi + lo, ~104-bit significand) from its
 * Maclaurin series
 *     Phi(x) = 1/2 + (1/sqrt(2 pi)) * sum_n (-1)^n x^(2n+1) / (2^n n! (2n+1)),
 * which converges for every x; for |x| <= 3 its terms stay below 2^7, so the
 * sum keeps about 90 correct bits. */
typedef struct { double hi, lo; } dd_t;

static dd_t dd_from_sum(double a, double b)             /* exact a + b (two-sum) */
{
    dd_t r;
    double s = a + b, v = s - a;
    r.hi = s;
    r.lo = (a - (s - v)) + (b - v);
    return r;
}
static dd_t dd_renorm(double a, double b)               /* |a| >= |b| */
{
    dd_t r;
    double s = a + b;
    r.hi = s;
    r.lo = b - (s - a);
    return r;
}
static dd_t dd_add(dd_t a, dd_t b)
{
    dd_t s = dd_from_sum(a.hi, b.hi), t = dd_from_sum(a.lo, b.lo);
    s.lo += t.hi;
    s = dd_renorm(s.hi, s.lo);
    s.lo += t.lo;
    return dd_renorm(s.hi, s.lo);
}
static dd_t dd_mul(dd_t a, dd_t b)
{
    double p = a.hi * b.hi;
    double e = fma(a.hi, b.hi, -p);                      /* exact error of the product */
    e += a.hi * b.lo + a.lo * b.hi;
    return dd_renorm(p, e);
}
static dd_t dd_div_d(dd_t a, double b)                   /* a / b, b a double */
{
    double q1 = a.hi / b;
    double p = q1 * b, pe = fma(q1, b, -p);              /* q1 * b exactly: p + pe */
    dd_t r = dd_add(a, dd_renorm(-p, -pe));
    double q2 = r.hi / b;
    return dd_renorm(q1, q2);
}

/* 1/sqrt(2 pi) as a double-double: pi = 3.141592653589793116 +
 * 1.2246467991473532e-16 (the double nearest pi, then the double nearest
 * the rest); sqrt by one Newton step from the double root, and the
 * reciprocal by one more. */
static dd_t inv_sqrt_two_pi(void)
{
    dd_t two_pi = {2.0 * 3.141592653589793116, 2.0 * 1.2246467991473532e-16};
    double s = sqrt(two_pi.hi);
    dd_t s2 = {s * s, fma(s, s, -(s * s))};
    dd_t rem = dd_add(two_pi, (dd_t){-s2.hi, -s2.lo});
    dd_t root = dd_renorm(s, rem.hi / (2.0 * s));         /* sqrt(2 pi) */
    double r0 = 1.0 / root.hi;
    dd_t prod = dd_mul(root, (dd_t){r0, 0.0});            /* root * r0 = 1 - e */
    dd_t e = dd_add((dd_t){1.0, 0.0}, (dd_t){-prod.hi, -prod.lo});
    return dd_renorm(r0, r0 * e.hi);                      /* r0 (1 + e) */
}

/* Phi(x) - p for a double-double x with |x| <= 3 (p exact in double). */
static dd_t cdf_minus_dd(dd_t x, double p)
{
    dd_t half_x2 = dd_mul(dd_mul(x, x), (dd_t){0.5, 0.0});
    dd_t power = x;                                       /* (-1)^n x^(2n+1) / (2^n n!) */
    dd_t sum = x;
    for (int n = 1; n < 200; ++n) {
        power = dd_div_d(dd_mul(power, (dd_t){-half_x2.hi, -half_x2.lo}), (double)n);
        dd_t term = dd_div_d(power, (double)(2 * n + 1));
        sum = dd_add(sum, term);
        if (fabs(term.hi) < 1e-40) break;
    }
    dd_t phi = dd_add((dd_t){0.5, 0.0}, dd_mul(inv_sqrt_two_pi(), sum));
    return dd_add(phi, (dd_t){-p, 0.0});
}

/* The double nearest PhiInv(p), 0 < p < 1/2: bisection on doubles in
 * [-3, 0] (the CDF's sign decides each step) down to two adjacent doubles
 * lo < hi around the quantile, then the one nearer it -- hi if the CDF at
 * their midpoint (lo + hi)/2, held exactly as a double-double, is below p. */
static double std_normal_quantile(double p)
{
    double lo = -3.0, hi = 0.0;
    for (int it = 0; it < 4000; ++it) {
        double mid = lo + 0.5 * (hi - lo);
        if (mid <= lo || mid >= hi) break;
        dd_t g = cdf_minus_dd((dd_t){mid, 0.0}, p);
        if (g.hi < 0.0) lo = mid; else hi = mid;
    }
    dd_t m = dd_renorm(lo, 0.5 * (hi - lo));
    return cdf_minus_dd(m, p).hi < 0.0 ? hi : lo;
}

void orc_breakpoints(int card, double *beta)
{
    /* Lower half by bisection (p < 1/2, where the CDF minus p keeps its
     * relative accuracy); the upper half by the symmetry of N(0,1),
     * PhiInv(1 - p) = -PhiInv(p), which maps nearest doubles to nearest
     * doubles; the median is 0. */
    for (int j = 1; 2 * j < card; ++j)
        beta[j - 1] = std_normal_quantile((double)j / (double)card);
    for (int j = 1; j < card; ++j) {
        if (2 * j == card) beta[j - 1] = 0.0;
        else if (2 * j > card) beta[j - 1] = -beta[card - j - 1];
    }
}

void orc_paa(const float *x, int n, int w, double *paa)
{
    int m = n / w;
    for (int s = 0; s < w; ++s) {
        double sum = 0.0;
        for (int t = s * m; t < (s + 1) * m; ++t) sum += (double)x[t];
        paa[s] = sum / (double)m;
    }
}

void orc_sax(const double *paa, int w, int card, const double *beta, uint8_t *sym)
{
    for (int s = 0; s < w; ++s) {
        int count = 0;
        for (int j = 1; j < card; ++j)
            if (beta[j - 1] <= paa[s]) ++count;
        sym[s] = (uint8_t)count;
    }
}

void orc_summarize(const float *data, int64_t N, int n, int w, int card,
                   const double *beta, uint8_t *sax)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        double paa[64];
        orc_paa(data + i * (int64_t)n, n, w, paa);
        orc_sax(paa, w, card, beta, sax + i * (int64_t)w);
    }
}

static int log2_card(int card)
{
    int b = 0;
    while ((1 << b) < card) ++b;
    return b;
}

void orc_isax_key(const uint8_t *sym, int w, int card, uint32_t key[4])
{
    int b = log2_card(card);
    key[0] = key[1] = key[2] = key[3] = 0u;
    for (int j = 0; j < b; ++j)
        for (int s = 0; s < w; ++s) {
            int p = j * w + s;                          /* position from the MSB */
            uint32_t bit = (sym[s] >> (b - 1 - j)) & 1u;
            key[p / 32] |= bit << (31 - (p % 32));
        }
}

/* ---------------------------------------------------------------- Sec. 2.1 */

double orc_ed2(const float *q, const float *x, int n)
{
    double s = 0.0;
    for (int t = 0; t < n; ++t) {
        double d = (double)q[t] - (double)x[t];
        s += d * d;
    }
    return s;
}

/* ------------------------------------------------------ Property 1, Sec. 4 */

/* Region [lo, hi] of symbol v: lo = beta_v (-inf for v = 0),
 * hi = beta_{v+1} (+inf for v = c-1). */
static double region_lo(int v, const double *beta) { return v == 0 ? -INFINITY : beta[v - 1]; }
static double region_hi(int v, int card, const double *beta) { return v == card - 1 ? INFINITY : beta[v]; }

double orc_mindist_ed2(const double *paa_q, const uint8_t *sym, int w, int m,
                       int card, const double *beta)
{
    double s = 0.0;
    for (int k = 0; k < w; ++k) {
        double lo = region_lo(sym[k], beta), hi = region_hi(sym[k], card, beta);
        double d = 0.0;
        if (paa_q[k] < lo) d = lo - paa_q[k];
        else if (paa_q[k] > hi) d = paa_q[k] - hi;
        s += d * d;
    }
    return (double)m * s;
}

/* ---------------------------------------------------------------- Sec. 3.4 */

void orc_envelope(const float *q, int n, int r, double *U, double *L)
{
    for (int i = 0; i < n; ++i) {
        int a = i - r < 0 ? 0 : i - r;
        int b = i + r > n - 1 ? n - 1 : i + r;
        double hi = (double)q[a], lo = (double)q[a];
        for (int j = a + 1; j <= b; ++j) {
            if ((double)q[j] > hi) hi = (double)q[j];
            if ((double)q[j] < lo) lo = (double)q[j];
        }
        U[i] = hi;
        L[i] = lo;
    }
}

double orc_lb_keogh2(const double *U, const double *L, const float *x, int n)
{
    double s = 0.0;
    for (int i = 0; i < n; ++i) {
        double c = (double)x[i], d = 0.0;
        if (c > U[i]) d = c - U[i];
        else if (c < L[i]) d = c - L[i];
        s += d * d;
    }
    return s;
}

double orc_mindist_dtw2(const double *paaU, const double *paaL, const uint8_t *sym,
                        int w, int m, int card, const double *beta)
{
    double s = 0.0;
    for (int k = 0; k < w; ++k) {
        double lo = region_lo(sym[k], beta), hi = region_hi(sym[k], card, beta);
        double d = 0.0;
        if (paaU[k] < lo) d = lo - paaU[k];          /* ABOVE */
        else if (paaL[k] > hi) d = paaL[k] - hi;     /* BELOW */
        s += d * d;                                  /* IN: 0 */
    }
    return (double)m * s;
}

/* LB_Improved (Lemire): LB_Keogh of x against the query's envelope [L, U],
 * plus the query against the envelope (same window) of h = x clamped into
 * [L, U].  A lower bound of the banded squared DTW; the DTW filter of the
 * query path uses it after LB_Keogh (Sec. 3.4 lower-bounds before real
 * distances).  Plain loops over the definition. */
double orc_lb_improved2(const float *q, const double *U, const double *L, const float *x, int n, int r)
{
    double first = orc_lb_keogh2(U, L, x, n), second = 0.0;
    double *h = (double *)malloc(sizeof(double) * (size_t)n);
    if (!h) return first;
    for (int i = 0; i < n; ++i) {
        double c = (double)x[i];
        h[i] = c > U[i] ? U[i] : (c < L[i] ? L[i] : c);
    }
    for (int i = 0; i < n; ++i) {
        int a = i - r < 0 ? 0 : i - r;
        int b = i + r > n - 1 ? n - 1 : i + r;
        double hi = h[a], lo = h[a];
        for (int j = a + 1; j <= b; ++j) {
            if (h[j] > hi) hi = h[j];
            if (h[j] < lo) lo = h[j];
        }
        double v = (double)q[i], d = 0.0;
        if (v > hi) d = v - hi;
        else if (v < lo) d = v - lo;
        second += d * d;
    }
    free(h);
    return first + second;
}

double orc_dtw2(const float *q, const float *x, int n, int r)
{
    /* D is an n x n table; only cells inside the window are ever written or
     * read (a cell outside the window is +inf and never the minimum). */
    static __thread double *D = NULL;
    static __thread size_t cap = 0;
    size_t need = (size_t)n * (size_t)n;
    if (need > cap) {
        free(D);
        D = (double *)malloc(sizeof(double) * need);
        cap = need;
    }
    if (r > n - 1) r = n - 1;
    for (int i = 0; i < n; ++i) {
        int jlo = i - r < 0 ? 0 : i - r;
        int jhi = i + r > n - 1 ? n - 1 : i + r;
        for (int j = jlo; j <= jhi; ++j) {
            double d = (double)q[i] - (double)x[j];
            double cost = d * d;
            double best;
            if (i == 0 && j == 0) best = 0.0;
            else {
                best = INFINITY;
                if (i > 0 && abs(i - 1 - j) <= r && D[(size_t)(i - 1) * n + j] < best)
                    best = D[(size_t)(i - 1) * n + j];
                if (j > 0 && abs(i - (j - 1)) <= r && D[(size_t)i * n + j - 1] < best)
                    best = D[(size_t)i * n + j - 1];
                if (i > 0 && j > 0 && D[(size_t)(i - 1) * n + j - 1] < best)
                    best = D[(size_t)(i - 1) * n + j - 1];
            }
            D[(size_t)i * n + j] = cost + best;
        }
    }
    return D[need - 1];
}

/* ------------------------------------------------------- k-NN, Sec. 5.4 */

/* (d2, id) lexicographic order. */
static int before(double da, int64_t ia, double db, int64_t ib)
{
    return da < db || (da == db && ia < ib);
}

/* Insert (d, id) into a sorted array of capacity k holding *cnt entries. */
static void topk_insert(double *kd, int64_t *ki, int *cnt, int k, double d, int64_t id)
{
    if (*cnt == k && !before(d, id, kd[k - 1], ki[k - 1])) return;
    int pos = (*cnt < k) ? (*cnt)++ : k - 1;
    while (pos > 0 && before(d, id, kd[pos - 1], ki[pos - 1])) {
        kd[pos] = kd[pos - 1];
        ki[pos] = ki[pos - 1];
        --pos;
    }
    kd[pos] = d;
    ki[pos] = id;
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_knn(const float *data, int64_t N, int n, const float *queries, int nq,
             int k, int dist, int r, int64_t id_base, int threads,
             int64_t *ids, double *d2)
{
    int T = threads > 0 ? threads : orc_max_threads();
    if (T < 1) T = 1;
    /* Each worker scans a contiguous block of rows and keeps its own k best
     * per query; the blocks partition the rows, so the k best of the union
     * of the per-block results is the k best of all rows. */
    size_t slots = (size_t)T * (size_t)nq * (size_t)k;
    double *bd = (double *)malloc(sizeof(double) * slots);
    int64_t *bi = (int64_t *)malloc(sizeof(int64_t) * slots);
    int *bc = (int *)calloc((size_t)T * (size_t)nq, sizeof(int));

#pragma omp parallel num_threads(T)
    {
        int t = 0;
#ifdef _OPENMP
        t = omp_get_thread_num();
        int nt = omp_get_num_threads();
#else
        int nt = 1;
#endif
        int64_t lo = N * t / nt, hi = N * (t + 1) / nt;
        for (int64_t row = lo; row < hi; ++row) {
            const float *x = data + row * (int64_t)n;
            for (int qi = 0; qi < nq; ++qi) {
                const float *q = queries + (int64_t)qi * n;
                double d = (dist == 0) ? orc_ed2(q, x, n) : orc_dtw2(q, x, n, r);
                size_t base = ((size_t)t * nq + qi) * (size_t)k;
                topk_insert(bd + base, bi + base, &bc[(size_t)t * nq + qi], k, d, id_base + row);
            }
        }
    }

    for (int qi = 0; qi < nq; ++qi) {
        int cnt = 0;
        double *od = d2 + (size_t)qi * k;
        int64_t *oi = ids + (size_t)qi * k;
        for (int t = 0; t < T; ++t) {
            size_t base = ((size_t)t * nq + qi) * (size_t)k;
            for (int e = 0; e < bc[(size_t)t * nq + qi]; ++e)
                topk_insert(od, oi, &cnt, k, bd[base + e], bi[base + e]);
        }
        for (int e = cnt; e < k; ++e) { od[e] = INFINITY; oi[e] = -1; }
    }
    free(bd);
    free(bi);
    free(bc);
}

int64_t orc_windows(const float *series, int64_t length, int n, int stride, int znorm, float *out)
{
    const int64_t count = (length - n) / stride + 1;
    for (int64_t i = 0; i < count; ++i) {
        const float *x = series + i * stride;
        float *o = out + i * (int64_t)n;
        if (!znorm) {
            for (int j = 0; j < n; ++j) o[j] = x[j];
            continue;
        }
        double sum = 0.0;
        for (int j = 0; j < n; ++j) sum = sum + (double)x[j];
        const double mean = sum / (double)n;
        double ss = 0.0;
        for (int j = 0; j < n; ++j) {
            const double d = (double)x[j] - mean;
            ss = ss + d * d;
        }
        const double var = ss / (double)n;
        const double inv = var > 0.0 ? 1.0 / sqrt(var) : 0.0;
        for (int j = 0; j < n; ++j) o[j] = (float)(((double)x[j] - mean) * inv);
    }
    return count;
}
