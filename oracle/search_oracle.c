/*
 * Search-stage oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain CPU statements of the steps the paper applies after dedispersion
 * (paper Section 2.3, "Other algorithms"): baseline removal, matched
 * filtering with boxcars of growing width, and peak finding by a sigma cut
 * followed by grouping contiguous regions into events; plus the cut-out of a
 * DM-time snippet around each event for the candidate classifier.  Only the
 * test-suite, the smoke check and the CPU-baseline leg of the benchmark may
 * load this library; it shares nothing with the CUDA path.
 *
 * Readings (the paper gives these steps in words only):
 *  - Baseline: y[t] = x[t] - median of x over [t-half, t+half) clipped to the
 *    row, the LOWER median (element of rank floor((m-1)/2), 0-based, of the m
 *    sorted values).  The paper subtracts a running mean; the running median
 *    is the robust variant used here; oracle_running_mean keeps the paper's
 *    mean form, and oracle_baseline_mean_row the mean baseline as the
 *    pipeline's integer option (mean rounded half up).
 *  - Noise: sigma_d = sqrt(sum_t y^2 / n) per DM row, the integer sum exact in
 *    int64 and the rest in double.
 *  - Boxcar of width w: S_w[t] = sum_{i<w} y[t+i] for t + w <= n (leading
 *    window); snr_w[t] = (float)S_w / (float)(sigma * sqrt(w)), 0 when the row
 *    is constant (sigma == 0).
 *  - Peaks: per cell the largest snr over the valid widths (ties keep the
 *    smaller width); cells with snr >= thresh are grouped by 4-connectivity in
 *    (DM, time); each group is reported once, at its cell of largest snr (ties:
 *    lower DM index, then earlier time); groups ordered by that cell's (d, t).
 *  - Snippet: 64 DM rows centred on the event's row (rows d-32 .. d+31) by 64
 *    time bins of w samples, bin k starting at t + (k-32)*w; a bin holds
 *    (float)(sum of the y samples inside the row) / (float)(sigma_row*sqrt(w))
 *    rounded to bfloat16 (round to nearest even); rows outside the data are 0.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---- baseline removal --------------------------------------------------- */

/* Running lower median by counting: a histogram of the window is kept and,
 * for every output sample, walked from the smallest value until the count
 * passes the median rank. */
int oracle_running_median(const int32_t *x, int64_t n, int64_t half, int32_t *med)
{
    if (n <= 0 || half <= 0) return -1;
    int32_t vmin = x[0], vmax = x[0];
    for (int64_t i = 1; i < n; ++i) {
        if (x[i] < vmin) vmin = x[i];
        if (x[i] > vmax) vmax = x[i];
    }
    int64_t range = (int64_t)vmax - vmin + 1;
    int64_t *hist = (int64_t *)calloc((size_t)range, sizeof(int64_t));
    if (!hist) return -2;
    int64_t lo = 0, hi = 0; /* window is [lo, hi) */
    for (int64_t t = 0; t < n; ++t) {
        int64_t want_lo = t - half < 0 ? 0 : t - half;
        int64_t want_hi = t + half > n ? n : t + half;
        while (hi < want_hi) { hist[x[hi] - vmin]++; hi++; }
        while (lo < want_lo) { hist[x[lo] - vmin]--; lo++; }
        int64_t m = hi - lo;
        int64_t rank = (m - 1) / 2;
        int64_t seen = 0;
        for (int64_t v = 0; v < range; ++v) {
            seen += hist[v];
            if (seen > rank) { med[t] = (int32_t)(v + vmin); break; }
        }
    }
    free(hist);
    return 0;
}

/* y = x - running lower median, for a uint32 dedispersed row. */
int oracle_baseline_row(const uint32_t *row, int64_t n, int64_t half, int32_t *y)
{
    int32_t *x = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int32_t *med = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    if (!x || !med) { free(x); free(med); return -2; }
    for (int64_t i = 0; i < n; ++i) x[i] = (int32_t)row[i];
    int rc = oracle_running_median(x, n, half, med);
    if (rc == 0)
        for (int64_t i = 0; i < n; ++i) y[i] = x[i] - med[i];
    free(x);
    free(med);
    return rc;
}

/* oracle_baseline_row applied to each of ndm independent rows (row d at
 * rows + d*ld_rows, result at y + d*n), the rows shared out over OpenMP
 * threads.  Returns the first failing row's status, else 0. */
int oracle_baseline_rows(const uint32_t *rows, int ndm, int64_t n, int64_t ld_rows, int64_t half, int32_t *y)
{
    int rc = 0;
#pragma omp parallel for schedule(dynamic, 1)
    for (int d = 0; d < ndm; ++d) {
        int r = oracle_baseline_row(rows + (size_t)d * (size_t)ld_rows, n, half, y + (size_t)d * (size_t)n);
        if (r != 0) {
#pragma omp critical
            rc = rc ? rc : r;
        }
    }
    return rc;
}

/* The paper's own baseline as an integer pipeline step: y = x - the running
 * mean over the same clipped window rounded half up, floor((2 s + m) / (2 m))
 * for the window sum s of its m values (exact integer arithmetic). */
int oracle_baseline_mean_row(const uint32_t *row, int64_t n, int64_t half, int32_t *y)
{
    if (n <= 0 || half <= 0) return -1;
    for (int64_t t = 0; t < n; ++t) {
        int64_t lo = t - half < 0 ? 0 : t - half;
        int64_t hi = t + half > n ? n : t + half;
        int64_t s = 0;
        for (int64_t i = lo; i < hi; ++i) s += row[i];
        const int64_t m = hi - lo;
        y[t] = (int32_t)((int64_t)row[t] - (2 * s + m) / (2 * m));
    }
    return 0;
}

/* The paper's own baseline: x minus the running mean over the same clipped
 * window, written as a double. */
int oracle_running_mean(const int32_t *x, int64_t n, int64_t half, double *mean)
{
    if (n <= 0 || half <= 0) return -1;
    for (int64_t t = 0; t < n; ++t) {
        int64_t lo = t - half < 0 ? 0 : t - half;
        int64_t hi = t + half > n ? n : t + half;
        int64_t s = 0;
        for (int64_t i = lo; i < hi; ++i) s += x[i];
        mean[t] = (double)s / (double)(hi - lo);
    }
    return 0;
}

/* ---- matched filter ------------------------------------------------------ */

int64_t oracle_sumsq(const int32_t *y, int64_t n)
{
    int64_t s = 0;
    for (int64_t i = 0; i < n; ++i) s += (int64_t)y[i] * y[i];
    return s;
}

double oracle_sigma(const int32_t *y, int64_t n)
{
    return sqrt((double)oracle_sumsq(y, n) / (double)n);
}

/* The denominator sigma*sqrt(w) as the float that divides the boxcar sum. */
static float snr_denominator(double sigma, int w)
{
    return (float)(sigma * sqrt((double)w));
}

/* snr[t] for t + w <= n; entries t > n - w are left untouched. */
int oracle_boxcar_snr(const int32_t *y, int64_t n, int w, float *snr)
{
    if (w <= 0 || w > n) return -1;
    int64_t sumsq = oracle_sumsq(y, n);
    double sigma = sqrt((double)sumsq / (double)n);
    float den = snr_denominator(sigma, w);
    for (int64_t t = 0; t + w <= n; ++t) {
        int64_t s = 0;
        for (int i = 0; i < w; ++i) s += y[t + i];
        snr[t] = sumsq == 0 ? 0.0f : (float)s / den;
    }
    return 0;
}

/* Best snr over the widths list, per cell, for one row. */
int oracle_best_snr_row(const int32_t *y, int64_t n, int nw, const int *widths,
                        float *best, int32_t *bestw)
{
    float *tmp = (float *)malloc((size_t)n * sizeof(float));
    if (!tmp) return -2;
    for (int64_t t = 0; t < n; ++t) { best[t] = -INFINITY; bestw[t] = 0; }
    for (int k = 0; k < nw; ++k) {
        int w = widths[k];
        if (w > n) continue;
        oracle_boxcar_snr(y, n, w, tmp);
        for (int64_t t = 0; t + w <= n; ++t) {
            if (tmp[t] > best[t] || bestw[t] == 0) { best[t] = tmp[t]; bestw[t] = w; }
        }
    }
    free(tmp);
    return 0;
}

/* oracle_best_snr_row for each of ndm independent rows of y (n values each),
 * the rows shared out over OpenMP threads. */
int oracle_best_snr_rows(const int32_t *y, int ndm, int64_t n, int nw, const int *widths,
                         float *best, int32_t *bestw)
{
    int rc = 0;
#pragma omp parallel for schedule(dynamic, 1)
    for (int d = 0; d < ndm; ++d) {
        int r = oracle_best_snr_row(y + (size_t)d * (size_t)n, n, nw, widths, best + (size_t)d * (size_t)n,
                                    bestw + (size_t)d * (size_t)n);
        if (r != 0) {
#pragma omp critical
            rc = rc ? rc : r;
        }
    }
    return rc;
}

/* ---- peak finding -------------------------------------------------------- */

typedef struct {
    int32_t d;
    int32_t t;
    int32_t w;
    float snr;
    int64_t ncells;
} oracle_cand;

static int better(float s1, int d1, int64_t t1, float s2, int d2, int64_t t2)
{
    if (s1 != s2) return s1 > s2;
    if (d1 != d2) return d1 < d2;
    return t1 < t2;
}

static int cmp_cand(const void *a, const void *b)
{
    const oracle_cand *x = (const oracle_cand *)a, *y = (const oracle_cand *)b;
    if (x->d != y->d) return x->d < y->d ? -1 : 1;
    if (x->t != y->t) return x->t < y->t ? -1 : 1;
    return 0;
}

/* Flood fill over the hot cells of an ndm x n map.  Returns the number of
 * groups (up to max_out are written), or a negative error. */
int64_t oracle_find_peaks(const float *best, const int32_t *bestw, int ndm, int64_t n,
                          float thresh, oracle_cand *out, int64_t max_out)
{
    size_t cells = (size_t)ndm * (size_t)n;
    uint8_t *seen = (uint8_t *)calloc(cells, 1);
    int64_t *stack = (int64_t *)malloc(cells * sizeof(int64_t));
    if (!seen || !stack) { free(seen); free(stack); return -2; }
    int64_t ngroups = 0;
    oracle_cand *all = NULL;
    int64_t cap = 0;
    for (size_t start = 0; start < cells; ++start) {
        if (seen[start] || !(best[start] >= thresh)) continue;
        int64_t sp = 0;
        stack[sp++] = (int64_t)start;
        seen[start] = 1;
        oracle_cand g;
        g.d = (int32_t)(start / n);
        g.t = (int32_t)(start % n);
        g.w = bestw[start];
        g.snr = best[start];
        g.ncells = 0;
        while (sp > 0) {
            int64_t i = stack[--sp];
            int d = (int)(i / n);
            int64_t t = i % n;
            g.ncells++;
            if (better(best[i], d, t, g.snr, g.d, g.t)) {
                g.d = d; g.t = (int32_t)t; g.w = bestw[i]; g.snr = best[i];
            }
            int64_t nb[4] = {d > 0 ? i - n : -1, d + 1 < ndm ? i + n : -1,
                             t > 0 ? i - 1 : -1, t + 1 < n ? i + 1 : -1};
            for (int k = 0; k < 4; ++k) {
                int64_t j = nb[k];
                if (j >= 0 && !seen[j] && best[j] >= thresh) { seen[j] = 1; stack[sp++] = j; }
            }
        }
        if (ngroups == cap) {
            cap = cap ? 2 * cap : 64;
            oracle_cand *na = (oracle_cand *)realloc(all, (size_t)cap * sizeof(oracle_cand));
            if (!na) { free(all); free(seen); free(stack); return -2; }
            all = na;
        }
        all[ngroups++] = g;
    }
    if (ngroups > 0) qsort(all, (size_t)ngroups, sizeof(oracle_cand), cmp_cand);
    for (int64_t k = 0; k < ngroups && k < max_out; ++k) out[k] = all[k];
    free(all);
    free(seen);
    free(stack);
    return ngroups;
}

/* ---- snippets ------------------------------------------------------------ */

static uint16_t float_to_bf16_rne(float f)
{
    uint32_t u;
    memcpy(&u, &f, 4);
    if ((u & 0x7f800000u) == 0x7f800000u && (u & 0x007fffffu)) return (uint16_t)((u >> 16) | 0x40);
    u += 0x7fffu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}

/* y: ndm rows of n int32 (baseline-removed), sumsq: per-row sum of squares.
 * out: ncand x 64 x 64 bfloat16 bit patterns. */
int oracle_snippets(const int32_t *y, const int64_t *sumsq, int ndm, int64_t n,
                    int64_t ncand, const int32_t *cd, const int32_t *ct, const int32_t *cw,
                    uint16_t *out)
{
    for (int64_t k = 0; k < ncand; ++k) {
        int w = cw[k];
        for (int r = 0; r < 64; ++r) {
            int dd = cd[k] - 32 + r;
            for (int b = 0; b < 64; ++b) {
                float v = 0.0f;
                if (dd >= 0 && dd < ndm && sumsq[dd] != 0) {
                    const int32_t *row = y + (size_t)dd * n;
                    int64_t s0 = (int64_t)ct[k] + (int64_t)(b - 32) * w;
                    int64_t s = 0;
                    for (int i = 0; i < w; ++i) {
                        int64_t t = s0 + i;
                        if (t >= 0 && t < n) s += row[t];
                    }
                    double sigma = sqrt((double)sumsq[dd] / (double)n);
                    v = (float)s / snr_denominator(sigma, w);
                }
                out[((size_t)k * 64 + r) * 64 + b] = float_to_bf16_rne(v);
            }
        }
    }
    return 0;
}
