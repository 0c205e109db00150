/*
 * FP64 oracle for the BFAST Monitor per-pixel path.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
 * CUDA path is checked against.  Only the tests, the package smoke check and
 * the benchmark's CPU-baseline leg may load it.  It shares no code, header or
 * table with the CUDA library.
 *
 * What it computes, per pixel p (time series y_1..y_N of one pixel):
 *   1. Keep the valid (cloud-free) observations in date order; n_p of them
 *      fall in the stable history (date index < n_hist), N_p in total.
 *   2. Regressors x_t of the season-trend model (Section 2.1, Eq. 1-2):
 *      x_t = (1, t, sin(2 pi t/f), cos(2 pi t/f), ..., sin(2 pi k t/f),
 *      cos(2 pi k t/f)), K = 2 + 2k, with t the actual date value.
 *   3. Ordinary least squares on the history (Eq. 5-6), solved by Householder
 *      QR (no normal equations).
 *   4. Residuals y_t - x_t' beta for every valid observation (sign of Eq. 3).
 *   5. sigma-hat = sqrt(sum of squared history residuals / (n_p - K))
 *      (Algorithm 1, step 5).
 *   6. MOSUM with bandwidth h_p = clamp(floor(h_frac * n_p), 1, n_p) over the
 *      valid observations (Eq. 3): for j = n_p+1 .. N_p,
 *      MO_j = sum_{s=j-h_p+1..j} r_s / (sigma-hat * sqrt(n_p)), by direct sums.
 *   7. Boundary b_j = lambda * sqrt(log+(j/n_p)) (Eq. 4), log+ x = 1 for x <= e.
 *   8. Break = original date index of the first j with |MO_j| > b_j (strict,
 *      Algorithm 1, step 12), else -1.  Mean MOSUM = mean of MO_j.
 *
 * Readings where the paper is silent (the complete-series case is unchanged):
 *   - missing values: positions j, n and h count valid observations only;
 *   - n_p <= K: status INSUFFICIENT_HISTORY (outputs NaN / -1);
 *   - rank test: with the trend column written as (t - c)/s (c, s the midpoint
 *     and half-range of the date set), QR of the history design gives R; the
 *     pixel is SINGULAR when min_k R_kk^2 / ||column k||^2 < 1e-5;
 *   - sigma-hat <= 1e-6 * max |y_hist| (or max = 0): DEGENERATE, MO = 0, no
 *     break, mean 0;
 *   - N_p = n_p: NO_MONITOR, mean NaN, no break.
 *
 * Also: the critical value lambda by Monte-Carlo of the limiting MOSUM
 * process Z(t) = W(t) - W(t-h) - h W(1) on t in [1, T] (lambda depends on
 * alpha, h and the horizon T = N/n, Section 2.1 after Eq. 4).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_PI 3.14159265358979323846
#define OR_E 2.71828182845904523536

enum { OR_OK = 0, OR_INSUFFICIENT = 1, OR_SINGULAR = 2, OR_DEGENERATE = 3, OR_NO_MONITOR = 4 };

/* Eq. 2: regressor vector for date value t */
static void eq2_regressors(double t, int k, double f, double *x) {
    x[0] = 1.0;
    x[1] = t;
    for (int j = 1; j <= k; ++j) {
        double a = 2.0 * OR_PI * (double)j * t / f;
        x[2 * j] = sin(a);
        x[2 * j + 1] = cos(a);
    }
}

/* Design matrix X (row t = x_t, Algorithm 1 step 1), row-major [N][K]. */
void oracle_design(const double *dates, int N, int k, double f, double *X) {
    int K = 2 + 2 * k;
    for (int t = 0; t < N; ++t) eq2_regressors(dates[t], k, f, X + (size_t)t * K);
}

/*
 * Least squares min ||A b - y|| by Householder QR (A: n x K, row-major, n >= K;
 * both are overwritten).  rdiag receives the diagonal of R.  Returns 0, or 1
 * when a column is exactly dependent (zero R_kk), in which case beta is NaN.
 */
int oracle_lstsq_qr(int n, int K, double *A, double *y, double *beta, double *rdiag) {
    int dep = 0;
    for (int j = 0; j < K; ++j) {
        double ss = 0.0;
        for (int i = j; i < n; ++i) ss += A[(size_t)i * K + j] * A[(size_t)i * K + j];
        double nrm = sqrt(ss);
        if (nrm == 0.0) {
            rdiag[j] = 0.0;
            dep = 1;
            continue;
        }
        double ajj = A[(size_t)j * K + j];
        double alpha = (ajj > 0.0) ? -nrm : nrm; /* reflect onto -sign(ajj)*||x|| e1 */
        double v0 = ajj - alpha;
        double vtv = v0 * v0 + (ss - ajj * ajj);
        /* Householder vector v = (v0, A[j+1..n-1][j]) */
        for (int c = j + 1; c < K; ++c) {
            double s = v0 * A[(size_t)j * K + c];
            for (int i = j + 1; i < n; ++i) s += A[(size_t)i * K + j] * A[(size_t)i * K + c];
            double g = 2.0 * s / vtv;
            A[(size_t)j * K + c] -= g * v0;
            for (int i = j + 1; i < n; ++i) A[(size_t)i * K + c] -= g * A[(size_t)i * K + j];
        }
        {
            double s = v0 * y[j];
            for (int i = j + 1; i < n; ++i) s += A[(size_t)i * K + j] * y[i];
            double g = 2.0 * s / vtv;
            y[j] -= g * v0;
            for (int i = j + 1; i < n; ++i) y[i] -= g * A[(size_t)i * K + j];
        }
        A[(size_t)j * K + j] = alpha;
        rdiag[j] = alpha;
    }
    if (dep) {
        for (int j = 0; j < K; ++j) beta[j] = NAN;
        return 1;
    }
    for (int j = K - 1; j >= 0; --j) {
        double s = y[j];
        for (int c = j + 1; c < K; ++c) s -= A[(size_t)j * K + c] * beta[c];
        beta[j] = s / A[(size_t)j * K + j];
    }
    return 0;
}

/*
 * Least squares through the normal equations of Eq. 6: G = A'A and A'y as
 * plain sums, Cholesky G = L L', two triangular solves.  Used only to cross-
 * check the QR path.  Returns 1 if a pivot is not positive.
 */
int oracle_lstsq_normal(int n, int K, const double *A, const double *y, double *beta) {
    double G[16 * 16], L[16 * 16], b[16], z[16];
    if (K > 16) return 2;
    for (int a = 0; a < K; ++a) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += A[(size_t)i * K + a] * y[i];
        b[a] = s;
        for (int c = 0; c < K; ++c) {
            double g = 0.0;
            for (int i = 0; i < n; ++i) g += A[(size_t)i * K + a] * A[(size_t)i * K + c];
            G[a * K + c] = g;
        }
    }
    memset(L, 0, sizeof(L));
    for (int j = 0; j < K; ++j) {
        double d = G[j * K + j];
        for (int c = 0; c < j; ++c) d -= L[j * K + c] * L[j * K + c];
        if (!(d > 0.0)) return 1;
        L[j * K + j] = sqrt(d);
        for (int i = j + 1; i < K; ++i) {
            double s = G[i * K + j];
            for (int c = 0; c < j; ++c) s -= L[i * K + c] * L[j * K + c];
            L[i * K + j] = s / L[j * K + j];
        }
    }
    for (int i = 0; i < K; ++i) {
        double s = b[i];
        for (int c = 0; c < i; ++c) s -= L[i * K + c] * z[c];
        z[i] = s / L[i * K + i];
    }
    for (int i = K - 1; i >= 0; --i) {
        double s = z[i];
        for (int c = i + 1; c < K; ++c) s -= L[c * K + i] * beta[c];
        beta[i] = s / L[i * K + i];
    }
    return 0;
}

/* log+ of Eq. 4 */
double oracle_logplus(double x) { return (x <= OR_E) ? 1.0 : log(x); }

/* boundary b_j of Eq. 4 at monitoring position j with history size n */
double oracle_boundary(double lambda, int j, int n) {
    return lambda * sqrt(oracle_logplus((double)j / (double)n));
}

/*
 * The monitoring path for m pixels.
 *   Y:     [N][m] values (double), valid: [N][m] 0/1.
 *   out:   brk[m] int32, mean_mo[m], sigma[m], beta[K][m], status[m] uint8,
 *          n_p[m], N_p[m], h_p[m] int32, margin[m] = min over the monitoring
 *          positions up to the break (all of them without a break) of
 *          | |MO_j| - b_j |, mo_trace (nullable) [m][N]: MO of the monitoring
 *          positions in order (NaN after the last).
 */
void oracle_monitor(int64_t m, int N, const double *dates, int k, double f, const double *Y,
                    const uint8_t *valid, int n_hist, double h_frac, double lambda, int32_t *brk,
                    double *mean_mo, double *sigma, double *beta, uint8_t *status, int32_t *n_out,
                    int32_t *Nv_out, int32_t *h_out, double *margin, double *mo_trace) {
    const int K = 2 + 2 * k;
    const double c = 0.5 * (dates[0] + dates[N - 1]);
    const double s = (N > 1 && dates[N - 1] > dates[0]) ? 0.5 * (dates[N - 1] - dates[0]) : 1.0;
#pragma omp parallel
    {
        int *idx = (int *)malloc(sizeof(int) * (size_t)N);
        double *A = (double *)malloc(sizeof(double) * (size_t)N * (size_t)K);
        double *yv = (double *)malloc(sizeof(double) * (size_t)N);
        double *r = (double *)malloc(sizeof(double) * (size_t)N);
        double x[16], bt[16], rd[16];
#pragma omp for schedule(dynamic, 64)
        for (int64_t p = 0; p < m; ++p) {
            int Np = 0, np = 0;
            for (int t = 0; t < N; ++t)
                if (valid[(size_t)t * (size_t)m + (size_t)p]) {
                    idx[Np++] = t;
                    if (t < n_hist) ++np;
                }
            n_out[p] = np;
            Nv_out[p] = Np;
            brk[p] = -1;
            margin[p] = INFINITY;
            if (mo_trace)
                for (int j = 0; j < N; ++j) mo_trace[(size_t)p * N + j] = NAN;
            int hp = (int)floor(h_frac * (double)np);
            if (hp < 1) hp = 1;
            if (hp > np) hp = np;
            h_out[p] = hp;
            for (int a = 0; a < K; ++a) beta[(size_t)a * m + p] = NAN;
            sigma[p] = NAN;
            mean_mo[p] = NAN;
            if (np <= K) {
                status[p] = OR_INSUFFICIENT;
                continue;
            }
            /* rank test on the design with the trend column (t - c)/s */
            double colss[16];
            for (int a = 0; a < K; ++a) colss[a] = 0.0;
            for (int j = 0; j < np; ++j) {
                eq2_regressors(dates[idx[j]], k, f, x);
                x[1] = (dates[idx[j]] - c) / s;
                for (int a = 0; a < K; ++a) {
                    A[(size_t)j * K + a] = x[a];
                    colss[a] += x[a] * x[a];
                }
                yv[j] = 0.0;
            }
            oracle_lstsq_qr(np, K, A, yv, bt, rd);
            double minratio = INFINITY;
            for (int a = 0; a < K; ++a) {
                double ratio = (colss[a] > 0.0) ? rd[a] * rd[a] / colss[a] : 0.0;
                if (ratio < minratio) minratio = ratio;
            }
            if (!(minratio >= 1e-5)) {
                status[p] = OR_SINGULAR;
                continue;
            }
            /* Eq. 5-6: least squares on the raw Eq. 2 design by Householder QR */
            double ymax = 0.0;
            for (int j = 0; j < np; ++j) {
                eq2_regressors(dates[idx[j]], k, f, A + (size_t)j * K);
                yv[j] = Y[(size_t)idx[j] * (size_t)m + (size_t)p];
                if (fabs(yv[j]) > ymax) ymax = fabs(yv[j]);
            }
            oracle_lstsq_qr(np, K, A, yv, bt, rd);
            for (int a = 0; a < K; ++a) beta[(size_t)a * m + p] = bt[a];
            /* residuals y - x'beta for every valid observation (Eq. 3) */
            for (int j = 0; j < Np; ++j) {
                eq2_regressors(dates[idx[j]], k, f, x);
                double fit = 0.0;
                for (int a = 0; a < K; ++a) fit += x[a] * bt[a];
                r[j] = Y[(size_t)idx[j] * (size_t)m + (size_t)p] - fit;
            }
            double ss = 0.0;
            for (int j = 0; j < np; ++j) ss += r[j] * r[j];
            double sg = sqrt(ss / (double)(np - K));
            sigma[p] = sg;
            if (!(sg > 1e-6 * ymax) || ymax == 0.0) {
                status[p] = OR_DEGENERATE;
                mean_mo[p] = 0.0;
                continue;
            }
            if (Np == np) {
                status[p] = OR_NO_MONITOR;
                continue;
            }
            status[p] = OR_OK;
            double scale = sg * sqrt((double)np);
            double sum_mo = 0.0, mg = INFINITY;
            int found = 0;
            for (int j = np + 1; j <= Np; ++j) { /* 1-based monitoring position */
                double w = 0.0;
                for (int q = j - hp + 1; q <= j; ++q) w += r[q - 1];
                double mo = w / scale;
                double b = oracle_boundary(lambda, j, np);
                sum_mo += mo;
                if (mo_trace) mo_trace[(size_t)p * N + (j - np - 1)] = mo;
                if (!found) {
                    double d = fabs(fabs(mo) - b);
                    if (d < mg) mg = d;
                    if (fabs(mo) > b) {
                        found = 1;
                        brk[p] = idx[j - 1];
                    }
                }
            }
            mean_mo[p] = sum_mo / (double)(Np - np);
            margin[p] = mg;
        }
        free(idx);
        free(A);
        free(yv);
        free(r);
    }
}

/* ---- critical value by simulation ------------------------------------- */

static inline uint64_t or_sm64(uint64_t *st) {
    uint64_t z = (*st += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static inline double or_normal(uint64_t *st) {
    double u1 = ((double)(or_sm64(st) >> 11) + 1.0) * 0x1.0p-53;
    double u2 = (double)(or_sm64(st) >> 11) * 0x1.0p-53;
    return sqrt(-2.0 * log(u1)) * cos(2.0 * OR_PI * u2);
}

static int cmp_double(const void *a, const void *b) {
    double x = *(const double *)a, y = *(const double *)b;
    return (x < y) ? -1 : (x > y);
}

/*
 * sup_{t in [1, T]} |W(t) - W(t-h) - h W(1)| / sqrt(log+ t) for `reps`
 * Brownian paths sampled on a grid of G steps per unit; stats[reps] receives
 * the suprema, the return value is their (1 - alpha) empirical quantile.
 */
double oracle_lambda(double alpha, double h, double T, int G, int reps, uint64_t seed, double *stats) {
    int nsteps = (int)llround(T * (double)G);
    int ih = (int)llround(h * (double)G);
    double *st = stats ? stats : (double *)malloc(sizeof(double) * (size_t)reps);
#pragma omp parallel
    {
        double *W = (double *)malloc(sizeof(double) * (size_t)(nsteps + 1));
        double sd = 1.0 / sqrt((double)G);
#pragma omp for schedule(static)
        for (int rr = 0; rr < reps; ++rr) {
            uint64_t s = seed * 0xA0761D6478BD642FULL + (uint64_t)rr * 0xE7037ED1A0B428DBULL + 1ULL;
            or_sm64(&s);
            W[0] = 0.0;
            for (int i = 1; i <= nsteps; ++i) W[i] = W[i - 1] + sd * or_normal(&s);
            double w1 = W[G], best = 0.0;
            for (int i = G; i <= nsteps; ++i) {
                double tt = (double)i / (double)G;
                double z = W[i] - W[i - ih] - h * w1;
                double v = fabs(z) / sqrt(oracle_logplus(tt));
                if (v > best) best = v;
            }
            st[rr] = best;
        }
        free(W);
    }
    double *srt = (double *)malloc(sizeof(double) * (size_t)reps);
    memcpy(srt, st, sizeof(double) * (size_t)reps);
    qsort(srt, (size_t)reps, sizeof(double), cmp_double);
    long q = (long)ceil((1.0 - alpha) * (double)reps) - 1;
    if (q < 0) q = 0;
    if (q >= reps) q = reps - 1;
    double lam = srt[q];
    free(srt);
    if (!stats) free(st);
    return lam;
}
