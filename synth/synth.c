/*
 * Seeded synthetic NDVI-like scenes for BFAST Monitor workloads.
 *
 * This file only draws inputs: acquisition dates, a season-trend signal with
 * noise, a cloud (missing-value) pattern and injected level shifts.  It holds
 * none of the monitoring method's arithmetic (no design matrix, no fit, no
 * MOSUM).  Both the CUDA path's tests/benchmark and the FP64 oracle's tests
 * take their inputs from here.
 *
 * Random numbers: SplitMix64 (Steele, Lea & Flood, OOPSLA 2014), one stream
 * per pixel keyed by (seed, pixel), so a scene does not depend on the number
 * of threads that generate it.  Normals by the Box-Muller transform.
 *
 * Layout of Y: time-major [N][m] (row t holds date t for all m pixels), the
 * layout of the paper's matrix Y (Section 3, Eq. 7).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define SYN_PI 3.14159265358979323846

static inline uint64_t sm64_next(uint64_t *s) {
    uint64_t z = (*s += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* uniform in [0, 1) with 53 random bits */
static inline double u01(uint64_t *s) { return (double)(sm64_next(s) >> 11) * 0x1.0p-53; }

/* uniform in (0, 1] */
static inline double u01_open0(uint64_t *s) { return ((double)(sm64_next(s) >> 11) + 1.0) * 0x1.0p-53; }

static inline double normal01(uint64_t *s) {
    double u1 = u01_open0(s), u2 = u01(s);
    return sqrt(-2.0 * log(u1)) * cos(2.0 * SYN_PI * u2);
}

static inline uint64_t stream_seed(uint64_t seed, uint64_t key) {
    uint64_t s = seed ^ 0x6A09E667F3BCC909ULL;
    uint64_t a = sm64_next(&s);
    uint64_t b = key * 0xD1B54A32D192ED03ULL + 0x9E3779B97F4A7C15ULL;
    uint64_t t = a ^ b;
    return sm64_next(&t);
}

/* dates t_i = (16*i + U{-3..3}) / 16 for i = 1..N: a 16-day revisit with a
 * few days of jitter, in units of the revisit interval (23 per year). */
void synth_dates(uint64_t seed, int N, double *dates) {
    uint64_t s = stream_seed(seed, 0xDA7E5ULL);
    for (int i = 0; i < N; ++i) {
        int jitter = (int)(sm64_next(&s) % 7ULL) - 3;
        dates[i] = (16.0 * (double)(i + 1) + (double)jitter) / 16.0;
    }
}

/*
 * One scene.
 *   k_gen harmonics in the signal; coef_fixed (2*k_gen values, sin/cos of
 *   harmonic j at [2j], [2j+1]) or, if NULL, each coefficient ~ U(0, coef_umax).
 *   miss_kind: 0 none, 1 i.i.d. with probability p_a, 2 two-state Markov chain
 *   with P(missing -> clear) = p_a and P(clear -> missing) = p_b, first state
 *   from the stationary law.
 *   A fraction break_frac of pixels gets a level shift ~ U(step_lo, step_hi)
 *   from a date index drawn uniformly from [n_hist, N) onwards.
 * Outputs (each nullable): Yf float [N][m] (NaN = missing), Yi int16 [N][m]
 * (round(y*1e4), -32768 = missing), brk int32 [m] (shift date index or -1).
 */
void synth_scene(uint64_t seed, int64_t m, int N, const double *dates, double f, int n_hist,
                 int k_gen, double intercept, double slope, const double *coef_fixed,
                 double coef_umax, double noise_sd, int miss_kind, double p_a, double p_b,
                 double break_frac, double step_lo, double step_hi, float *Yf, int16_t *Yi,
                 int32_t *brk) {
    double *harm = (double *)malloc(sizeof(double) * (size_t)N * (size_t)(2 * k_gen + 1));
    for (int t = 0; t < N; ++t)
        for (int j = 1; j <= k_gen; ++j) {
            double a = 2.0 * SYN_PI * (double)j * dates[t] / f;
            harm[(size_t)t * (2 * k_gen + 1) + 2 * (j - 1)] = sin(a);
            harm[(size_t)t * (2 * k_gen + 1) + 2 * (j - 1) + 1] = cos(a);
        }
    const int64_t B = 256;
    const int64_t nblk = (m + B - 1) / B;
#pragma omp parallel
    {
        uint64_t st[256];
        double coef[256][6];
        int32_t bdate[256];
        double step[256];
        int state[256];
#pragma omp for schedule(static)
        for (int64_t blk = 0; blk < nblk; ++blk) {
            int64_t p0 = blk * B;
            int64_t nb = (m - p0 < B) ? (m - p0) : B;
            for (int64_t q = 0; q < nb; ++q) {
                uint64_t *s = &st[q];
                *s = stream_seed(seed, (uint64_t)(p0 + q) + 1ULL);
                for (int j = 0; j < 2 * k_gen && j < 6; ++j)
                    coef[q][j] = coef_fixed ? coef_fixed[j] : coef_umax * u01(s);
                double ub = u01(s);
                int64_t span = (int64_t)N - (int64_t)n_hist;
                int32_t bd = (int32_t)n_hist + (int32_t)(span > 0 ? (int64_t)(sm64_next(s) % (uint64_t)span) : 0);
                double stp = step_lo + (step_hi - step_lo) * u01(s);
                bdate[q] = (ub < break_frac && span > 0) ? bd : -1;
                step[q] = stp;
                double pi_miss = (p_a + p_b > 0.0) ? p_b / (p_a + p_b) : 0.0;
                state[q] = (miss_kind == 2) ? (u01(s) < pi_miss) : 0;
                if (brk) brk[p0 + q] = bdate[q];
            }
            for (int t = 0; t < N; ++t) {
                const double *h = harm + (size_t)t * (2 * k_gen + 1);
                double base = intercept + slope * dates[t];
                for (int64_t q = 0; q < nb; ++q) {
                    uint64_t *s = &st[q];
                    int miss;
                    if (miss_kind == 1) {
                        miss = u01(s) < p_a;
                    } else if (miss_kind == 2) {
                        if (t > 0) {
                            double u = u01(s);
                            state[q] = state[q] ? !(u < p_a) : (u < p_b);
                        }
                        miss = state[q];
                    } else {
                        miss = 0;
                    }
                    double y = base;
                    for (int j = 0; j < 2 * k_gen && j < 6; ++j) y += coef[q][j] * h[j];
                    y += noise_sd * normal01(s);
                    if (bdate[q] >= 0 && t >= bdate[q]) y += step[q];
                    size_t o = (size_t)t * (size_t)m + (size_t)(p0 + q);
                    if (Yf) Yf[o] = miss ? NAN : (float)y;
                    if (Yi) {
                        double v = nearbyint(y * 1e4);
                        if (v > 32767.0) v = 32767.0;
                        if (v < -32767.0) v = -32767.0;
                        Yi[o] = miss ? (int16_t)-32768 : (int16_t)v;
                    }
                }
            }
        }
    }
    free(harm);
}
