// Per-pixel arithmetic of the CUDA-core path, written once for the device
// kernel (one thread per pixel) and for host-side checks of the same code.
//
// Steps for one pixel (Section 2.1, Eq. 3-6, Algorithm 1 with missing values
// masked):
//   pass 1   masked sums of the basis functions of bfm::Basis over the
//            history dates -> Gram matrix G and X'My (normal equations, Eq. 6)
//   solve    K x K Cholesky of G, two triangular solves
//   pass 1b  one step of iterative refinement: beta += G^-1 X'M(y - X beta)
//   pass 2a  history residuals y - x'beta (sign of Eq. 3), stored compacted;
//            sigma-hat (Algorithm 1, step 5); the last h of them open the
//            first MOSUM window
//   pass 2b  monitoring residuals; the window of h valid residuals slides by
//            one add and one subtract (Algorithm 3's update, over valid
//            positions), kept as a compensated sum; first crossing of
//            lambda*sqrt(log+(j/n)) * sigma*sqrt(n) (Eq. 3-4) and the mean
#pragma once

#include <math.h>
#include <stdint.h>

#include "bfm_internal.cuh"

namespace bfm {

constexpr float kSingularRatio = 1e-5f;
constexpr float kDegenerateRatio = 1e-6f;
constexpr double kEuler = 2.71828182845904523536;

__host__ __device__ __forceinline__ float qnanf() {
#ifdef __CUDA_ARCH__
    return __int_as_float(0x7fc00000);
#else
    return NAN;
#endif
}

// Compensated (Neumaier) accumulation s += x with error term c.
__host__ __device__ __forceinline__ void comp_add(float& s, float& c, float x) {
    const float t = s + x;
    if (fabsf(s) >= fabsf(x))
        c += (s - t) + x;
    else
        c += (x - t) + s;
    s = t;
}

// Gram matrix from the masked basis sums a[] (see Basis).  Every entry is
// written explicitly in both triangles.
template <int KH>
__host__ __device__ __forceinline__ void gram_from_sums(const float (&a)[Basis<KH>::NBR],
                                                        float (&G)[Basis<KH>::K][Basis<KH>::K]) {
    using B = Basis<KH>;
    auto Cs = [&](int j) -> float { return j == 0 ? a[0] : a[B::C(j)]; };
    auto Ss = [&](int j) -> float { return j == 0 ? 0.f : (j > 0 ? a[B::S(j)] : -a[B::S(-j)]); };
    auto set = [&](int r, int c, float v) {
        G[r][c] = v;
        G[c][r] = v;
    };
    set(0, 0, a[0]);
    set(0, 1, a[1]);
    set(1, 1, a[B::TT]);
#pragma unroll
    for (int j = 1; j <= KH; ++j) {
        set(0, B::S(j), a[B::S(j)]);
        set(0, B::C(j), a[B::C(j)]);
        set(1, B::S(j), a[B::TS(j)]);
        set(1, B::C(j), a[B::TC(j)]);
#pragma unroll
        for (int b = 1; b <= KH; ++b) {
            const int dm = j > b ? j - b : b - j;
            // sin(ja)sin(ba), cos(ja)cos(ba), sin(ja)cos(ba) as single harmonics
            set(B::S(j), B::S(b), 0.5f * (Cs(dm) - Cs(j + b)));
            set(B::C(j), B::C(b), 0.5f * (Cs(dm) + Cs(j + b)));
            set(B::S(j), B::C(b), 0.5f * (Ss(j + b) + Ss(j - b)));
        }
    }
}

// In-register Cholesky G = L L' (lower; reciprocal diagonal in dinv).
// Returns false when a pivot relative to its diagonal entry is below
// kSingularRatio (the rank test).
template <int K>
__host__ __device__ __forceinline__ bool cholesky(const float (&G)[K][K], float (&L)[K][K], float (&dinv)[K]) {
    bool ok = true;
#pragma unroll
    for (int j = 0; j < K; ++j) {
        float d = G[j][j];
#pragma unroll
        for (int c = 0; c < j; ++c) d = fmaf(-L[j][c], L[j][c], d);
        ok = ok && (d >= kSingularRatio * G[j][j]) && (G[j][j] > 0.f);
        const float inv = 1.0f / sqrtf(fmaxf(d, 1e-30f));
        dinv[j] = inv;
        L[j][j] = d * inv;
#pragma unroll
        for (int i = j + 1; i < K; ++i) {
            float s = G[i][j];
#pragma unroll
            for (int c = 0; c < j; ++c) s = fmaf(-L[i][c], L[j][c], s);
            L[i][j] = s * inv;
        }
    }
    return ok;
}

template <int K>
__host__ __device__ __forceinline__ void chol_solve(const float (&L)[K][K], const float (&dinv)[K], const float (&b)[K],
                                                    float (&x)[K]) {
    float z[K];
#pragma unroll
    for (int i = 0; i < K; ++i) {
        float s = b[i];
#pragma unroll
        for (int c = 0; c < i; ++c) s = fmaf(-L[i][c], z[c], s);
        z[i] = s * dinv[i];
    }
#pragma unroll
    for (int i = K - 1; i >= 0; --i) {
        float s = z[i];
#pragma unroll
        for (int c = i + 1; c < K; ++c) s = fmaf(-L[c][i], x[c], s);
        x[i] = s * dinv[i];
    }
}

template <int KH>
struct PixelOut {
    uint8_t status;
    int32_t brk;
    float mean, sigma;
    float beta[Basis<KH>::K];
};

struct PixelParams {
    int N, n_hist;
    double h_frac;
    float lambda, c_over_s, inv_s;
};

// x_t . beta as two interleaved chains
template <int K>
__host__ __device__ __forceinline__ float dot_x(const float (&x)[K], const float (&beta)[K]) {
    float f0 = 0.f, f1 = 0.f;
#pragma unroll
    for (int i = 0; i < K; i += 2) {
        f0 = fmaf(x[i], beta[i], f0);
        f1 = fmaf(x[i + 1], beta[i + 1], f1);
    }
    return f0 + f1;
}

// obs(t, y) -> validity of date t (y set when valid); row(t, q) fills the NB
// basis values of date t; rowx(t, x) the first K of them; store_r(j, r) and
// load_r(j) hold compacted residual j (load_r only asks for j it was given
// within the last h stores).
template <int KH, class Obs, class Row, class RowX, class Store, class Load>
__host__ __device__ __forceinline__ void process_pixel(const PixelParams& P, Obs obs, Row row, RowX rowx,
                                                       Store store_r, Load load_r, PixelOut<KH>& o) {
    using B = Basis<KH>;
    constexpr int K = B::K, NB = B::NB, NBR = B::NBR;
    const int N = P.N, n_hist = P.n_hist;

    // ---- pass 1 ----
    float a[NBR], bb[K];
#pragma unroll
    for (int i = 0; i < NBR; ++i) a[i] = 0.f;
#pragma unroll
    for (int i = 0; i < K; ++i) bb[i] = 0.f;
    float ymax = 0.f;
#pragma unroll 2
    for (int t = 0; t < n_hist; ++t) {
        float y = 0.f;
        const bool v = obs(t, y);
        const float w = v ? 1.f : 0.f, yw = v ? y : 0.f;
        ymax = fmaxf(ymax, fabsf(yw));
        float q[NB];
        row(t, q);
        a[0] += w;
#pragma unroll
        for (int l = 1; l < NBR; ++l) a[l] = fmaf(w, q[l], a[l]);
        bb[0] += yw;
#pragma unroll
        for (int i = 1; i < K; ++i) bb[i] = fmaf(yw, q[i], bb[i]);
    }
    const int n_i = (int)a[0];

    // ---- solve ----
    float G[K][K], L[K][K], dinv[K], beta[K];
    gram_from_sums<KH>(a, G);
    const bool nonsingular = cholesky<K>(G, L, dinv);
    chol_solve<K>(L, dinv, bb, beta);

    // ---- pass 1b: one refinement step ----
    {
        float cc[K];
#pragma unroll
        for (int i = 0; i < K; ++i) cc[i] = 0.f;
#pragma unroll 2
        for (int t = 0; t < n_hist; ++t) {
            float y = 0.f;
            const bool v = obs(t, y);
            float x[K];
            rowx(t, x);
            const float r = v ? (y - dot_x<K>(x, beta)) : 0.f;
#pragma unroll
            for (int i = 0; i < K; ++i) cc[i] = fmaf(r, x[i], cc[i]);
        }
        float dl[K];
        chol_solve<K>(L, dinv, cc, dl);
#pragma unroll
        for (int i = 0; i < K; ++i) beta[i] += dl[i];
    }

    int h = (int)floor(P.h_frac * (double)n_i);
    if (h < 1) h = 1;
    if (h > n_i) h = n_i;  // 0 when n_i = 0: every index below stays >= 0
    const int wstart = n_i - h;

    // ---- pass 2a ----
    int j = 0;
    float ss = 0.f, W = 0.f, Wc = 0.f;
#pragma unroll 2
    for (int t = 0; t < n_hist; ++t) {
        float y = 0.f;
        const bool v = obs(t, y);
        float x[K];
        rowx(t, x);
        const float r = y - dot_x<K>(x, beta);
        if (v) {
            ss = fmaf(r, r, ss);
            store_r(j, r);
            if (j >= wstart) comp_add(W, Wc, r);
            ++j;
        }
    }
    const float sigma = sqrtf(ss / (float)(n_i - K));
    const bool degenerate = !(sigma > kDegenerateRatio * ymax) || ymax == 0.f;
    const float scale = sigma * sqrtf((float)n_i);
    const float thr = P.lambda * scale;
    const int jlim = (int)floor(kEuler * (double)n_i);  // j/n_i <= e  <=>  j <= jlim

    // ---- pass 2b ----
    int brk = -1;
    float sumW = 0.f, sumWc = 0.f;
#pragma unroll 2
    for (int t = n_hist; t < N; ++t) {
        float y = 0.f;
        const bool v = obs(t, y);
        float x[K];
        rowx(t, x);
        const float r = y - dot_x<K>(x, beta);
        if (v) {
            const float lag = load_r(j - h);
            store_r(j, r);
            comp_add(W, Wc, r - lag);
            const float wv = W + Wc;
            const int J = j + 1;  // 1-based position of this observation
            float th = thr;
            if (J > jlim) th = thr * sqrtf(logf((float)J / (float)n_i));
            if (brk < 0 && fabsf(wv) > th) brk = t;
            comp_add(sumW, sumWc, wv);
            ++j;
        }
    }
    const int N_i = j;

    const float qnan = qnanf();
    bool fitted = true;
    o.brk = -1;
    o.sigma = sigma;
    if (n_i <= K) {
        o.status = BFM_PX_INSUFFICIENT_HISTORY;
        fitted = false;
    } else if (!nonsingular) {
        o.status = BFM_PX_SINGULAR;
        fitted = false;
    } else if (degenerate) {
        o.status = BFM_PX_DEGENERATE;
        o.mean = 0.f;
    } else if (N_i == n_i) {
        o.status = BFM_PX_NO_MONITOR;
        o.mean = qnan;
    } else {
        o.status = BFM_PX_OK;
        o.brk = brk;
        o.mean = (sumW + sumWc) / ((float)(N_i - n_i) * scale);
    }
    if (!fitted) {
        o.mean = qnan;
        o.sigma = qnan;
    }
    // beta of the centred trend -> raw parameterisation of Eq. 2
#pragma unroll
    for (int i = 0; i < K; ++i) o.beta[i] = fitted ? beta[i] : qnan;
    if (fitted) {
        o.beta[0] = fmaf(-beta[1], P.c_over_s, beta[0]);
        o.beta[1] = beta[1] * P.inv_s;
    }
}

}  // namespace bfm
