// Per-pixel arithmetic of the CUDA-core path, split into phases that NW
// warps run on one 32-pixel tile.  Lane = pixel; warp w owns a contiguous
// segment of the history dates (phases 1 and 3) and of all dates (phases
// 5 to 7).  Warps exchange per-pixel partial results through a shared
// buffer between phases; every phase writes only locations no other warp
// reads during that phase, so a barrier between phases is the only
// synchronisation.  The functions are __host__ __device__ so the same code
// can be run warp by warp on the host.
//
// Steps for one pixel (Section 2.1, Eq. 3-6, Algorithm 1 with missing values
// masked; readings of the paper as in the library header):
//   1  masked sums of the basis functions of bfm::Basis over the history
//      -> Gram matrix G and X'My (normal equations, Eq. 6)        [segments]
//   2  Cholesky of G, solve for beta0                                [every warp]
//   3  refinement sums c = X'M(y - X beta0), s0 = sum r0^2          [segments]
//   4  beta = beta0 + G^-1 c; sum of squared history residuals
//      s1 = s0 - delta'c (residuals y - x'beta are orthogonal to X), sigma-hat
//      (Algorithm 1, step 5)                                         [every warp]
//   5  residuals r = y - x'beta (sign of Eq. 3) at every valid date and their
//      compacted prefix sums within the segment, stored in the segment's own
//      slots; segment count, sum and validity words                 [segments]
//   6  segment offsets (exclusive sums of counts and sums)           [every warp]
//   7  MOSUM MO_J = (S_J - S_{J-h}) / (sigma sqrt(n)) for monitoring J, with
//      S_J = r_1 + ... + r_J over valid positions (Eq. 3, window of h valid
//      residuals); first J with |MO_J| > lambda sqrt(log+(J/n)) (Eq. 4,
//      strict) and the sum of MO_J                                   [segments]
//   8  combine: earliest crossing, mean MOSUM, status, outputs       [one warp]
#pragma once

#include <math.h>
#include <stdint.h>

#include "bfm_internal.cuh"

namespace bfm {

constexpr float kSingularRatio = 1e-5f;
constexpr float kDegenerateRatio = 1e-6f;
constexpr double kEuler = 2.71828182845904523536;
constexpr int kNW = 4;  // warps (date segments) per 32-pixel tile

constexpr float kLn2f = 0.693147180559945309f;

// log2 for the boundary of Eq. 4: the hardware approximation on the device
// (absolute error near 2^-22 for these arguments), the library function on the host.
__host__ __device__ __forceinline__ float log2_fast(float x) {
#ifdef __CUDA_ARCH__
    return __log2f(x);
#else
    return log2f(x);
#endif
}

__host__ __device__ __forceinline__ float qnanf() {
#ifdef __CUDA_ARCH__
    return __int_as_float(0x7fc00000);
#else
    return NAN;
#endif
}

// Compensated (Kahan) accumulation s += x with error term c (s + c is the sum).
__host__ __device__ __forceinline__ void comp_add(float& s, float& c, float x) {
    const float y = x + c;
    const float t = s + y;
    c = y - (t - s);
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

struct SegParams {
    int N, n_hist;
    double h_frac;
    float lambda, c_over_s, inv_s;
};

// contiguous segment w of [0, n) split into kNW parts
__host__ __device__ __forceinline__ void segment(int n, int w, int& s0, int& s1) {
    const int L = (n + kNW - 1) / kNW;
    s0 = w * L < n ? w * L : n;
    s1 = s0 + L < n ? s0 + L : n;
}

// Validity words per segment kept in the partials buffer (segments of up to
// 32 * kSegWords dates, i.e. N <= kNW * 32 * kSegWords).
constexpr int kSegWords = 14;

// Floats per lane and warp in the partials buffer: the phase-1 sums
// (a[], bb[], ymax), or count/sum/crossing fields plus validity words.
template <int KH>
struct Partials {
    static constexpr int kGram = Basis<KH>::NBR + Basis<KH>::K + 1;
    static constexpr int kMaxMo = 3 + kSegWords;  // phase 7: the segment's MO of largest magnitude
    static constexpr int kStride = kGram > kMaxMo + 1 ? kGram : kMaxMo + 1;
};

// Per-lane state carried across phases (registers on the device).
template <int KH>
struct Lane {
    static constexpr int K = Basis<KH>::K;
    float beta[K];
    float L[K][K];
    float dinv[K];
    float ymax;
    int n_i;
    bool nonsingular;
    float sigma, scale, inv_scale, lam2, lg_n;
    int h, jlim;
    // segment bookkeeping of phases 5-7
    int cnt_off[kNW];                  // valid observations before each all-date segment
    float sum_off_hi[kNW], sum_off_lo[kNW];  // residual sums before each segment
    int mycnt, myoff;                  // this warp's segment: valid observations, and before it
    int N_i;
};

// PART(w, i) -> float& : partial slot i of warp w for this lane.

// ---- phase 1: masked basis sums over this warp's history segment -------------------
template <int KH, class Obs, class Row, class Part>
__host__ __device__ __forceinline__ void phase1_gram(const SegParams& P, int w, Obs obs, Row row, Part part) {
    using B = Basis<KH>;
    constexpr int K = B::K, NB = B::NB, NBR = B::NBR;
    int s0, s1;
    segment(P.n_hist, w, s0, s1);
    float a[NBR], bb[K];
#pragma unroll
    for (int i = 0; i < NBR; ++i) a[i] = 0.f;
#pragma unroll
    for (int i = 0; i < K; ++i) bb[i] = 0.f;
    float ymax = 0.f;
#pragma unroll 2
    for (int t = s0; t < s1; ++t) {
        float y = 0.f;
        const bool v = obs(t, y);
        const float wt = v ? 1.f : 0.f, yw = v ? y : 0.f;
        ymax = fmaxf(ymax, fabsf(yw));
        float q[NB];
        row(t, q);
        a[0] += wt;
#pragma unroll
        for (int l = 1; l < NBR; ++l) a[l] = fmaf(wt, q[l], a[l]);
        bb[0] += yw;
#pragma unroll
        for (int i = 1; i < K; ++i) bb[i] = fmaf(yw, q[i], bb[i]);
    }
#pragma unroll
    for (int i = 0; i < NBR; ++i) part(w, i) = a[i];
#pragma unroll
    for (int i = 0; i < K; ++i) part(w, NBR + i) = bb[i];
    part(w, NBR + K) = ymax;
}

// ---- phase 2: combine, Cholesky, beta0 -------------------------------------------
template <int KH, class Part>
__host__ __device__ __forceinline__ void phase2_solve(Lane<KH>& S, Part part) {
    using B = Basis<KH>;
    constexpr int K = B::K, NBR = B::NBR;
    float a[NBR], bb[K];
    float ymax = 0.f;
#pragma unroll
    for (int i = 0; i < NBR; ++i) a[i] = 0.f;
#pragma unroll
    for (int i = 0; i < K; ++i) bb[i] = 0.f;
#pragma unroll
    for (int w = 0; w < kNW; ++w) {
#pragma unroll
        for (int i = 0; i < NBR; ++i) a[i] += part(w, i);
#pragma unroll
        for (int i = 0; i < K; ++i) bb[i] += part(w, NBR + i);
        ymax = fmaxf(ymax, part(w, NBR + K));
    }
    S.n_i = (int)a[0];
    S.ymax = ymax;
    float G[K][K];
    gram_from_sums<KH>(a, G);
    S.nonsingular = cholesky<K>(G, S.L, S.dinv);
    chol_solve<K>(S.L, S.dinv, bb, S.beta);
}

// ---- phase 3: refinement sums over this warp's history segment ------------------
template <int KH, class Obs, class RowX, class Part>
__host__ __device__ __forceinline__ void phase3_refine(const SegParams& P, int w, const Lane<KH>& S, Obs obs,
                                                       RowX rowx, Part part) {
    constexpr int K = Basis<KH>::K;
    int s0, s1;
    segment(P.n_hist, w, s0, s1);
    float cc[K];
#pragma unroll
    for (int i = 0; i < K; ++i) cc[i] = 0.f;
    float ss = 0.f;
#pragma unroll 2
    for (int t = s0; t < s1; ++t) {
        float y = 0.f;
        const bool v = obs(t, y);
        float x[K];
        rowx(t, x);
        const float r = v ? (y - dot_x<K>(x, S.beta)) : 0.f;
        ss = fmaf(r, r, ss);
#pragma unroll
        for (int i = 0; i < K; ++i) cc[i] = fmaf(r, x[i], cc[i]);
    }
#pragma unroll
    for (int i = 0; i < K; ++i) part(w, i) = cc[i];
    part(w, K) = ss;
}

// ---- phase 4: refined beta, sigma-hat, bandwidth ---------------------------------
template <int KH, class Part>
__host__ __device__ __forceinline__ void phase4_sigma(const SegParams& P, Lane<KH>& S, Part part) {
    constexpr int K = Basis<KH>::K;
    float cc[K], ss = 0.f;
#pragma unroll
    for (int i = 0; i < K; ++i) cc[i] = 0.f;
#pragma unroll
    for (int w = 0; w < kNW; ++w) {
#pragma unroll
        for (int i = 0; i < K; ++i) cc[i] += part(w, i);
        ss += part(w, K);
    }
    float dl[K];
    chol_solve<K>(S.L, S.dinv, cc, dl);
    float dc = 0.f;
#pragma unroll
    for (int i = 0; i < K; ++i) {
        S.beta[i] += dl[i];
        dc = fmaf(dl[i], cc[i], dc);
    }
    const float s1 = fmaxf(ss - dc, 0.f);
    const int n_i = S.n_i;
    S.sigma = sqrtf(s1 / (float)(n_i - K));
    S.scale = S.sigma * sqrtf((float)n_i);
    S.inv_scale = 1.f / S.scale;
    S.lam2 = P.lambda * P.lambda;
    S.lg_n = log2f((float)n_i);
    int h = (int)floor(P.h_frac * (double)n_i);
    if (h < 1) h = 1;
    if (h > n_i) h = n_i;  // 0 when n_i = 0
    S.h = h;
    S.jlim = (int)floor(kEuler * (double)n_i);  // J/n_i <= e  <=>  J <= jlim
}

// ---- phase 5: residuals, segment-local compacted prefix sums ------------------------
// put_s(slot, v) writes slot (always <= the date being read, inside the
// segment); putw(w, i, bits) stores validity word i of this warp's segment.
template <int KH, class Obs, class RowX, class PutS, class Part, class PutW>
__host__ __device__ __forceinline__ void phase5_resid(const SegParams& P, int w, const Lane<KH>& S, Obs obs,
                                                      RowX rowx, PutS put_s, Part part, PutW putw) {
    constexpr int K = Basis<KH>::K;
    int s0, s1;
    segment(P.N, w, s0, s1);
    int jl = 0;
    float sh = 0.f, sl = 0.f;
    uint32_t bits = 0u;
#pragma unroll 2
    for (int t = s0; t < s1; ++t) {
        float y = 0.f;
        const bool v = obs(t, y);
        float x[K];
        rowx(t, x);
        const float r = y - dot_x<K>(x, S.beta);
        if (v) {
            comp_add(sh, sl, r);
            put_s(s0 + jl, sh + sl);
            ++jl;
        }
        bits |= (v ? 1u : 0u) << ((t - s0) & 31);
        if (((t - s0) & 31) == 31 || t == s1 - 1) {
            putw(w, (t - s0) >> 5, bits);
            bits = 0u;
        }
    }
    part(w, 0) = (float)jl;
    part(w, 1) = sh;
    part(w, 2) = sl;
}

// ---- phase 6: segment offsets ---------------------------------------------------------
template <int KH, class Part>
__host__ __device__ __forceinline__ void phase6_offsets(int w, Lane<KH>& S, Part part) {
    int off = 0;
    float sh = 0.f, sl = 0.f;
#pragma unroll
    for (int v = 0; v < kNW; ++v) {
        const int c = (int)part(v, 0);
        S.cnt_off[v] = off;
        S.sum_off_hi[v] = sh;
        S.sum_off_lo[v] = sl;
        if (v == w) {
            S.mycnt = c;
            S.myoff = off;
        }
        off += c;
        comp_add(sh, sl, part(v, 1));
        sl += part(v, 2);
    }
    S.N_i = off;
}

// Date slot (offset from the segment start) of the n-th (0-based) valid date
// of warp w's segment, from its validity words.
template <class GetW>
__host__ __device__ __forceinline__ int nth_valid(int w, int n, int nwords, GetW getw) {
    for (int i = 0; i < nwords; ++i) {
        uint32_t x = getw(w, i);
#ifdef __CUDA_ARCH__
        const int c = __popc(x);
#else
        const int c = __builtin_popcount(x);
#endif
        if (n < c) {
            for (int k = 0; k < n; ++k) x &= x - 1;  // drop the lowest n set bits
#ifdef __CUDA_ARCH__
            return 32 * i + __ffs(x) - 1;
#else
            return 32 * i + __builtin_ctz(x);
#endif
        }
        n -= c;
    }
    return -1;
}

// ---- phase 7: MOSUM over this warp's compacted entries ----------------------------
// get_s(slot) reads slot; seg_start(v) is the first date of all-date segment v.
// Writes the first crossing (date, or -1) and the compensated sum of MO.
// Loops jl over [jlo, jhi) (the warp's range of the lanes' monitoring entries).
template <int KH, class GetS, class Part, class GetW>
__host__ __device__ __forceinline__ void phase7_mosum(const SegParams& P, int w, const Lane<KH>& S, GetS get_s,
                                                      int jlo, int jhi, Part part, GetW getw) {
    int s0, s1;
    segment(P.N, w, s0, s1);
    const int n_i = S.n_i, h = S.h;
    const int mycnt = S.mycnt, off = S.myoff;
    float myoh = 0.f, myol = 0.f;
#pragma unroll
    for (int u = 0; u < kNW; ++u)
        if (u == w) {
            myoh = S.sum_off_hi[u];
            myol = S.sum_off_lo[u];
        }
    int first = -1;
    float mh = 0.f, ml = 0.f;
    float mx = 0.f;  // MO of largest magnitude in this segment (the first of equals)
    for (int jl = jlo; jl < jhi; ++jl) {
        const int J = off + jl + 1;  // 1-based valid position
        if (jl < mycnt && J > n_i) {
            const float sj = get_s(s0 + jl);
            const int g = J - h;  // >= 1 because J > n_i >= h
            int v = 0, offv = 0;  // segment holding valid position g (select chain, no indexing)
            float oh = 0.f, ol = 0.f;
#pragma unroll
            for (int u = 1; u < kNW; ++u)
                if (S.cnt_off[u] < g) {
                    v = u;
                    offv = S.cnt_off[u];
                    oh = S.sum_off_hi[u];
                    ol = S.sum_off_lo[u];
                }
            int g0, g1;
            segment(P.N, v, g0, g1);
            const float sg = get_s(g0 + (g - offv - 1));
            // S_J - S_g with both prefix sums split into segment offset + local sum
            const float W = (sj - sg) + ((myoh - oh) + (myol - ol));
            // Eq. 4 squared: MO_J^2 > lambda^2 log+(J/n), MO_J = W / (sigma-hat sqrt(n))
            const float mo = W * S.inv_scale;
            const float b2 = J > S.jlim ? S.lam2 * kLn2f * (log2_fast((float)J) - S.lg_n) : S.lam2;
            if (first < 0 && mo * mo > b2) first = jl;
            if (fabsf(mo) > fabsf(mx)) mx = mo;
            comp_add(mh, ml, W);
        }
    }
    part(w, 0) = first < 0 ? -1.f : (float)(s0 + nth_valid(w, first, (s1 - s0 + 31) >> 5, getw));
    part(w, 1) = mh;
    part(w, 2) = ml;
    part(w, Partials<KH>::kMaxMo) = mx;
}

template <int KH>
struct PixelOut {
    uint8_t status;
    int32_t brk;
    float mean, sigma, maxmo;
    float beta[Basis<KH>::K];
};

// ---- phase 8: combine and outputs -----------------------------------------------------
template <int KH, class Part>
__host__ __device__ __forceinline__ void phase8_out(const SegParams& P, const Lane<KH>& S, Part part,
                                                    PixelOut<KH>& o) {
    constexpr int K = Basis<KH>::K;
    int brk = -1;
    float mh = 0.f, ml = 0.f, mx = 0.f;
#pragma unroll
    for (int w = 0; w < kNW; ++w) {
        const float f = part(w, 0);
        if (brk < 0 && f >= 0.f) brk = (int)f;
        comp_add(mh, ml, part(w, 1));
        ml += part(w, 2);
        const float x = part(w, Partials<KH>::kMaxMo);
        if (fabsf(x) > fabsf(mx)) mx = x;  // segments in date order: the first of equals
    }
    const int n_i = S.n_i, N_i = S.N_i;
    const bool degenerate = !(S.sigma > kDegenerateRatio * S.ymax) || S.ymax == 0.f;
    const float qnan = qnanf();
    bool fitted = true;
    o.brk = -1;
    o.sigma = S.sigma;
    if (n_i <= K) {
        o.status = BFM_PX_INSUFFICIENT_HISTORY;
        fitted = false;
    } else if (!S.nonsingular) {
        o.status = BFM_PX_SINGULAR;
        fitted = false;
    } else if (degenerate) {
        o.status = BFM_PX_DEGENERATE;
        o.mean = 0.f;
        o.maxmo = 0.f;
    } else if (N_i == n_i) {
        o.status = BFM_PX_NO_MONITOR;
        o.mean = qnan;
        o.maxmo = qnan;
    } else {
        o.status = BFM_PX_OK;
        o.brk = brk;
        o.mean = (mh + ml) / ((float)(N_i - n_i) * S.scale);
        o.maxmo = mx;
    }
    if (!fitted) {
        o.mean = qnan;
        o.sigma = qnan;
        o.maxmo = qnan;
    }
    // beta of the centred trend -> raw parameterisation of Eq. 2
#pragma unroll
    for (int i = 0; i < K; ++i) o.beta[i] = fitted ? S.beta[i] : qnan;
    if (fitted) {
        o.beta[0] = fmaf(-S.beta[1], P.c_over_s, S.beta[0]);
        o.beta[1] = S.beta[1] * P.inv_s;
    }
}

}  // namespace bfm
