// Residuals and MOSUM process of selected pixels (bfm_trace).
//
// The many-core path returns the breaks and per-pixel summaries only; the
// residuals or the MOSUM process of an individual series can be examined
// afterwards, once the breaks say which series are of interest (Section 3.2,
// the remarks after Algorithm 2).  This file does that examination on the
// device for a list of pixels, one warp per pixel:
//   1. compaction of the pixel's valid observations (ballot + popcount over
//      32-date groups), n_p = valid history observations, N_p = all;
//   2. the least-squares fit of Eq. 5-6 on the valid history observations,
//      redone in FP64 from the Eq. 2 regressors of the actual dates (trend
//      centred and scaled) by Cholesky on the normal equations;
//   3. residuals y - x'beta (the sign of Eq. 3) of every valid observation,
//      sigma-hat with n_p - K degrees of freedom (Algorithm 1 step 5);
//   4. MO_j of Eq. 3 for every valid monitoring observation: the sum of the
//      h_p residuals ending at position j over sigma-hat * sqrt(n_p), from
//      FP64 prefix sums (the difference of two FP64 prefix sums is exact to
//      well below the float output).
// The pixel statuses written by bfm_monitor for the same data decide which
// pixels have a fit (OK, DEGENERATE, NO_MONITOR) so that the two calls agree
// on them; DEGENERATE pixels get MO = 0 at their monitoring dates.
#include <cmath>

#include "bfm_internal.cuh"

namespace bfm {
namespace {

struct TraceParams {
    const void* Y;
    const uint32_t* mask;
    int64_t m, mask_words;
    int N, n_hist, dtype;
    double h_frac, f, c, s;
    const double* dates;
    const int64_t* pixels;
    int64_t count;
    const uint8_t* status;
    float* mo;
    float* resid;
};

// Shared memory of one warp: compacted values (double), their date indices
// and the compacted position of every date (-1 when missing).
constexpr int kBytesPerDate = 16;
constexpr int kMaxWarps = 4;
constexpr size_t kSmemTarget = 48 * 1024;

// Eq. 2 regressors of date t with the trend column (t - c)/s.
template <int KH>
__device__ __forceinline__ void regressors(double t, const TraceParams& P, double* x) {
    x[0] = 1.0;
    x[1] = (t - P.c) / P.s;
#pragma unroll
    for (int j = 1; j <= KH; ++j) {
        double sj, cj;
        sincospi(2.0 * (double)j * t / P.f, &sj, &cj);  // sin/cos(2 pi j t / f)
        x[2 * j] = sj;
        x[2 * j + 1] = cj;
    }
}

template <int KH>
__global__ void __launch_bounds__(32 * kMaxWarps) trace_kernel(const TraceParams P) {
    constexpr int K = 2 + 2 * KH;
    constexpr int NG = K * (K + 1) / 2;  // packed lower triangle, row a at a(a+1)/2
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
    if (i >= P.count) return;
    const int N = P.N;
    double* val = reinterpret_cast<double*>(smem + (size_t)wib * kBytesPerDate * N);
    int* tix = reinterpret_cast<int*>(val + N);
    int* pos = tix + N;
    float* mo_row = P.mo ? P.mo + i * N : nullptr;
    float* rs_row = P.resid ? P.resid + i * N : nullptr;
    const float qnan = __int_as_float(0x7fc00000);

    const int64_t p = P.pixels ? P.pixels[i] : i;
    int st = -1;
    if (p >= 0 && p < P.m) st = P.status[p];
    bool fit = st == BFM_PX_OK || st == BFM_PX_DEGENERATE || st == BFM_PX_NO_MONITOR;

    // 1. compaction
    int nv = 0, np = 0;
    if (fit) {
        for (int t0 = 0; t0 < N; t0 += 32) {
            const int t = t0 + lane;
            bool v = false;
            double y = 0.0;
            if (t < N) {
                const size_t o = (size_t)t * (size_t)P.m + (size_t)p;
                if (P.dtype == BFM_F32) {
                    const float yf = static_cast<const float*>(P.Y)[o];
                    v = !isnan(yf);
                    y = (double)yf;
                } else {
                    const int16_t yq = static_cast<const int16_t*>(P.Y)[o];
                    v = yq != (int16_t)-32768;
                    y = (double)yq;
                }
                if (v && P.mask) v = (P.mask[(size_t)t * (size_t)P.mask_words + (size_t)(p >> 5)] >> (p & 31)) & 1u;
            }
            const unsigned b = __ballot_sync(~0u, v);
            const int q = nv + __popc(b & ((1u << lane) - 1u));
            if (t < N) pos[t] = v ? q : -1;
            if (v) {
                val[q] = y;
                tix[q] = t;
            }
            nv += __popc(b);
            const int hl = P.n_hist - t0;  // history dates in this group
            const unsigned hm = hl >= 32 ? ~0u : (hl > 0 ? (1u << hl) - 1u : 0u);
            np += __popc(b & hm);
        }
        __syncwarp();
        fit = np > K;
    }

    // 2. normal equations of the history (every lane ends with the full sums)
    double beta[K];
    if (fit) {
        double g[NG], rhs[K];
#pragma unroll
        for (int a = 0; a < NG; ++a) g[a] = 0.0;
#pragma unroll
        for (int a = 0; a < K; ++a) rhs[a] = 0.0;
        for (int j = lane; j < np; j += 32) {
            double x[K];
            regressors<KH>(P.dates[tix[j]], P, x);
            const double y = val[j];
#pragma unroll
            for (int a = 0; a < K; ++a) {
#pragma unroll
                for (int b = 0; b <= a; ++b) g[a * (a + 1) / 2 + b] = fma(x[a], x[b], g[a * (a + 1) / 2 + b]);
                rhs[a] = fma(x[a], y, rhs[a]);
            }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
            for (int a = 0; a < NG; ++a) g[a] += __shfl_xor_sync(~0u, g[a], off);
#pragma unroll
            for (int a = 0; a < K; ++a) rhs[a] += __shfl_xor_sync(~0u, rhs[a], off);
        }
        // Cholesky G = L L' in place (every lane, identical), then two triangular solves
#pragma unroll
        for (int a = 0; a < K; ++a) {
#pragma unroll
            for (int b = 0; b <= a; ++b) {
                double v = g[a * (a + 1) / 2 + b];
#pragma unroll
                for (int c = 0; c < b; ++c) v -= g[a * (a + 1) / 2 + c] * g[b * (b + 1) / 2 + c];
                if (a == b) {
                    fit = fit && v > 0.0;
                    g[a * (a + 1) / 2 + a] = sqrt(v > 0.0 ? v : 1.0);
                } else {
                    g[a * (a + 1) / 2 + b] = v / g[b * (b + 1) / 2 + b];
                }
            }
        }
#pragma unroll
        for (int a = 0; a < K; ++a) {
            double v = rhs[a];
#pragma unroll
            for (int c = 0; c < a; ++c) v -= g[a * (a + 1) / 2 + c] * rhs[c];
            rhs[a] = v / g[a * (a + 1) / 2 + a];
        }
#pragma unroll
        for (int a = K - 1; a >= 0; --a) {
            double v = rhs[a];
#pragma unroll
            for (int c = a + 1; c < K; ++c) v -= g[c * (c + 1) / 2 + a] * beta[c];
            beta[a] = v / g[a * (a + 1) / 2 + a];
        }
    }

    if (!fit) {
        for (int t = lane; t < N; t += 32) {
            if (mo_row) mo_row[t] = qnan;
            if (rs_row) rs_row[t] = qnan;
        }
        return;
    }

    // 3. residuals of every valid observation, sigma-hat from the history part
    double ss = 0.0;
    for (int j = lane; j < nv; j += 32) {
        double x[K];
        regressors<KH>(P.dates[tix[j]], P, x);
        double yhat = 0.0;
#pragma unroll
        for (int a = 0; a < K; ++a) yhat = fma(x[a], beta[a], yhat);
        const double r = val[j] - yhat;
        val[j] = r;
        if (j < np) ss = fma(r, r, ss);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) ss += __shfl_xor_sync(~0u, ss, off);
    __syncwarp();
    if (rs_row)
        for (int t = lane; t < N; t += 32) {
            const int q = pos[t];
            rs_row[t] = q >= 0 ? (float)val[q] : qnan;
        }
    if (!mo_row) return;
    __syncwarp();

    // 4. prefix sums of the residuals in place, then the windows of h_p terms
    double carry = 0.0;
    for (int j0 = 0; j0 < nv; j0 += 32) {
        const int j = j0 + lane;
        double v = j < nv ? val[j] : 0.0;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const double u = __shfl_up_sync(~0u, v, off);
            if (lane >= off) v += u;
        }
        v += carry;
        if (j < nv) val[j] = v;
        carry = __shfl_sync(~0u, v, 31);
    }
    __syncwarp();
    int hp = (int)floor(P.h_frac * (double)np);
    hp = hp < 1 ? 1 : (hp > np ? np : hp);
    const double scale = sqrt(ss / (double)(np - K)) * sqrt((double)np);
    const bool degenerate = st == BFM_PX_DEGENERATE;
    for (int t = lane; t < N; t += 32) {
        const int q = pos[t];  // 0-based position: the window holds positions q-hp+1..q
        float out = qnan;
        if (q >= np) out = degenerate ? 0.0f : (float)((val[q] - val[q - hp]) / scale);
        mo_row[t] = out;
    }
}

}  // namespace
}  // namespace bfm

using namespace bfm;

extern "C" bfm_status bfm_trace(bfm_design_t d, const void* Y, int dtype, const uint32_t* mask_bits, int64_t m,
                                int n_hist, double h_frac, const int64_t* pixels, int64_t count,
                                const uint8_t* status, float* mo, float* resid, void* stream) {
    if (!d) {
        set_error("bfm_trace: design handle is NULL");
        return BFM_EINVAL;
    }
    if (dtype != BFM_F32 && dtype != BFM_I16) {
        set_error("bfm_trace: dtype is not BFM_F32 or BFM_I16");
        return BFM_EINVAL;
    }
    if (m < 1 || count < 0) {
        set_error("bfm_trace: needs m >= 1 and count >= 0");
        return BFM_EINVAL;
    }
    if (!(n_hist >= 1 && n_hist < d->N)) {
        set_error("bfm_trace: n_hist outside 1 <= n_hist < N");
        return BFM_EINVAL;
    }
    if (!(h_frac > 0.0 && h_frac <= 1.0)) {
        set_error("bfm_trace: h_frac outside (0, 1]");
        return BFM_EINVAL;
    }
    if (count == 0) return BFM_OK;
    if (!Y || !status || (!mo && !resid)) {
        set_error("bfm_trace: Y, status and at least one of mo, resid must be non-NULL device pointers");
        return BFM_EINVAL;
    }
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != d->device) {
        set_error("bfm_trace: the design belongs to another device");
        return BFM_EINVAL;
    }
    TraceParams P{};
    P.Y = Y;
    P.mask = mask_bits;
    P.m = m;
    P.mask_words = (m + 31) / 32;
    P.N = d->N;
    P.n_hist = n_hist;
    P.dtype = dtype;
    P.h_frac = h_frac;
    P.f = d->f;
    P.c = d->c;
    P.s = d->s;
    P.dates = d->d_dates;
    P.pixels = pixels;
    P.count = count;
    P.status = status;
    P.mo = mo;
    P.resid = resid;
    const size_t per_warp = (size_t)kBytesPerDate * (size_t)d->N;
    int warps = (int)(kSmemTarget / per_warp);
    warps = warps < 1 ? 1 : (warps > kMaxWarps ? kMaxWarps : warps);
    const int64_t grid = (count + warps - 1) / warps;
    if (grid > 0x7fffffffLL) {
        set_error("bfm_trace: count too large for one call");
        return BFM_EUNSUPPORTED;
    }
    const size_t smem = per_warp * (size_t)warps;
    cudaStream_t st = (cudaStream_t)stream;
    if (d->k == 1)
        trace_kernel<1><<<(unsigned)grid, 32 * warps, smem, st>>>(P);
    else if (d->k == 2)
        trace_kernel<2><<<(unsigned)grid, 32 * warps, smem, st>>>(P);
    else
        trace_kernel<3><<<(unsigned)grid, 32 * warps, smem, st>>>(P);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "bfm_trace: launch");
    return BFM_OK;
}
