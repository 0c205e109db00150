// Fast path for complete series: one shared pseudo-inverse (BFM_ALGO_COMPLETE).
//
// Section 3 (Eq. 8-11): when no observation is missing, every pixel's history
// regression has the same design X_h, so beta = M y_h with one matrix
// M = (X_h' X_h)^-1 X_h' for all pixels (the paper forms beta_all = M Y as one
// tall product).  Here M is built once per (design, n_hist) on the host in
// FP64 and the rest is one streaming kernel, one thread per pixel, in three
// passes over the pixel's column of Y:
//   1. beta0 = M y over the history dates (FP32), max |y|, and the
//      completeness check (NaN / -32768 / mask bit);
//   2. history residuals r0_t = y_t - x_t'beta0 (re-read from L2: the pass-1
//      loads carry an evict-last hint and the grid is sized so that the
//      history of the resident pixels fits L2) and one step of iterative
//      refinement, beta = beta0 + M r0: the FP32 sum M y cancels (its partial
//      sums are several times the result), M r0 does not; sigma-hat^2 =
//      sum r0^2 / (n - K), which differs from sum r^2 only by a term of second
//      order in beta - beta0; the first h - 1 residuals of the first window;
//   3. monitoring dates t = n..N-1: the window sum gains r_t and, from t = n+1
//      on, drops r_{t-h}, recomputed from y_{t-h} as the paper's moving_sums
//      kernel recomputes residuals instead of storing them (Algorithm 3);
//      residuals there use the intercept and trend coefficients as hi + lo
//      pairs (beta0 and the refinement step), since a rounding of those enters
//      all h residuals of a window alike;
//      MO_t = W / (sigma-hat sqrt(n)) is tested against lambda^2 log+((t+1)/n)
//      (Eq. 4, squared, table per CTA), and the mean and the largest |MO|
//      are kept.
// With no missing data, n_p = n_hist, N_p = N and h_p = clamp(floor(h_frac n),
// 1, n) for every pixel, and positions are date indices, so this is exactly
// the general definition.  A pixel that meets a missing value anywhere gets
// status BFM_PX_INCOMPLETE and NaN outputs (the general forms handle it).
#include <cudaTypedefs.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <type_traits>
#include <vector>

#include "bfm_internal.cuh"
#include "ptx.cuh"
#include "stage.cuh"

namespace bfm {

__device__ unsigned int g_bfm_complete_err = 0;  // bit 0: a stage wait gave up

cudaError_t complete_read_clear_errors(cudaStream_t s, unsigned int* bits) {
    unsigned int v = 0;
    cudaError_t e = cudaMemcpyFromSymbolAsync(&v, g_bfm_complete_err, sizeof v, 0, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    const unsigned int zero = 0;
    e = cudaMemcpyToSymbolAsync(g_bfm_complete_err, &zero, sizeof zero, 0, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    *bits = v;
    return e;
}

namespace {

using namespace stage;

constexpr int kThreads = 256;
constexpr int kU1 = 16;  // history dates per load batch (16 loads in flight per thread)
constexpr int kU3 = 8;   // monitoring dates per load batch (two loads per date)
constexpr double kL2Budget = 80e6;  // bytes of history the resident pixels may hold in L2
constexpr size_t kSmemMax = 112 * 1024;  // shared memory per CTA of the staged form (two CTAs per SM)
constexpr int kStageBytes = 8192;         // one stage: 8 (float) or 16 (int16) dates of a 256-pixel tile
constexpr int kStages = 4;                // stages in flight per CTA
constexpr uint64_t kWaitNs = 2000000000ull;  // bound of every stage wait

struct CompleteParams {
    const void* Y;
    const uint32_t* mask;
    int64_t m, mask_words;
    int N, n, h, shared_status;
    const float* tab;  // M' [n][K] (row t = column t of M), then X [N][K]
    double lam2;
    float c_over_s, inv_s;
    int32_t* brk;
    float* mean;
    float* sigma;
    float* beta;
    uint8_t* status;
    float* maxmo;
};

// One stored value with an L2 policy (no use of the result here, so that a
// batch of these loads is in flight together).
__device__ __forceinline__ float ld_hint(const float* p, uint64_t pol) {
    float v;
    asm("ld.global.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
    return v;
}

__device__ __forceinline__ int16_t ld_hint(const int16_t* p, uint64_t pol) {
    unsigned short q;
    asm("ld.global.L2::cache_hint.u16 %0, [%1], %2;" : "=h"(q) : "l"(p), "l"(pol));
    return (int16_t)q;
}

// The value of an observation, NaN when it is missing (float: NaN already;
// int16: -32768).  A missing value then poisons beta0 (history) or the window
// sum (monitoring), and a pixel is complete exactly when neither is NaN.
__device__ __forceinline__ float obs_value(float v) { return v; }
__device__ __forceinline__ float obs_value(int16_t q) {
    return q == (int16_t)-32768 ? __int_as_float(0x7fc00000) : (float)q;
}

// Error-free sum: hi + lo gains x exactly (TwoSum), lo collects the errors.
__device__ __forceinline__ void comp_add(float& hi, float& lo, float x) {
    const float s = hi + x;
    const float bp = s - hi;
    lo += (hi - (s - bp)) + (x - bp);
    hi = s;
}

// Shared-memory layout of one CTA: M' [n][K], X [N][K], the squared boundary
// [N - n] and the window sums of the regressors [K] (floats); then, in the
// staged form, 128-byte aligned: the last h residuals of each thread
// [h][kThreads] floats, kStages stages of kStageBytes of Y, the stages' full
// and empty mbarriers, and an abort flag.
__host__ __device__ inline size_t ring_offset(int N, int n, int K) {
    return ((size_t)(n + N) * K + (size_t)(N - n) + (size_t)K + 31) & ~(size_t)31;  // 128-byte aligned
}

// kStaged: Y reaches the threads through shared-memory stages filled by 1-D
// bulk copies, one per date row of the 256-pixel tile, issued by a ninth
// (producer) warp up to kStages stages ahead across passes and tiles; each
// stage has a full barrier (the copies landed) and an empty barrier (all
// eight consumer warps are done with it), so the warps meet only through
// those.  The residuals leaving the MOSUM window come from a per-thread ring
// in shared memory.  Otherwise each thread loads its own values in register
// batches and recomputes the leaving residual from y_{t-h}.
template <int KH, typename T, bool kMask, bool kStaged>
__global__ void __launch_bounds__(kStaged ? kThreads + 32 : kThreads, 2)
    complete_kernel(const __grid_constant__ CUtensorMap tmap, const CompleteParams P) {
    constexpr int K = 2 + 2 * KH;
    constexpr int G1 = kStaged ? kStageBytes / (kThreads * (int)sizeof(T)) : kU1;  // dates per batch, history
    constexpr int G3 = kStaged ? G1 : kU3;                                          // dates per batch, monitoring
    extern __shared__ __align__(128) float sm[];
    const int n = P.n, N = P.N, h = P.h;
    const int64_t m = P.m;
    float* sM = sm;             // [n][K]
    float* sX = sm + n * K;     // [N][K]
    float* sB = sX + N * K;     // [N - n]: lambda^2 log+((t + 1) / n) for t = n..N-1
    float* sXW = sB + (N - n);  // [K]: sum of x_t over the first window's history dates t = w0..n-1
    float* ring = sm + ring_offset(N, n, K) + threadIdx.x;  // slot s at ring[s * kThreads]
    unsigned char* stages = reinterpret_cast<unsigned char*>(sm + ring_offset(N, n, K) + (size_t)h * kThreads);
    uint64_t* full = reinterpret_cast<uint64_t*>(stages + kStages * kStageBytes);
    uint64_t* empty = full + kStages;
    volatile uint32_t* abort_flag = reinterpret_cast<volatile uint32_t*>(empty + kStages);
    const int w0 = n - h + 1;
    for (int i = threadIdx.x; i < (n + N) * K; i += blockDim.x) sm[i] = P.tab[i];
    for (int i = threadIdx.x; i < N - n; i += blockDim.x) {
        const double x = (double)(n + 1 + i) / (double)n;
        sB[i] = (float)(P.lam2 * (x <= 2.718281828459045235360287 ? 1.0 : log(x)));
    }
    if (kStaged && threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            ptx::mbar_init(full + s, 1);
            ptx::mbar_init(empty + s, kThreads / 32);
        }
        *abort_flag = 0u;
        ptx::fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x < K) {
        float acc = 0.f;
        for (int t = w0; t < n; ++t) acc += sX[t * K + threadIdx.x];
        sXW[threadIdx.x] = acc;
    }
    __syncthreads();
    const float qnan = __int_as_float(0x7fc00000);
    const uint64_t keep = l2_evict_last(), normal = l2_evict_normal(), drop = l2_evict_first();
    const int64_t ntiles = (m + kThreads - 1) / kThreads;
    auto write_unfitted = [&](int64_t p, int st) {
        P.brk[p] = -1;
        P.mean[p] = qnan;
        P.sigma[p] = qnan;
#pragma unroll
        for (int a = 0; a < K; ++a) P.beta[(size_t)a * m + p] = qnan;
        P.status[p] = (uint8_t)st;
        if (P.maxmo) P.maxmo[p] = qnan;
    };
    if (P.shared_status != BFM_PX_OK) {
        if (kStaged && threadIdx.x >= kThreads) return;
        for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
            const int64_t p = tile * kThreads + threadIdx.x;
            if (p < m) write_unfitted(p, P.shared_status);
        }
        return;
    }

    // stage sequence of one tile: pass 1 and pass 2 (history, ng1 batches
    // each), pass 3 (monitoring, ng3 batches); stage j of this CTA is batch
    // j % Q of its tile j / Q, in ring slot j % kStages
    const int ng1 = (n + G1 - 1) / G1, ng3 = (N - n + G3 - 1) / G3, Q = 2 * ng1 + ng3;
    const int64_t my_tiles = (int64_t)blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const int64_t total = my_tiles * Q;
    bool bad = false;
    auto issue = [&](int64_t js) {  // producer: fill the slot of stage js with one box (256 pixels x G dates)
        const int64_t tl = js / Q;
        const int k = (int)(js - tl * Q);
        const int px0 = (int)((blockIdx.x + tl * gridDim.x) * kThreads);
        const int d0 = k < 2 * ng1 ? (k < ng1 ? k : k - ng1) * G1 : n + (k - 2 * ng1) * G3;
        const int slot = (int)(js % kStages);
        // pass 1 keeps the history in L2 for pass 2, pass 2 drops it (the
        // ring holds the residuals the first windows need)
        const uint64_t pol = k < ng1 ? keep : (k < 2 * ng1 ? drop : normal);
        // pixels past m and dates past N arrive as zeros; the box is always full
        ptx::mbar_arrive_expect_tx(full + slot, (uint32_t)kStageBytes);
        tma_box(stages + slot * kStageBytes, &tmap, full + slot, px0, d0, pol);
    };
    if (kStaged && threadIdx.x >= kThreads) {  // the producer warp: one lane issues
        if (threadIdx.x == kThreads) {
            ptx::prefetch_tmap(&tmap);
            int64_t js = 0;
            for (; js < total; ++js) {
                const int slot = (int)(js % kStages);
                if (js >= kStages &&
                    !wait_released(empty + slot, (uint32_t)(((js / kStages) - 1) & 1), abort_flag, kWaitNs)) {
                    *abort_flag = 1u;
                    atomicOr(&g_bfm_complete_err, 1u);
                    break;
                }
                if (*abort_flag) break;
                issue(js);
            }
            // copies still in flight land before the CTA's shared memory is released
            for (int64_t i = js > kStages ? js - kStages : 0; i < js; ++i)
                ptx::mbar_wait_bounded(full + (i % kStages), (uint32_t)((i / kStages) & 1), kWaitNs);
        }
        return;
    }
    // the consumers' stage j kept as (slot, lap parity): slot = j % kStages, phase = (j / kStages) & 1
    int cslot = 0;
    uint32_t cphase = 0;
    // Wait for stage j and return this thread's column in it.  Fast path: one
    // look at the barrier and a warp vote; the bounded wait, which also ends
    // when another warp or the producer has raised the abort flag, runs only
    // when some lane finds the stage not yet landed.  A warp whose wait gives up
    // raises the abort flag and is `bad` from then on (warp-uniform): it may
    // still read stages, whose contents no longer matter (its pixels end as
    // TIMEOUT), but it releases none, so the producer never refills a slot whose
    // copy may still be in flight.
    auto acquire = [&]() -> const T* {
        const int slot = cslot;
        bool ok = ptx::mbar_try_wait(full + slot, cphase);
        if (!__all_sync(~0u, ok)) {
            if (!ok) ok = wait_released(full + slot, cphase, abort_flag, kWaitNs);
            if (__any_sync(~0u, !ok)) {
                if ((threadIdx.x & 31) == 0 && !bad) {
                    *abort_flag = 1u;
                    atomicOr(&g_bfm_complete_err, 1u);
                }
                bad = true;
            }
        }
        return reinterpret_cast<const T*>(stages + slot * kStageBytes) + threadIdx.x;
    };
    auto release = [&]() {  // this warp is done with stage j
        __syncwarp();
        if ((threadIdx.x & 31) == 0 && !bad) mbar_arrive(empty + cslot);
        if (++cslot == kStages) {
            cslot = 0;
            cphase ^= 1u;
        }
    };

    int64_t tile = blockIdx.x;
    for (; tile < ntiles; tile += gridDim.x) {
        const int64_t p = tile * kThreads + threadIdx.x;
        const bool active = p < m;
        if (!kStaged && !active) continue;
        const T* yp = static_cast<const T*>(P.Y) + (active ? p : 0);
        const uint32_t* mp = kMask ? P.mask + (active ? (p >> 5) : 0) : nullptr;
        const uint32_t mbit = 1u << (p & 31);
        const size_t ms = (size_t)m, mws = (size_t)P.mask_words;

        // Batches of dates: every value of a batch is loaded (or its stage
        // waited for) before any is used; full batches carry no bounds
        // checks, the last one of a pass neutralises the dates past its end.
        // pass 1: first solution beta0 = M y, max |y|, completeness of the history
        float b0[K];
#pragma unroll
        for (int a = 0; a < K; ++a) b0[a] = 0.f;
        float ymax = 0.f;
        auto pass1 = [&](int d0, auto full_c) {
            constexpr bool full = decltype(full_c)::value;
            const int cnt = full ? G1 : n - d0;
            T raw[G1];
            uint32_t mw[G1];
            if constexpr (kStaged) {
                const T* st = acquire();
#pragma unroll
                for (int u = 0; u < G1; ++u) raw[u] = (full || u < cnt) ? st[u * kThreads] : T(0);
            } else {
                const T* q = yp + (size_t)d0 * ms;
#pragma unroll
                for (int u = 0; u < G1; ++u) {
                    raw[u] = (full || u < cnt) ? ld_hint(q, keep) : T(0);
                    q += ms;
                }
            }
            if (kMask) {
                const uint32_t* qm = mp + (size_t)d0 * mws;
#pragma unroll
                for (int u = 0; u < G1; ++u) {
                    mw[u] = (full || u < cnt) ? *qm : ~0u;
                    qm += mws;
                }
            }
#pragma unroll
            for (int u = 0; u < G1; ++u) {
                // past the end of a partial batch raw = 0 and the mask word is all ones
                float v = obs_value(raw[u]);
                if (kMask && !(mw[u] & mbit)) v = __int_as_float(0x7fc00000);
                ymax = fmaxf(ymax, fabsf(v));
                const float* mt = sM + (full ? d0 + u : min(d0 + u, n - 1)) * K;
#pragma unroll
                for (int a = 0; a < K; ++a) b0[a] = fmaf(mt[a], v, b0[a]);
            }
            if constexpr (kStaged) release();
        };
        int d0 = 0;
        for (; d0 + G1 <= n && !bad; d0 += G1) pass1(d0, std::true_type{});
        if (d0 < n && !bad) pass1(d0, std::false_type{});

        // pass 2: residuals r0 = y - x'beta0 of the history; one refinement
        // step for the intercept and the trend, whose FP32 sums M y cancel
        // (partial sums several times the result; the harmonic rows of M
        // oscillate and do not): c = (M r0)_{0,1}; sigma-hat from sum r0^2 (it
        // differs from sum r^2 by a second-order term); the first window's
        // h - 1 oldest residuals (kept in the ring in the staged form).
        float c0 = 0.f, c1 = 0.f, ss = 0.f, W0 = 0.f;
        auto pass2 = [&](int d0, auto full_c, auto win_c) {
            constexpr bool full = decltype(full_c)::value;
            constexpr bool win = decltype(win_c)::value;  // the batch may reach the first window (t >= w0)
            const int cnt = full ? G1 : n - d0;
            T raw[G1];
            if constexpr (kStaged) {
                const T* st = acquire();
#pragma unroll
                for (int u = 0; u < G1; ++u) raw[u] = (full || u < cnt) ? st[u * kThreads] : T(0);
            } else {
                const T* q = yp + (size_t)d0 * ms;
#pragma unroll
                for (int u = 0; u < G1; ++u) {
                    raw[u] = (full || u < cnt) ? ld_hint(q, d0 + u < w0 ? drop : keep) : T(0);
                    q += ms;
                }
            }
#pragma unroll
            for (int u = 0; u < G1; ++u) {
                const int t = d0 + u, tc = full ? t : min(t, n - 1);
                float r = residual<K>(obs_value(raw[u]), sX + tc * K, b0);
                if (!full) r = u < cnt ? r : 0.f;
                ss = fmaf(r, r, ss);
                c0 = fmaf(sM[tc * K], r, c0);
                c1 = fmaf(sM[tc * K + 1], r, c1);
                if (win && t >= w0 && (full || u < cnt)) {
                    W0 += r;
                    if (kStaged) ring[(t - w0) * kThreads] = r;
                }
            }
            if constexpr (kStaged) release();
        };
        for (d0 = 0; d0 + G1 <= n && !bad; d0 += G1) {
            if (d0 + G1 <= w0)
                pass2(d0, std::true_type{}, std::false_type{});
            else
                pass2(d0, std::true_type{}, std::true_type{});
        }
        if (d0 < n && !bad) pass2(d0, std::false_type{}, std::true_type{});
        // residuals from here on: beta0 with the intercept and trend corrected
        // by (c0, c1), kept apart (a float rounding of those two would enter
        // all h residuals of a window alike)
        float W = W0 - fmaf(sXW[1], c1, sXW[0] * c0);
        if (kStaged)
            for (int d = w0; d < n; ++d) ring[(d - w0) * kThreads] -= fmaf(sX[d * K + 1], c1, c0);
        const float sig = sqrtf(ss / (float)(n - K));
        const bool degenerate = !(sig > 1e-6f * ymax) || ymax == 0.f;
        const float inv_scale = degenerate ? 0.f : 1.f / (sig * sqrtf((float)n));
        const float inv2 = inv_scale * inv_scale;

        // pass 3: monitoring dates.  The residual leaving the window is the
        // ring slot of date t - h (the same slot as date t), or, in the plain
        // form, recomputed from y_{t-h} (re-read from L2/L1).
        int brk = -1;
        float sh = 0.f, sl = 0.f, wmax = -INFINITY, wmin = INFINITY;
        int slot = h - 1;  // ring slot of date t: (t - w0) mod h
        auto pass3 = [&](int d0, auto full_c) {
            constexpr bool full = decltype(full_c)::value;
            const int cnt = full ? G3 : N - d0;
            T raw[G3], old[kStaged ? 1 : G3];  // old: y_{t-h} of the plain form
            uint32_t mw[G3];
            if constexpr (kStaged) {
                (void)old;
                const T* st = acquire();
#pragma unroll
                for (int u = 0; u < G3; ++u) raw[u] = (full || u < cnt) ? st[u * kThreads] : T(0);
            } else {
                const T* q = yp + (size_t)d0 * ms;
#pragma unroll
                for (int u = 0; u < G3; ++u) {
                    raw[u] = (full || u < cnt) ? ld_hint(q, normal) : T(0);
                    old[u] = (full || u < cnt) ? ld_hint(q - (size_t)h * ms, drop) : T(0);
                    q += ms;
                }
            }
            if (kMask) {
                const uint32_t* qm = mp + (size_t)d0 * mws;
#pragma unroll
                for (int u = 0; u < G3; ++u) {
                    mw[u] = (full || u < cnt) ? *qm : ~0u;
                    qm += mws;
                }
            }
            // boundary test MO^2 > b^2 as W^2 inv_scale^2 - b^2 > 0: its maximum over
            // the batch, and the first crossing searched only in a batch that has one
            float blk = 0.f, cmax = -INFINITY, wv[G3];
#pragma unroll
            for (int u = 0; u < G3; ++u) {
                const int t = d0 + u;
                wv[u] = 0.f;
                if (full || u < cnt) {
                    float v = obs_value(raw[u]);
                    if (kMask && !(mw[u] & mbit)) v = __int_as_float(0x7fc00000);
                    const float r = residual2<K>(v, sX + t * K, b0, c0, c1);
                    float ro;
                    if constexpr (kStaged) {
                        ro = t > n ? ring[slot * kThreads] : 0.f;
                        ring[slot * kThreads] = r;
                        slot = slot + 1 == h ? 0 : slot + 1;
                    } else {
                        ro = t > n ? residual2<K>(obs_value(old[u]), sX + (t - h) * K, b0, c0, c1) : 0.f;
                    }
                    W = (W + r) - ro;
                    wv[u] = W;
                    cmax = fmaxf(cmax, fmaf(W * W, inv2, -sB[t - n]));
                    blk += W;
                    wmax = fmaxf(wmax, W);
                    wmin = fminf(wmin, W);
                }
            }
            if (brk < 0 && cmax > 0.f) {
#pragma unroll
                for (int u = 0; u < G3; ++u)
                    if ((full || u < cnt) && brk < 0 && fmaf(wv[u] * wv[u], inv2, -sB[d0 + u - n]) > 0.f) brk = d0 + u;
            }
            comp_add(sh, sl, blk);
            if constexpr (kStaged) release();
        };
        for (d0 = n; d0 + G3 <= N && !bad; d0 += G3) pass3(d0, std::true_type{});
        if (d0 < N && !bad) pass3(d0, std::false_type{});
        if (bad) break;
        if (!active) continue;

        if (isnan(b0[0]) || isnan(sh)) {  // a missing value met in the history or the monitoring period
            write_unfitted(p, BFM_PX_INCOMPLETE);
            continue;
        }
        P.brk[p] = degenerate ? -1 : brk;
        P.mean[p] = degenerate ? 0.f : (sh + sl) * inv_scale / (float)(N - n);
        P.sigma[p] = sig;
        // beta of the centred trend -> raw parameterisation of Eq. 2
        const float beta0 = b0[0] + c0, beta1 = b0[1] + c1;
        P.beta[p] = fmaf(-beta1, P.c_over_s, beta0);
        P.beta[(size_t)m + p] = beta1 * P.inv_s;
#pragma unroll
        for (int a = 2; a < K; ++a) P.beta[(size_t)a * m + p] = b0[a];
        P.status[p] = degenerate ? BFM_PX_DEGENERATE : BFM_PX_OK;
        // largest |MO| (positive on an exact tie of opposite signs)
        if (P.maxmo) P.maxmo[p] = degenerate ? 0.f : (wmax >= -wmin ? wmax : wmin) * inv_scale;
    }
    if (bad) {
        // a stage wait gave up: report it, stop the producer (which lets its
        // copies in flight land before the CTA ends) and mark this warp's
        // unfinished pixels
        if ((threadIdx.x & 31) == 0) {
            *abort_flag = 1u;
            atomicOr(&g_bfm_complete_err, 1u);
        }
        for (; tile < ntiles; tile += gridDim.x) {
            const int64_t p = tile * kThreads + threadIdx.x;
            if (p < m) write_unfitted(p, BFM_PX_TIMEOUT);
        }
    }
}

template <int KH, typename T, bool kMask, bool kStaged>
bfm_status launch_variant(const CUtensorMap& tm, const CompleteParams& P, int grid, size_t smem, cudaStream_t st) {
    auto* fn = complete_kernel<KH, T, kMask, kStaged>;
    if (smem > 48 * 1024) {
        // the opt-in maximum, not this launch's size: launches of other sizes (other
        // scenes, other host threads) never find a smaller limit in place
        const cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        if (e != cudaSuccess) return cuda_fail(e, "bfm_monitor (complete): shared memory attribute");
    }
    fn<<<grid, kStaged ? kThreads + 32 : kThreads, smem, st>>>(tm, P);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "bfm_monitor (complete): launch");
    return BFM_OK;
}

template <int KH, bool kStaged>
bfm_status launch_kh(const CUtensorMap& tm, const CompleteParams& P, int dtype, int grid, size_t smem,
                     cudaStream_t st) {
    if (dtype == BFM_F32)
        return P.mask ? launch_variant<KH, float, true, kStaged>(tm, P, grid, smem, st)
                      : launch_variant<KH, float, false, kStaged>(tm, P, grid, smem, st);
    return P.mask ? launch_variant<KH, int16_t, true, kStaged>(tm, P, grid, smem, st)
                  : launch_variant<KH, int16_t, false, kStaged>(tm, P, grid, smem, st);
}

// The shared table of (design, n_hist): M' and X in float, built in FP64.
// Status BFM_PX_INSUFFICIENT_HISTORY for n <= K, BFM_PX_SINGULAR when a
// Cholesky pivot of X_h'X_h falls below 1e-5 of its diagonal entry (the rank
// test of the general forms).
bfm_status complete_table(bfm_design_s* d, int n, const float** tab, int* status) {
    std::lock_guard<std::mutex> lk(d->complete_mu);
    for (const auto& e : d->complete)
        if (e.n_hist == n) {
            *tab = e.d_tab;
            *status = e.status;
            return BFM_OK;
        }
    const int K = d->K, N = d->N, k = d->k;
    std::vector<double> X((size_t)N * K);
    const double two_pi = 6.283185307179586476925286766559;
    for (int t = 0; t < N; ++t) {
        double* x = X.data() + (size_t)t * K;
        x[0] = 1.0;
        x[1] = (d->dates[t] - d->c) / d->s;
        for (int j = 1; j <= k; ++j) {
            const double a = two_pi * (double)j * d->dates[t] / d->f;
            x[2 * j] = std::sin(a);
            x[2 * j + 1] = std::cos(a);
        }
    }
    std::vector<float> host((size_t)(n + N) * K, 0.f);
    int st = BFM_PX_OK;
    if (n <= K) {
        st = BFM_PX_INSUFFICIENT_HISTORY;
    } else {
        std::vector<double> G((size_t)K * K, 0.0), L((size_t)K * K, 0.0);
        for (int t = 0; t < n; ++t)
            for (int a = 0; a < K; ++a)
                for (int b = 0; b < K; ++b) G[a * K + b] += X[(size_t)t * K + a] * X[(size_t)t * K + b];
        for (int j = 0; j < K && st == BFM_PX_OK; ++j) {
            double v = G[j * K + j];
            for (int c = 0; c < j; ++c) v -= L[j * K + c] * L[j * K + c];
            if (!(G[j * K + j] > 0.0) || !(v >= 1e-5 * G[j * K + j])) {
                st = BFM_PX_SINGULAR;
                break;
            }
            L[j * K + j] = std::sqrt(v);
            for (int i = j + 1; i < K; ++i) {
                double s = G[i * K + j];
                for (int c = 0; c < j; ++c) s -= L[i * K + c] * L[j * K + c];
                L[i * K + j] = s / L[j * K + j];
            }
        }
        if (st == BFM_PX_OK) {
            // row t of M' = G^-1 x_t (forward and back substitution)
            std::vector<double> z(K);
            for (int t = 0; t < n; ++t) {
                const double* x = X.data() + (size_t)t * K;
                for (int i = 0; i < K; ++i) {
                    double s = x[i];
                    for (int c = 0; c < i; ++c) s -= L[i * K + c] * z[c];
                    z[i] = s / L[i * K + i];
                }
                for (int i = K - 1; i >= 0; --i) {
                    double s = z[i];
                    for (int c = i + 1; c < K; ++c) s -= L[c * K + i] * z[c];
                    z[i] = s / L[i * K + i];
                }
                for (int i = 0; i < K; ++i) host[(size_t)t * K + i] = (float)z[i];
            }
        }
    }
    for (size_t i = 0; i < (size_t)N * K; ++i) host[(size_t)n * K + i] = (float)X[i];
    float* dtab = nullptr;
    cudaError_t e = cudaMalloc(&dtab, host.size() * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpy(dtab, host.data(), host.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        if (dtab) cudaFree(dtab);
        return cuda_fail(e, "bfm_monitor (complete): shared table");
    }
    d->complete.push_back({n, st, dtab});
    *tab = dtab;
    *status = st;
    return BFM_OK;
}

}  // namespace

// Shared memory of the complete-series kernel (staged form: ring, stages,
// their barriers and the abort flag on top of the tables).
size_t complete_smem_bytes(int N, int n, int K, int h, bool staged) {
    return sizeof(float) * ring_offset(N, n, K) +
           (staged ? sizeof(float) * (size_t)h * kThreads + (size_t)kStages * (kStageBytes + 16) + 16 : 0);
}

bfm_status launch_complete(bfm_design_s* d, int dtype, const void* Y, const uint32_t* mask, int64_t m, int n_hist,
                           double h_frac, double lambda, int32_t* brk, float* mean, float* sigma, float* beta,
                           uint8_t* status, cudaStream_t stream, float* maxmo) {
    const float* tab = nullptr;
    int shared = BFM_PX_OK;
    bfm_status rc = complete_table(d, n_hist, &tab, &shared);
    if (rc != BFM_OK) return rc;
    CompleteParams P{};
    P.Y = Y;
    P.mask = mask;
    P.m = m;
    P.mask_words = (m + 31) / 32;
    P.N = d->N;
    P.n = n_hist;
    int h = (int)std::floor(h_frac * (double)n_hist);
    P.h = h < 1 ? 1 : (h > n_hist ? n_hist : h);
    P.shared_status = shared;
    P.tab = tab;
    P.lam2 = lambda * lambda;
    P.c_over_s = (float)(d->c / d->s);
    P.inv_s = (float)(1.0 / d->s);
    P.brk = brk;
    P.mean = mean;
    P.sigma = sigma;
    P.beta = beta;
    P.status = status;
    P.maxmo = maxmo;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "bfm_monitor (complete): device attributes");
    // CTAs per SM: 2, or 1 when two CTAs' pixels would hold more history than the L2 budget
    const size_t elt = dtype == BFM_F32 ? 4 : 2;
    const int per_sm = 2.0 * kThreads * n_hist * (double)elt * sms <= kL2Budget ? 2 : 1;
    const int64_t ntiles = (m + kThreads - 1) / kThreads;
    const int grid = (int)(ntiles < (int64_t)per_sm * sms ? ntiles : (int64_t)per_sm * sms);
    // staged form: bulk copies need 16-byte aligned rows (base and m * elt), and
    // the ring, stages and tables must leave room for two CTAs per SM
    const bool aligned = ((uintptr_t)Y % 16 == 0) && ((size_t)m * elt % 16 == 0);
    bool staged = aligned && complete_smem_bytes(d->N, n_hist, d->K, P.h, true) <= kSmemMax;
    CUtensorMap tm;
    std::memset(&tm, 0, sizeof tm);
    if (staged) {  // Y as a 2-D tensor (pixels innermost), boxes of 256 pixels x one stage of dates
        auto enc = encode_tiled();
        const cuuint64_t gdim[2] = {(cuuint64_t)m, (cuuint64_t)d->N};
        const cuuint64_t gstride[1] = {(cuuint64_t)m * elt};
        const cuuint32_t box[2] = {(cuuint32_t)kThreads, (cuuint32_t)(kStageBytes / (kThreads * elt))};
        const cuuint32_t es[2] = {1u, 1u};
        staged = enc && enc(&tm, elt == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_UINT16, 2,
                            const_cast<void*>(Y), gdim, gstride, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    }
    const size_t smem = complete_smem_bytes(d->N, n_hist, d->K, P.h, staged);
    if (staged) {
        if (d->k == 1) return launch_kh<1, true>(tm, P, dtype, grid, smem, stream);
        if (d->k == 2) return launch_kh<2, true>(tm, P, dtype, grid, smem, stream);
        return launch_kh<3, true>(tm, P, dtype, grid, smem, stream);
    }
    if (d->k == 1) return launch_kh<1, false>(tm, P, dtype, grid, smem, stream);
    if (d->k == 2) return launch_kh<2, false>(tm, P, dtype, grid, smem, stream);
    return launch_kh<3, false>(tm, P, dtype, grid, smem, stream);
}

}  // namespace bfm
