// Streaming CUDA-core form of the general path (BFM_ALGO_STREAM): one thread
// per pixel, missing values allowed.
//
// Each pixel's column of Y is streamed four times through shared memory
// (pass A, A', B over the history, pass C over the monitoring dates), in
// stages filled by 2-D TMA boxes (256 pixels x 8 dates: three float or six
// int16 stages) that a producer warp issues up to a full ring ahead; the history stays
// in L2 between its passes (evict-last hints, a grid sized to the L2), so Y
// is read once from DRAM.  Per pixel (Section 2.1, Eq. 3-6, Algorithm 1 with
// missing values masked, as in the other forms):
//   A   masked sums of the basis functions of bfm::Basis over the valid
//       history dates -> Gram matrix G (identities of gram_from_sums) and
//       X'My; valid count n_p; max |y|.  Cholesky of G with the rank test of
//       the other forms, beta0 = G^-1 X'My.
//   A'  r0 = y - x'beta0 at the valid history dates: s0 = sum r0^2 and
//       c = X'M r0; delta = G^-1 c, beta = beta0 + delta, sum of squared
//       residuals s1 = s0 - delta'c (Algorithm 1 step 5), sigma-hat, h_p.
//   B   residuals of the first window's h_p - 1 valid history observations
//       (valid ranks n_p - h_p + 1 .. n_p - 1, 0-based) into a per-thread
//       ring in shared memory, and their sum.
//   C   at each valid monitoring observation (position J = n_p + 1 ..): the
//       window sum gains its residual and loses the ring slot it replaces
//       (the observation h_p positions earlier); MO_J = W / (sigma-hat
//       sqrt(n_p)) against lambda^2 log+(J / n_p) (Eq. 4, squared; the
//       first crossing's date is the break), the mean and the largest |MO|.
// Residuals in B and C hold the intercept and trend coefficients as beta0 +
// delta (hi + lo): a float rounding of those two would enter all h_p
// residuals of a window alike.
#include <cudaTypedefs.h>

#include <atomic>
#include <cmath>
#include <cstring>
#include <mutex>
#include <type_traits>

#include "bfm_internal.cuh"
#include "ptx.cuh"
#include "simt_seg.cuh"
#include "stage.cuh"

namespace bfm {

__device__ unsigned int g_bfm_stream_err = 0;  // bit 0: a stage wait gave up

namespace {
std::atomic<uint64_t> g_stage_wait_ns{2000000000ull};
}

uint64_t stage_wait_ns() { return g_stage_wait_ns.load(std::memory_order_relaxed); }
void set_stage_wait_ns(uint64_t ns) { g_stage_wait_ns.store(ns ? ns : 2000000000ull, std::memory_order_relaxed); }

cudaError_t stream_read_clear_errors(cudaStream_t s, unsigned int* bits) {
    unsigned int v = 0;
    cudaError_t e = cudaMemcpyFromSymbolAsync(&v, g_bfm_stream_err, sizeof v, 0, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    const unsigned int zero = 0;
    e = cudaMemcpyToSymbolAsync(g_bfm_stream_err, &zero, sizeof zero, 0, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    *bits = v;
    return e;
}

namespace {

using namespace stage;

constexpr int kThreads = 256;                // pixels per CTA (eight consumer warps)
constexpr int kDates = 8;                    // dates per stage (one TMA box of 256 pixels x 8 dates)
constexpr int kStageArea = 24576;            // bytes of stages per CTA: 3 float or 6 int16 stages
constexpr int kMaxStages = 6;

template <typename T>
struct Stage {
    static constexpr int kBytes = kDates * kThreads * (int)sizeof(T);
    static constexpr int kCount = kStageArea / kBytes;
};
constexpr size_t kSmemMax = 112 * 1024;      // two CTAs per SM
constexpr double kL2Budget = 80e6;           // bytes of history the resident pixels may hold in L2
constexpr uint64_t kWaitNs = 2000000000ull;  // bound of every wait

struct StreamParams {
    uint64_t wait_ns;  // bound of the consumers' stage waits (bfm_stage_wait_limit)
    const uint32_t* mask;
    int64_t m, mask_words;
    int N, n, hmax;
    double h_frac;
    const float* basis;  // device [N][NB] (bfm::Basis rows, centred trend)
    float lam2, c_over_s, inv_s;
    int32_t* brk;
    float* mean;
    float* sigma;
    float* beta;
    uint8_t* status;
    float* maxmo;
};

// Observation value and validity (float: NaN missing; int16: -32768 missing).
__device__ __forceinline__ bool obs(float raw, float& y) {
    y = raw;
    return !isnan(raw);
}
__device__ __forceinline__ bool obs(int16_t raw, float& y) {
    y = (float)raw;
    return raw != (int16_t)-32768;
}

// Shared-memory layout (bytes, each part 128-byte aligned): basis rows of the
// history [n][NB], regressors of the monitoring dates [N - n][K], the ring
// [hmax][kThreads], the stages, full and empty barriers, the abort flag.
struct Layout {
    size_t phi, xm, ring, stages, bars, total;
};

__host__ __device__ inline size_t up128(size_t x) { return (x + 127) & ~(size_t)127; }

__host__ __device__ inline Layout stream_layout(int N, int n, int K, int NB, int hmax) {
    Layout L{};
    L.phi = 0;
    L.xm = up128(sizeof(float) * (size_t)n * NB);
    L.ring = L.xm + up128(sizeof(float) * (size_t)(N - n) * K);
    L.stages = L.ring + up128(sizeof(float) * (size_t)hmax * kThreads);
    L.bars = L.stages + (size_t)kStageArea;
    L.total = L.bars + 2 * kMaxStages * sizeof(uint64_t) + 16;
    return L;
}

template <int KH, typename T, bool kMask>
__global__ void __launch_bounds__(kThreads + 32, 2)
    stream_kernel(const __grid_constant__ CUtensorMap tmap, const StreamParams P) {
    using B = Basis<KH>;
    constexpr int K = B::K, NB = B::NB, NBR = B::NBR;
    constexpr int G = kDates;                    // dates per stage
    constexpr int kStageBytes = Stage<T>::kBytes;
    constexpr int kStages = Stage<T>::kCount;    // stages in flight
    extern __shared__ __align__(128) unsigned char smem[];
    const int n = P.n, N = P.N, hmax = P.hmax;
    const int64_t m = P.m;
    const Layout Lo = stream_layout(N, n, K, NB, hmax);
    float* sPhi = reinterpret_cast<float*>(smem + Lo.phi);  // [n][NB]
    float* sXm = reinterpret_cast<float*>(smem + Lo.xm);    // [N - n][K], row t - n
    float* ring = reinterpret_cast<float*>(smem + Lo.ring) + threadIdx.x;  // slot s at ring[s * kThreads]
    unsigned char* stages = smem + Lo.stages;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + Lo.bars);
    uint64_t* empty = full + kMaxStages;
    volatile uint32_t* abort_flag = reinterpret_cast<volatile uint32_t*>(empty + kMaxStages);
    for (int i = threadIdx.x; i < n * NB; i += blockDim.x) sPhi[i] = P.basis[i];
    for (int i = threadIdx.x; i < (N - n) * K; i += blockDim.x) {
        const int r = i / K;
        sXm[i] = P.basis[(size_t)(n + r) * NB + (i - r * K)];
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            ptx::mbar_init(full + s, 1);
            ptx::mbar_init(empty + s, kThreads / 32);
        }
        *abort_flag = 0u;
        ptx::fence_mbar_init();
    }
    __syncthreads();

    // stage sequence of one tile: passes A, A', B over the history (ng1
    // boxes each), pass C over the monitoring dates (ng3 boxes); stage j of
    // this CTA is box j % Q of its tile j / Q, in slot j % kStages
    const int64_t ntiles = (m + kThreads - 1) / kThreads;
    const int ng1 = (n + G - 1) / G, ng3 = (N - n + G - 1) / G, Q = 3 * ng1 + ng3;
    const int64_t my_tiles = (int64_t)blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const int64_t total = my_tiles * Q;

    if (threadIdx.x >= kThreads) {  // the producer warp: one lane issues the boxes
        if (threadIdx.x == kThreads) {
            ptx::prefetch_tmap(&tmap);
            const uint64_t keep = l2_evict_last(), normal = l2_evict_normal(), drop = l2_evict_first();
            int64_t js = 0;
            for (; js < total; ++js) {
                const int slot = (int)(js % kStages);
                // the slot's previous stage released by every consumer warp
                if (js >= kStages &&
                    !wait_released(empty + slot, (uint32_t)(((js / kStages) - 1) & 1), abort_flag, kWaitNs)) {
                    *abort_flag = 1u;
                    atomicOr(&g_bfm_stream_err, 1u);
                    break;
                }
                if (*abort_flag) break;
                const int64_t tl = js / Q;
                const int k = (int)(js - tl * Q);
                const int px0 = (int)((blockIdx.x + tl * gridDim.x) * kThreads);
                const int d0 = k < 3 * ng1 ? (k % ng1) * G : n + (k - 3 * ng1) * G;
                // passes A and A' keep the history in L2 for the next history
                // pass; pass B is its last use
                const uint64_t pol = k < 2 * ng1 ? keep : (k < 3 * ng1 ? drop : normal);
                ptx::mbar_arrive_expect_tx(full + slot, (uint32_t)kStageBytes);  // boxes are always full
                tma_box(stages + slot * kStageBytes, &tmap, full + slot, px0, d0, pol);
            }
            // copies still in flight land before the CTA's shared memory is released
            for (int64_t i = js > kStages ? js - kStages : 0; i < js; ++i)
                ptx::mbar_wait_bounded(full + (i % kStages), (uint32_t)((i / kStages) & 1), kWaitNs);
        }
        return;
    }

    bool bad = false;
    // the consumers' stage j kept as (slot, lap parity): slot = j % kStages, phase = (j / kStages) & 1
    int cslot = 0;
    uint32_t cphase = 0;
    // Wait for stage j and return this thread's column in it.  Fast path: one
    // look at the barrier and a warp vote.  The bounded wait, which also ends
    // when another warp or the producer has raised the abort flag, runs only
    // when some lane finds the stage not yet landed; a bound below 1 us (a test
    // of the failure path) makes the first look a non-blocking one and the only
    // one.  A warp whose wait gives up raises the abort flag and is `bad` from
    // then on (warp-uniform): it may still read stages, whose contents no longer
    // matter (its pixels end as TIMEOUT), but it releases none, so the producer
    // never refills a slot whose copy may still be in flight.
    const bool test_mode = P.wait_ns < 1000u;
    auto acquire = [&]() -> const T* {
        const int slot = cslot;
        bool ok = !test_mode && ptx::mbar_try_wait(full + slot, cphase);
        if (!__all_sync(~0u, ok)) {
            if (!ok) ok = test_mode ? ptx::mbar_test_wait(full + slot, cphase)
                                    : wait_released(full + slot, cphase, abort_flag, P.wait_ns);
            if (__any_sync(~0u, !ok)) {
                if ((threadIdx.x & 31) == 0 && !bad) {
                    *abort_flag = 1u;
                    atomicOr(&g_bfm_stream_err, 1u);
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
    const float qnan = __int_as_float(0x7fc00000);
    auto write_unfitted = [&](int64_t p, int st) {
        P.brk[p] = -1;
        P.mean[p] = qnan;
        P.sigma[p] = qnan;
#pragma unroll
        for (int a = 0; a < K; ++a) P.beta[(size_t)a * m + p] = qnan;
        P.status[p] = (uint8_t)st;
        if (P.maxmo) P.maxmo[p] = qnan;
    };

    int64_t tile = blockIdx.x;
    for (; tile < ntiles; tile += gridDim.x) {
        const int64_t p = tile * kThreads + threadIdx.x;
        const bool active = p < m;
        const uint32_t* mp = kMask ? P.mask + (active ? (p >> 5) : 0) : nullptr;
        const uint32_t mbit = 1u << (p & 31);
        const size_t mws = (size_t)P.mask_words;
        // observation u of a stage whose dates start at d0: value (0 when
        // missing) and 1/0 for valid/missing; in a partial batch (full =
        // false) the dates from cnt on do not belong to the pass
        auto get = [&](const T* st, int d0, int u, int cnt, bool full, float& y) -> float {
            bool ok = obs(st[u * kThreads], y);
            if (!full) ok = ok && u < cnt;
            if (kMask) ok = ok && (mp[(size_t)(d0 + u) * mws] & mbit);
            y = ok ? y : 0.f;
            return ok ? 1.f : 0.f;
        };

        // pass A: masked basis sums (S[0] is n_p), X'My, max |y| over the history
        float S[NBR], Bv[K];
#pragma unroll
        for (int i = 0; i < NBR; ++i) S[i] = 0.f;
#pragma unroll
        for (int a = 0; a < K; ++a) Bv[a] = 0.f;
        float ymax = 0.f;
        auto passA = [&](int d0, auto full_c) {
            constexpr bool full = decltype(full_c)::value;
            const int cnt = full ? G : n - d0;
            const T* st = acquire();
#pragma unroll
            for (int u = 0; u < G; ++u) {
                float y;
                const float v = get(st, d0, u, cnt, full, y);
                const float* ph = sPhi + (full ? d0 + u : min(d0 + u, n - 1)) * NB;
#pragma unroll
                for (int i = 0; i < NBR; ++i) S[i] = fmaf(ph[i], v, S[i]);
#pragma unroll
                for (int a = 0; a < K; ++a) Bv[a] = fmaf(ph[a], y, Bv[a]);
                ymax = fmaxf(ymax, fabsf(y));
            }
            release();
        };
        int d0 = 0;
        for (; d0 + G <= n && !bad; d0 += G) passA(d0, std::true_type{});
        if (d0 < n && !bad) passA(d0, std::false_type{});
        const int np = (int)S[0];  // basis row 0 is 1: S[0] counts the valid history dates
        float b0[K];
        bool nonsingular;
        {
            float Gm[K][K], Lc[K][K], dinv[K];
            gram_from_sums<KH>(S, Gm);
            nonsingular = cholesky<K>(Gm, Lc, dinv);
            chol_solve<K>(Lc, dinv, Bv, b0);
        }

        // pass A': residuals r0 of the first solution, refinement sums c = X'M r0
        float cr[K];
#pragma unroll
        for (int a = 0; a < K; ++a) cr[a] = 0.f;
        float ss0 = 0.f;
        auto passA2 = [&](int d0, auto full_c) {
            constexpr bool full = decltype(full_c)::value;
            const int cnt = full ? G : n - d0;
            const T* st = acquire();
#pragma unroll
            for (int u = 0; u < G; ++u) {
                float y;
                const float v = get(st, d0, u, cnt, full, y);
                const float* ph = sPhi + (full ? d0 + u : min(d0 + u, n - 1)) * NB;
                const float r = residual<K>(y, ph, b0) * v;
                ss0 = fmaf(r, r, ss0);
#pragma unroll
                for (int a = 0; a < K; ++a) cr[a] = fmaf(ph[a], r, cr[a]);
            }
            release();
        };
        for (d0 = 0; d0 + G <= n && !bad; d0 += G) passA2(d0, std::true_type{});
        if (d0 < n && !bad) passA2(d0, std::false_type{});
        float dl[K];
        {
            float Gm[K][K], Lc[K][K], dinv[K];
            gram_from_sums<KH>(S, Gm);
            cholesky<K>(Gm, Lc, dinv);
            chol_solve<K>(Lc, dinv, cr, dl);
        }
        float dc = 0.f;
#pragma unroll
        for (int a = 0; a < K; ++a) dc = fmaf(dl[a], cr[a], dc);
        const bool fit = np > K && nonsingular;
        const float sig = sqrtf(fmaxf(ss0 - dc, 0.f) / (float)(np - K));
        const bool degenerate = !(sig > kDegenerateRatio * ymax) || ymax == 0.f;
        int hp = (int)floor(P.h_frac * (double)np);
        hp = hp < 1 ? 1 : (hp > np ? np : hp);
        if (!fit) hp = 1;  // keeps the ring arithmetic in range; nothing of it is used
        float bres[K];  // coefficients of the residuals: intercept and trend as hi (bres) + lo (dl)
#pragma unroll
        for (int a = 0; a < K; ++a) bres[a] = a < 2 ? b0[a] : b0[a] + dl[a];
        const float lo0 = dl[0], lo1 = dl[1];
        const float inv_scale = (fit && !degenerate) ? 1.f / (sig * sqrtf((float)np)) : 0.f;
        const float inv2 = inv_scale * inv_scale;
        const float lam2ln2 = P.lam2 * kLn2f, blg = lam2ln2 * log2f((float)np);
        const float jlimf = (float)floor(kEuler * (double)np);  // J / n_p <= e  <=>  J <= jlim

        // pass B: the first window's h_p - 1 valid history residuals into the
        // ring (valid ranks wq .. n_p - 1 -> slots 0 .. h_p - 2), branch-free
        const int wq = fit ? np - hp + 1 : np;  // 0-based valid rank of the window's oldest history observation
        float W = 0.f;
        int q = -wq;  // valid rank minus wq: the slot of the next valid observation when >= 0
        auto passB = [&](int d0, auto full_c) {
            constexpr bool full = decltype(full_c)::value;
            const int cnt = full ? G : n - d0;
            const T* st = acquire();
            if (__any_sync(~0u, q + G > 0)) {  // some pixel of the warp may reach its window in this batch
#pragma unroll
                for (int u = 0; u < G; ++u) {
                    float y;
                    const float v = get(st, d0, u, cnt, full, y);
                    const float r =
                        residual2<K>(y, sPhi + (full ? d0 + u : min(d0 + u, n - 1)) * NB, bres, lo0, lo1);
                    const bool take = v != 0.f && q >= 0;
                    if (take) ring[q * kThreads] = r;
                    W += take ? r : 0.f;
                    q += v != 0.f ? 1 : 0;
                }
            } else {  // only count the valid observations
#pragma unroll
                for (int u = 0; u < G; ++u) {
                    float y;
                    q += get(st, d0, u, cnt, full, y) != 0.f ? 1 : 0;
                }
            }
            release();
        };
        for (d0 = 0; d0 + G <= n && !bad; d0 += G) passB(d0, std::true_type{});
        if (d0 < n && !bad) passB(d0, std::false_type{});

        // pass C: the monitoring observations, branch-free per date
        float Jf = (float)(np + 1);  // position of the next valid monitoring observation (exact in float)
        int slot = hp - 1;  // ring slot of the next observation
        int brk = -1;
        float sh = 0.f, sl = 0.f, wmax = -INFINITY, wmin = INFINITY;
        auto passC = [&](int d0, auto full_c) {
            constexpr bool full = decltype(full_c)::value;
            const int cnt = full ? G : N - d0;
            const T* st = acquire();
            // boundary test W^2 inv_scale^2 - b^2 > 0 (MO^2 > b^2): its maximum over
            // the batch, the first crossing searched only in a batch that has one
            float cv[G], blk = 0.f, cmax = -INFINITY;
#pragma unroll
            for (int u = 0; u < G; ++u) {
                float y;
                const float v = get(st, d0, u, cnt, full, y);
                const bool take = v != 0.f;
                const float r =
                    residual2<K>(y, sXm + (full ? d0 + u - n : min(d0 + u, N - 1) - n) * K, bres, lo0, lo1);
                const float old = ring[slot * kThreads];
                const float ro = Jf > (float)(np + 1) ? old : 0.f;
                if (take) ring[slot * kThreads] = r;
                const int nslot = slot + 1 == hp ? 0 : slot + 1;
                slot = take ? nslot : slot;
                const float Wn = (W + r) - ro;
                W = take ? Wn : W;
                const float b2 = Jf > jlimf ? fmaf(lam2ln2, log2_fast(Jf), -blg) : P.lam2;
                const float c = take ? fmaf(W * W, inv2, -b2) : -1.f;
                cv[u] = c;
                cmax = fmaxf(cmax, c);
                blk += take ? W : 0.f;
                wmax = take ? fmaxf(wmax, W) : wmax;
                wmin = take ? fminf(wmin, W) : wmin;
                Jf += v;
            }
            if (brk < 0 && cmax > 0.f) {
#pragma unroll
                for (int u = 0; u < G; ++u)
                    if (brk < 0 && cv[u] > 0.f) brk = d0 + u;
            }
            comp_add(sh, sl, blk);
            release();
        };
        for (d0 = n; d0 + G <= N && !bad; d0 += G) passC(d0, std::true_type{});
        if (d0 < N && !bad) passC(d0, std::false_type{});
        if (bad) break;
        if (!active) continue;

        const int Np = (int)Jf - 1;
        if (np <= K) {
            write_unfitted(p, BFM_PX_INSUFFICIENT_HISTORY);
        } else if (!nonsingular) {
            write_unfitted(p, BFM_PX_SINGULAR);
        } else {
            P.sigma[p] = sig;
            // beta of the centred trend -> raw parameterisation of Eq. 2
            const float beta0 = b0[0] + dl[0], beta1 = b0[1] + dl[1];
            P.beta[p] = fmaf(-beta1, P.c_over_s, beta0);
            P.beta[(size_t)m + p] = beta1 * P.inv_s;
#pragma unroll
            for (int a = 2; a < K; ++a) P.beta[(size_t)a * m + p] = bres[a];
            if (degenerate) {
                P.status[p] = BFM_PX_DEGENERATE;
                P.brk[p] = -1;
                P.mean[p] = 0.f;
                if (P.maxmo) P.maxmo[p] = 0.f;
            } else if (Np == np) {
                P.status[p] = BFM_PX_NO_MONITOR;
                P.brk[p] = -1;
                P.mean[p] = qnan;
                if (P.maxmo) P.maxmo[p] = qnan;
            } else {
                P.status[p] = BFM_PX_OK;
                P.brk[p] = brk;
                P.mean[p] = (sh + sl) * inv_scale / (float)(Np - np);
                // largest |MO| (positive on an exact tie of opposite signs)
                if (P.maxmo) P.maxmo[p] = (wmax >= -wmin ? wmax : wmin) * inv_scale;
            }
        }
    }
    if (bad) {
        // a stage wait gave up: report it, stop the producer (which lets its
        // copies in flight land before the CTA ends) and mark this thread's
        // unfinished pixels
        if ((threadIdx.x & 31) == 0) {
            *abort_flag = 1u;
            atomicOr(&g_bfm_stream_err, 1u);
        }
        for (; tile < ntiles; tile += gridDim.x) {
            const int64_t p = tile * kThreads + threadIdx.x;
            if (p < m) write_unfitted(p, BFM_PX_TIMEOUT);
        }
    }
}

template <int KH, typename T, bool kMask>
bfm_status launch_one(const CUtensorMap& tm, const StreamParams& P, int grid, size_t smem, cudaStream_t st) {
    auto* fn = stream_kernel<KH, T, kMask>;
    if (smem > 48 * 1024) {
        // the opt-in maximum, not this launch's size: launches of other sizes (other
        // scenes, other host threads) never find a smaller limit in place
        const cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        if (e != cudaSuccess) return cuda_fail(e, "bfm_monitor (stream): shared memory attribute");
    }
    fn<<<grid, kThreads + 32, smem, st>>>(tm, P);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "bfm_monitor (stream): launch");
    return BFM_OK;
}

template <int KH>
bfm_status launch_kh(const CUtensorMap& tm, const StreamParams& P, int dtype, int grid, size_t smem,
                     cudaStream_t st) {
    if (dtype == BFM_F32)
        return P.mask ? launch_one<KH, float, true>(tm, P, grid, smem, st)
                      : launch_one<KH, float, false>(tm, P, grid, smem, st);
    return P.mask ? launch_one<KH, int16_t, true>(tm, P, grid, smem, st)
                  : launch_one<KH, int16_t, false>(tm, P, grid, smem, st);
}

int stream_hmax(int n_hist, double h_frac) {
    int h = (int)std::floor(h_frac * (double)n_hist);
    return h < 1 ? 1 : (h > n_hist ? n_hist : h);
}

}  // namespace

bool stream_supported(const bfm_design_s* d, int dtype, int n_hist, double h_frac, const void* Y, int64_t m) {
    const size_t elt = dtype == BFM_F32 ? 4 : 2;
    if (m < 1 || (uintptr_t)Y % 16 != 0 || ((size_t)m * elt) % 16 != 0) return false;
    const int NB = basis_stride(d->k);
    return stream_layout(d->N, n_hist, d->K, NB, stream_hmax(n_hist, h_frac)).total <= kSmemMax;
}

bfm_status launch_stream(const bfm_design_s* d, int dtype, const void* Y, const uint32_t* mask, int64_t m,
                         int n_hist, double h_frac, double lambda, int32_t* brk, float* mean, float* sigma,
                         float* beta, uint8_t* status, cudaStream_t stream, float* maxmo) {
    if (!stream_supported(d, dtype, n_hist, h_frac, Y, m)) {
        set_error("bfm_monitor: the streaming form needs Y with a 16-byte aligned base and rows of a multiple of "
                  "16 bytes, and basis tables plus a residual ring of floor(h_frac * n_hist) slots per pixel "
                  "within 112 KB of shared memory");
        return BFM_EUNSUPPORTED;
    }
    auto enc = encode_tiled();
    if (!enc) {
        set_error("bfm_monitor (stream): cuTensorMapEncodeTiled is not available");
        return BFM_ECUDA;
    }
    const size_t elt = dtype == BFM_F32 ? 4 : 2;
    StreamParams P{};
    P.wait_ns = stage_wait_ns();
    P.mask = mask;
    P.m = m;
    P.mask_words = (m + 31) / 32;
    P.N = d->N;
    P.n = n_hist;
    P.hmax = stream_hmax(n_hist, h_frac);
    P.h_frac = h_frac;
    P.basis = d->d_basis;
    P.lam2 = (float)(lambda * lambda);
    P.c_over_s = (float)(d->c / d->s);
    P.inv_s = (float)(1.0 / d->s);
    P.brk = brk;
    P.mean = mean;
    P.sigma = sigma;
    P.beta = beta;
    P.status = status;
    P.maxmo = maxmo;
    CUtensorMap tm;
    std::memset(&tm, 0, sizeof tm);
    const cuuint64_t gdim[2] = {(cuuint64_t)m, (cuuint64_t)d->N};
    const cuuint64_t gstride[1] = {(cuuint64_t)m * elt};
    const cuuint32_t box[2] = {(cuuint32_t)kThreads, (cuuint32_t)kDates};
    const cuuint32_t es[2] = {1u, 1u};
    if (enc(&tm, elt == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_UINT16, 2,
            const_cast<void*>(Y), gdim, gstride, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS) {
        set_error("bfm_monitor (stream): cuTensorMapEncodeTiled failed for Y");
        return BFM_ECUDA;
    }
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "bfm_monitor (stream): device attributes");
    // CTAs per SM: 2, or 1 when two CTAs' pixels would hold more history than the L2 budget
    const int per_sm = 2.0 * kThreads * n_hist * (double)elt * sms <= kL2Budget ? 2 : 1;
    const int64_t ntiles = (m + kThreads - 1) / kThreads;
    const int grid = (int)(ntiles < (int64_t)per_sm * sms ? ntiles : (int64_t)per_sm * sms);
    const size_t smem = stream_layout(d->N, n_hist, d->K, basis_stride(d->k), P.hmax).total;
    if (d->k == 1) return launch_kh<1>(tm, P, dtype, grid, smem, stream);
    if (d->k == 2) return launch_kh<2>(tm, P, dtype, grid, smem, stream);
    return launch_kh<3>(tm, P, dtype, grid, smem, stream);
}

}  // namespace bfm
