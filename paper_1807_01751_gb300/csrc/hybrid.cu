// Hybrid form of the general path (BFM_ALGO_HYBRID): one thread per pixel for
// the per-date scan, the tensor cores for every contraction over dates.
//
// A CTA owns 512 pixels (four 128-pixel M-tiles = four TMEM lane sets) and
// runs one per SM, so that one copy of the basis tables, three 16 KB stages
// and a residual ring of floor(h_frac n_hist) slots for all 512 pixels share
// the SM's shared memory.  Warps 0..15 own 32 pixels each (the pixel's TMEM
// lane is its thread's lane), warp 16 issues the 2-D TMA boxes of Y (128
// pixels x 8 float or 16 int16 dates, one per M-tile and stage), warp 17
// issues the tensor-core work and owns the tensor memory.  Per work block of
// 512 pixels (Section 2.1, Eq. 3-6, Algorithm 1 with missing values masked):
//
//   A   history, 16 dates per chunk: each pixel thread writes its row of the
//       chunk's A operands into TMEM -- the 0/1 validity mask as fp16 and the
//       masked y as tf32 -- and the MMA warp accumulates
//         G  += mask x [basis hi | basis lo]   (the 3 + 6k masked basis sums
//                                               of bfm::Basis, fp16, N = 32)
//         b  += y x [x hi | x lo]              (X'My, tf32, N = 16)
//       The pixel thread reads G and b, forms the Gram matrix (identities of
//       gram_from_sums), FP32 Cholesky with the rank test of the other forms,
//       beta0 = G^-1 X'My, and writes beta0 (scaled by a power of two, split
//       fp16 hi + lo) as an A operand.
//   B'  history again (from L2): yhat0 = X beta0 in TMEM pieces of 32 dates
//       (fp16 MMA, B = the regressors hi and lo read MN-major); the thread
//       forms r0 = y - yhat0 at valid dates, s0 = sum r0^2, and writes r0
//       (scaled, fp16 hi + lo) as an A operand for c += r0 x [x hi | x lo]
//       (X'M r0, the refinement step).  It also notes the date of the oldest
//       history observation of its first MOSUM window.  Then delta = G^-1 c,
//       beta = beta0 + delta, sigma-hat^2 = (s0 - delta'c) / (n_p - K)
//       (Algorithm 1 step 5), and delta is written as a further A operand.
//   C   dates from the earliest window start of the tile to N: yhat = X
//       (beta0 + delta) in TMEM pieces; residuals r = y - yhat; history dates
//       of the first window fill the ring, monitoring dates slide the window
//       (Eq. 3) and test MO against the boundary of Eq. 4: the exact test
//       runs only on stages whose largest |MO| reaches the boundary at the
//       stage's first position (the boundary grows with the position), and
//       only until the first crossing.
//
// Precision: the Gram sums use the basis split into fp16 hi + lo (22 bits);
// X'My uses tf32 y (beta0 is only the start of the refinement); r0 and the
// coefficients are split hi + lo with per-pixel power-of-two scales, and the
// regressors of the fitted values, scaled by 2^12, three ways (hi, mid, lo),
// so that the fitted values carry ~22 bits of beta0 and of delta separately
// and lose no more to the regressors: the float rounding of an intercept or
// trend would otherwise enter every residual of a window alike.
#include <cuda_fp16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <mutex>
#include <type_traits>
#include <vector>

#include "bfm_internal.cuh"
#include "ptx.cuh"
#include "simt_seg.cuh"
#include "stage.cuh"

namespace bfm {

__device__ unsigned int g_bfm_hybrid_err = 0;  // bit 0: a bounded wait gave up

cudaError_t hybrid_read_clear_errors(cudaStream_t s, unsigned int* bits) {
    unsigned int v = 0;
    cudaError_t e = cudaMemcpyFromSymbolAsync(&v, g_bfm_hybrid_err, sizeof v, 0, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    const unsigned int zero = 0;
    e = cudaMemcpyToSymbolAsync(g_bfm_hybrid_err, &zero, sizeof zero, 0, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    *bits = v;
    return e;
}

namespace {

using namespace stage;

constexpr int kMT = 4;                    // 128-pixel M-tiles per CTA
constexpr int kPx = 128 * kMT;            // pixels per CTA tile
constexpr int kCons = 4 * kMT;            // pixel warps
constexpr int kProdWarp = kCons;          // TMA producer warp
constexpr int kMmaWarp = kCons + 1;       // tensor-core issuing warp (owns TMEM)
constexpr int kThreads = 32 * (kCons + 2);
constexpr int kStages = 3;
constexpr int kBoxPx = 128;               // TMA box width (one M-tile)
constexpr int kStageBytes = 16384;        // kMT boxes
constexpr int kBoxBytes = kStageBytes / kMT;
constexpr uint32_t kTmemCols = 512;
constexpr uint64_t kWaitNs = 2000000000ull;
constexpr size_t kSmemCap = 232448;       // opt-in dynamic shared memory per block

// TMEM columns within an M-tile's 128 (the phases reuse them in turn):
//   pass A : G sums [0, 32), X'My [32, 48), A buffers 2 x (mask 8 | y 16) [48, 96)
//   pass B': c [0, 16), beta0 coefficients (24) [16, 40), r0 buffers 2 x (hi 8 | lo 8) [40, 72),
//            fitted-value pieces 2 x 16 [72, 104), the basis sums kept for the second solve [104, 128)
//   pass C : beta0 coefficients [16, 40), delta coefficients (24) [40, 64), pieces 2 x 32 [64, 128)
constexpr uint32_t kColG = 0, kColB = 32, kColA = 48, kColC = 0, kColB0 = 16, kColR = 40, kColY0 = 72, kColDl = 40,
                   kColY = 64;
// Pass B' keeps the pixel's basis sums (up to 21) in [104, 128), free until pass C, for the
// second solve, so that they do not occupy registers through the pass.
constexpr uint32_t kColS = 104;
// Coefficient operands: 24 columns per set, A_hi (K = 32: 16 columns) then A_lo (K = 16: 8 columns).
constexpr uint32_t kCoefLo = 16;
// The regressors of the fitted-value table are scaled by 2^12 before their three-way fp16 split.
constexpr float kYScale = 4096.f, kInvYScale = 1.f / 4096.f;

template <typename T>
struct Dt {
    static constexpr int G = kBoxBytes / (kBoxPx * (int)sizeof(T));  // dates per stage: 8 float, 16 int16
};

struct HybridParams {
    uint64_t wait_ns;            // bound of the pixel warps' stage waits (bfm_stage_wait_limit)
    const uint32_t* mask;
    int64_t m, mask_words;
    int N, n, hmax, npad;
    double h_frac;
    const unsigned char* tabs;   // design tables (hybrid_tables), npad dates
    float lam2, c_over_s, inv_s;
    int32_t* brk;
    float* mean;
    float* sigma;
    float* beta;
    uint8_t* status;
    float* maxmo;
};

// Byte offsets of the design tables in global memory for npad dates.
__host__ __device__ inline size_t tab_gram_lo(int npad) { return (size_t)npad * 48; }
__host__ __device__ inline size_t tab_x(int npad) { return (size_t)npad * 96; }
__host__ __device__ inline size_t tab_yhat(int npad) { return (size_t)npad * 160; }
__host__ __device__ inline size_t tab_yhat_bytes(int npad) { return (size_t)npad * 48 + 384; }
__host__ __device__ inline size_t tab_bytes(int npad) { return tab_yhat(npad) + tab_yhat_bytes(npad); }

struct HLayout {
    size_t gh, gl, xt, yh, stages, ring, bars, total;
};

// One tile of a batched launch (bfm_batch): its tensor map, parameters and
// first 512-pixel work block within its group.
struct HybBatchTile {
    CUtensorMap tm;  // 64-byte aligned type
    HybridParams P;
    int64_t block0;
};

// The batch side of a launch: the group's tiles (device memory), its work
// blocks and the shared-memory layout that holds the largest tables and ring
// among them.
struct HybBatch {
    const HybBatchTile* tiles;
    int ntiles;
    int64_t blocks;
    HLayout lo;
};

__host__ __device__ inline size_t up1024(size_t x) { return (x + 1023) & ~(size_t)1023; }

// Shared memory: Gram table hi and lo and the tf32 regressor table over the
// history (16-date chunks), the fitted-value table over all npad dates, the
// stages, the ring [hmax][kPx], barriers and a few words.
__host__ __device__ inline HLayout hyb_layout(int n, int npad, int hmax) {
    const size_t nh16 = (size_t)((n + 15) & ~15);
    HLayout L{};
    L.gh = 0;
    L.gl = L.gh + nh16 / 8 * 384;
    L.xt = L.gl + nh16 / 8 * 384;
    L.yh = L.xt + nh16 / 4 * 256;
    L.stages = up1024(L.yh + tab_yhat_bytes(npad));
    L.ring = L.stages + (size_t)kStages * kStageBytes;
    L.bars = L.ring + (size_t)hmax * kPx * 4;
    L.total = L.bars + (size_t)(2 * kStages + 14) * 8 + 16;
    return L;
}

__device__ __forceinline__ float obs_y(float raw, bool& ok) {
    ok = !isnan(raw);
    return raw;
}
__device__ __forceinline__ float obs_y(int16_t raw, bool& ok) {
    ok = raw != (int16_t)-32768;
    return (float)raw;
}

// 2^(T - e) for v = 1.x * 2^e (so |v| * scale lies in [2^T, 2^(T+1))); 1 for
// zero, subnormal, infinite or NaN v.
__device__ __forceinline__ float pow2_scale(float v, int T) {
    const int e = (__float_as_int(v) >> 23) & 0xff;
    if (e == 0 || e == 0xff) return 1.f;
    int r = 254 + T - e;
    r = r < 1 ? 1 : (r > 254 ? 254 : r);
    return __int_as_float(r << 23);
}

__device__ __forceinline__ uint32_t h2bits(__half lo, __half hi) {
    return (uint32_t)__half_as_ushort(lo) | ((uint32_t)__half_as_ushort(hi) << 16);
}

// x = hi + lo exactly in float, hi the fp16 rounding of x; lo is rounded to fp16 by the caller.
__device__ __forceinline__ void split_h(float x, __half& hi, float& lo) {
    hi = __float2half_rn(x);
    lo = x - __half2float(hi);
}

// Coefficient A operands (fp16) for the fitted-value table, whose K rows are
// the regressors' three-way split [hi; mid; lo] (rows 24..31 are read from the
// next date group and meet zeros here): A_hi = [c_hi | c_hi | c_hi | 0]
// (K = 32, words 0..15) and A_lo = [c_lo | c_lo] (K = 16, words 16..23), so
// that the products cover c_hi (hi + mid + lo) + c_lo (hi + mid).  Returns in
// rep the value the products represent, c_hi + c_lo, in float.
template <int K>
__device__ __forceinline__ void coef_words(const float (&c)[K], float scale, uint32_t (&w)[24], float (&rep)[K]) {
    __half hi[8], lo[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        if (i < K) {
            float l;
            split_h(c[i] * scale, hi[i], l);
            lo[i] = __float2half_rn(l);
            rep[i < K ? i : 0] = __half2float(hi[i]) + __half2float(lo[i]);
        } else {
            hi[i] = __float2half_rn(0.f);
            lo[i] = hi[i];
        }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        w[j] = h2bits(hi[2 * j], hi[2 * j + 1]);
        w[4 + j] = w[j];
        w[8 + j] = w[j];
        w[12 + j] = 0u;
        w[16 + j] = h2bits(lo[2 * j], lo[2 * j + 1]);
        w[20 + j] = w[16 + j];
    }
}

__device__ __forceinline__ void coef_store(uint32_t taddr, const uint32_t (&w)[24]) {
    uint32_t a[16], b[8];
#pragma unroll
    for (int i = 0; i < 16; ++i) a[i] = w[i];
#pragma unroll
    for (int i = 0; i < 8; ++i) b[i] = w[16 + i];
    ptx::tmem_st16(taddr, a);
    ptx::tmem_st8(taddr + kCoefLo, b);
}

// Bounded wait that also ends when the CTA aborts; false when it gave up.
__device__ __forceinline__ bool wait_bar(uint64_t* bar, uint32_t parity, volatile uint32_t* abort_flag,
                                         uint64_t limit_ns) {
    if (ptx::mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = ptx::globaltimer_ns();
    while (true) {
        if (ptx::mbar_try_wait_hint(bar, parity, 20000u)) return true;
        if (*abort_flag || ptx::globaltimer_ns() - t0 > limit_ns) return false;
    }
}

__device__ __forceinline__ void raise_abort(volatile uint32_t* abort_flag) {
    if (!*abort_flag) {
        *abort_flag = 1u;
        atomicOr(&g_bfm_hybrid_err, 1u);
    }
}

// Validity of one observation of this thread's pixel: the in-band marker
// (float NaN, int16 -32768) and, with an explicit mask, the pixel's bit of
// the date's mask row.  `in_range` false makes the date invalid (and skips
// the mask read).
template <typename T, bool kMask>
struct Obs {
    const uint32_t* mp;
    size_t mws;
    uint32_t mbit;
    __device__ __forceinline__ bool valid(T raw, int d, bool in_range) const {
        bool ok;
        (void)obs_y(raw, ok);
        ok = ok && in_range;
        if (kMask) ok = ok && in_range && (mp[(size_t)d * mws] & mbit) != 0u;
        return ok;
    }
    // value (0 when invalid) and validity
    __device__ __forceinline__ float value(T raw, int d, bool in_range, bool& ok) const {
        const float y = obs_y(raw, ok);
        ok = ok && in_range;
        if (kMask) ok = ok && in_range && (mp[(size_t)d * mws] & mbit) != 0u;
        return y;
    }
};

// Pass A, 8 dates from d8: masked y as tf32 bits, the 0/1 mask as 4 fp16
// pairs (even date in the low half), and max |y|.
template <bool kFull, typename T, bool kMask>
__device__ __forceinline__ void pass_a8(const Obs<T, kMask>& ob, const T* st, int d8, int n, uint32_t* yv,
                                        uint32_t* mk, float& ymax) {
    float vf[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        bool ok;
        float y = ob.value(st[u * kBoxPx], d8 + u, kFull || d8 + u < n, ok);
        y = ok ? y : 0.f;
        ymax = fmaxf(ymax, fabsf(y));
        yv[u] = __float_as_uint(y);
        vf[u] = ok ? 1.f : 0.f;
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const __half2 h = __floats2half2_rn(vf[2 * j], vf[2 * j + 1]);
        mk[j] = *reinterpret_cast<const uint32_t*>(&h);
    }
}

// Pass B', 8 dates from d8: r0 = y - yhat0 (0 where invalid), s0 += r0^2,
// r0 * s_r split into fp16 hi (11 leading bits) + lo as 4 + 4 packed pairs;
// with kScan, the date of valid rank `rem` (counted down) becomes wdate.
template <bool kFull, bool kScan, typename T, bool kMask>
__device__ __forceinline__ void pass_b8(const Obs<T, kMask>& ob, const T* st, int d8, int n, const float* yh,
                                        float inv_sb, float s_r, float& ss0, uint32_t* hw, uint32_t* lw, int& rem,
                                        int& wdate) {
    float hi[8], lo[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        bool ok;
        const float y = ob.value(st[u * kBoxPx], d8 + u, kFull || d8 + u < n, ok);
        const float r = ok ? fmaf(-yh[u], inv_sb, y) : 0.f;
        ss0 = fmaf(r, r, ss0);
        const float rs = r * s_r;
        hi[u] = __uint_as_float(__float_as_uint(rs) & 0xFFFFE000u);
        lo[u] = rs - hi[u];
        if (kScan) wdate = (ok && rem == 0) ? d8 + u : wdate;
        rem -= ok ? 1 : 0;
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const __half2 h = __floats2half2_rn(hi[2 * j], hi[2 * j + 1]);
        const __half2 l = __floats2half2_rn(lo[2 * j], lo[2 * j + 1]);
        hw[j] = *reinterpret_cast<const uint32_t*>(&h);
        lw[j] = *reinterpret_cast<const uint32_t*>(&l);
    }
}

// State of the monitoring scan of one pixel.
struct Mon {
    int slot = 0;         // ring slot (float offset) of the next residual
    int hp_off = 0;       // h_p slots
    int fill_end = 0;     // h_p - 1 slots: the first window's history part
    int wdate = 0;        // date of the first window's oldest history observation
    int cnt = 0;          // valid monitoring observations so far
    float inv_sb = 1.f;
    float W = 0.f;        // window sum of h_p residuals
    float blk = 0.f;      // sum of W over this stretch's valid monitoring positions
    float amax = 0.f;     // largest |W| seen in this stretch (a bound for the boundary pre-test)
    float wmax = -INFINITY, wmin = INFINITY;  // extreme W over the monitoring positions
};

// History dates [d8, d8 + 8) before n: the first window's residuals into the ring.
template <typename T, bool kMask>
__device__ __forceinline__ void mon_hist8(const Obs<T, kMask>& ob, const T* st, int d8, const float* yh,
                                          float* ring_t, Mon& mo) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        bool ok;
        const float y = ob.value(st[u * kBoxPx], d8 + u, true, ok);
        const float r = fmaf(-yh[u], mo.inv_sb, y);
        const bool take = ok && d8 + u >= mo.wdate && mo.slot < mo.fill_end;
        if (take) ring_t[mo.slot] = r;
        mo.slot += take ? kPx : 0;
        mo.W += take ? r : 0.f;
    }
}

// One monitoring date: the window gains r and loses the ring slot it replaces.
template <bool kExt>
__device__ __forceinline__ void mon_step(bool ok, float r, float* ring_t, Mon& mo) {
    float* a = ring_t + mo.slot;
    const float old = *a;
    if (ok) *a = r;
    const int ns = mo.slot + (ok ? kPx : 0);
    mo.slot = ns == mo.hp_off ? 0 : ns;
    mo.W += ok ? r - old : 0.f;
    mo.cnt += ok ? 1 : 0;
    mo.blk += ok ? mo.W : 0.f;
    mo.amax = fmaxf(mo.amax, fabsf(mo.W));
    if (kExt) {
        mo.wmax = ok ? fmaxf(mo.wmax, mo.W) : mo.wmax;
        mo.wmin = ok ? fminf(mo.wmin, mo.W) : mo.wmin;
    }
}

// Monitoring dates [d8, d8 + 8), all >= n (kFull: all < N).
template <bool kFull, bool kExt, typename T, bool kMask>
__device__ __forceinline__ void mon8(const Obs<T, kMask>& ob, const T* st, int d8, int N, const float* yh,
                                     float* ring_t, Mon& mo, float (&Wu)[8]) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        bool ok;
        const float y = ob.value(st[u * kBoxPx], d8 + u, kFull || d8 + u < N, ok);
        mon_step<kExt>(ok, fmaf(-yh[u], mo.inv_sb, y), ring_t, mo);
        Wu[u] = mo.W;
    }
}

// Dates [d8, d8 + 8) that hold n (or N): history dates fill the ring, later ones are monitored.
template <typename T, bool kMask>
__device__ __forceinline__ void mon_mixed8(const Obs<T, kMask>& ob, const T* st, int d8, int n, int N,
                                        const float* yh, float* ring_t, Mon& mo, float (&Wu)[8], bool ext) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        const int d = d8 + u;
        bool ok;
        const float y = ob.value(st[u * kBoxPx], d, d < N, ok);
        const float r = fmaf(-yh[u], mo.inv_sb, y);
        if (d < n) {
            const bool take = ok && d >= mo.wdate && mo.slot < mo.fill_end;
            if (take) ring_t[mo.slot] = r;
            mo.slot += take ? kPx : 0;
            mo.W += take ? r : 0.f;
        } else if (ext) {
            mon_step<true>(ok, r, ring_t, mo);
        } else {
            mon_step<false>(ok, r, ring_t, mo);
        }
        Wu[u] = mo.W;
    }
}

// kBatch: the work blocks of several tiles (Bt; tmap and P are unused but for
// P.wait_ns), the tables of a block's tile loaded by the MMA warp when its
// previous block belonged to another tile; otherwise the blocks of one tile.
template <int KH, typename T, bool kMask, bool kBatch>
__global__ void __launch_bounds__(kThreads, 1)
    hybrid_kernel(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ HybridParams P,
                  const HybBatch Bt) {
    using B = Basis<KH>;
    constexpr int K = B::K, NBR = B::NBR;
    constexpr int G = Dt<T>::G;         // dates per stage
    extern __shared__ __align__(1024) unsigned char smem[];
    const HLayout Lo = kBatch ? Bt.lo : hyb_layout(P.n, P.npad, P.hmax);
    unsigned char* s_gh = smem + Lo.gh;
    unsigned char* s_gl = smem + Lo.gl;
    unsigned char* s_xt = smem + Lo.xt;
    unsigned char* s_yh = smem + Lo.yh;
    unsigned char* stages = smem + Lo.stages;
    float* ring = reinterpret_cast<float*>(smem + Lo.ring);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + Lo.bars);
    uint64_t* full = bars;                  // [kStages] stage landed
    uint64_t* empty = full + kStages;       // [kStages] stage released by every pixel warp
    uint64_t* afull = empty + kStages;      // [2] A buffer written by every pixel warp
    uint64_t* aempty = afull + 2;           // [2] MMAs reading the A buffer done
    uint64_t* yfull = aempty + 2;           // [2] fitted-value piece computed
    uint64_t* yempty = yfull + 2;           // [2] fitted-value piece read by every pixel warp
    uint64_t* accd = yempty + 2;            // pass A sums complete
    uint64_t* cdone = accd + 1;             // refinement sums complete
    uint64_t* coefb = cdone + 1;            // coefficient operands written (two uses per block)
    uint64_t* dminb = coefb + 1;            // earliest window start of the block published
    uint64_t* finb = dminb + 1;             // the MMA warp's last MMAs done
    uint64_t* tabb = finb + 1;              // batch: earlier MMAs done / a tile's tables landed
    uint32_t* s_tmem = reinterpret_cast<uint32_t*>(tabb + 1);
    int* s_dstart = reinterpret_cast<int*>(s_tmem + 1);  // [2], by block parity
    volatile uint32_t* abort_flag = s_tmem + 3;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if constexpr (!kBatch) {
        const int npad = P.npad;
        const size_t nh16 = (size_t)((P.n + 15) & ~15);
        auto copy = [&](unsigned char* dst, size_t src_off, size_t bytes) {
            const uint4* s = reinterpret_cast<const uint4*>(P.tabs + src_off);
            uint4* d = reinterpret_cast<uint4*>(dst);
            for (size_t i = tid; i < bytes / 16; i += kThreads) d[i] = __ldg(s + i);
        };
        copy(s_gh, 0, nh16 / 8 * 384);
        copy(s_gl, tab_gram_lo(npad), nh16 / 8 * 384);
        copy(s_xt, tab_x(npad), nh16 / 4 * 256);
        copy(s_yh, tab_yhat(npad), tab_yhat_bytes(npad));
    }
    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            ptx::mbar_init(full + s, 1);
            ptx::mbar_init(empty + s, kCons);
        }
        for (int b = 0; b < 2; ++b) {
            ptx::mbar_init(afull + b, kCons);
            ptx::mbar_init(aempty + b, 1);
            ptx::mbar_init(yfull + b, 1);
            ptx::mbar_init(yempty + b, kCons);
        }
        ptx::mbar_init(accd, 1);
        ptx::mbar_init(cdone, 1);
        ptx::mbar_init(coefb, kCons);
        ptx::mbar_init(dminb, kCons);
        ptx::mbar_init(finb, 1);
        ptx::mbar_init(tabb, 1);
        s_dstart[0] = INT_MAX;
        s_dstart[1] = INT_MAX;
        *abort_flag = 0u;
        ptx::fence_mbar_init();
    }
    if (warp == kMmaWarp) ptx::tmem_alloc(s_tmem, kTmemCols);
    ptx::fence_async_smem();  // tables written by the threads, read by the tensor cores
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem = *s_tmem;

    // 512-pixel work blocks; the tile of block wb and the block's first pixel in it
    const int64_t nwork = kBatch ? Bt.blocks : (P.m + kPx - 1) / kPx;
    auto locate = [&](int64_t wb, int& ti, int64_t& px0) {
        if constexpr (kBatch) {
            int lo = 0, hi = Bt.ntiles - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (Bt.tiles[mid].block0 <= wb)
                    lo = mid;
                else
                    hi = mid - 1;
            }
            ti = lo;
            px0 = (wb - Bt.tiles[lo].block0) * kPx;
        } else {
            ti = 0;
            px0 = wb * kPx;
        }
    };
    auto dstart_of = [](int v, int n) -> int {
        const int d = v < n ? v : n;
        return d / G * G;
    };

    if (warp == kProdWarp) {
        // ---------------- TMA producer: passes A, B' over the history, C from the window start
        if (lane == 0) {
            if constexpr (!kBatch) ptx::prefetch_tmap(&tmap);
            const uint64_t keep = l2_evict_last(), normal = l2_evict_normal(), drop = l2_evict_first();
            int64_t js = 0;
            bool ok = true;
            uint32_t dpar = 0;
            auto issue = [&](const CUtensorMap* tm, int64_t px0, int d0, uint64_t pol) -> bool {
                const int slot = (int)(js % kStages);
                if (js >= kStages &&
                    !wait_released(empty + slot, (uint32_t)(((js / kStages) - 1) & 1), abort_flag, kWaitNs)) {
                    raise_abort(abort_flag);
                    return false;
                }
                if (*abort_flag) return false;
                unsigned char* dst = stages + slot * kStageBytes;
                ptx::mbar_arrive_expect_tx(full + slot, (uint32_t)kStageBytes);
#pragma unroll
                for (int g = 0; g < kMT; ++g) tma_box(dst + g * kBoxBytes, tm, full + slot, (int)(px0 + g * kBoxPx), d0, pol);
                ++js;
                return true;
            };
            int it = 0, cur = -1;
            for (int64_t wb = blockIdx.x; wb < nwork && ok; wb += gridDim.x, ++it) {
                int ti;
                int64_t px0;
                locate(wb, ti, px0);
                const CUtensorMap* tm = &tmap;
                if constexpr (kBatch) {
                    tm = &Bt.tiles[ti].tm;
                    if (ti != cur) ptx::fence_tmap_acquire(tm);  // a map in global memory
                    cur = ti;
                }
                const HybridParams& Q = kBatch ? Bt.tiles[ti].P : P;
                const int n = Q.n, N = Q.N;
                const int nst_h = (n + G - 1) / G;  // stages of one history pass
                for (int s = 0; s < nst_h && ok; ++s) ok = issue(tm, px0, s * G, keep);
                for (int s = 0; s < nst_h && ok; ++s) ok = issue(tm, px0, s * G, drop);
                if (!ok) break;
                if (!wait_bar(dminb, dpar, abort_flag, kWaitNs)) {
                    raise_abort(abort_flag);
                    break;
                }
                dpar ^= 1u;
                const int ds = dstart_of(s_dstart[it & 1], n);
                for (int d0 = ds; d0 < N && ok; d0 += G) ok = issue(tm, px0, d0, normal);
            }
            // copies still in flight land before the CTA's shared memory is released
            for (int64_t i = js > kStages ? js - kStages : 0; i < js; ++i)
                ptx::mbar_wait_bounded(full + (i % kStages), (uint32_t)((i / kStages) & 1), kWaitNs);
        }
        __syncwarp();
    } else if (warp == kMmaWarp) {
        // ---------------- tensor-core issuer
        if (lane == 0) {
            const uint32_t id_g = ptx::idesc_f16(128, 32, false), id_c = ptx::idesc_f16(128, 16, false);
            const uint32_t id_x = ptx::idesc_tf32(128, 16);
            const uint32_t id_y16 = ptx::idesc_f16(128, 16, true), id_y32 = ptx::idesc_f16(128, 32, true);
            uint32_t cc = 0, pc = 0, cpar = 0;
            bool ok = true;
            // fitted values into piece buffer pc & 1: 16 dates of beta0 in pass B', 32 dates of
            // beta0 + delta in pass C.  Per coefficient set: A_hi x rows 0..15, A_hi x rows 16..31,
            // A_lo x rows 0..15 of the table (rows 16..31 start 256 bytes on).
            auto piece = [&](int d0, bool pass_c) -> bool {
                const uint32_t b = pc & 1u;
                if (pc >= 2 && !wait_bar(yempty + b, ((pc >> 1) - 1) & 1u, abort_flag, kWaitNs)) return false;
                ptx::tc_fence_after();
                const uint64_t y01 = ptx::smem_desc(s_yh + (size_t)(d0 / 8) * 384, 128, 384);
                const uint64_t y23 = ptx::smem_desc(s_yh + (size_t)(d0 / 8) * 384 + 256, 128, 384);
                const uint32_t idy = pass_c ? id_y32 : id_y16;
#pragma unroll
                for (int g = 0; g < kMT; ++g) {
                    const uint32_t base = tmem + 128u * g;
                    const uint32_t dcol = pass_c ? base + kColY + 32u * b : base + kColY0 + 16u * b;
                    ptx::mma_f16_ta(dcol, base + kColB0, y01, idy, false);
                    ptx::mma_f16_ta(dcol, base + kColB0 + 8, y23, idy, true);
                    ptx::mma_f16_ta(dcol, base + kColB0 + kCoefLo, y01, idy, true);
                    if (pass_c) {
                        ptx::mma_f16_ta(dcol, base + kColDl, y01, idy, true);
                        ptx::mma_f16_ta(dcol, base + kColDl + 8, y23, idy, true);
                        ptx::mma_f16_ta(dcol, base + kColDl + kCoefLo, y01, idy, true);
                    }
                }
                ptx::mma_commit(yfull + b);
                ++pc;
                return true;
            };
            auto wait_a = [&]() -> bool {
                const uint32_t b = cc & 1u;
                if (!wait_bar(afull + b, (cc >> 1) & 1u, abort_flag, kWaitNs)) return false;
                ptx::tc_fence_after();
                return true;
            };
            int it = 0, cur = -1;
            uint32_t tpar = 0;
            bool tab_pending = false;  // a table copy not seen to land
            for (int64_t wb = blockIdx.x; wb < nwork && ok; wb += gridDim.x, ++it) {
                int ti;
                int64_t px0;
                locate(wb, ti, px0);
                const HybridParams& Q = kBatch ? Bt.tiles[ti].P : P;
                const int n = Q.n, N = Q.N;
                const int nck = (n + 15) / 16;  // 16-date chunks of the history
                if constexpr (kBatch) {
                    if (ti != cur) {
                        // the MMAs of the previous tile have read its tables before they are replaced
                        if (cur >= 0) {
                            ptx::mma_commit(tabb);
                            if (!(ok = wait_bar(tabb, tpar, abort_flag, kWaitNs))) break;
                            tpar ^= 1u;
                        }
                        const int npad = Q.npad;
                        const uint32_t bg = (uint32_t)((n + 15) & ~15) / 8 * 384, bx = (uint32_t)((n + 15) & ~15) / 4 * 256;
                        const uint32_t by = (uint32_t)tab_yhat_bytes(npad);
                        ptx::mbar_arrive_expect_tx(tabb, 2 * bg + bx + by);
                        ptx::bulk_g2s(s_gh, Q.tabs, bg, tabb);
                        ptx::bulk_g2s(s_gl, Q.tabs + tab_gram_lo(npad), bg, tabb);
                        ptx::bulk_g2s(s_xt, Q.tabs + tab_x(npad), bx, tabb);
                        ptx::bulk_g2s(s_yh, Q.tabs + tab_yhat(npad), by, tabb);
                        tab_pending = true;
                        if (!(ok = wait_bar(tabb, tpar, abort_flag, kWaitNs))) break;
                        tab_pending = false;
                        tpar ^= 1u;
                        cur = ti;
                    }
                }
                // pass A: masked basis sums and X'My
                for (int c = 0; c < nck && ok; ++c) {
                    if (!(ok = wait_a())) break;
                    const uint32_t b = cc & 1u;
                    const uint64_t gh = ptx::smem_desc(s_gh + (size_t)(2 * c) * 384, 384, 128);
                    const uint64_t gl = ptx::smem_desc(s_gl + (size_t)(2 * c) * 384, 384, 128);
                    const uint64_t x0 = ptx::smem_desc(s_xt + (size_t)(4 * c) * 256, 256, 128);
                    const uint64_t x1 = ptx::smem_desc(s_xt + (size_t)(4 * c + 2) * 256, 256, 128);
#pragma unroll
                    for (int g = 0; g < kMT; ++g) {
                        const uint32_t base = tmem + 128u * g, a = base + kColA + 24u * b;
                        ptx::mma_f16_ta(base + kColG, a, gh, id_g, c > 0);
                        ptx::mma_f16_ta(base + kColG, a, gl, id_g, true);
                        ptx::mma_tf32_ta(base + kColB, a + 8, x0, id_x, c > 0);
                        ptx::mma_tf32_ta(base + kColB, a + 16, x1, id_x, true);
                    }
                    ptx::mma_commit(aempty + b);
                    ++cc;
                }
                if (!ok) break;
                ptx::mma_commit(accd);
                // pass B': fitted values of beta0, refinement sums X'M r0
                if (!(ok = wait_bar(coefb, cpar, abort_flag, kWaitNs))) break;
                cpar ^= 1u;
                ptx::tc_fence_after();
                for (int c = 0; c < 2 && c < nck && ok; ++c) ok = piece(16 * c, false);
                for (int c = 0; c < nck && ok; ++c) {
                    if (!(ok = wait_a())) break;
                    const uint32_t b = cc & 1u;
                    const uint64_t gh = ptx::smem_desc(s_gh + (size_t)(2 * c) * 384, 384, 128);
                    const uint64_t gl = ptx::smem_desc(s_gl + (size_t)(2 * c) * 384, 384, 128);
#pragma unroll
                    for (int g = 0; g < kMT; ++g) {
                        const uint32_t base = tmem + 128u * g, a = base + kColR + 16u * b;
                        ptx::mma_f16_ta(base + kColC, a, gh, id_c, c > 0);
                        ptx::mma_f16_ta(base + kColC, a + 8, gh, id_c, true);
                        ptx::mma_f16_ta(base + kColC, a, gl, id_c, true);
                    }
                    ptx::mma_commit(aempty + b);
                    ++cc;
                    // the pixel warps read chunk c's fitted values before they wrote its A operands
                    if (c + 2 < nck) ok = piece(16 * (c + 2), false);
                }
                if (!ok) break;
                ptx::mma_commit(cdone);
                // pass C: fitted values of beta0 + delta from the block's earliest window start
                if (!(ok = wait_bar(coefb, cpar, abort_flag, kWaitNs))) break;
                cpar ^= 1u;
                ptx::tc_fence_after();
                const int ds = dstart_of(s_dstart[it & 1], n);
                for (int d0 = ds; d0 < N && ok; d0 += 32) ok = piece(d0, true);
            }
            if (!ok) raise_abort(abort_flag);
            // a table copy in flight lands before the CTA's shared memory is released
            if (tab_pending) ptx::mbar_wait_bounded(tabb, tpar, kWaitNs);
            // every MMA issued has completed before the tensor memory is released
            ptx::mma_commit(finb);
            ptx::mbar_wait_bounded(finb, 0u, kWaitNs);
        }
        __syncwarp();
    } else {
        // ---------------- pixel warps
        const int w = warp, g = w >> 2, q = w & 3;
        const int pl = 32 * w + lane;                       // pixel within the block
        const uint32_t tl = (uint32_t)(32 * q) << 16;       // TMEM lane field of this warp
        const uint32_t tcol = tmem + 128u * (uint32_t)g;    // this M-tile's columns
        float* ring_t = ring + pl;
        const T* sbase = reinterpret_cast<const T*>(stages + (pl >> 7) * kBoxBytes) + (pl & 127);
        const float qnan = __int_as_float(0x7fc00000);
        bool bad = false;
        int cslot = 0;
        uint32_t cphase = 0;
        uint32_t cc = 0, pc = 0, accpar = 0, cdpar = 0, dpar = 0;
        // Wait for the next stage and return this thread's column in it.  Fast path:
        // one look at the barrier and a warp vote; the bounded wait (which also ends
        // on the abort flag) only when some lane finds the stage not yet landed.  A
        // bound below 1 us (a test of the failure path) makes that look a
        // non-blocking one and the only one.  A warp whose wait gives up raises the
        // abort flag and is `bad` from then on (warp-uniform): it may finish reading
        // the chunk it is in, whose contents no longer matter (its pixels end as
        // TIMEOUT), but it releases no stage, so the producer never refills a slot
        // whose copy may still be in flight.
        const bool test_mode = P.wait_ns < 1000u;
        auto acquire = [&]() -> const T* {
            const int slot = cslot;
            bool ok = !test_mode && ptx::mbar_try_wait(full + slot, cphase);
            if (!__all_sync(~0u, ok)) {
                if (!ok)
                    ok = test_mode ? ptx::mbar_test_wait(full + slot, cphase)
                                   : wait_bar(full + slot, cphase, abort_flag, P.wait_ns);
                if (__any_sync(~0u, !ok)) {
                    if (lane == 0) raise_abort(abort_flag);
                    bad = true;
                }
            }
            return sbase + slot * (kStageBytes / (int)sizeof(T));
        };
        auto release = [&]() {
            __syncwarp();
            if (lane == 0 && !bad) mbar_arrive(empty + cslot);
            const int ns = cslot + 1;
            cphase ^= ns == kStages ? 1u : 0u;
            cslot = ns == kStages ? 0 : ns;
        };
        auto wait_w = [&](uint64_t* bar, uint32_t parity) -> bool {  // warp-uniform bounded wait
            bool ok = ptx::mbar_try_wait(bar, parity);
            if (!__all_sync(~0u, ok)) {
                if (!ok) ok = wait_bar(bar, parity, abort_flag, kWaitNs);
                if (__any_sync(~0u, !ok)) {
                    if (lane == 0) raise_abort(abort_flag);
                    bad = true;
                    return false;
                }
            }
            return true;
        };
        auto arrive = [&](uint64_t* bar) {  // after this warp's TMEM accesses
            ptx::tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(bar);
        };
        auto write_unfitted = [&](const HybridParams& Q, int64_t p, int st) {
            Q.brk[p] = -1;
            Q.mean[p] = qnan;
            Q.sigma[p] = qnan;
#pragma unroll
            for (int a = 0; a < K; ++a) Q.beta[(size_t)a * Q.m + p] = qnan;
            Q.status[p] = (uint8_t)st;
            if (Q.maxmo) Q.maxmo[p] = qnan;
        };

        int it = 0;
        int64_t wb = blockIdx.x;
        for (; wb < nwork; wb += gridDim.x, ++it) {
            int ti;
            int64_t px0;
            locate(wb, ti, px0);
            const HybridParams& Q = kBatch ? Bt.tiles[ti].P : P;
            const int n = Q.n, N = Q.N, hmax = Q.hmax;
            const int nck = (n + 15) / 16;  // 16-date chunks of the history
            const int64_t m = Q.m;
            const int64_t p = px0 + pl;
            const bool active = p < m;
            Obs<T, kMask> ob{kMask ? Q.mask + (active ? (p >> 5) : 0) : nullptr, (size_t)Q.mask_words,
                             1u << (p & 31)};

            // ---- pass A: A operands of the masked basis sums and X'My
            float ymax = 0.f;
            for (int c = 0; c < nck && !bad; ++c) {
                const uint32_t b = cc & 1u;
                if (cc >= 2 && !wait_w(aempty + b, ((cc >> 1) - 1) & 1u)) break;
                ptx::tc_fence_after();
                uint32_t yv[16], mk[8];
                const T* stg = nullptr;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int d8 = 16 * c + 8 * h;
                    if (d8 < n) {  // warp-uniform: the dates exist
                        if (h == 0 || G == 8) stg = acquire();
                        const T* st = stg + (G == 16 ? h * 8 * kBoxPx : 0);
                        if (d8 + 8 <= n)
                            pass_a8<true>(ob, st, d8, n, yv + 8 * h, mk + 4 * h, ymax);
                        else
                            pass_a8<false>(ob, st, d8, n, yv + 8 * h, mk + 4 * h, ymax);
                        if (G == 8 || h == 1 || d8 + 8 >= n) release();
                    } else {
#pragma unroll
                        for (int u = 0; u < 8; ++u) yv[8 * h + u] = 0u;
#pragma unroll
                        for (int j = 0; j < 4; ++j) mk[4 * h + j] = 0u;
                    }
                }
                if (bad) break;
                const uint32_t a = tl + tcol + kColA + 24u * b;
                ptx::tmem_st8(a, mk);
                ptx::tmem_st16(a + 8, yv);
                ptx::tmem_wait_st();
                arrive(afull + b);
                ++cc;
            }
            if (bad) break;
            if (!wait_w(accd, accpar)) break;
            accpar ^= 1u;
            ptx::tc_fence_after();
            float S[NBR], Bv[K];
            {
                float v32[32], v16[16];
                ptx::tmem_ld32(tl + tcol + kColG, v32);
                ptx::tmem_ld16(tl + tcol + kColB, v16);
#pragma unroll
                for (int i = 0; i < NBR; ++i) S[i] = v32[i];
#pragma unroll
                for (int a = 0; a < K; ++a) Bv[a] = v16[a] + v16[8 + a];
            }
            const int np = (int)S[0];  // basis row 0 is 1: the count of valid history dates
            {
                uint32_t w16[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) w16[i] = i < NBR ? __float_as_uint(S[i]) : 0u;
                ptx::tmem_st16(tl + tcol + kColS, w16);
                if constexpr (NBR > 16) {
                    uint32_t w8[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) w8[i] = 16 + i < NBR ? __float_as_uint(S[16 + i]) : 0u;
                    ptx::tmem_st8(tl + tcol + kColS + 16, w8);
                }
            }
            float b0[K];
            bool nonsingular;
            {
                float Gm[K][K], Lc[K][K], dinv[K];
                gram_from_sums<KH>(S, Gm);
                nonsingular = cholesky<K>(Gm, Lc, dinv);
                chol_solve<K>(Lc, dinv, Bv, b0);
            }
            // operand scales (powers of two): |beta0| * s_b < 2^13; |r0| <= max|y| + sum|beta0|
            // (|x_i| <= 1 with the centred trend), so |r0| * s_r < 2^13
            float s_b, s_r;
            {
                float bm = 0.f, bs = 0.f;
#pragma unroll
                for (int a = 0; a < K; ++a) {
                    bm = fmaxf(bm, fabsf(b0[a]));
                    bs += fabsf(b0[a]);
                }
                s_b = pow2_scale(bm, 12);
                s_r = pow2_scale(ymax + bs, 12);
                if (!(bs < INFINITY)) {  // a singular pixel: keep every operand finite
                    s_b = 1.f;
                    s_r = 1.f;
#pragma unroll
                    for (int a = 0; a < K; ++a) b0[a] = 0.f;
                }
            }
            const float inv_sb = 1.f / s_b, inv_sr = 1.f / s_r;
            const float inv_fit = inv_sb * kInvYScale;  // the fitted values come out scaled by s_b 2^12
            {
                uint32_t wv[24];
                float rep[K];
                coef_words<K>(b0, s_b, wv, rep);
                coef_store(tl + tcol + kColB0, wv);
                ptx::tmem_wait_st();
                arrive(coefb);
            }
            const bool fit = np > K && nonsingular;
            int hp = (int)floor(Q.h_frac * (double)np);
            hp = hp < 1 ? 1 : (hp > np ? np : hp);
            if (!fit) hp = 1;  // keeps the ring arithmetic in range; nothing of it is used
            hp = hp > hmax ? hmax : hp;  // n_p <= n_hist, so this never binds: the ring holds hmax slots
            const int wq = fit ? np - hp + 1 : np;  // 0-based valid rank of the first window's oldest history obs

            // ---- pass B': r0 = y - yhat0, s0, A operands of X'M r0, the window's start date
            float ss0 = 0.f;
            int rem = wq, wdate = n;
            for (int c = 0; c < nck && !bad; ++c) {
                if (!wait_w(yfull + (pc & 1u), (pc >> 1) & 1u)) break;
                ptx::tc_fence_after();
                float yh[16];
                ptx::tmem_ld16(tl + tcol + kColY0 + 16u * (pc & 1u), yh);
                arrive(yempty + (pc & 1u));
                ++pc;
                const uint32_t b = cc & 1u;
                if (cc >= 2 && !wait_w(aempty + b, ((cc >> 1) - 1) & 1u)) break;
                ptx::tc_fence_after();
                uint32_t hw[8], lw[8];
                const T* stg = nullptr;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int d8 = 16 * c + 8 * h;
                    if (d8 < n) {
                        if (h == 0 || G == 8) stg = acquire();
                        const T* st = stg + (G == 16 ? h * 8 * kBoxPx : 0);
                        const bool scan = __any_sync(~0u, rem < 8);  // a pixel may reach its window start
                        const bool fullb = d8 + 8 <= n;
                        if (scan) {
                            if (fullb)
                                pass_b8<true, true>(ob, st, d8, n, yh + 8 * h, inv_fit, s_r, ss0, hw + 4 * h,
                                                    lw + 4 * h, rem, wdate);
                            else
                                pass_b8<false, true>(ob, st, d8, n, yh + 8 * h, inv_fit, s_r, ss0, hw + 4 * h,
                                                     lw + 4 * h, rem, wdate);
                        } else {
                            if (fullb)
                                pass_b8<true, false>(ob, st, d8, n, yh + 8 * h, inv_fit, s_r, ss0, hw + 4 * h,
                                                     lw + 4 * h, rem, wdate);
                            else
                                pass_b8<false, false>(ob, st, d8, n, yh + 8 * h, inv_fit, s_r, ss0, hw + 4 * h,
                                                      lw + 4 * h, rem, wdate);
                        }
                        if (G == 8 || h == 1 || d8 + 8 >= n) release();
                    } else {
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            hw[4 * h + j] = 0u;
                            lw[4 * h + j] = 0u;
                        }
                    }
                }
                if (bad) break;
                const uint32_t a = tl + tcol + kColR + 16u * b;
                ptx::tmem_st8(a, hw);
                ptx::tmem_st8(a + 8, lw);
                ptx::tmem_wait_st();
                arrive(afull + b);
                ++cc;
            }
            if (bad) break;
            if (!wait_w(cdone, cdpar)) break;
            cdpar ^= 1u;
            ptx::tc_fence_after();
            float cr[K];
            {
                float v16[16];
                ptx::tmem_ld16(tl + tcol + kColC, v16);
#pragma unroll
                for (int a = 0; a < K; ++a) cr[a] = v16[a] * inv_sr;
            }
            float dl[K];
            {
                float S2[NBR];
                {
                    float v16[16];
                    ptx::tmem_ld16(tl + tcol + kColS, v16);
#pragma unroll
                    for (int i = 0; i < 16 && i < NBR; ++i) S2[i] = v16[i];
                    if constexpr (NBR > 16) {
                        float v8[8];
                        ptx::tmem_ld8(tl + tcol + kColS + 16, v8);
#pragma unroll
                        for (int i = 16; i < NBR; ++i) S2[i] = v8[i - 16];
                    }
                }
                float Gm[K][K], Lc[K][K], dinv[K];
                gram_from_sums<KH>(S2, Gm);
                cholesky<K>(Gm, Lc, dinv);
                chol_solve<K>(Lc, dinv, cr, dl);
            }
            float dc = 0.f;
#pragma unroll
            for (int a = 0; a < K; ++a) dc = fmaf(dl[a], cr[a], dc);
            const float sig = sqrtf(fmaxf(ss0 - dc, 0.f) / (float)(np - K));
            const bool degenerate = !(sig > kDegenerateRatio * ymax) || ymax == 0.f;
            // beta of the centred trend: beta0 as the MMAs see it (c_hi + c_lo of its coefficient
            // words, unscaled; read back rather than kept in registers through pass B') plus delta.
            // The TMEM loads are warp-collective, so every lane takes them, before any branch.
            float bt[K];
            {
                float wh[8], wl[8];
                ptx::tmem_ld8(tl + tcol + kColB0, wh);
                ptx::tmem_ld8(tl + tcol + kColB0 + kCoefLo, wl);
#pragma unroll
                for (int a = 0; a < K; ++a) {
                    const uint32_t uh = __float_as_uint(wh[a >> 1]), ul = __float_as_uint(wl[a >> 1]);
                    const float h = __half2float(__ushort_as_half((unsigned short)((a & 1) ? uh >> 16 : uh)));
                    const float l = __half2float(__ushort_as_half((unsigned short)((a & 1) ? ul >> 16 : ul)));
                    bt[a] = (h + l) * inv_sb + dl[a];
                }
            }
            // outputs known now (the rest after the monitoring scan)
            if (active) {
                if (np <= K) {
                    write_unfitted(Q, p, BFM_PX_INSUFFICIENT_HISTORY);
                } else if (!nonsingular) {
                    write_unfitted(Q, p, BFM_PX_SINGULAR);
                } else {
                    Q.sigma[p] = sig;
                    // -> raw parameterisation of Eq. 2
                    Q.beta[p] = fmaf(-bt[1], Q.c_over_s, bt[0]);
                    Q.beta[(size_t)m + p] = bt[1] * Q.inv_s;
#pragma unroll
                    for (int a = 2; a < K; ++a) Q.beta[(size_t)a * m + p] = bt[a];
                }
            }
            {
                float dfin[K];
#pragma unroll
                for (int a = 0; a < K; ++a) dfin[a] = (fit && isfinite(dl[a])) ? dl[a] : 0.f;
                uint32_t wv[24];
                float rep[K];
                coef_words<K>(dfin, s_b, wv, rep);
                coef_store(tl + tcol + kColDl, wv);
            }
            // the block's earliest window start, for the producer and the MMA warp
            {
                const unsigned v = active ? (unsigned)wdate : (unsigned)n;
                const unsigned wmn = __reduce_min_sync(~0u, v);
                if (lane == 0) atomicMin(&s_dstart[it & 1], (int)wmn);
            }
            ptx::tmem_wait_st();
            ptx::tc_fence_before();
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(dminb);
                mbar_arrive(coefb);
            }
            if (!wait_w(dminb, dpar)) break;
            dpar ^= 1u;
            const int ds = dstart_of(s_dstart[it & 1], n);
            if (tid == 0) s_dstart[(it + 1) & 1] = INT_MAX;

            // ---- pass C: window fill from the history, then the monitoring scan
            const float inv_scale = (fit && !degenerate) ? 1.f / (sig * sqrtf((float)np)) : 0.f;
            const float inv2 = inv_scale * inv_scale;
            const float lam2 = Q.lam2, lam2ln2 = lam2 * kLn2f, blg = lam2ln2 * log2_fast((float)np);
            float* const maxmo = Q.maxmo;
            const float jlimf = (float)floor(kEuler * (double)np);  // J / n_p <= e  <=>  J <= jlim
            Mon mo{};
            mo.hp_off = hp * kPx;
            mo.fill_end = (hp - 1) * kPx;
            mo.wdate = wdate;
            mo.inv_sb = inv_fit;
            ring_t[(hp - 1) * kPx] = 0.f;  // the first monitoring step finds h_p - 1 residuals
            int brk = -1;
            float sh = 0.f, sl = 0.f;
            const T* stg = nullptr;
            for (int d8 = ds; d8 < N && !bad; d8 += 8) {
                const int off = d8 - ds;
                if ((off & 31) == 0 && !wait_w(yfull + (pc & 1u), (pc >> 1) & 1u)) break;
                ptx::tc_fence_after();
                if (off % G == 0) {
                    stg = acquire();
                }
                const T* st = stg + (off % G);  // dates of the stage are rows of kBoxPx elements
                const T* st8 = stg + (off % G) * kBoxPx;
                (void)st;
                float yh[8];
                ptx::tmem_ld8(tl + tcol + kColY + 32u * (pc & 1u) + (uint32_t)(off & 31), yh);
                if ((off & 31) == 24 || d8 + 8 >= N) {
                    arrive(yempty + (pc & 1u));
                    ++pc;
                }
                if (d8 + 8 <= n) {
                    mon_hist8(ob, st8, d8, yh, ring_t, mo);
                } else {
                    const int J0 = np + 1 + mo.cnt;
                    float Wu[8];
                    mo.blk = 0.f;
                    mo.amax = 0.f;
                    if (d8 >= n && d8 + 8 <= N) {
                        if (maxmo)
                            mon8<true, true>(ob, st8, d8, N, yh, ring_t, mo, Wu);
                        else
                            mon8<true, false>(ob, st8, d8, N, yh, ring_t, mo, Wu);
                    } else {
                        mon_mixed8(ob, st8, d8, n, N, yh, ring_t, mo, Wu, maxmo != nullptr);
                    }
                    comp_add(sh, sl, mo.blk);
                    // the boundary grows with the position: a stretch whose largest |MO| stays
                    // within the boundary at its first position holds no crossing (lowered by
                    // 1e-6 relative, so that rounding of the boundary never hides a crossing)
                    if (brk < 0) {
                        const float Jf0 = (float)J0;
                        const float b2f = (Jf0 > jlimf ? fmaf(lam2ln2, log2_fast(Jf0), -blg) : lam2) * 0.999999f;
                        if (fmaf(mo.amax * mo.amax, inv2, -b2f) > 0.f) {
                            float Jc = Jf0;
#pragma unroll
                            for (int u = 0; u < 8; ++u) {
                                const int d = d8 + u;
                                if (d >= n && ob.valid(st8[u * kBoxPx], d, d < N)) {
                                    const float b2 = Jc > jlimf ? fmaf(lam2ln2, log2_fast(Jc), -blg) : lam2;
                                    if (brk < 0 && fmaf(Wu[u] * Wu[u], inv2, -b2) > 0.f) brk = d;
                                    Jc += 1.f;
                                }
                            }
                        }
                    }
                }
                if ((off % G) + 8 == G || d8 + 8 >= N) release();
            }
            if (bad) break;
            if (!active) continue;

            const int Np = np + mo.cnt;
            if (fit) {
                if (degenerate) {
                    Q.status[p] = BFM_PX_DEGENERATE;
                    Q.brk[p] = -1;
                    Q.mean[p] = 0.f;
                    if (maxmo) maxmo[p] = 0.f;
                } else if (Np == np) {
                    Q.status[p] = BFM_PX_NO_MONITOR;
                    Q.brk[p] = -1;
                    Q.mean[p] = qnan;
                    if (maxmo) maxmo[p] = qnan;
                } else {
                    Q.status[p] = BFM_PX_OK;
                    Q.brk[p] = brk;
                    Q.mean[p] = (sh + sl) * inv_scale / (float)(Np - np);
                    // largest |MO| (positive on an exact tie of opposite signs)
                    if (maxmo) maxmo[p] = (mo.wmax >= -mo.wmin ? mo.wmax : mo.wmin) * inv_scale;
                }
            }
        }
        if (bad) {
            // a wait gave up: mark this thread's unfinished pixels
            for (; wb < nwork; wb += gridDim.x) {
                int ti;
                int64_t px0;
                locate(wb, ti, px0);
                const HybridParams& Q = kBatch ? Bt.tiles[ti].P : P;
                if (px0 + pl < Q.m) write_unfitted(Q, px0 + pl, BFM_PX_TIMEOUT);
            }
        }
    }
    ptx::tc_fence_before();
    __syncthreads();
    if (warp == kMmaWarp) {
        ptx::tc_fence_after();
        ptx::tmem_dealloc(tmem, kTmemCols);
    }
}

template <int KH, typename T, bool kMask>
bfm_status launch_one(const CUtensorMap& tm, const HybridParams& P, int grid, size_t smem, cudaStream_t st) {
    auto* fn = hybrid_kernel<KH, T, kMask, false>;
    // the opt-in maximum, not this launch's size: launches of other sizes (other
    // scenes, other host threads) never find a smaller limit in place
    const cudaError_t ea = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemCap);
    if (ea != cudaSuccess) return cuda_fail(ea, "bfm_monitor (hybrid): shared memory attribute");
    fn<<<grid, kThreads, smem, st>>>(tm, P, HybBatch{});
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "bfm_monitor (hybrid): launch");
    return BFM_OK;
}

template <int KH>
bfm_status launch_kh(const CUtensorMap& tm, const HybridParams& P, int dtype, int grid, size_t smem,
                     cudaStream_t st) {
    if (dtype == BFM_F32)
        return P.mask ? launch_one<KH, float, true>(tm, P, grid, smem, st)
                      : launch_one<KH, float, false>(tm, P, grid, smem, st);
    return P.mask ? launch_one<KH, int16_t, true>(tm, P, grid, smem, st)
                  : launch_one<KH, int16_t, false>(tm, P, grid, smem, st);
}

int hyb_hmax(int n_hist, double h_frac) {
    int h = (int)std::floor(h_frac * (double)n_hist);
    return h < 1 ? 1 : (h > n_hist ? n_hist : h);
}

int hyb_npad(int N) { return (N + 31) / 32 * 32 + 32; }

}  // namespace

// Design tables of the hybrid form for npad = hyb_npad(N) dates (zero beyond N):
//   Gram hi, Gram lo: the 3 + 6k basis functions (bfm::Basis order) split fp16
//     hi + lo, K-major over dates, three 8-row groups per 8-date group:
//     (t/8)*384 + (r/8)*128 + (r%8)*16 + (t%8)*2 (an MMA with N = 32 reads its
//     fourth row group from the next date group: accumulator columns 24..31,
//     which nothing reads);
//   X: the K regressors as tf32 hi (rows 0..7) and lo = x - hi (rows 8..15),
//     K-major over dates: (t/4)*256 + (r/8)*128 + (r%8)*16 + (t%4)*4;
//   fitted values: the K regressors times 2^12 split three ways into fp16 hi
//     (rows 0..7), mid (8..15) and lo (16..23), read MN-major:
//     (t/8)*384 + (r/8)*128 + (r%8)*16 + (t%8)*2, plus one group of zeros at
//     the end (rows 24..31 of the last group are read from it and meet zero
//     coefficients).
void hybrid_tables(const bfm_design_s& d, const std::vector<double>& rows, std::vector<unsigned char>& out) {
    const int npad = hyb_npad(d.N), nbr = 3 + 6 * d.k, K = d.K;
    out.assign(tab_bytes(npad), 0);
    unsigned char* gh = out.data();
    unsigned char* gl = out.data() + tab_gram_lo(npad);
    unsigned char* xt = out.data() + tab_x(npad);
    unsigned char* yh = out.data() + tab_yhat(npad);
    for (int t = 0; t < d.N; ++t) {
        for (int r = 0; r < nbr; ++r) {
            const double v = rows[(size_t)t * d.NB + r];
            const __half hi = __double2half(v);
            const __half lo = __double2half(v - (double)__half2float(hi));
            const size_t o = (size_t)(t / 8) * 384 + (size_t)(r / 8) * 128 + (size_t)(r % 8) * 16 + (size_t)(t % 8) * 2;
            std::memcpy(gh + o, &hi, 2);
            std::memcpy(gl + o, &lo, 2);
        }
        for (int r = 0; r < K; ++r) {
            const double v = rows[(size_t)t * d.NB + r];
            // tf32 keeps the top 10 stored mantissa bits: hi by truncation, lo exact in float
            uint32_t bits;
            const float vf = (float)v;
            std::memcpy(&bits, &vf, 4);
            bits &= 0xFFFFE000u;
            float hif;
            std::memcpy(&hif, &bits, 4);
            const float lof = (float)(v - (double)hif);
            std::memcpy(xt + (size_t)(t / 4) * 256 + (size_t)(r % 8) * 16 + (size_t)(t % 4) * 4, &hif, 4);
            std::memcpy(xt + (size_t)(t / 4) * 256 + 128 + (size_t)(r % 8) * 16 + (size_t)(t % 4) * 4, &lof, 4);
            const double vs = v * (double)kYScale;
            const __half h1 = __double2half(vs);
            const double r1 = vs - (double)__half2float(h1);
            const __half h2 = __double2half(r1);
            const __half h3 = __double2half(r1 - (double)__half2float(h2));
            const size_t oy = (size_t)(t / 8) * 384 + (size_t)(r % 8) * 16 + (size_t)(t % 8) * 2;
            std::memcpy(yh + oy, &h1, 2);
            std::memcpy(yh + oy + 128, &h2, 2);
            std::memcpy(yh + oy + 256, &h3, 2);
        }
    }
}

size_t hybrid_table_bytes(int N) { return tab_bytes(hyb_npad(N)); }

bool hybrid_supported(const bfm_design_s* d, int dtype, int n_hist, double h_frac, const void* Y, int64_t m) {
    const size_t elt = dtype == BFM_F32 ? 4 : 2;
    if (!d->d_hyb || m < 1 || (uintptr_t)Y % 16 != 0 || ((size_t)m * elt) % 16 != 0) return false;
    return hyb_layout(n_hist, hyb_npad(d->N), hyb_hmax(n_hist, h_frac)).total <= kSmemCap;
}

namespace {

// Parameters and tensor map of one tile (false, with a message, when the
// hybrid form does not take it).
bool hyb_fill(const bfm_design_s* d, int dtype, const void* Y, const uint32_t* mask, int64_t m, int n_hist,
              double h_frac, double lambda, int32_t* brk, float* mean, float* sigma, float* beta, uint8_t* status,
              float* maxmo, HybridParams* Pout, CUtensorMap* tm) {
    if (!hybrid_supported(d, dtype, n_hist, h_frac, Y, m)) {
        set_error("the hybrid form needs Y with a 16-byte aligned base and rows of a multiple of 16 bytes, and "
                  "basis tables, stages and a residual ring of floor(h_frac * n_hist) slots for 512 pixels within "
                  "the shared memory of one SM");
        return false;
    }
    auto enc = encode_tiled();
    if (!enc) {
        set_error("hybrid form: cuTensorMapEncodeTiled is not available");
        return false;
    }
    const size_t elt = dtype == BFM_F32 ? 4 : 2;
    HybridParams P{};
    P.wait_ns = stage_wait_ns();
    P.mask = mask;
    P.m = m;
    P.mask_words = (m + 31) / 32;
    P.N = d->N;
    P.n = n_hist;
    P.hmax = hyb_hmax(n_hist, h_frac);
    P.npad = hyb_npad(d->N);
    P.h_frac = h_frac;
    P.tabs = static_cast<const unsigned char*>(d->d_hyb);
    P.lam2 = (float)(lambda * lambda);
    P.c_over_s = (float)(d->c / d->s);
    P.inv_s = (float)(1.0 / d->s);
    P.brk = brk;
    P.mean = mean;
    P.sigma = sigma;
    P.beta = beta;
    P.status = status;
    P.maxmo = maxmo;
    std::memset(tm, 0, sizeof *tm);
    const int G = dtype == BFM_F32 ? Dt<float>::G : Dt<int16_t>::G;
    const cuuint64_t gdim[2] = {(cuuint64_t)m, (cuuint64_t)d->N};
    const cuuint64_t gstride[1] = {(cuuint64_t)m * elt};
    const cuuint32_t box[2] = {(cuuint32_t)kBoxPx, (cuuint32_t)G};
    const cuuint32_t es[2] = {1u, 1u};
    if (enc(tm, elt == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_UINT16, 2,
            const_cast<void*>(Y), gdim, gstride, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS) {
        set_error("hybrid form: cuTensorMapEncodeTiled failed for Y");
        return false;
    }
    *Pout = P;
    return true;
}

int sm_count_cur() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 1;
    return sms;
}

}  // namespace

bfm_status launch_hybrid(const bfm_design_s* d, int dtype, const void* Y, const uint32_t* mask, int64_t m,
                         int n_hist, double h_frac, double lambda, int32_t* brk, float* mean, float* sigma,
                         float* beta, uint8_t* status, cudaStream_t stream, float* maxmo) {
    HybridParams P;
    CUtensorMap tm;
    if (!hyb_fill(d, dtype, Y, mask, m, n_hist, h_frac, lambda, brk, mean, sigma, beta, status, maxmo, &P, &tm))
        return BFM_EUNSUPPORTED;
    const int sms = sm_count_cur();
    const int64_t ntiles = (m + kPx - 1) / kPx;
    const int grid = (int)(ntiles < (int64_t)sms ? ntiles : (int64_t)sms);
    const size_t smem = hyb_layout(n_hist, P.npad, P.hmax).total;
    if (d->k == 1) return launch_kh<1>(tm, P, dtype, grid, smem, stream);
    if (d->k == 2) return launch_kh<2>(tm, P, dtype, grid, smem, stream);
    return launch_kh<3>(tm, P, dtype, grid, smem, stream);
}

// ---- batched launch (bfm_batch) --------------------------------------------------------------

struct HybGroup {
    int k, dtype;
    bool mask;
    int nmax = 0, npadmax = 0, hmaxmax = 0;  // the layout holds the largest of each
    int64_t blocks = 0;
    std::vector<HybBatchTile> tiles;
    HybBatchTile* d_tiles = nullptr;
    bool dirty = true;
};

HybGroup* hyb_group_create(int k, int dtype, bool has_mask) {
    auto* g = new HybGroup;
    g->k = k;
    g->dtype = dtype;
    g->mask = has_mask;
    return g;
}

void hyb_group_destroy(HybGroup* g) {
    if (!g) return;
    if (g->d_tiles) cudaFree(g->d_tiles);
    delete g;
}

bool hyb_group_variant(const HybGroup* g, int k, int dtype, bool has_mask) {
    return g->k == k && g->dtype == dtype && g->mask == has_mask;
}

int hyb_group_add(HybGroup* g, const bfm_design_s* d, const void* Y, const uint32_t* mask, int64_t m, int n_hist,
                  double h_frac, double lambda, int32_t* brk, float* mean, float* sigma, float* beta,
                  uint8_t* status) {
    HybBatchTile t;
    if (!hyb_fill(d, g->dtype, Y, mask, m, n_hist, h_frac, lambda, brk, mean, sigma, beta, status, nullptr, &t.P,
                  &t.tm))
        return -1;
    const int nmax = std::max(g->nmax, n_hist), npadmax = std::max(g->npadmax, t.P.npad),
              hmaxmax = std::max(g->hmaxmax, t.P.hmax);
    if (hyb_layout(nmax, npadmax, hmaxmax).total > kSmemCap) return 0;
    g->nmax = nmax;
    g->npadmax = npadmax;
    g->hmaxmax = hmaxmax;
    t.block0 = g->blocks;
    g->blocks += (m + kPx - 1) / kPx;
    g->tiles.push_back(t);
    g->dirty = true;
    return 1;
}

bfm_status hyb_group_upload(HybGroup* g) {
    if (!g->dirty) return BFM_OK;
    if (g->d_tiles) cudaFree(g->d_tiles);
    g->d_tiles = nullptr;
    cudaError_t e = cudaMalloc(&g->d_tiles, sizeof(HybBatchTile) * g->tiles.size());
    if (e == cudaSuccess)
        e = cudaMemcpy(g->d_tiles, g->tiles.data(), sizeof(HybBatchTile) * g->tiles.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "bfm_batch: uploading hybrid tile descriptors");
    g->dirty = false;
    return BFM_OK;
}

namespace {
template <int KH, typename T, bool kMask>
void* hyb_batch_fn() {
    return (void*)hybrid_kernel<KH, T, kMask, true>;
}
}  // namespace

bfm_status hyb_group_node(HybGroup* g, cudaGraph_t graph, const cudaGraphNode_t* dep, cudaGraphNode_t* node) {
    void* fn = nullptr;
    const bool f32 = g->dtype == BFM_F32;
    switch (g->k) {
        case 1:
            fn = f32 ? (g->mask ? hyb_batch_fn<1, float, true>() : hyb_batch_fn<1, float, false>())
                     : (g->mask ? hyb_batch_fn<1, int16_t, true>() : hyb_batch_fn<1, int16_t, false>());
            break;
        case 2:
            fn = f32 ? (g->mask ? hyb_batch_fn<2, float, true>() : hyb_batch_fn<2, float, false>())
                     : (g->mask ? hyb_batch_fn<2, int16_t, true>() : hyb_batch_fn<2, int16_t, false>());
            break;
        default:
            fn = f32 ? (g->mask ? hyb_batch_fn<3, float, true>() : hyb_batch_fn<3, float, false>())
                     : (g->mask ? hyb_batch_fn<3, int16_t, true>() : hyb_batch_fn<3, int16_t, false>());
            break;
    }
    HybBatch bt{};
    bt.tiles = g->d_tiles;
    bt.ntiles = (int)g->tiles.size();
    bt.blocks = g->blocks;
    bt.lo = hyb_layout(g->nmax, g->npadmax, g->hmaxmax);
    const size_t smem = bt.lo.total;
    // the opt-in maximum: other groups of the same variant may need more than this one
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemCap);
    if (e != cudaSuccess) return cuda_fail(e, "bfm_batch: hybrid kernel shared memory attribute");
    // the single-tile parameters are unused but for the stage-wait bound
    static CUtensorMap tm_unused;  // zero; never read by the batched kernel
    HybridParams P{};
    P.wait_ns = g->tiles.empty() ? stage_wait_ns() : g->tiles[0].P.wait_ns;
    void* args[3] = {&tm_unused, &P, &bt};
    const int sms = sm_count_cur();
    cudaKernelNodeParams kp{};
    kp.func = fn;
    kp.gridDim = dim3((unsigned)std::min<int64_t>(g->blocks, sms));
    kp.blockDim = dim3(kThreads);
    kp.sharedMemBytes = (unsigned)smem;
    kp.kernelParams = args;
    e = cudaGraphAddKernelNode(node, graph, dep, dep ? 1 : 0, &kp);
    if (e != cudaSuccess) return cuda_fail(e, "bfm_batch: hybrid kernel node");
    return BFM_OK;
}

int64_t hyb_group_blocks(const HybGroup* g) { return g->blocks; }

}  // namespace bfm
