// Tensor-core form of the per-pixel path (int16 or float storage).
//
// One CTA = 128 pixels = the M of every tcgen05.mma = the 128 TMEM lanes,
// held by 256 threads: pixel px by the pair (px, px + 128), warps w and w + 4,
// which reach the same TMEM lane quarter.  Y arrives by TMA in [16 dates][128
// px] blocks through a ring of S shared-memory stages (3 for float, 6 for
// int16; full/empty mbarriers, one producer thread), with L2 hints: the
// history is kept (evict-last) for its second read, later dates are dropped.
// The basis tables (fp16 hi/lo, the B operand of every MMA) sit in shared
// memory: table A = basis rows 0..15 over all dates, table B = rows 16..31
// over the history.  Per tile:
//
//   normal   per 16-date chunk of the history each thread of a pair writes
//            the fp16 A-operand rows of its 8-date group: the 0/1 mask and
//            y*s_y split hi + lo (masked).  One thread issues
//              TMEM[G] += mask x (Phi_hi + Phi_lo)       (3+6k basis sums, Eq. 6)
//              TMEM[b] += (y_hi + y_lo) x (Phi_hi + Phi_lo)   (X'My, Eq. 6)
//            double-buffered against the next chunk's operand writes
//   solve    both threads of a pair: Gram from the basis sums, Cholesky,
//            beta0 (FP32)
//   refine   TMEM[Y] = [beta0_hi | beta0_lo] x Phi (table A read MN-major:
//            rows = coefficients, columns = dates), 192 dates per piece;
//            r0 = y - yhat0 on valid history dates, split hi + lo, then
//            TMEM[c] += r0 x Phi: one refinement step beta = beta0 + G^-1 c;
//            sum r^2 = sum r0^2 - delta'c (sigma-hat, Eq. 5)
//   MOSUM    per 192-date piece TMEM[Y] = X beta0 + X delta; the first
//            thread of a pair forms r = y - yhat 8 dates at a time and
//            compensated prefix sums S over valid positions in a ring; the
//            second, one group behind, the windows of h valid residuals
//            W = S_J - S_{J-h} (Eq. 3), the first crossing of
//            lambda*sqrt(log+(j/n)) (Eq. 4) and the mean
//
// Scaling: every A operand row is one pixel, so each thread scales its own
// rows by powers of two (exact) chosen from its data, keeping fp16 hi + lo
// splits inside fp16's range; results are scaled back exactly.  TMEM use is
// 256 columns per CTA and shared memory about 109 KB at 414 dates, so two
// CTAs share an SM.
#include <cuda_fp16.h>
#include <cudaTypedefs.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "bfm_internal.cuh"
#include "ptx.cuh"
#include "simt_seg.cuh"

namespace bfm {

__device__ unsigned int g_bfm_mma_err = 0;

cudaError_t mma_read_clear_errors(cudaStream_t s, unsigned int* bits) {
    unsigned int v = 0;
    cudaError_t e = cudaMemcpyFromSymbolAsync(&v, g_bfm_mma_err, sizeof v, 0, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    const unsigned int zero = 0;
    e = cudaMemcpyToSymbolAsync(g_bfm_mma_err, &zero, sizeof zero, 0, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    *bits = v;
    return e;
}

namespace {

constexpr int kTile = 128;                  // pixels per CTA
constexpr int kBlk = 16;                    // dates per Y block (TMA box height) and per A chunk
constexpr int kPlane = kTile * kBlk * 2;    // bytes of one fp16 A plane (128 x 16)
constexpr int kBufBytes = 3 * kPlane;       // one A buffer (three planes)
constexpr int kMaxStages = 8;
constexpr int kCoefPlane = kTile * 16 * 2;  // one [128 x 16] coefficient plane
constexpr uint32_t kColG = 0, kColB = 32, kColC = 48, kColY = 64;
constexpr int kPiece = 192;                 // fitted-value dates per TMEM piece
constexpr uint32_t kTmemCols = 256;         // 64 + kPiece: two CTAs fit one SM's TMEM
constexpr uint64_t kWaitNs = 2000000000ull;
constexpr uint32_t kALbo = 2048;            // A: K-direction core stride (16 row groups x 128 B)
constexpr uint32_t kTabLbo = 256;           // B tables: date-group stride (16 rows x 16 B)

__device__ __forceinline__ uint32_t pack_h2(float a, float b) {
    const __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&h);
}

// A-operand row segment: 8 consecutive K elements of row m, group g (K-major,
// core-matrix column g at g*2048 bytes).
__device__ __forceinline__ void st_a(unsigned char* plane, int m, int g, const float (&v)[8]) {
    uint4 u;
    u.x = pack_h2(v[0], v[1]);
    u.y = pack_h2(v[2], v[3]);
    u.z = pack_h2(v[4], v[5]);
    u.w = pack_h2(v[6], v[7]);
    *reinterpret_cast<uint4*>(plane + (size_t)g * kALbo + (size_t)m * 16) = u;
}

// x = hi + lo with hi exactly representable in fp16 (11 significant bits by
// truncation) and lo = x - hi exact in float; packed conversion rounds lo only.
__device__ __forceinline__ void split_hi_lo(float x, float& hi, float& lo) {
    hi = __int_as_float(__float_as_int(x) & 0xFFFFE000);
    lo = x - hi;
}

__device__ __forceinline__ uint64_t l2_policy_evict_last() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ uint64_t l2_policy_evict_first() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
// 2^(T - e) for v = 1.x * 2^e, so that |v| * scale lies in [2^T, 2^(T+1));
// 1 for zero, subnormal, infinite or NaN v.
__device__ __forceinline__ float pow2_scale(float v, int T) {
    const int e = (__float_as_int(v) >> 23) & 0xff;
    if (e == 0 || e == 0xff) return 1.f;
    int r = 254 + T - e;
    r = r < 1 ? 1 : (r > 254 ? 254 : r);
    return __int_as_float(r << 23);
}

// D (+)= A x Phi for one 16-date k-block; Phi table (K-major: dates = K,
// 16 rows = N): date-group stride 256 B, row-group stride 128 B.
__device__ __forceinline__ void mma_kb(uint32_t dcol, const unsigned char* aplane, int kb_in_chunk,
                                       const unsigned char* tab, int d0, bool acc) {
    const uint64_t ad = ptx::smem_desc(aplane + (size_t)kb_in_chunk * 2 * kALbo, kALbo, 128);
    const uint64_t bd = ptx::smem_desc(tab + (size_t)(d0 / 8) * kTabLbo, kTabLbo, 128);
    ptx::mma_f16(dcol, ad, bd, ptx::idesc_f16(kTile, 16, false), acc);
}

// X c over dates [d0, d0 + n) into TMEM column dcol: A = [c_hi | 0], [c_lo | 0]
// (K = 16 coefficient slots), B = table A read MN-major (N = dates): K-direction
// (row-group) stride 128 B, N-direction (date-group) stride 256 B.
__device__ __forceinline__ void mma_xc(uint32_t dcol, const unsigned char* chi, const unsigned char* clo,
                                       const unsigned char* tab_hi, const unsigned char* tab_lo, int d0, int n,
                                       bool accumulate) {
    const uint64_t ah = ptx::smem_desc(chi, kALbo, 128), al = ptx::smem_desc(clo, kALbo, 128);
    const uint32_t id = ptx::idesc_f16(kTile, n, true);
    const uint64_t bh = ptx::smem_desc(tab_hi + (size_t)(d0 / 8) * kTabLbo, 128, kTabLbo);
    const uint64_t bl = ptx::smem_desc(tab_lo + (size_t)(d0 / 8) * kTabLbo, 128, kTabLbo);
    ptx::mma_f16(dcol, ah, bh, id, accumulate);
    ptx::mma_f16(dcol, al, bh, id, true);
    ptx::mma_f16(dcol, ah, bl, id, true);
}

template <typename T>
struct YSmem;
template <>
struct YSmem<float> {
    static __device__ __forceinline__ float get(const unsigned char* st, int idx, bool& valid) {
        const float v = reinterpret_cast<const float*>(st)[idx];
        valid = v == v;
        return v;
    }
};
template <>
struct YSmem<int16_t> {
    static __device__ __forceinline__ float get(const unsigned char* st, int idx, bool& valid) {
        const int v = reinterpret_cast<const int16_t*>(st)[idx];
        valid = v != -32768;
        return (float)v;
    }
};

__device__ __forceinline__ void tma_load_2d_hint(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y,
                                                 uint64_t pol) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1, {%2, %3}], [%4], %5;" ::"r"(ptx::smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(ptx::smem_u32(bar)), "l"(pol)
        : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(ptx::smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_cnt(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0], %1;" ::"r"(ptx::smem_u32(bar)), "r"(count) : "memory");
}

// 256 threads per 128-pixel tile: pixel px = tid % 128 is held by the thread
// pair (px, px + 128), warps w and w + 4, which reach the same TMEM lane
// quarter.  In the two history passes each thread of the pair takes one of
// the two 8-date groups of every 16-date chunk; the MOSUM pass runs on the
// first thread of each pair.
constexpr int kThreads = 2 * kTile;

constexpr int kHdr = 1024;  // fixed shared-memory header: TMEM address slot, work-block broadcast

// One 128-pixel block `blk` of a tile, on a CTA of kThreads threads that
// holds kTmemCols TMEM columns at `tmem`; smem_base is the dynamic shared
// memory (header, then the layout of mma_layout).
template <int KH, typename T, bool kMask>
__device__ __forceinline__ void mma_block(const CUtensorMap* tmap, const MmaParams& P, int64_t blk,
                                          unsigned char* smem_base, uint32_t tmem) {
    using B = Basis<KH>;
    constexpr int K = B::K, NBR = B::NBR;
    constexpr bool kInt = sizeof(T) == 2;
    constexpr int kStageBytes = kBlk * kTile * (int)sizeof(T);
    unsigned char* smem_raw = smem_base + kHdr;
    const size_t ta = (size_t)(P.npad / 8) * kTabLbo, tb = NBR > 16 ? (size_t)(P.nhpad / 8) * kTabLbo : 0;
    unsigned char* tA_hi = smem_raw;
    unsigned char* tA_lo = tA_hi + ta;
    unsigned char* region = tA_lo + ta;  // table B and the A buffers; the MOSUM ring after the solve
    unsigned char* tB_hi = region;
    unsigned char* tB_lo = tB_hi + tb;
    unsigned char* sA = tB_lo + tb;
    unsigned char* sC = region + P.region_bytes;  // beta0 hi, beta0 lo, delta hi, delta lo planes
    unsigned char* sY = sC + 4 * kCoefPlane;      // Y blocks [16 dates][128 px]
    const int S = P.stages;
    // per-chunk valid bytes [nbh][2][128], then a float per thread: in the delta
    // planes (free until the delta is known) when they fit there, else after the stages
    unsigned char* sVb = P.vb_extra ? sY + (size_t)S * kStageBytes : sC + 2 * kCoefPlane;
    float* sX = reinterpret_cast<float*>(sVb + (size_t)((P.n_hist + kBlk - 1) / kBlk) * 2 * kTile);
    uint64_t* bars = reinterpret_cast<uint64_t*>(sY + (size_t)S * kStageBytes + P.vb_extra);
    uint64_t* bar_buf = bars + 0;  // [2] A-buffer reuse
    uint64_t* bar_done = bars + 2;
    uint64_t* full = bars + 3;                 // [S] Y block landed
    uint64_t* empty = bars + 3 + kMaxStages;   // [S] Y block released (256 arrivals)
    uint64_t* rdy = bars + 3 + 2 * kMaxStages;  // [2] MOSUM group published by the first threads
    uint64_t* cons = rdy + 2;                    // [2] MOSUM group consumed by the second threads
    int* s_dstart = reinterpret_cast<int*>(cons + 2);

    const int tid = threadIdx.x, warp = tid >> 5;
    const int px = tid & (kTile - 1), half = tid >> 7;
    const int64_t p0 = blk * kTile;
    const int64_t p = p0 + px;
    const bool active = p < P.m;
    const int N = P.N, n_hist = P.n_hist;
    const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;

    if (tid == 0) {
        for (int i = 0; i < 3; ++i) ptx::mbar_init(bars + i, 1);
        for (int i = 0; i < S; ++i) {
            ptx::mbar_init(full + i, 1);
            ptx::mbar_init(empty + i, kThreads);
        }
        for (int i = 0; i < 2; ++i) {
            ptx::mbar_init(rdy + i, kTile);
            ptx::mbar_init(cons + i, kTile);
        }
        ptx::fence_mbar_init();
        *s_dstart = N;
        ptx::prefetch_tmap(tmap);
    }
    {
        // basis tables: A over all npad dates; B (rows 16..31) over the history
        const uint4* gA = P.phi;
        uint4* dA = reinterpret_cast<uint4*>(tA_hi);
        for (size_t i = tid; i < 2 * ta / 16; i += kThreads) dA[i] = __ldg(gA + i);
        if constexpr (NBR > 16) {
            const uint4* gB = P.phi + 2 * ta / 16;
            const size_t nb1 = tb / 16;
            uint4* dB = reinterpret_cast<uint4*>(tB_hi);
            for (size_t i = tid; i < nb1; i += kThreads) {
                dB[i] = __ldg(gB + i);
                dB[nb1 + i] = __ldg(gB + ta / 16 + i);
            }
        }
    }
    ptx::fence_async_smem();
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    bool ok = true;

    const uint64_t keep = l2_policy_evict_last(), last = l2_policy_evict_first();
    const uint32_t* mrow = P.mask + (p0 >> 5) + (px >> 5);

    // ---- Y stream: passes over date blocks [b0, b1) -------------------------------------------
    // Block q of the kernel's sequence sits in stage q % S; the producer
    // thread keeps S blocks in flight and refills a stage once its empty
    // barrier has seen 256 arrivals (the producer's 256 after a chunk barrier
    // in the history passes, 2 from each first thread in the MOSUM pass).
    uint32_t q_next = 0, s_q0 = 0;
    int s_b0 = 0, s_b1 = 0, s_tlim = 0;
    int producer = 0;  // thread 0 in the history passes, thread 128 in the MOSUM pass
    uint64_t s_pol = keep;
    auto issue = [&](uint32_t q, int bd) {  // the producer thread
        const int st = (int)(q % (uint32_t)S);
        if (q >= (uint32_t)S) ok &= ptx::mbar_wait_bounded(empty + st, ((q / S) - 1u) & 1u, kWaitNs);
        ptx::mbar_arrive_expect_tx(full + st, kStageBytes);
        tma_load_2d_hint(sY + (size_t)st * kStageBytes, tmap, full + st, (int)p0, bd * kBlk, s_pol);
    };
    auto open = [&](int b0, int b1, int tlim, uint64_t pol) {
        s_b0 = b0;
        s_b1 = b1;
        s_q0 = q_next;
        q_next += (uint32_t)(b1 - b0);
        s_pol = pol;
        s_tlim = tlim;
        if (tid == producer)
            for (int j = 0; j < S && b0 + j < b1; ++j) issue(s_q0 + (uint32_t)j, b0 + j);
    };
    // the stage of date block bd, waited for
    auto block_wait = [&](int bd) -> const unsigned char* {
        const uint32_t q = s_q0 + (uint32_t)(bd - s_b0);
        const int st = (int)(q % (uint32_t)S);
        ok &= ptx::mbar_wait_bounded(full + st, (q / S) & 1u, kWaitNs);
        return sY + (size_t)st * kStageBytes;
    };
    // done with block bd: `count` arrivals (the producer refills the stage later)
    auto block_release = [&](int bd, uint32_t count) {
        const uint32_t q = s_q0 + (uint32_t)(bd - s_b0);
        mbar_arrive_cnt(empty + (int)(q % (uint32_t)S), count);
    };
    auto block_refill = [&](int bd) {  // the producer thread
        const uint32_t q = s_q0 + (uint32_t)(bd - s_b0);
        if (bd + S < s_b1) issue(q + (uint32_t)S, bd + S);
    };
    // dates [t0, t0 + 8) of this pixel from a waited stage: values (0 where
    // invalid) and valid bits (missing, masked, t >= tlim, pixel beyond m)
    auto read8 = [&](const unsigned char* sb, int t0, float (&y)[8]) -> uint32_t {
        const int r0 = t0 & (kBlk - 1);
        const int nt = s_tlim - t0;  // dates of the group before tlim
        const uint32_t lim = !active || nt <= 0 ? 0u : (nt >= 8 ? 0xffu : (1u << nt) - 1u);
        uint32_t vb = 0u;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            bool v;
            y[e] = YSmem<T>::get(sb, (r0 + e) * kTile + px, v);
            vb |= (v ? 1u : 0u) << e;
        }
        vb &= lim;
        if constexpr (kMask) {
#pragma unroll
            for (int e = 0; e < 8; ++e)
                if ((vb >> e) & 1u)
                    vb &= ~((((__ldg(mrow + (size_t)(t0 + e) * P.mask_words) >> (px & 31)) & 1u) ^ 1u) << e);
        }
#pragma unroll
        for (int e = 0; e < 8; ++e) y[e] = ((vb >> e) & 1u) ? y[e] : 0.f;
        return vb;
    };
    // history passes: after the chunk's barrier every thread is done with
    // block c, so thread 0 completes its empty phase at once and refills it
    auto chunk_release = [&](int bd) {
        if (tid == producer) {
            block_release(bd, kThreads);
            block_refill(bd);
        }
    };

    uint32_t done_uses = 0, buf_uses[2] = {0u, 0u};
    auto wait_done = [&]() {
        ok &= ptx::mbar_wait_bounded(bar_done, done_uses & 1u, kWaitNs);
        ++done_uses;
        ptx::tc_fence_after();
    };
    // before rewriting A buffer b: the MMAs that read its previous contents are done
    auto acquire = [&](int b) {
        if (buf_uses[b]) ok &= ptx::mbar_wait_bounded(bar_buf + b, (buf_uses[b] - 1u) & 1u, kWaitNs);
    };
    // the pair partner's value of x (both threads call it)
    auto pair_exchange = [&](float x) -> float {
        sX[tid] = x;
        __syncthreads();
        const float o = sX[tid ^ kTile];
        __syncthreads();
        return o;
    };
    const int nbh = (n_hist + kBlk - 1) / kBlk;  // history blocks

    // ---- normal equations (Eq. 6): masked basis sums and X'My over the history --------------
    // A rows per 16-date chunk (this thread: group `half`): the 0/1 mask, and
    // y*s_y split into fp16 hi + lo (int16: 256*(y >> 8) and y & 255, both
    // exact; float: a per-pixel power of two s_y from the first group of
    // eight dates holding a valid value (both threads of the pair look at
    // both groups until then), redone from the history maximum if a value of
    // the tile leaves the range where the split keeps 22 bits).
    float ymax = 0.f, s_y = 1.f;
    bool s_set = kInt;
    for (int attempt = 0; attempt < 2; ++attempt) {
        open(0, nbh, n_hist, keep);
        float ym = 0.f;
        for (int c = 0; c < nbh; ++c) {
            const int buf = c & 1;
            unsigned char* pl = sA + (size_t)buf * kBufBytes;
            acquire(buf);
            const unsigned char* sb = block_wait(c);
            float yc[8];
            if (!s_set) {  // float: the first group with a valid value sets s_y (earlier rows are 0)
#pragma unroll
                for (int g = 0; g < 2; ++g) {
                    float yg[8];
                    read8(sb, c * kBlk + g * 8, yg);
                    float gm = 0.f;
#pragma unroll
                    for (int e = 0; e < 8; ++e) gm = fmaxf(gm, fabsf(yg[e]));
                    if (!s_set && gm > 0.f) {
                        s_y = pow2_scale(gm, 4);
                        s_set = true;
                    }
                }
            }
            const uint32_t vc = read8(sb, c * kBlk + half * 8, yc);
            float mk[8], a1[8], a2[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const bool v = (vc >> e) & 1u;
                mk[e] = v ? 1.f : 0.f;
                const float y = yc[e];
                ym = fmaxf(ym, fabsf(y));
                if constexpr (kInt) {
                    const int yi = (int)y;
                    a1[e] = (float)((yi >> 8) * 256);
                    a2[e] = (float)(yi & 255);
                } else {
                    split_hi_lo(y * s_y, a1[e], a2[e]);
                }
            }
            st_a(pl, px, half, mk);
            st_a(pl + kPlane, px, half, a1);
            st_a(pl + 2 * kPlane, px, half, a2);
            ptx::fence_async_smem();
            ptx::tc_fence_before();
            __syncthreads();
            chunk_release(c);
            if (tid == 0) {
                ptx::tc_fence_after();
                const int d0 = c * kBlk;
                const bool first = c == 0;
                mma_kb(tmem + kColG, pl, 0, tA_hi, d0, !first);
                mma_kb(tmem + kColG, pl, 0, tA_lo, d0, true);
                if constexpr (NBR > 16) {
                    mma_kb(tmem + kColG + 16, pl, 0, tB_hi, d0, !first);
                    mma_kb(tmem + kColG + 16, pl, 0, tB_lo, d0, true);
                }
                mma_kb(tmem + kColB, pl + kPlane, 0, tA_hi, d0, !first);
                mma_kb(tmem + kColB, pl + kPlane, 0, tA_lo, d0, true);
                mma_kb(tmem + kColB, pl + 2 * kPlane, 0, tA_hi, d0, true);
                mma_kb(tmem + kColB, pl + 2 * kPlane, 0, tA_lo, d0, true);
                ptx::mma_commit(bar_buf + buf);
                if (c == nbh - 1) ptx::mma_commit(bar_done);
            }
            ++buf_uses[buf];
        }
        wait_done();
        ymax = fmaxf(ym, pair_exchange(ym));
        if (kInt) break;
        const float qy = ymax * s_y;
        const bool redo = ymax > 0.f && !(qy < 32768.f && qy >= 4.f);
        if (!__syncthreads_or(redo ? 1 : 0) || attempt == 1) break;
        s_y = pow2_scale(ymax, 8);
        s_set = true;
    }

    // ---- solve (both threads of the pair, identically) -------------------------------------------
    float a[NBR], bb[K];
    {
        float v32[32], v16[16];
        ptx::tmem_ld32(tmem + lane_base + kColG, v32);
        ptx::tmem_ld16(tmem + lane_base + kColB, v16);
#pragma unroll
        for (int i = 0; i < NBR; ++i) a[i] = v32[i];
        const float inv_sy = 1.f / s_y;
#pragma unroll
        for (int i = 0; i < K; ++i) bb[i] = v16[i] * inv_sy;
    }
    const int n_i = (int)a[0];
    float G[K][K], L[K][K], dinv[K], beta[K];
    gram_from_sums<KH>(a, G);
    const bool nonsingular = cholesky<K>(G, L, dinv);
    chol_solve<K>(L, dinv, bb, beta);
    // Per-pixel operand scales (powers of two, exact): |beta| * s_b < 2^13 and,
    // since |x_i| <= 1 (centred trend), |r0| * s_r <= (max|y| + sum|beta|) * s_r < 2^13.
    float s_b, s_r;
    {
        float bm = 0.f, bsum = 0.f;
#pragma unroll
        for (int i = 0; i < K; ++i) {
            bm = fmaxf(bm, fabsf(beta[i]));
            bsum += fabsf(beta[i]);
        }
        s_b = pow2_scale(bm, 12);
        s_r = pow2_scale(ymax + bsum, 12);
    }
    auto write_coef = [&](const float (&coef)[K], unsigned char* hi_plane, unsigned char* lo_plane) {
        float h[8], l[8], z[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const float cs = i < K ? coef[i] * s_b : 0.f;
            split_hi_lo(cs, h[i], l[i]);
            z[i] = 0.f;
        }
        st_a(hi_plane, px, 0, h);
        st_a(hi_plane, px, 1, z);
        st_a(lo_plane, px, 0, l);
        st_a(lo_plane, px, 1, z);
    };
    if (half == 0) write_coef(beta, sC, sC + kCoefPlane);
    const float inv_b = 1.f / s_b;

    // ---- one refinement step: r0 = y - X beta0 on the history, c = X'M r0 ------------------
    // X beta0 comes from the tensor cores, kPiece dates per TMEM piece; each
    // thread of the pair takes its group of every chunk and records the
    // group's valid bits.
    float ss = 0.f;
    open(0, nbh, n_hist, keep);
    for (int d0 = 0; d0 < nbh * kBlk; d0 += kPiece) {
        const int w = nbh * kBlk - d0 < kPiece ? nbh * kBlk - d0 : kPiece;
        ptx::fence_async_smem();
        ptx::tc_fence_before();
        __syncthreads();  // coefficient planes written; previous piece's TMEM reads done
        if (tid == 0) {
            ptx::tc_fence_after();
            mma_xc(tmem + kColY, sC, sC + kCoefPlane, tA_hi, tA_lo, d0, w, false);
            ptx::mma_commit(bar_done);
        }
        wait_done();
        uint32_t rq[8];
        ptx::tmem_ld8_issue(tmem + lane_base + kColY + (uint32_t)(half * 8), rq);
#pragma unroll 1
        for (int c = d0 / kBlk; c < (d0 + w) / kBlk; ++c) {
            const int buf = c & 1;
            const int t0 = c * kBlk + half * 8;
            unsigned char* pl = sA + (size_t)buf * kBufBytes;
            acquire(buf);
            float yc[8], yh[8];
            const unsigned char* sb = block_wait(c);
            const uint32_t vc = read8(sb, t0, yc);
            ptx::tmem_wait_ld8(rq);
#pragma unroll
            for (int e = 0; e < 8; ++e) yh[e] = __uint_as_float(rq[e]);
            if (t0 + kBlk < d0 + w) ptx::tmem_ld8_issue(tmem + lane_base + kColY + (uint32_t)(t0 + kBlk - d0), rq);
            float rh[8], rl[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const bool v = (vc >> e) & 1u;
                const float r0 = v ? (yc[e] - yh[e] * inv_b) : 0.f;
                ss = fmaf(r0, r0, ss);
                split_hi_lo(r0 * s_r, rh[e], rl[e]);
            }
            sVb[(c * 2 + half) * kTile + px] = (unsigned char)vc;
            st_a(pl, px, half, rh);
            st_a(pl + kPlane, px, half, rl);
            ptx::fence_async_smem();
            ptx::tc_fence_before();
            __syncthreads();
            chunk_release(c);
            if (tid == 0) {
                ptx::tc_fence_after();
                const int dd = c * kBlk;
                const bool first = c == 0;
                mma_kb(tmem + kColC, pl, 0, tA_hi, dd, !first);
                mma_kb(tmem + kColC, pl, 0, tA_lo, dd, true);
                mma_kb(tmem + kColC, pl + kPlane, 0, tA_hi, dd, true);
                ptx::mma_commit(bar_buf + buf);
                if (c == nbh - 1) ptx::mma_commit(bar_done);
            }
            ++buf_uses[buf];
        }
    }
    wait_done();
    ss += pair_exchange(ss);
    // Bandwidth h (Eq. 3, missing-data reading) and the date of the earliest
    // history observation a monitoring window reaches back to: the h-th valid
    // one from the end of the history.
    int h = (int)floor(P.h_frac * (double)n_i);
    if (h < 1) h = 1;
    if (h > n_i) h = n_i;
    int dfirst = N;
    {
        int cnt = 0;
        for (int q = 2 * nbh - 1; q >= 0 && cnt < h; --q) {
            uint32_t byte = sVb[q * kTile + px];
            const int pc = __popc(byte);
            if (cnt + pc >= h) {
                for (int k = cnt; k < h - 1; ++k) byte &= ~(0x80000000u >> __clz(byte));  // drop the top set bits
                dfirst = q * 8 + (31 - __clz(byte));
            }
            cnt += pc;
        }
    }
    float sigma, scale;
    int jlim;
    float dl[K];
    {
        float v16[16], cc[K];
        ptx::tmem_ld16(tmem + lane_base + kColC, v16);
        const float inv_r = 1.f / s_r;
#pragma unroll
        for (int i = 0; i < K; ++i) cc[i] = v16[i] * inv_r;
        chol_solve<K>(L, dinv, cc, dl);
        float dc = 0.f;
#pragma unroll
        for (int i = 0; i < K; ++i) {
            beta[i] += dl[i];
            dc = fmaf(dl[i], cc[i], dc);
        }
        sigma = sqrtf(fmaxf(ss - dc, 0.f) / (float)(n_i - K));
        scale = sigma * sqrtf((float)n_i);
        jlim = (int)floor(kEuler * (double)n_i);
    }
    __syncthreads();  // valid bytes read by both threads before the delta planes overwrite them
    if (half == 0) write_coef(dl, sC + 2 * kCoefPlane, sC + 3 * kCoefPlane);
    const bool degenerate = !(sigma > kDegenerateRatio * ymax) || ymax == 0.f;
    // The MOSUM pass starts at the earliest such date over the tile's pixels
    // that get a break test (prefix sums from there on differ from those
    // from date 0 by a constant, which the window differences cancel).
    if (half == 0 && active && n_i > K && nonsingular && !degenerate) atomicMin(s_dstart, dfirst);
    __syncthreads();
    int d_start = *s_dstart;
    d_start = (d_start < n_hist ? d_start : n_hist) / kBlk * kBlk;

    // ---- MOSUM from d_start, 8 dates at a time, as a two-stage pipeline per pixel ----------------
    // First thread of the pair: yhat = X beta0 + X delta per kPiece-date TMEM
    // piece (the fp16 split error of beta0 lies in the span of X and cancels
    // against the refinement); per 8-date group the residuals, then
    // prefix sums S over valid positions (the group's own running sum, then
    // S = base_hi + (base_lo + local) for every date, the base carried as an
    // unevaluated sum and advanced by one TwoSum per group) into a ring of
    // R >= h + 17 slots, and a mailbox word
    // (group's first slot, valid bits).  Second thread, one group behind:
    // the windows W_J = S_J - S_{J-h} (Eq. 3) of the group's monitoring
    // positions J = n + 1, n + 2, ..., MO_J = W_J / (sigma-hat sqrt(n)),
    // the test MO_J^2 > lambda^2 log+(J/n) (Eq. 4, squared) and the mean.
    // The ring can hold one group in flight between the two: the first
    // thread waits for the second to finish group g - 2 before group g.
    float* ring = reinterpret_cast<float*>(region);  // [P.ring][128]; table B and the A buffers are free now
    uint32_t* mbox = reinterpret_cast<uint32_t*>(region + (size_t)P.ring * kTile * 4);  // [2][128]
    const int R = P.ring;
    int jm = 0, slot = 0, brk = -1;
    float Sh = 0.f, Sc = 0.f;
    float m0 = 0.f, m0c = 0.f;
    float mx = 0.f;  // MO of largest magnitude (the first of equals), when asked for
    const bool want_mx = P.maxmo != nullptr;
    const float inv_scale = 1.f / scale, lam2 = P.lambda * P.lambda;
    const float lg_n = log2f((float)n_i);
    const int nball = (N + kBlk - 1) / kBlk;
    uint32_t grp = 0;  // MOSUM group sequence number (the same in both threads)
    producer = kTile;  // the second threads trail the first ones: refills stay off the first threads' path
    open(d_start / kBlk, nball, N, last);
    for (int d0 = d_start; d0 < P.npad; d0 += kPiece) {
        const int w = P.npad - d0 < kPiece ? P.npad - d0 : kPiece;
        ptx::fence_async_smem();
        ptx::tc_fence_before();
        __syncthreads();
        if (tid == 0) {
            ptx::tc_fence_after();
            mma_xc(tmem + kColY, sC, sC + kCoefPlane, tA_hi, tA_lo, d0, w, false);
            mma_xc(tmem + kColY, sC + 2 * kCoefPlane, sC + 3 * kCoefPlane, tA_hi, tA_lo, d0, w, true);
            ptx::mma_commit(bar_done);
        }
        wait_done();
        const int dend = d0 + w < nball * kBlk ? d0 + w : nball * kBlk;  // whole Y blocks
        if (half == 0) {
            uint32_t rq[8];
            if (d0 < dend) ptx::tmem_ld8_issue(tmem + lane_base + kColY, rq);
            const unsigned char* sb = nullptr;
#pragma unroll 1
            for (int c0 = d0; c0 < dend; c0 += 8, ++grp) {
                float yc[8], yh[8];
                const int bd = c0 / kBlk;
                if ((c0 & 8) == 0) sb = block_wait(bd);
                const uint32_t vb = read8(sb, c0, yc);
                if (c0 & 8) block_release(bd, 2);
                ptx::tmem_wait_ld8(rq);
#pragma unroll
                for (int e = 0; e < 8; ++e) yh[e] = __uint_as_float(rq[e]);
                if (c0 + 8 < dend) ptx::tmem_ld8_issue(tmem + lane_base + kColY + (uint32_t)(c0 + 8 - d0), rq);
                float loc[8], Sv[8];
                float acc = 0.f;
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    acc += ((vb >> e) & 1u) ? (yc[e] - yh[e] * inv_b) : 0.f;
                    loc[e] = acc;
                }
                // the base is the unevaluated sum Sh + Sc: each S is rounded once
                // from it, and the base moves on by one TwoSum per group
#pragma unroll
                for (int e = 0; e < 8; ++e) Sv[e] = Sh + (Sc + loc[e]);
                {
                    const float b = Sc + loc[7];
                    const float t = Sh + b;
                    const float bv = t - Sh;
                    Sc = (Sh - (t - bv)) + (b - bv);
                    Sh = t;
                }
                if (grp >= 2) ok &= ptx::mbar_wait_bounded(cons + (grp & 1), ((grp >> 1) - 1u) & 1u, kWaitNs);
                if (slot <= R - 8) {  // the group's slots do not wrap
                    float* wp = ring + slot * kTile + px;
#pragma unroll
                    for (int e = 0; e < 8; ++e)
                        if ((vb >> e) & 1u) wp[__popc(vb & ((1u << e) - 1u)) * kTile] = Sv[e];
                } else {
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        int se = slot + __popc(vb & ((1u << e) - 1u));
                        se -= se >= R ? R : 0;
                        if ((vb >> e) & 1u) ring[se * kTile + px] = Sv[e];
                    }
                }
                mbox[(grp & 1) * kTile + px] = ((uint32_t)slot << 8) | vb;
                slot += __popc(vb);
                slot -= slot >= R ? R : 0;
                mbar_arrive(rdy + (grp & 1));
            }
        } else {
#pragma unroll 1
            for (int c0 = d0; c0 < dend; c0 += 8, ++grp) {
                ok &= ptx::mbar_wait_bounded(rdy + (grp & 1), (grp >> 1) & 1u, kWaitNs);
                const int dm = n_hist - c0;  // monitoring dates of the group: e >= dm
                const uint32_t mon = dm <= 0 ? 0xffu : (dm >= 8 ? 0u : (0xffu << dm) & 0xffu);
                if (mon) {  // the same for every thread: a group with monitoring dates
                    const uint32_t word = mbox[(grp & 1) * kTile + px];
                    const uint32_t vb = word & 0xffu, mv = vb & mon;
                    const int sl0 = (int)(word >> 8);
                    float wv[8], mo2[8];
                    const bool nowrap = sl0 <= R - 8 && sl0 >= h;  // neither the slots nor their lags wrap
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        int se = sl0 + __popc(vb & ((1u << e) - 1u));
                        int ls = se - h;
                        if (!nowrap) {
                            se -= se >= R ? R : 0;
                            ls = se - h;
                            ls += ls < 0 ? R : 0;
                        }
                        const float W = ring[se * kTile + px] - ring[ls * kTile + px];
                        const float mo = W * inv_scale;
                        const bool mm = (mv >> e) & 1u;
                        wv[e] = mm ? W : 0.f;
                        mo2[e] = mm ? mo * mo : 0.f;
                    }
                    // log+ >= 1: |MO| <= lambda never crosses; the exact boundary
                    // only for candidates before the first crossing
                    uint32_t cand = 0u;
#pragma unroll
                    for (int e = 0; e < 8; ++e) cand |= (mo2[e] > lam2 ? 1u : 0u) << e;
                    if (brk < 0 && cand) {
                        int jb = jm;
#pragma unroll
                        for (int e = 0; e < 8; ++e) {
                            if (brk < 0 && ((cand >> e) & 1u)) {
                                const int J = n_i + jb + 1;
                                const float b2 = J > jlim ? lam2 * kLn2f * (log2_fast((float)J) - lg_n) : lam2;
                                if (mo2[e] > b2) brk = c0 + e;
                            }
                            jb += (mv >> e) & 1u;
                        }
                    }
                    if (want_mx) {
#pragma unroll
                        for (int e = 0; e < 8; ++e)
                            if (((mv >> e) & 1u) && mo2[e] > mx * mx) mx = wv[e] * inv_scale;
                    }
                    jm += __popc(mv);
                    // the group's windows summed as a tree, then one compensated add
                    const float gsum = ((wv[0] + wv[1]) + (wv[2] + wv[3])) + ((wv[4] + wv[5]) + (wv[6] + wv[7]));
                    comp_add(m0, m0c, gsum);
                }
                mbar_arrive(cons + (grp & 1));
                if (tid == producer && (c0 & 8)) block_refill(c0 / kBlk);
            }
        }
    }
    const float sumW = m0, sumWc = m0c;

    // ---- outputs ------------------------------------------------------------------------------
    ptx::tc_fence_before();
    __syncthreads();
    if (!__syncthreads_and(ok ? 1 : 0)) ok = false;
    if (!active || half == 0) return;  // the second thread of the pair holds the MOSUM results
    if (!ok) {
        P.status[p] = BFM_PX_TIMEOUT;
        atomicOr(&g_bfm_mma_err, 2u);
        return;
    }
    const float qnan = qnanf();
    uint8_t st;
    float o_mean = qnan, o_sigma = sigma;
    int o_brk = -1;
    bool fitted = true;
    if (n_i <= K) {
        st = BFM_PX_INSUFFICIENT_HISTORY;
        fitted = false;
    } else if (!nonsingular) {
        st = BFM_PX_SINGULAR;
        fitted = false;
    } else if (degenerate) {
        st = BFM_PX_DEGENERATE;
        o_mean = 0.f;
    } else if (jm == 0) {
        st = BFM_PX_NO_MONITOR;
    } else {
        st = BFM_PX_OK;
        o_brk = brk;
        o_mean = (sumW + sumWc) / ((float)jm * scale);
    }
    if (!fitted) o_sigma = qnan;
    P.status[p] = st;
    P.brk[p] = o_brk;
    P.mean[p] = o_mean;
    P.sigma[p] = o_sigma;
    if (want_mx) P.maxmo[p] = st == BFM_PX_OK ? mx : (st == BFM_PX_DEGENERATE ? 0.f : qnan);
#pragma unroll
    for (int i = 0; i < K; ++i) {
        float bi = beta[i];
        if (i == 0) bi = fmaf(-beta[1], P.c_over_s, beta[0]);
        if (i == 1) bi = beta[1] * P.inv_s;
        P.beta[(size_t)i * P.m + p] = fitted ? bi : qnan;
    }
}

template <int KH, typename T, bool kMask>
__global__ void __launch_bounds__(kThreads, 2) mma_kernel(const __grid_constant__ CUtensorMap tmap,
                                                          const __grid_constant__ MmaParams P) {
    extern __shared__ __align__(1024) unsigned char smem[];
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem);
    if ((threadIdx.x >> 5) == 0) ptx::tmem_alloc(tslot, kTmemCols);
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem = *tslot;
    mma_block<KH, T, kMask>(&tmap, P, (int64_t)blockIdx.x, smem, tmem);
    ptx::tc_fence_before();
    __syncthreads();
    if ((threadIdx.x >> 5) == 0) ptx::tmem_dealloc(tmem, kTmemCols);
}

// Ring of prefix sums: the h slots behind the oldest position of the group
// the second thread reads, that group and the one the first thread writes.
int ring_len(int n_hist, double h_frac) {
    int hmax = (int)std::floor(h_frac * (double)n_hist);
    if (hmax < 1) hmax = 1;
    if (hmax > n_hist) hmax = n_hist;
    return hmax + 17;
}

struct MmaLayout {
    int stages, region_bytes, vb_extra;
    size_t smem;
};

// Shared memory: tables A (hi, lo) over npad dates; a region holding tables B
// (only with more than 16 basis sums) and two A buffers, later the MOSUM ring;
// four coefficient planes; the Y stages (TMA loader); barriers.
MmaLayout mma_layout(int npad, int nhpad, int k, int ring, int elt, bool tma) {
    MmaLayout L{};
    const size_t ta = (size_t)(npad / 8) * kTabLbo;
    const size_t tb = 3 + 6 * k > 16 ? (size_t)(nhpad / 8) * kTabLbo : 0;
    size_t region = 2 * tb + 2 * (size_t)kBufBytes;
    const size_t rb = (size_t)ring * kTile * 4 + 2 * kTile * 4;  // ring and mailbox
    if (rb > region) region = rb;
    region = (region + 1023) & ~(size_t)1023;
    L.region_bytes = (int)region;
    L.stages = tma ? (elt == 4 ? 3 : 6) : 0;
    // valid bytes (2 per history block and pixel) and the pair exchange floats
    const int nbh = (nhpad + kBlk - 1) / kBlk;
    const size_t vb = (size_t)nbh * 2 * kTile + 2 * kTile * 4;
    L.vb_extra = vb <= 2 * (size_t)kCoefPlane ? 0 : (int)((vb + 127) & ~(size_t)127);
    L.smem = kHdr + 2 * ta + region + 4 * (size_t)kCoefPlane + (size_t)L.stages * kBlk * kTile * elt + L.vb_extra +
             256;
    return L;
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn_mma() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
    });
    return fn;
}

template <int KH, typename T>
bfm_status launch_t(const CUtensorMap& tm, const MmaParams& P, size_t smem, cudaStream_t stream) {
    auto kern = P.mask ? mma_kernel<KH, T, true> : mma_kernel<KH, T, false>;
    static thread_local int configured[2] = {-1, -1};
    int dev = 0;
    cudaGetDevice(&dev);
    if (configured[P.mask ? 1 : 0] != dev) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(mma_kernel)");
        configured[P.mask ? 1 : 0] = dev;
    }
    const unsigned grid = (unsigned)((P.m + kTile - 1) / kTile);
    kern<<<grid, kThreads, smem, stream>>>(tm, P);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "mma kernel launch");
    return BFM_OK;
}

}  // namespace

// Y must be describable by a tensor map with boxes of 128 pixels x 16 dates.
bool mma_layout_ok(const void* Y, int dtype, int64_t m) {
    const int elt = dtype == BFM_F32 ? 4 : 2;
    return m == 0 || (((uintptr_t)Y % 16 == 0) && ((m * elt) % 16 == 0) && m >= kTile);
}

bool mma_supported(const bfm_design_s* d, int dtype, int n_hist, double h_frac, const void* Y, int64_t m,
                   size_t* smem_out) {
    if ((dtype != BFM_I16 && dtype != BFM_F32) || !d->d_phi_tc) return false;
    if (!mma_layout_ok(Y, dtype, m)) return false;
    const MmaLayout L = mma_layout(d->npad_tc, (n_hist + 31) / 32 * 32, d->k, ring_len(n_hist, h_frac),
                                   dtype == BFM_F32 ? 4 : 2, true);
    if (smem_out) *smem_out = L.smem;
    return L.smem <= 227 * 1024;
}

namespace {

// P, the tensor map and the shared memory of one tile (false, with a message,
// when the tensor-core form does not take it).
bool mma_prepare(const bfm_design_s* d, int dtype, const void* Y, const uint32_t* mask, int64_t m, int n_hist,
                 double h_frac, double lambda, int32_t* brk, float* mean, float* sigma, float* beta,
                 uint8_t* status, float* maxmo, MmaParams* Pout, CUtensorMap* tm, size_t* smem_out) {
    const int elt = dtype == BFM_F32 ? 4 : 2;
    if (!mma_supported(d, dtype, n_hist, h_frac, Y, m, nullptr) || m < kTile) {
        set_error("tensor-core form: needs basis tables and a MOSUM ring that fit shared memory, and Y with a "
                  "16-byte aligned base, m >= 128 and rows of a multiple of 16 bytes");
        return false;
    }
    auto enc = encode_fn_mma();
    if (!enc) {
        set_error("tensor-core form: cuTensorMapEncodeTiled is not available");
        return false;
    }
    MmaParams P{};
    P.Y = Y;
    P.mask = mask;
    P.m = m;
    P.mask_words = (m + 31) / 32;
    P.N = d->N;
    P.n_hist = n_hist;
    P.npad = d->npad_tc;
    P.nhpad = (n_hist + 31) / 32 * 32;
    P.phi = static_cast<const uint4*>(d->d_phi_tc);
    P.h_frac = h_frac;
    P.lambda = (float)lambda;
    P.c_over_s = (float)(d->c / d->s);
    P.inv_s = (float)(1.0 / d->s);
    P.ring = ring_len(n_hist, h_frac);
    P.brk = brk;
    P.mean = mean;
    P.sigma = sigma;
    P.beta = beta;
    P.status = status;
    P.maxmo = maxmo;
    std::memset(tm, 0, sizeof *tm);
    cuuint64_t gdim[2] = {(cuuint64_t)m, (cuuint64_t)d->N};
    cuuint64_t gstride[1] = {(cuuint64_t)m * elt};
    cuuint32_t box[2] = {(cuuint32_t)kTile, (cuuint32_t)kBlk};
    cuuint32_t es[2] = {1u, 1u};
    const CUresult r = enc(tm, elt == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_UINT16, 2,
                           const_cast<void*>(Y), gdim, gstride, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("tensor-core form: cuTensorMapEncodeTiled failed for Y");
        return false;
    }
    const MmaLayout L = mma_layout(P.npad, P.nhpad, d->k, P.ring, elt, true);
    P.stages = L.stages;
    P.region_bytes = L.region_bytes;
    P.vb_extra = L.vb_extra;
    // At least 80 KB, so that at most two CTAs (2 x 256 TMEM columns) share an SM.
    *smem_out = L.smem < 80 * 1024 ? 80 * 1024 : L.smem;
    *Pout = P;
    return true;
}

}  // namespace

bfm_status launch_mma(const bfm_design_s* d, int dtype, const void* Y, const uint32_t* mask, int64_t m,
                      int n_hist, double h_frac, double lambda, int32_t* brk, float* mean, float* sigma,
                      float* beta, uint8_t* status, cudaStream_t stream, float* maxmo) {
    if (m == 0) return BFM_OK;
    MmaParams P;
    CUtensorMap tm;
    size_t smem = 0;
    if (!mma_prepare(d, dtype, Y, mask, m, n_hist, h_frac, lambda, brk, mean, sigma, beta, status, maxmo, &P, &tm,
                     &smem))
        return BFM_EUNSUPPORTED;
    const bool i16 = dtype == BFM_I16;
    switch (d->k) {
        case 1: return i16 ? launch_t<1, int16_t>(tm, P, smem, stream) : launch_t<1, float>(tm, P, smem, stream);
        case 2: return i16 ? launch_t<2, int16_t>(tm, P, smem, stream) : launch_t<2, float>(tm, P, smem, stream);
        default: return i16 ? launch_t<3, int16_t>(tm, P, smem, stream) : launch_t<3, float>(tm, P, smem, stream);
    }
}

bool mma_fill_tile(const bfm_design_s* d, int dtype, const void* Y, const uint32_t* mask, int64_t m, int n_hist,
                   double h_frac, double lambda, int32_t* brk, float* mean, float* sigma, float* beta,
                   uint8_t* status, MmaBatchTile* out, size_t* smem) {
    std::memset(out, 0, sizeof *out);
    if (!mma_prepare(d, dtype, Y, mask, m, n_hist, h_frac, lambda, brk, mean, sigma, beta, status, nullptr, &out->P,
                     &out->tm, smem))
        return false;
    out->kh = d->k;
    out->dtype = dtype;
    out->has_mask = mask != nullptr;
    return true;
}

namespace {
template <int KH, typename T, bool kMask>
void* tile_kernel_fn() {
    return (void*)mma_kernel<KH, T, kMask>;
}
}  // namespace

int mma_variant(int k, int dtype, bool has_mask) { return ((k - 1) * 2 + (dtype == BFM_I16 ? 1 : 0)) * 2 + (has_mask ? 1 : 0); }

bfm_status mma_tile_node(const MmaBatchTile& t, size_t smem, cudaGraph_t graph, const cudaGraphNode_t* dep,
                         cudaGraphNode_t* node_out) {
    static void* const fns[12] = {
        tile_kernel_fn<1, float, false>(),   tile_kernel_fn<1, float, true>(),
        tile_kernel_fn<1, int16_t, false>(), tile_kernel_fn<1, int16_t, true>(),
        tile_kernel_fn<2, float, false>(),   tile_kernel_fn<2, float, true>(),
        tile_kernel_fn<2, int16_t, false>(), tile_kernel_fn<2, int16_t, true>(),
        tile_kernel_fn<3, float, false>(),   tile_kernel_fn<3, float, true>(),
        tile_kernel_fn<3, int16_t, false>(), tile_kernel_fn<3, int16_t, true>()};
    const int variant = mma_variant(t.kh, t.dtype, t.has_mask != 0);
    if (variant < 0 || variant >= 12) {
        set_error("bfm_batch: bad tensor-core variant");
        return BFM_EINVAL;
    }
    cudaError_t e = cudaFuncSetAttribute(fns[variant], cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(mma_kernel)");
    // the arguments are copied into the node: the tile's tensor map and parameters
    void* args[] = {(void*)&t.tm, (void*)&t.P};
    cudaKernelNodeParams kp{};
    kp.func = fns[variant];
    kp.gridDim = dim3((unsigned)((t.P.m + kTile - 1) / kTile));
    kp.blockDim = dim3(kThreads);
    kp.sharedMemBytes = (unsigned)smem;
    kp.kernelParams = args;
    e = cudaGraphAddKernelNode(node_out, graph, dep, dep ? 1 : 0, &kp);
    if (e != cudaSuccess) return cuda_fail(e, "bfm_batch: tensor-core kernel node");
    return BFM_OK;
}

}  // namespace bfm
