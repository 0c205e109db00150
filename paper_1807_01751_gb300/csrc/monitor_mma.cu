// Tensor-core ("precision") form of the per-pixel path for int16 storage.
//
// One CTA = 128 pixels = the M of every tcgen05.mma = the 128 TMEM lanes;
// thread m owns pixel m (TMEM lane m).  Per tile:
//
//   stage    Y[N][128] int16 by 2-D TMA; the basis table (fp16 hi/lo, the
//            B operand of every MMA) by plain loads
//   A        for 32-date chunks of the history, each thread writes three
//            fp16 A-operand rows: the 0/1 mask, 256*(y >> 8) and (y & 255)
//            (both exact: y = 256*hi + lo), masked.  The single issuing thread
//            runs, per 16 dates,
//              TMEM[G] += mask  x Phi_hi + mask x Phi_lo   (32 basis sums, Eq. 6)
//              TMEM[b] += hi|lo x Phi_hi|lo                (X'My, Eq. 6)
//            double-buffered against the next chunk's operand writes
//   solve    every thread: Gram from the basis sums, Cholesky, beta0 (FP32)
//   yhat0    TMEM[Y] = [beta_hi | beta_lo] x Phi (Phi read MN-major: rows =
//            coefficients, columns = dates) over all dates
//   refine   r0 = y - yhat0 on valid history dates, split fp16 hi/lo, then
//            TMEM[c] += r0 x Phi: one refinement step beta = beta0 + G^-1 c;
//            sum r^2 = sum r0^2 - delta'c (sigma-hat, Algorithm 1 step 5)
//   yhat     TMEM[Y] += [delta_hi | delta_lo] x Phi (yhat = yhat0 + X delta)
//   MOSUM    per thread, 8 dates at a time: r = y - yhat, compensated
//            prefix sums S over valid positions in a ring, windows of h
//            valid residuals W = S_J - S_{J-h} (Eq. 3), first crossing of
//            lambda*sqrt(log+(j/n)) (Eq. 4) and the mean
//
// Scaling: A operands carry beta/16 and r0/4 (exact powers of two) so that
// fp16 holds any int16-scale value; results are scaled back exactly.
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

constexpr int kTile = 128;              // pixels per CTA
constexpr int kChunk = 32;              // dates per A-operand chunk
constexpr int kPlane = kTile * kChunk * 2;  // bytes of one fp16 A plane (128 x 32)
constexpr int kBufBytes = 3 * kPlane;   // one A buffer (three planes)
constexpr uint32_t kColG = 0, kColB = 32, kColC = 48, kColY = 64;
constexpr uint64_t kWaitNs = 2000000000ull;
constexpr uint32_t kALbo = 2048;        // A: K-direction core stride (16 row groups x 128 B)
constexpr uint32_t kPhiLbo = 512;       // Phi as K-major B (dates = K): date-group stride
constexpr uint32_t kPhiSbo = 128;       //   row-group stride

struct MmaParams {
    const int16_t* Y;
    const uint32_t* mask;
    int64_t m, mask_words;
    int N, n_hist, npad, nhp;  // npad = N padded to 32, nhp = history dates padded to 16
    const uint4* phi;          // hi table then lo table
    double h_frac;
    float lambda, c_over_s, inv_s;
    int box_rows, nbox, ring;
    uint32_t tmem_cols;  // power of two >= 64 + npad
    int32_t* brk;
    float* mean;
    float* sigma;
    float* beta;
    uint8_t* status;
};

__device__ __forceinline__ uint32_t pack_h2(float a, float b) {
    const __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&h);
}

// A-operand row segment: 8 consecutive K elements of row m, group g.
__device__ __forceinline__ void st_a(unsigned char* plane, int m, int g, const float (&v)[8]) {
    uint4 u;
    u.x = pack_h2(v[0], v[1]);
    u.y = pack_h2(v[2], v[3]);
    u.z = pack_h2(v[4], v[5]);
    u.w = pack_h2(v[6], v[7]);
    *reinterpret_cast<uint4*>(plane + (size_t)g * kALbo + (size_t)m * 16) = u;
}

// Issue D (+)= A x Phi over one A buffer region for the rows [r0, r0 + n) of Phi
// (Phi as K-major B: rows = N, dates = K), K range = dates [d0, d0 + 16).
__device__ __forceinline__ void mma_kblock(uint32_t dcol, const unsigned char* aplane, int kb_in_chunk,
                                           const unsigned char* phi, int d0, int n, bool acc) {
    const uint64_t ad = ptx::smem_desc(aplane + (size_t)kb_in_chunk * 2 * kALbo, kALbo, 128);
    const uint64_t bd = ptx::smem_desc(phi + (size_t)(d0 / 8) * kPhiLbo, kPhiLbo, kPhiSbo);
    ptx::mma_f16(dcol, ad, bd, ptx::idesc_f16(kTile, n, false), acc);
}

// X b over dates [0, ncols) into TMEM column base dcol (added to what is there
// when `accumulate`): A = [b_hi | 0], [b_lo | 0] (K = 16 coefficient slots),
// B = Phi rows 0..15 read MN-major (N = dates).
__device__ __forceinline__ void mma_yhat(uint32_t dcol, const unsigned char* bhi, const unsigned char* blo,
                                         const unsigned char* phi_hi, const unsigned char* phi_lo, int ncols,
                                         bool accumulate) {
    const uint64_t ah = ptx::smem_desc(bhi, kALbo, 128), al = ptx::smem_desc(blo, kALbo, 128);
    for (int n0 = 0; n0 < ncols; n0 += 256) {
        const int n = ncols - n0 < 256 ? ncols - n0 : 256;
        const uint32_t id = ptx::idesc_f16(kTile, n, true);
        // MN-major B: K-direction (coefficient) core stride 128 B, N-direction (date) stride 512 B
        const uint64_t bh = ptx::smem_desc(phi_hi + (size_t)(n0 / 8) * kPhiLbo, kPhiSbo, kPhiLbo);
        const uint64_t bl = ptx::smem_desc(phi_lo + (size_t)(n0 / 8) * kPhiLbo, kPhiSbo, kPhiLbo);
        ptx::mma_f16(dcol + (uint32_t)n0, ah, bh, id, accumulate);
        ptx::mma_f16(dcol + (uint32_t)n0, al, bh, id, true);
        ptx::mma_f16(dcol + (uint32_t)n0, ah, bl, id, true);
    }
}

template <int KH, bool kTMA, bool kMask>
__global__ void __launch_bounds__(kTile, 1) mma_kernel(const __grid_constant__ CUtensorMap tmap, const MmaParams P) {
    using B = Basis<KH>;
    constexpr int K = B::K, NBR = B::NBR;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const int rows = P.nbox * P.box_rows;
    const size_t y_bytes = ((size_t)rows * kTile * 2 + 1023) & ~(size_t)1023;
    const size_t phi_one = (size_t)(P.npad / 8) * 512;
    int16_t* sY = reinterpret_cast<int16_t*>(smem_raw);
    unsigned char* sPhi = smem_raw + y_bytes;  // hi table, then lo table
    unsigned char* sA = sPhi + 2 * phi_one;    // two A buffers (also beta planes, ring)
    uint64_t* bars = reinterpret_cast<uint64_t*>(sA + 2 * kBufBytes);
    uint64_t* bar_load = bars + 0;
    uint64_t* bar_a = bars + 1;  // [2] A-buffer reuse, Gram phase
    uint64_t* bar_r = bars + 3;  // [2] A-buffer reuse, refinement phase
    uint64_t* bar_done = bars + 5;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 6);
    const unsigned char* phi_hi = sPhi;
    const unsigned char* phi_lo = sPhi + phi_one;

    const int tid = threadIdx.x, warp = tid >> 5;
    const int64_t p0 = (int64_t)blockIdx.x * kTile;
    const int64_t p = p0 + tid;
    const bool active = p < P.m;
    const int N = P.N, n_hist = P.n_hist;
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;

    if (tid == 0) {
        ptx::mbar_init(bar_load, 1);
        for (int i = 1; i < 6; ++i) ptx::mbar_init(bars + i, 1);
        ptx::fence_mbar_init();
    }
    if (warp == 0) ptx::tmem_alloc(tslot, P.tmem_cols);
    {
        const size_t n16 = 2 * phi_one / 16;
        uint4* dst = reinterpret_cast<uint4*>(sPhi);
        for (size_t i = tid; i < n16; i += kTile) dst[i] = __ldg(P.phi + i);
    }
    ptx::fence_async_smem();
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem = *tslot;
    bool ok = true;

    // ---- stage Y ----------------------------------------------------------------------
    if constexpr (kTMA) {
        if (tid == 0) {
            ptx::prefetch_tmap(&tmap);
            ptx::mbar_arrive_expect_tx(bar_load, (uint32_t)(rows * kTile * 2));
            for (int b = 0; b < P.nbox; ++b)
                ptx::tma_load_2d(sY + (size_t)b * P.box_rows * kTile, &tmap, bar_load, (int)p0, b * P.box_rows);
        }
        if (!ptx::mbar_wait_bounded(bar_load, 0, kWaitNs)) {
            ok = false;
            if (tid == 0) atomicOr(&g_bfm_mma_err, 1u);
            ptx::mbar_wait_bounded(bar_load, 0, kWaitNs);
        }
    } else {
        for (int idx = tid; idx < N * kTile; idx += kTile) {
            const int t = idx / kTile, l = idx % kTile;
            sY[idx] = (p0 + l < P.m) ? P.Y[(size_t)t * P.m + p0 + l] : (int16_t)-32768;
        }
        __syncthreads();
    }
    if (!__syncthreads_and(ok)) {
        if (active) P.status[p] = BFM_PX_TIMEOUT;
        ptx::tc_fence_before();
        __syncthreads();
        if (warp == 0) ptx::tmem_dealloc(tmem, P.tmem_cols);
        return;
    }

    const uint32_t* mrow = P.mask + (p0 >> 5) + (tid >> 5);
    auto obs = [&](int t, int& y) -> bool {
        y = sY[t * kTile + tid];
        bool v = y != -32768;
        if constexpr (kMask) v = v && ((__ldg(mrow + (size_t)t * P.mask_words) >> (tid & 31)) & 1u);
        return v;
    };
    uint32_t wait_phase_done = 0;
    auto wait_done = [&]() -> bool {
        const bool r = ptx::mbar_wait_bounded(bar_done, wait_phase_done & 1u, kWaitNs);
        ++wait_phase_done;
        ptx::tc_fence_after();
        return r;
    };

    // ---- A: masked basis sums and X'My over the history --------------------------------
    const int nch = (n_hist + kChunk - 1) / kChunk;
    float ymax = 0.f;
    for (int c = 0; c < nch; ++c) {
        const int buf = c & 1;
        unsigned char* pl = sA + (size_t)buf * kBufBytes;
        if (c >= 2) ok &= ptx::mbar_wait_bounded(bar_a + buf, (uint32_t)(((c >> 1) - 1) & 1), kWaitNs);
#pragma unroll 1
        for (int g = 0; g < kChunk / 8; ++g) {
            float mk[8], a1[8], a2[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int t = c * kChunk + g * 8 + e;
                int y = -32768;
                bool v = false;
                if (t < n_hist) v = obs(t, y);
                mk[e] = v ? 1.f : 0.f;
                a1[e] = v ? (float)((y >> 8) * 256) : 0.f;
                a2[e] = v ? (float)(y & 255) : 0.f;
                ymax = fmaxf(ymax, v ? fabsf((float)y) : 0.f);
            }
            st_a(pl, tid, g, mk);
            st_a(pl + kPlane, tid, g, a1);
            st_a(pl + 2 * kPlane, tid, g, a2);
        }
        ptx::fence_async_smem();
        ptx::tc_fence_before();
        __syncthreads();
        if (tid == 0) {
            ptx::tc_fence_after();
#pragma unroll
            for (int kb = 0; kb < kChunk / 16; ++kb) {
                const int d0 = c * kChunk + kb * 16;
                const bool first = (c == 0 && kb == 0);
                mma_kblock(tmem + kColG, pl, kb, phi_hi, d0, 32, !first);
                mma_kblock(tmem + kColG, pl, kb, phi_lo, d0, 32, true);
                mma_kblock(tmem + kColB, pl + kPlane, kb, phi_hi, d0, 16, !first);
                mma_kblock(tmem + kColB, pl + kPlane, kb, phi_lo, d0, 16, true);
                mma_kblock(tmem + kColB, pl + 2 * kPlane, kb, phi_hi, d0, 16, true);
                mma_kblock(tmem + kColB, pl + 2 * kPlane, kb, phi_lo, d0, 16, true);
            }
            ptx::mma_commit(bar_a + buf);
            if (c == nch - 1) ptx::mma_commit(bar_done);
        }
    }
    ok &= wait_done();

    // ---- solve -------------------------------------------------------------------------
    float a[NBR], bb[K];
    {
        float v32[32], v16[16];
        ptx::tmem_ld32(tmem + lane_base + kColG, v32);
        ptx::tmem_ld16(tmem + lane_base + kColB, v16);
#pragma unroll
        for (int i = 0; i < NBR; ++i) a[i] = v32[i];
#pragma unroll
        for (int i = 0; i < K; ++i) bb[i] = v16[i];
    }
    const int n_i = (int)a[0];
    float G[K][K], L[K][K], dinv[K], beta[K];
    gram_from_sums<KH>(a, G);
    const bool nonsingular = cholesky<K>(G, L, dinv);
    chol_solve<K>(L, dinv, bb, beta);

    // coef/16 as fp16 hi and lo A rows (coefficient slots 0..K-1, 8..15 zero) in buffer 0
    auto write_beta = [&](const float (&coef)[K]) {
        float h[8], l[8], z[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const float b16 = i < K ? coef[i] * 0.0625f : 0.f;
            h[i] = __half2float(__float2half_rn(b16));
            l[i] = b16 - h[i];
            z[i] = 0.f;
        }
        st_a(sA, tid, 0, h);
        st_a(sA, tid, 1, z);
        st_a(sA + kPlane, tid, 0, l);
        st_a(sA + kPlane, tid, 1, z);
        ptx::fence_async_smem();
        ptx::tc_fence_before();
        __syncthreads();
    };

    // ---- yhat0 = X beta0 over all dates ------------------------------------------------------
    write_beta(beta);
    if (tid == 0) {
        ptx::tc_fence_after();
        mma_yhat(tmem + kColY, sA, sA + kPlane, phi_hi, phi_lo, P.npad, false);
        ptx::mma_commit(bar_done);
    }
    ok &= wait_done();

    // ---- refinement: r0 = y - yhat0, X'M r0 by MMA ------------------------------------------
    float ss = 0.f;
    for (int c = 0; c < nch; ++c) {
        const int buf = c & 1;
        unsigned char* pl = sA + (size_t)buf * kBufBytes;
        if (c >= 2) ok &= ptx::mbar_wait_bounded(bar_r + buf, (uint32_t)(((c >> 1) - 1) & 1), kWaitNs);
#pragma unroll 1
        for (int g = 0; g < kChunk / 8; ++g) {
            float yh[8], rh[8], rl[8];
            ptx::tmem_ld8(tmem + lane_base + kColY + (uint32_t)(c * kChunk + g * 8), yh);
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int t = c * kChunk + g * 8 + e;
                int y = 0;
                bool v = false;
                if (t < n_hist) v = obs(t, y);
                const float r0 = v ? ((float)y - 16.f * yh[e]) : 0.f;
                ss = fmaf(r0, r0, ss);
                const float r4 = r0 * 0.25f;
                rh[e] = __half2float(__float2half_rn(r4));
                rl[e] = r4 - rh[e];
            }
            st_a(pl, tid, g, rh);
            st_a(pl + kPlane, tid, g, rl);
        }
        ptx::fence_async_smem();
        ptx::tc_fence_before();
        __syncthreads();
        if (tid == 0) {
            ptx::tc_fence_after();
#pragma unroll
            for (int kb = 0; kb < kChunk / 16; ++kb) {
                const int d0 = c * kChunk + kb * 16;
                const bool first = (c == 0 && kb == 0);
                mma_kblock(tmem + kColC, pl, kb, phi_hi, d0, 16, !first);
                mma_kblock(tmem + kColC, pl, kb, phi_lo, d0, 16, true);
                mma_kblock(tmem + kColC, pl + kPlane, kb, phi_hi, d0, 16, true);
            }
            ptx::mma_commit(bar_r + buf);
            if (c == nch - 1) ptx::mma_commit(bar_done);
        }
    }
    ok &= wait_done();
    float sigma, scale, thr;
    int h, jlim;
    float dl[K];
    {
        float v16[16], cc[K];
        ptx::tmem_ld16(tmem + lane_base + kColC, v16);
#pragma unroll
        for (int i = 0; i < K; ++i) cc[i] = 4.f * v16[i];
        chol_solve<K>(L, dinv, cc, dl);
        float dc = 0.f;
#pragma unroll
        for (int i = 0; i < K; ++i) {
            beta[i] += dl[i];
            dc = fmaf(dl[i], cc[i], dc);
        }
        sigma = sqrtf(fmaxf(ss - dc, 0.f) / (float)(n_i - K));
        scale = sigma * sqrtf((float)n_i);
        thr = P.lambda * scale;
        h = (int)floor(P.h_frac * (double)n_i);
        if (h < 1) h = 1;
        if (h > n_i) h = n_i;
        jlim = (int)floor(kEuler * (double)n_i);
    }

    // ---- yhat = yhat0 + X delta over all dates ---------------------------------------------------
    // Adding the correction to the stored yhat0 (rather than forming X beta
    // again) makes the fp16 split error of beta0 -- which lies in the span of
    // X -- cancel between the refinement residuals and the final residuals.
    write_beta(dl);
    if (tid == 0) {
        ptx::tc_fence_after();
        mma_yhat(tmem + kColY, sA, sA + kPlane, phi_hi, phi_lo, P.npad, true);
        ptx::mma_commit(bar_done);
    }
    ok &= wait_done();

    // ---- MOSUM, 8 dates at a time ---------------------------------------------------------
    // Per group: residuals and validity independently; the compensated prefix
    // sums S_J over valid positions go to a ring of R >= h + 9 slots (the
    // group's writes all land before its reads); then each window
    // W_J = S_J - S_{J-h} of the group's monitoring positions (Eq. 3) is an
    // independent difference tested against lambda*sqrt(log+(J/n)) (Eq. 4).
    // Branch-free: invalid dates add 0 and their (in-range) lag reads are masked.
    float* ring = reinterpret_cast<float*>(sA);  // [P.ring][128], free now
    const int R = P.ring;
    int j = 0, slot = 0, brk = -1;
    float Sh = 0.f, Sc = 0.f;                       // running prefix sum (compensated)
    float m0 = 0.f, m0c = 0.f, m1 = 0.f, m1c = 0.f;  // two interleaved sums of W
#pragma unroll 1
    for (int c0 = 0; c0 < N; c0 += 8) {
        float yh[8];
        ptx::tmem_ld8(tmem + lane_base + kColY + (uint32_t)c0, yh);
        float r[8];
        uint32_t vb = 0u;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int t = c0 + e;
            int y = 0;
            const bool v = t < N && obs(t, y);
            r[e] = (float)y - 16.f * yh[e];
            vb |= (v ? 1u : 0u) << e;
        }
        float Sv[8];
        int sl[8], jj[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int v = (vb >> e) & 1u;
            comp_add(Sh, Sc, v ? r[e] : 0.f);
            Sv[e] = Sh + Sc;
            if (v) ring[slot * kTile + tid] = Sv[e];
            sl[e] = slot;
            jj[e] = j;
            j += v;
            slot += v;
            slot = slot == R ? 0 : slot;
        }
        const int d = n_hist - c0;  // monitoring dates of the group: e >= d
        const uint32_t mon = d <= 0 ? 0xffu : (d >= 8 ? 0u : (0xffu << d) & 0xffu);
        const uint32_t mv = vb & mon;
        uint32_t cross = 0u;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            int ls = sl[e] - h;
            ls += ls < 0 ? R : 0;
            const float W = Sv[e] - ring[ls * kTile + tid];
            const int J = jj[e] + 1;
            float th = thr;
            if (J > jlim) th = thr * sqrtf(logf((float)J / (float)n_i));
            const bool m = (mv >> e) & 1u;
            cross |= ((m && fabsf(W) > th) ? 1u : 0u) << e;
            if (e & 1)
                comp_add(m1, m1c, m ? W : 0.f);
            else
                comp_add(m0, m0c, m ? W : 0.f);
        }
        if (brk < 0 && cross) brk = c0 + __ffs(cross) - 1;
    }
    float sumW = m0, sumWc = m0c;
    comp_add(sumW, sumWc, m1);
    sumWc += m1c;
    const int N_i = j;

    // ---- outputs ------------------------------------------------------------------------------
    ptx::tc_fence_before();
    __syncthreads();
    if (warp == 0) ptx::tmem_dealloc(tmem, P.tmem_cols);
    if (!active) return;
    if (!ok) {
        P.status[p] = BFM_PX_TIMEOUT;
        atomicOr(&g_bfm_mma_err, 2u);
        return;
    }
    const bool degenerate = !(sigma > kDegenerateRatio * ymax) || ymax == 0.f;
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
    } else if (N_i == n_i) {
        st = BFM_PX_NO_MONITOR;
    } else {
        st = BFM_PX_OK;
        o_brk = brk;
        o_mean = (sumW + sumWc) / ((float)(N_i - n_i) * scale);
    }
    if (!fitted) o_sigma = qnan;
    P.status[p] = st;
    P.brk[p] = o_brk;
    P.mean[p] = o_mean;
    P.sigma[p] = o_sigma;
#pragma unroll
    for (int i = 0; i < K; ++i) {
        float bi = beta[i];
        if (i == 0) bi = fmaf(-beta[1], P.c_over_s, beta[0]);
        if (i == 1) bi = beta[1] * P.inv_s;
        P.beta[(size_t)i * P.m + p] = fitted ? bi : qnan;
    }
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

size_t mma_smem(int N, int npad, int* box_rows, int* nbox) {
    const int nb = (N + 255) / 256;
    const int br = (N + nb - 1) / nb;
    const size_t y = (((size_t)nb * br * kTile * 2) + 1023) & ~(size_t)1023;
    if (box_rows) *box_rows = br;
    if (nbox) *nbox = nb;
    return y + tc_phi_bytes(npad) + 2 * (size_t)kBufBytes + 64;
}

// Ring of prefix sums: the h slots behind the oldest new position of an
// 8-date group must survive the group's writes.
int ring_len(int n_hist, double h_frac) {
    int hmax = (int)std::floor(h_frac * (double)n_hist);
    if (hmax < 1) hmax = 1;
    if (hmax > n_hist) hmax = n_hist;
    return hmax + 9;
}

template <int KH, bool kTMA>
bfm_status launch_t(const CUtensorMap& tm, const MmaParams& P, size_t smem, cudaStream_t stream) {
    auto kern = P.mask ? mma_kernel<KH, kTMA, true> : mma_kernel<KH, kTMA, false>;
    static thread_local int configured[2] = {-1, -1};
    int dev = 0;
    cudaGetDevice(&dev);
    if (configured[P.mask ? 1 : 0] != dev) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(mma_kernel)");
        configured[P.mask ? 1 : 0] = dev;
    }
    const unsigned grid = (unsigned)((P.m + kTile - 1) / kTile);
    kern<<<grid, kTile, smem, stream>>>(tm, P);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "mma kernel launch");
    return BFM_OK;
}

}  // namespace

bool mma_supported(const bfm_design_s* d, int dtype, int n_hist, double h_frac, size_t* smem_out) {
    if (dtype != BFM_I16 || !d->d_phi_tc || d->N > kTcMaxDates) return false;
    if (ring_len(n_hist, h_frac) * kTile * 4 > 2 * kBufBytes) return false;
    const size_t smem = mma_smem(d->N, d->npad_tc, nullptr, nullptr);
    if (smem_out) *smem_out = smem;
    return smem <= 227 * 1024;
}

bfm_status launch_mma(const bfm_design_s* d, const void* Y, const uint32_t* mask, int64_t m, int n_hist,
                      double h_frac, double lambda, int32_t* brk, float* mean, float* sigma, float* beta,
                      uint8_t* status, cudaStream_t stream) {
    MmaParams P{};
    int br = 0, nb = 0;
    const size_t smem = mma_smem(d->N, d->npad_tc, &br, &nb);
    P.Y = static_cast<const int16_t*>(Y);
    P.mask = mask;
    P.m = m;
    P.mask_words = (m + 31) / 32;
    P.N = d->N;
    P.n_hist = n_hist;
    P.npad = d->npad_tc;
    P.nhp = (n_hist + 15) / 16 * 16;
    P.phi = static_cast<const uint4*>(d->d_phi_tc);
    P.h_frac = h_frac;
    P.lambda = (float)lambda;
    P.c_over_s = (float)(d->c / d->s);
    P.inv_s = (float)(1.0 / d->s);
    P.box_rows = br;
    P.nbox = nb;
    P.ring = ring_len(n_hist, h_frac);
    P.tmem_cols = (kColY + (uint32_t)d->npad_tc <= 256u) ? 256u : 512u;
    P.brk = brk;
    P.mean = mean;
    P.sigma = sigma;
    P.beta = beta;
    P.status = status;
    CUtensorMap tm;
    std::memset(&tm, 0, sizeof tm);
    bool tma = ((uintptr_t)Y % 16 == 0) && ((m * 2) % 16 == 0) && m >= kTile;
    if (tma) {
        auto enc = encode_fn_mma();
        if (!enc) {
            tma = false;
        } else {
            cuuint64_t gdim[2] = {(cuuint64_t)m, (cuuint64_t)d->N};
            cuuint64_t gstride[1] = {(cuuint64_t)m * 2};
            cuuint32_t box[2] = {(cuuint32_t)kTile, (cuuint32_t)br};
            cuuint32_t es[2] = {1u, 1u};
            CUresult r = enc(&tm, CU_TENSOR_MAP_DATA_TYPE_UINT16 /* same 16 bits */, 2, const_cast<void*>(Y), gdim,
                             gstride, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS) tma = false;
        }
    }
    switch (d->k) {
        case 1: return tma ? launch_t<1, true>(tm, P, smem, stream) : launch_t<1, false>(tm, P, smem, stream);
        case 2: return tma ? launch_t<2, true>(tm, P, smem, stream) : launch_t<2, false>(tm, P, smem, stream);
        default: return tma ? launch_t<3, true>(tm, P, smem, stream) : launch_t<3, false>(tm, P, smem, stream);
    }
}

}  // namespace bfm
