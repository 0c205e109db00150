// CUDA-core ("plain form") BFAST Monitor kernel: one thread per pixel, one
// warp per 32-pixel tile, the tile's whole series staged in shared memory.
//
// Per pixel (Section 2.1 and Algorithm 1, with missing values masked):
//   pass 1   masked sums of the basis functions of bfm_internal.cuh over the
//            history dates -> Gram matrix G and X'My (Eq. 5-6)
//   solve    K x K Cholesky of G, two triangular solves
//   pass 1b  one step of iterative refinement: beta += G^-1 X'M(y - X beta),
//            with the residual formed in float from the float data
//   pass 2   residuals y - x'beta (Eq. 3 sign) at every valid date, compacted
//            in place; sigma-hat from the history part (Algorithm 1, step 5);
//            the MOSUM window of h residuals kept as a compensated running
//            sum (the sliding update of Algorithm 3, over valid positions);
//            first crossing of lambda*sqrt(log+(j/n)) (Eq. 4) and the mean.
//
// Y is time-major (Eq. 7), so a warp's 32 pixels of one date are one
// 128-byte (float) or 64-byte (int16) row: the tile [N][32] arrives by 2-D
// TMA boxes of up to 256 dates, or by coalesced plain loads when the layout
// does not meet TMA's alignment rules.
#include <cudaTypedefs.h>

#include <cmath>
#include <mutex>

#include "bfm_internal.cuh"
#include "ptx.cuh"

namespace bfm {

__device__ unsigned int g_bfm_err = 0;

cudaError_t simt_read_clear_errors(cudaStream_t s, unsigned int* bits) {
    unsigned int v = 0;
    cudaError_t e = cudaMemcpyFromSymbolAsync(&v, g_bfm_err, sizeof v, 0, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    const unsigned int zero = 0;
    e = cudaMemcpyToSymbolAsync(g_bfm_err, &zero, sizeof zero, 0, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    *bits = v;
    return e;
}

namespace {

constexpr uint64_t kLoadWaitLimitNs = 2000000000ull;  // 2 s
constexpr float kSingularRatio = 1e-5f;
constexpr float kDegenerateRatio = 1e-6f;
constexpr double kE = 2.71828182845904523536;

template <typename T>
struct Obs;

template <>
struct Obs<float> {
    static __device__ __forceinline__ bool get(const float* tile, int idx, float& y) {
        float v = tile[idx];
        y = v;
        return v == v;  // not NaN
    }
    static __device__ __forceinline__ float missing() { return __int_as_float(0x7fc00000); }
};

template <>
struct Obs<int16_t> {
    static __device__ __forceinline__ bool get(const int16_t* tile, int idx, float& y) {
        int v = tile[idx];
        y = (float)v;
        return v != -32768;
    }
    static __device__ __forceinline__ int16_t missing() { return (int16_t)-32768; }
};

// Compensated (Neumaier) accumulation s += x with error term c.
__device__ __forceinline__ void comp_add(float& s, float& c, float x) {
    float t = s + x;
    if (fabsf(s) >= fabsf(x))
        c += (s - t) + x;
    else
        c += (x - t) + s;
    s = t;
}

template <int KH>
__device__ __forceinline__ void load_row(const float4* __restrict__ B4, int t, float (&q)[Basis<KH>::NB]) {
    constexpr int NB = Basis<KH>::NB;
#pragma unroll
    for (int i = 0; i < NB / 4; ++i) {
        float4 v = __ldg(B4 + (size_t)t * (NB / 4) + i);
        q[4 * i + 0] = v.x;
        q[4 * i + 1] = v.y;
        q[4 * i + 2] = v.z;
        q[4 * i + 3] = v.w;
    }
}

template <int KH>
__device__ __forceinline__ void load_x(const float4* __restrict__ B4, int t, float (&x)[Basis<KH>::K]) {
    constexpr int NB = Basis<KH>::NB, K = Basis<KH>::K;
    float q[(K + 3) & ~3];
#pragma unroll
    for (int i = 0; i < (K + 3) / 4; ++i) {
        float4 v = __ldg(B4 + (size_t)t * (NB / 4) + i);
        q[4 * i + 0] = v.x;
        q[4 * i + 1] = v.y;
        q[4 * i + 2] = v.z;
        q[4 * i + 3] = v.w;
    }
#pragma unroll
    for (int i = 0; i < K; ++i) x[i] = q[i];
}

// Gram matrix from the masked basis sums a[] (see Basis).
template <int KH>
__device__ __forceinline__ void gram_from_sums(const float (&a)[Basis<KH>::NBR], float (&G)[Basis<KH>::K][Basis<KH>::K]) {
    using B = Basis<KH>;
    auto Cs = [&](int j) -> float { return j == 0 ? a[0] : a[B::C(j)]; };
    auto Ss = [&](int j) -> float { return j == 0 ? 0.f : (j > 0 ? a[B::S(j)] : -a[B::S(-j)]); };
    G[0][0] = a[0];
    G[0][1] = a[1];
    G[1][1] = a[B::TT];
#pragma unroll
    for (int j = 1; j <= KH; ++j) {
        G[0][B::S(j)] = a[B::S(j)];
        G[0][B::C(j)] = a[B::C(j)];
        G[1][B::S(j)] = a[B::TS(j)];
        G[1][B::C(j)] = a[B::TC(j)];
#pragma unroll
        for (int b = 1; b <= KH; ++b) {
            int dm = j > b ? j - b : b - j;
            G[B::S(j)][B::S(b)] = 0.5f * (Cs(dm) - Cs(j + b));
            G[B::C(j)][B::C(b)] = 0.5f * (Cs(dm) + Cs(j + b));
            G[B::S(j)][B::C(b)] = 0.5f * (Ss(j + b) + Ss(j - b));
        }
    }
#pragma unroll
    for (int i = 0; i < B::K; ++i)
#pragma unroll
        for (int j = 0; j < i; ++j) G[i][j] = G[j][i];
    // the sin/cos blocks were written for all (j, b); make them symmetric too
#pragma unroll
    for (int i = 0; i < B::K; ++i)
#pragma unroll
        for (int j = i + 1; j < B::K; ++j) G[j][i] = G[i][j];
}

// In-register Cholesky G = L L' (lower, reciprocal diagonal kept in dinv).
// Returns false when a pivot relative to its diagonal entry is below kSingularRatio.
template <int K>
__device__ __forceinline__ bool cholesky(const float (&G)[K][K], float (&L)[K][K], float (&dinv)[K]) {
    bool ok = true;
#pragma unroll
    for (int j = 0; j < K; ++j) {
        float d = G[j][j];
#pragma unroll
        for (int c = 0; c < j; ++c) d = fmaf(-L[j][c], L[j][c], d);
        ok = ok && (d >= kSingularRatio * G[j][j]) && (G[j][j] > 0.f);
        float inv = rsqrtf(fmaxf(d, 1e-30f));
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
__device__ __forceinline__ void chol_solve(const float (&L)[K][K], const float (&dinv)[K], const float (&b)[K],
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

template <int KH, typename T, bool kTMA>
__global__ void __launch_bounds__(32) simt_kernel(const __grid_constant__ CUtensorMap tmap, const MonitorParams P) {
    using B = Basis<KH>;
    constexpr int K = B::K, NB = B::NB, NBR = B::NBR;
    constexpr bool kInPlace = sizeof(T) == sizeof(float);

    extern __shared__ __align__(128) unsigned char smem_raw[];
    T* tile = reinterpret_cast<T*>(smem_raw);
    const int rows = P.nbox * P.box_rows;
    const size_t tile_bytes = ((size_t)rows * 32 * sizeof(T) + 127) & ~(size_t)127;
    float* ring = reinterpret_cast<float*>(smem_raw + tile_bytes);
    const size_t ring_bytes = (size_t)P.ring * 32 * sizeof(float);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + tile_bytes + ring_bytes);

    const int lane = threadIdx.x;
    const int64_t p0 = (int64_t)blockIdx.x * 32;
    const int64_t p = p0 + lane;
    const bool active = p < P.m;
    const int N = P.N, n_hist = P.n_hist;

    // ---- stage the [N][32] tile -------------------------------------------------
    if constexpr (kTMA) {
        if (lane == 0) {
            ptx::prefetch_tmap(&tmap);
            ptx::mbar_init(bar, 1);
            ptx::fence_mbar_init();
        }
        __syncwarp();
        if (lane == 0) {
            ptx::mbar_arrive_expect_tx(bar, (uint32_t)(rows * 32 * sizeof(T)));
            for (int b = 0; b < P.nbox; ++b)
                ptx::tma_load_2d(tile + (size_t)b * P.box_rows * 32, &tmap, bar, (int)p0, b * P.box_rows);
        }
        if (!ptx::mbar_wait_bounded(bar, 0, kLoadWaitLimitNs)) {
            if (lane == 0) atomicOr(&g_bfm_err, 1u);
            if (active) P.status[p] = BFM_PX_TIMEOUT;
            ptx::mbar_wait_bounded(bar, 0, kLoadWaitLimitNs);  // let copies in flight land
            return;
        }
    } else {
        const T* Yp = reinterpret_cast<const T*>(P.Y);
        for (int t = 0; t < N; ++t) tile[t * 32 + lane] = active ? Yp[(size_t)t * P.m + p] : Obs<T>::missing();
        __syncwarp();
    }

    const float4* B4 = reinterpret_cast<const float4*>(P.basis);
    const uint32_t* mrow = P.mask ? P.mask + blockIdx.x : nullptr;

    auto obs = [&](int t, float& y) -> bool {
        bool v = Obs<T>::get(tile, t * 32 + lane, y);
        if (mrow) v = v && ((__ldg(mrow + (size_t)t * P.mask_words) >> lane) & 1u);
        return v;
    };

    // ---- pass 1: masked basis sums and X'My over the history ---------------------
    float a[NBR], bb[K];
#pragma unroll
    for (int i = 0; i < NBR; ++i) a[i] = 0.f;
#pragma unroll
    for (int i = 0; i < K; ++i) bb[i] = 0.f;
    float ymax = 0.f;
#pragma unroll 2
    for (int t = 0; t < n_hist; ++t) {
        float y;
        bool v = obs(t, y);
        float w = v ? 1.f : 0.f, yw = v ? y : 0.f;
        ymax = fmaxf(ymax, fabsf(yw));
        float q[NB];
        load_row<KH>(B4, t, q);
        a[0] += w;
#pragma unroll
        for (int l = 1; l < NBR; ++l) a[l] = fmaf(w, q[l], a[l]);
        bb[0] += yw;
#pragma unroll
        for (int i = 1; i < K; ++i) bb[i] = fmaf(yw, q[i], bb[i]);
    }
    const int n_i = (int)a[0];

    // ---- solve ---------------------------------------------------------------------
    float G[K][K], L[K][K], dinv[K], beta[K];
    gram_from_sums<KH>(a, G);
    const bool nonsingular = cholesky<K>(G, L, dinv);
    chol_solve<K>(L, dinv, bb, beta);

    // ---- pass 1b: one refinement step ------------------------------------------------
    {
        float cc[K];
#pragma unroll
        for (int i = 0; i < K; ++i) cc[i] = 0.f;
#pragma unroll 2
        for (int t = 0; t < n_hist; ++t) {
            float y;
            bool v = obs(t, y);
            float x[K];
            load_x<KH>(B4, t, x);
            float f0 = 0.f, f1 = 0.f;
#pragma unroll
            for (int i = 0; i < K; i += 2) {
                f0 = fmaf(x[i], beta[i], f0);
                f1 = fmaf(x[i + 1], beta[i + 1], f1);
            }
            float r = v ? (y - (f0 + f1)) : 0.f;
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
    const int wstart = n_i - h;  // first compacted index inside the first window

    auto store_r = [&](int j, float r) {
        if constexpr (kInPlace)
            reinterpret_cast<float*>(tile)[j * 32 + lane] = r;
        else
            ring[(j & (P.ring - 1)) * 32 + lane] = r;
    };
    auto load_r = [&](int j) -> float {
        if constexpr (kInPlace)
            return reinterpret_cast<float*>(tile)[j * 32 + lane];
        else
            return ring[(j & (P.ring - 1)) * 32 + lane];
    };

    // ---- pass 2a: history residuals, sigma-hat, first window -------------------------
    int j = 0;
    float ss = 0.f, W = 0.f, Wc = 0.f;
#pragma unroll 2
    for (int t = 0; t < n_hist; ++t) {
        float y;
        bool v = obs(t, y);
        float x[K];
        load_x<KH>(B4, t, x);
        float f0 = 0.f, f1 = 0.f;
#pragma unroll
        for (int i = 0; i < K; i += 2) {
            f0 = fmaf(x[i], beta[i], f0);
            f1 = fmaf(x[i + 1], beta[i + 1], f1);
        }
        float r = y - (f0 + f1);
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
    const int jlim = (int)floor(kE * (double)n_i);  // j/n_i <= e  <=>  j <= jlim

    // ---- pass 2b: monitoring MOSUM, first crossing, mean ------------------------------
    int brk = -1;
    float sumW = 0.f, sumWc = 0.f;
#pragma unroll 2
    for (int t = n_hist; t < N; ++t) {
        float y;
        bool v = obs(t, y);
        float x[K];
        load_x<KH>(B4, t, x);
        float f0 = 0.f, f1 = 0.f;
#pragma unroll
        for (int i = 0; i < K; i += 2) {
            f0 = fmaf(x[i], beta[i], f0);
            f1 = fmaf(x[i + 1], beta[i + 1], f1);
        }
        float r = y - (f0 + f1);
        if (v) {
            float lag = load_r(j - h);
            store_r(j, r);
            comp_add(W, Wc, r - lag);
            const float wv = W + Wc;
            const int J = j + 1;  // 1-based monitoring position
            float th = thr;
            if (J > jlim) th = thr * sqrtf(logf((float)J / (float)n_i));
            if (brk < 0 && fabsf(wv) > th) brk = t;
            comp_add(sumW, sumWc, wv);
            ++j;
        }
    }
    const int N_i = j;

    if (!active) return;
    uint8_t st;
    float o_mean, o_sigma = sigma;
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
        o_mean = __int_as_float(0x7fc00000);
    } else {
        st = BFM_PX_OK;
        o_brk = brk;
        o_mean = (sumW + sumWc) / ((float)(N_i - n_i) * scale);
    }
    const float qnan = __int_as_float(0x7fc00000);
    if (!fitted) {
        o_mean = qnan;
        o_sigma = qnan;
    }
    P.status[p] = st;
    P.brk[p] = o_brk;
    P.mean[p] = o_mean;
    P.sigma[p] = o_sigma;
    // beta of the centred trend -> raw parameterisation of Eq. 2
    float braw[K];
#pragma unroll
    for (int i = 0; i < K; ++i) braw[i] = beta[i];
    braw[0] = fmaf(-beta[1], P.c_over_s, beta[0]);
    braw[1] = beta[1] * P.inv_s;
#pragma unroll
    for (int i = 0; i < K; ++i) P.beta[(size_t)i * P.m + p] = fitted ? braw[i] : qnan;
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
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

template <int KH, typename T, bool kTMA>
bfm_status launch_one(const CUtensorMap& tm, const MonitorParams& P, size_t smem, cudaStream_t stream) {
    auto kern = simt_kernel<KH, T, kTMA>;
    static thread_local int configured_dev = -1;
    int dev = 0;
    cudaGetDevice(&dev);
    if (configured_dev != dev) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(MaxDynamicSharedMemorySize)");
        cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        configured_dev = dev;
    }
    const unsigned grid = (unsigned)((P.m + 31) / 32);
    kern<<<grid, 32, smem, stream>>>(tm, P);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "simt kernel launch");
    return BFM_OK;
}

template <int KH>
bfm_status dispatch_dtype(int dtype, bool tma, const CUtensorMap& tm, const MonitorParams& P, size_t smem,
                          cudaStream_t s) {
    if (dtype == BFM_F32)
        return tma ? launch_one<KH, float, true>(tm, P, smem, s) : launch_one<KH, float, false>(tm, P, smem, s);
    return tma ? launch_one<KH, int16_t, true>(tm, P, smem, s) : launch_one<KH, int16_t, false>(tm, P, smem, s);
}

}  // namespace

size_t simt_smem_bytes(int N, int dtype, int n_hist, double h_frac, int* box_rows, int* nbox, int* ring) {
    const int elt = dtype == BFM_F32 ? 4 : 2;
    const int nb = (N + 255) / 256;
    const int br = (N + nb - 1) / nb;
    const int rows = nb * br;
    size_t tile = ((size_t)rows * 32 * elt + 127) & ~(size_t)127;
    int rg = 0;
    if (dtype != BFM_F32) {
        int hmax = (int)std::floor(h_frac * (double)n_hist);
        if (hmax < 1) hmax = 1;
        if (hmax > n_hist) hmax = n_hist;
        rg = 1;
        while (rg < hmax + 1) rg <<= 1;
    }
    size_t total = tile + (size_t)rg * 32 * 4 + 16;
    if (box_rows) *box_rows = br;
    if (nbox) *nbox = nb;
    if (ring) *ring = rg;
    return total <= 227 * 1024 ? total : 0;
}

bfm_status launch_simt(const bfm_design_s* d, const void* Y, int dtype, const uint32_t* mask, int64_t m, int n_hist,
                       double h_frac, double lambda, int32_t* brk, float* mean, float* sigma, float* beta,
                       uint8_t* status, cudaStream_t stream) {
    MonitorParams P{};
    int br = 0, nb = 0, rg = 0;
    size_t smem = simt_smem_bytes(d->N, dtype, n_hist, h_frac, &br, &nb, &rg);
    if (smem == 0) {
        set_error("bfm_monitor: the series does not fit one on-chip tile (N or the bandwidth too large)");
        return BFM_EUNSUPPORTED;
    }
    P.Y = Y;
    P.mask = mask;
    P.m = m;
    P.mask_words = (m + 31) / 32;
    P.N = d->N;
    P.n_hist = n_hist;
    P.basis = d->d_basis;
    P.h_frac = h_frac;
    P.lambda = (float)lambda;
    P.c_over_s = (float)(d->c / d->s);
    P.inv_s = (float)(1.0 / d->s);
    P.box_rows = br;
    P.nbox = nb;
    P.ring = rg;
    P.brk = brk;
    P.mean = mean;
    P.sigma = sigma;
    P.beta = beta;
    P.status = status;

    const int elt = dtype == BFM_F32 ? 4 : 2;
    CUtensorMap tm;
    memset(&tm, 0, sizeof(tm));
    bool tma = ((uintptr_t)Y % 16 == 0) && (((int64_t)m * elt) % 16 == 0) && m >= 32;
    if (tma) {
        auto enc = encode_fn();
        if (!enc) {
            tma = false;
        } else {
            cuuint64_t gdim[2] = {(cuuint64_t)m, (cuuint64_t)d->N};
            cuuint64_t gstride[1] = {(cuuint64_t)m * elt};
            cuuint32_t box[2] = {32u, (cuuint32_t)br};
            cuuint32_t estride[2] = {1u, 1u};
            CUresult r = enc(&tm, dtype == BFM_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_UINT16 /* same 16 bits */, 2,
                             const_cast<void*>(Y), gdim, gstride, box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE,
                             CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS) tma = false;
        }
    }
    switch (d->k) {
        case 1: return dispatch_dtype<1>(dtype, tma, tm, P, smem, stream);
        case 2: return dispatch_dtype<2>(dtype, tma, tm, P, smem, stream);
        default: return dispatch_dtype<3>(dtype, tma, tm, P, smem, stream);
    }
}

}  // namespace bfm
