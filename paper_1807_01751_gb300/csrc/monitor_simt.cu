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
#include "simt_pixel.cuh"

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

template <int KH, typename T, bool kTMA>
__global__ void __launch_bounds__(32) simt_kernel(const __grid_constant__ CUtensorMap tmap, const MonitorParams P) {
    using B = Basis<KH>;
    constexpr int K = B::K, NB = B::NB;
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
    const int N = P.N;

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
    auto row = [&](int t, float (&q)[NB]) { load_row<KH>(B4, t, q); };
    auto rowx = [&](int t, float (&x)[K]) { load_x<KH>(B4, t, x); };
    auto store_r = [&](int j, float r) {
        if constexpr (kInPlace)
            reinterpret_cast<float*>(tile)[j * 32 + lane] = r;  // j <= t: overwrites consumed dates only
        else
            ring[(j & (P.ring - 1)) * 32 + lane] = r;
    };
    auto load_r = [&](int j) -> float {
        if constexpr (kInPlace)
            return reinterpret_cast<float*>(tile)[j * 32 + lane];
        else
            return ring[(j & (P.ring - 1)) * 32 + lane];
    };

    PixelParams pp{P.N, P.n_hist, P.h_frac, P.lambda, P.c_over_s, P.inv_s};
    PixelOut<KH> o;
    process_pixel<KH>(pp, obs, row, rowx, store_r, load_r, o);

    if (!active) return;
    P.status[p] = o.status;
    P.brk[p] = o.brk;
    P.mean[p] = o.mean;
    P.sigma[p] = o.sigma;
#pragma unroll
    for (int i = 0; i < K; ++i) P.beta[(size_t)i * P.m + p] = o.beta[i];
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
