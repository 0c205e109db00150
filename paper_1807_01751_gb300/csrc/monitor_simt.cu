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
#include "simt_seg.cuh"

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

bool make_tensor_map(CUtensorMap* tm, const void* Y, int dtype, int64_t m, int N, int box_rows);

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

// Shared-memory layout of one 32-pixel tile (see simt_smem_bytes).
struct TileSmem {
    unsigned char* tile;
    float* work;
    float* part;
};

template <int KH, typename T>
__device__ __forceinline__ TileSmem tile_smem(unsigned char* smem_raw, const MonitorParams& P) {
    constexpr int PS = Partials<KH>::kStride;
    const int rows = P.nbox * P.box_rows;
    const size_t tile_bytes = ((size_t)rows * 32 * sizeof(T) + 127) & ~(size_t)127;
    const size_t work_bytes = sizeof(T) == 4 ? 0 : (((size_t)P.N * 32 * sizeof(float) + 127) & ~(size_t)127);
    TileSmem L;
    L.tile = smem_raw;
    L.work = sizeof(T) == 4 ? reinterpret_cast<float*>(smem_raw) : reinterpret_cast<float*>(smem_raw + tile_bytes);
    L.part = reinterpret_cast<float*>(smem_raw + tile_bytes + work_bytes);
    (void)PS;
    return L;
}

// One 32-pixel block (pixels 32*block .. 32*block+31 of the scene in P) by the
// whole CTA (kNW warps).  tmap: tensor map of Y, or nullptr for plain loads.
// bar/bar_uses: the CTA's tile-load mbarrier and how often it has completed.
// Returns with every warp done with shared memory except for a final
// barrier the caller places before the next block.
template <int KH, typename T, bool kMask>
__device__ __forceinline__ void simt_block(const CUtensorMap* tmap, const MonitorParams& P, int64_t block,
                                           unsigned char* smem_raw, uint64_t* bar, uint32_t& bar_uses) {
    using B = Basis<KH>;
    constexpr int K = B::K, NB = B::NB, PS = Partials<KH>::kStride;
    const TileSmem L = tile_smem<KH, T>(smem_raw, P);
    T* tile = reinterpret_cast<T*>(L.tile);
    float* work = L.work;
    float* part = L.part;
    const int rows = P.nbox * P.box_rows;

    const int lane = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
    const int64_t p0 = block * 32;
    const int64_t p = p0 + lane;
    const bool active = p < P.m;
    const int N = P.N;

    // ---- stage the [N][32] tile -------------------------------------------------------
    if (tmap) {
        if (threadIdx.x == 0) {
            ptx::mbar_arrive_expect_tx(bar, (uint32_t)(rows * 32 * sizeof(T)));
            for (int b = 0; b < P.nbox; ++b)
                ptx::tma_load_2d(tile + (size_t)b * P.box_rows * 32, tmap, bar, (int)p0, b * P.box_rows);
        }
        const uint32_t parity = bar_uses & 1u;
        ++bar_uses;
        if (!__syncthreads_and(ptx::mbar_wait_bounded(bar, parity, kLoadWaitLimitNs))) {
            if (threadIdx.x == 0) atomicOr(&g_bfm_err, 1u);
            if (w == 0 && active) P.status[p] = BFM_PX_TIMEOUT;
            ptx::mbar_wait_bounded(bar, parity, kLoadWaitLimitNs);  // let copies in flight land
            return;
        }
    } else {
        const T* Yp = reinterpret_cast<const T*>(P.Y);
        for (int idx = threadIdx.x; idx < N * 32; idx += kNW * 32) {
            const int t = idx >> 5, l = idx & 31;
            tile[idx] = (p0 + l < P.m) ? Yp[(size_t)t * P.m + p0 + l] : Obs<T>::missing();
        }
        __syncthreads();
    }

    const float4* B4 = reinterpret_cast<const float4*>(P.basis);
    const uint32_t* mrow = P.mask + (p0 >> 5);
    auto obs = [&](int t, float& y) -> bool {
        bool v = Obs<T>::get(tile, t * 32 + lane, y);
        if constexpr (kMask) v = v && ((__ldg(mrow + (size_t)t * P.mask_words) >> lane) & 1u);
        return v;
    };
    auto row = [&](int t, float (&q)[NB]) { load_row<KH>(B4, t, q); };
    auto rowx = [&](int t, float (&x)[K]) { load_x<KH>(B4, t, x); };
    auto partf = [&](int ww, int i) -> float& { return part[(ww * PS + i) * 32 + lane]; };
    auto put_r = [&](int t, float r) { work[t * 32 + lane] = r; };
    auto get_r = [&](int t) -> float { return work[t * 32 + lane]; };
    auto putw = [&](int ww, int i, uint32_t bits) { partf(ww, 3 + i) = __uint_as_float(bits); };
    auto getw = [&](int ww, int i) -> uint32_t { return __float_as_uint(partf(ww, 3 + i)); };

    const SegParams sp{P.N, P.n_hist, P.h_frac, P.lambda, P.c_over_s, P.inv_s};
    Lane<KH> S;
    phase1_gram<KH>(sp, w, obs, row, partf);
    __syncthreads();
    phase2_solve<KH>(S, partf);
    __syncthreads();
    phase3_refine<KH>(sp, w, S, obs, rowx, partf);
    __syncthreads();
    phase4_sigma<KH>(sp, S, partf);
    __syncthreads();
    phase5_resid<KH>(sp, w, S, obs, rowx, put_r, partf, putw);
    __syncthreads();
    phase6_offsets<KH>(w, S, partf);
    __syncthreads();  // phase 7 overwrites the segment totals phase 6 reads in every warp
    int first_mon = S.n_i - S.myoff;
    first_mon = first_mon < 0 ? 0 : first_mon;
    const int jlo = __reduce_min_sync(0xffffffffu, first_mon);
    const int jhi = __reduce_max_sync(0xffffffffu, S.mycnt);
    phase7_mosum<KH>(sp, w, S, get_r, jlo, jhi, partf, getw);
    __syncthreads();
    if (w == 0) {
        PixelOut<KH> o;
        phase8_out<KH>(sp, S, partf, o);
        if (active) {
            P.status[p] = o.status;
            P.brk[p] = o.brk;
            P.mean[p] = o.mean;
            P.sigma[p] = o.sigma;
            if (P.maxmo) P.maxmo[p] = o.maxmo;
#pragma unroll
            for (int i = 0; i < K; ++i) P.beta[(size_t)i * P.m + p] = o.beta[i];
        }
    }
}

__device__ __forceinline__ uint64_t* tile_bar(unsigned char* smem_raw, size_t smem_bytes) {
    return reinterpret_cast<uint64_t*>(smem_raw + smem_bytes - 16);
}

template <int KH, typename T, bool kTMA, bool kMask>
__global__ void __launch_bounds__(kNW * 32) simt_kernel(const __grid_constant__ CUtensorMap tmap, const MonitorParams P,
                                                       size_t smem_bytes) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint64_t* bar = tile_bar(smem_raw, smem_bytes);
    if (kTMA && threadIdx.x == 0) {
        ptx::prefetch_tmap(&tmap);
        ptx::mbar_init(bar, 1);
        ptx::fence_mbar_init();
    }
    __syncthreads();
    uint32_t uses = 0;
    simt_block<KH, T, kMask>(kTMA ? &tmap : nullptr, P, blockIdx.x, smem_raw, bar, uses);
}

// Persistent batched kernel: CTAs take 32-pixel blocks of any tile from a
// device counter (`grab` at a time) until all `total` blocks are done.
__global__ void __launch_bounds__(kNW * 32) batch_kernel(const BatchTileDesc* __restrict__ tiles,
                                                        const CUtensorMap* __restrict__ tmaps, int ntiles,
                                                        long long total, unsigned long long* counter, int grab,
                                                        size_t smem_bytes) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ long long s_item;
    uint64_t* bar = tile_bar(smem_raw, smem_bytes);
    if (threadIdx.x == 0) {
        ptx::mbar_init(bar, 1);
        ptx::fence_mbar_init();
    }
    __syncthreads();
    uint32_t uses = 0;
    for (;;) {
        if (threadIdx.x == 0) s_item = (long long)atomicAdd(counter, (unsigned long long)grab);
        __syncthreads();
        const long long it0 = s_item;
        __syncthreads();
        if (it0 >= total) break;
        const long long it1 = it0 + grab < total ? it0 + grab : total;
        for (long long it = it0; it < it1; ++it) {
            int lo = 0, hi = ntiles - 1;  // last tile whose first block is <= it
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (tiles[mid].block0 <= it)
                    lo = mid;
                else
                    hi = mid - 1;
            }
            const BatchTileDesc& T = tiles[lo];
            const MonitorParams P = T.P;
            const long long block = it - T.block0;
            const CUtensorMap* tm = T.has_tma ? tmaps + lo : nullptr;
            if (tm && threadIdx.x == 0) ptx::fence_tmap_acquire(tm);  // the TMA-issuing thread
            const int sel = (T.kh - 1) * 4 + (T.dtype == BFM_I16 ? 2 : 0) + (T.has_mask ? 1 : 0);
            switch (sel) {
                case 0: simt_block<1, float, false>(tm, P, block, smem_raw, bar, uses); break;
                case 1: simt_block<1, float, true>(tm, P, block, smem_raw, bar, uses); break;
                case 2: simt_block<1, int16_t, false>(tm, P, block, smem_raw, bar, uses); break;
                case 3: simt_block<1, int16_t, true>(tm, P, block, smem_raw, bar, uses); break;
                case 4: simt_block<2, float, false>(tm, P, block, smem_raw, bar, uses); break;
                case 5: simt_block<2, float, true>(tm, P, block, smem_raw, bar, uses); break;
                case 6: simt_block<2, int16_t, false>(tm, P, block, smem_raw, bar, uses); break;
                case 7: simt_block<2, int16_t, true>(tm, P, block, smem_raw, bar, uses); break;
                case 8: simt_block<3, float, false>(tm, P, block, smem_raw, bar, uses); break;
                case 9: simt_block<3, float, true>(tm, P, block, smem_raw, bar, uses); break;
                case 10: simt_block<3, int16_t, false>(tm, P, block, smem_raw, bar, uses); break;
                default: simt_block<3, int16_t, true>(tm, P, block, smem_raw, bar, uses); break;
            }
            __syncthreads();
        }
    }
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
    auto kern = P.mask ? simt_kernel<KH, T, kTMA, true> : simt_kernel<KH, T, kTMA, false>;
    static thread_local int configured_dev[2] = {-1, -1};
    int dev = 0;
    cudaGetDevice(&dev);
    if (configured_dev[P.mask ? 1 : 0] != dev) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(MaxDynamicSharedMemorySize)");
        cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        configured_dev[P.mask ? 1 : 0] = dev;
    }
    const unsigned grid = (unsigned)((P.m + 31) / 32);
    kern<<<grid, kNW * 32, smem, stream>>>(tm, P, smem);
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

size_t simt_smem_bytes(int N, int k, int dtype, int* box_rows, int* nbox) {
    const int elt = dtype == BFM_F32 ? 4 : 2;
    const int nb = (N + 255) / 256;
    int br = (N + nb - 1) / nb;
    // every TMA box must start on a 128-byte boundary of shared memory: with
    // 64-byte int16 rows the box height has to be even
    if ((br * 32 * elt) % 128 != 0) ++br;
    const int rows = nb * br;
    const size_t tile = ((size_t)rows * 32 * elt + 127) & ~(size_t)127;
    const size_t work = dtype == BFM_F32 ? 0 : (((size_t)N * 32 * 4 + 127) & ~(size_t)127);
    const int ps = k == 1 ? Partials<1>::kStride : k == 2 ? Partials<2>::kStride : Partials<3>::kStride;
    const size_t total = tile + work + (size_t)kNW * ps * 32 * 4 + 16;
    if (box_rows) *box_rows = br;
    if (nbox) *nbox = nb;
    if ((N + kNW - 1) / kNW > 32 * kSegWords) return 0;
    return total <= 227 * 1024 ? total : 0;
}

bfm_status launch_simt(const bfm_design_s* d, const void* Y, int dtype, const uint32_t* mask, int64_t m, int n_hist,
                       double h_frac, double lambda, int32_t* brk, float* mean, float* sigma, float* beta,
                       uint8_t* status, cudaStream_t stream, float* maxmo) {
    MonitorParams P{};
    int br = 0, nb = 0;
    size_t smem = simt_smem_bytes(d->N, d->k, dtype, &br, &nb);
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
    P.brk = brk;
    P.mean = mean;
    P.sigma = sigma;
    P.beta = beta;
    P.status = status;
    P.maxmo = maxmo;

    CUtensorMap tm;
    memset(&tm, 0, sizeof(tm));
    const bool tma = make_tensor_map(&tm, Y, dtype, m, d->N, br);
    switch (d->k) {
        case 1: return dispatch_dtype<1>(dtype, tma, tm, P, smem, stream);
        case 2: return dispatch_dtype<2>(dtype, tma, tm, P, smem, stream);
        default: return dispatch_dtype<3>(dtype, tma, tm, P, smem, stream);
    }
}

bool make_tensor_map(CUtensorMap* tm, const void* Y, int dtype, int64_t m, int N, int box_rows) {
    const int elt = dtype == BFM_F32 ? 4 : 2;
    if ((uintptr_t)Y % 16 != 0 || ((int64_t)m * elt) % 16 != 0 || m < 32) return false;
    auto enc = encode_fn();
    if (!enc) return false;
    cuuint64_t gdim[2] = {(cuuint64_t)m, (cuuint64_t)N};
    cuuint64_t gstride[1] = {(cuuint64_t)m * elt};
    cuuint32_t box[2] = {32u, (cuuint32_t)box_rows};
    cuuint32_t estride[2] = {1u, 1u};
    CUresult r = enc(tm, dtype == BFM_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_UINT16, 2,
                     const_cast<void*>(Y), gdim, gstride, box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

bfm_status batch_launch_kernel(const void* tiles, const void* tmaps, int ntiles, int64_t total_blocks,
                               unsigned long long* counter, int grab, int grid, size_t smem, cudaStream_t s,
                               cudaGraph_t graph, const cudaGraphNode_t* dep, cudaGraphNode_t* node_out) {
    static thread_local int configured = -1;
    int dev = 0;
    cudaGetDevice(&dev);
    if (configured != dev) {
        cudaFuncAttributes fa{};
        cudaFuncGetAttributes(&fa, batch_kernel);  // static shared memory counts against the 227 KB
        cudaError_t e = cudaFuncSetAttribute(batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             227 * 1024 - (int)fa.sharedSizeBytes);
        if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(batch_kernel)");
        cudaFuncSetAttribute(batch_kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        configured = dev;
    }
    const BatchTileDesc* t = static_cast<const BatchTileDesc*>(tiles);
    const CUtensorMap* tm = static_cast<const CUtensorMap*>(tmaps);
    long long total = (long long)total_blocks;
    if (graph) {
        void* args[] = {(void*)&t, (void*)&tm, (void*)&ntiles, (void*)&total, (void*)&counter, (void*)&grab,
                        (void*)&smem};
        cudaKernelNodeParams kp{};
        kp.func = (void*)batch_kernel;
        kp.gridDim = dim3((unsigned)grid);
        kp.blockDim = dim3(kNW * 32);
        kp.sharedMemBytes = (unsigned)smem;
        kp.kernelParams = args;
        cudaError_t e = cudaGraphAddKernelNode(node_out, graph, dep, dep ? 1 : 0, &kp);
        if (e != cudaSuccess) return cuda_fail(e, "bfm_batch: kernel node");
        return BFM_OK;
    }
    batch_kernel<<<grid, kNW * 32, smem, s>>>(t, tm, ntiles, total, counter, grab, smem);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "batch kernel launch");
    return BFM_OK;
}

}  // namespace bfm
