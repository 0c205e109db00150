// Helpers shared by the kernels that stream Y through shared-memory stages
// filled by 2-D TMA boxes (complete.cu, stream.cu): L2 cache policies, the
// box load, the consumer-side mbarrier arrive, the residuals of the fitted
// model, and the host's tensor-map encoder.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "ptx.cuh"

namespace bfm {
namespace stage {

// L2 eviction priorities for the loads of a pass: keep (the data is read
// again by a later pass), normal, drop (last use).
__device__ __forceinline__ uint64_t l2_evict_last() {
    uint64_t pol;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

__device__ __forceinline__ uint64_t l2_evict_normal() {
    uint64_t pol;
    asm("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

__device__ __forceinline__ uint64_t l2_evict_first() {
    uint64_t pol;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

// 2-D tiled TMA load of the box at (x = pixel, y = date) into shared memory,
// completing its bytes on `bar`, with an L2 policy.
__device__ __forceinline__ void tma_box(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y,
                                        uint64_t pol) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1, {%2, %3}], [%4], %5;" ::"r"(ptx::smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(ptx::smem_u32(bar)), "l"(pol)
        : "memory");
}

// One arrival on `bar` (release: the arriving thread's earlier reads of a
// stage are done before the producer may refill it).
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(ptx::smem_u32(bar)) : "memory");
}

// The producer's wait for every consumer warp to release a slot: bounded by
// limit_ns, and ended early by the CTA's abort flag (a consumer whose own wait
// gave up raises it and never releases its stage).  False when it gave up.
__device__ __forceinline__ bool wait_released(uint64_t* bar, uint32_t parity, volatile uint32_t* abort_flag,
                                              uint64_t limit_ns) {
    if (ptx::mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = ptx::globaltimer_ns();
    while (true) {
        if (ptx::mbar_try_wait_hint(bar, parity, 20000u)) return true;
        if (*abort_flag || ptx::globaltimer_ns() - t0 > limit_ns) return false;
    }
}

// y - x'beta (the residual of Eq. 3) with x a regressor row in shared memory.
template <int K>
__device__ __forceinline__ float residual(float y, const float* x, const float (&beta)[K]) {
    float yhat = 0.f;
#pragma unroll
    for (int a = 0; a < K; ++a) yhat = fmaf(x[a], beta[a], yhat);
    return y - yhat;
}

// The same with the intercept and trend coefficients held as hi (beta) + lo
// (lo0, lo1): a float rounding of those two would enter every residual of a
// MOSUM window with the same sign, h times over.
template <int K>
__device__ __forceinline__ float residual2(float y, const float* x, const float (&beta)[K], float lo0, float lo1) {
    return residual<K>(y, x, beta) - fmaf(x[1], lo1, lo0);
}

// cuTensorMapEncodeTiled from the driver (nullptr when it is not available).
inline PFN_cuTensorMapEncodeTiled_v12000 encode_tiled() {
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

}  // namespace stage
}  // namespace bfm
