// Measured cost of the per-pixel K x K solve of Eq. 6 in FP64 and in FP32
// (bfm_solve_rate): the figure behind the choice of an FP32 Cholesky with one
// refinement step over an FP64 solve on this GPU.
//
// One thread per system: a symmetric positive definite K x K matrix and a
// right-hand side made from the thread index (a Gram matrix of K + 4
// hash-generated rows plus K on the diagonal), its Cholesky factor, and the
// forward and backward substitutions -- the work a pixel does twice (beta0,
// then the refinement delta).  Nothing of it touches memory except one
// never-taken store that keeps the result alive.
#include <cuda_runtime.h>

#include <cstdint>

#include "bfm_internal.cuh"

namespace bfm {
namespace {

__device__ double g_solve_sink;

__device__ __forceinline__ uint32_t mix32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

template <typename F, int K>
__global__ void __launch_bounds__(256) solve_kernel(int64_t systems, int reps) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= systems) return;
    // the system is built in float whatever F is, so that only the solve differs
    float Af[K][K], bf[K];
    uint32_t h = mix32((uint32_t)i * 2654435761u + 1u);
#pragma unroll
    for (int r = 0; r < K; ++r) {
        bf[r] = (float)((h = mix32(h)) & 0xffff) * (1.f / 65536.f);
#pragma unroll
        for (int c = 0; c < K; ++c) Af[r][c] = r == c ? (float)K : 0.f;
    }
#pragma unroll
    for (int t = 0; t < K + 4; ++t) {
        float row[K];
#pragma unroll
        for (int c = 0; c < K; ++c) row[c] = (float)((h = mix32(h)) & 0xffff) * (1.f / 65536.f) - 0.5f;
#pragma unroll
        for (int r = 0; r < K; ++r)
#pragma unroll
            for (int c = 0; c < K; ++c) Af[r][c] = fmaf(row[r], row[c], Af[r][c]);
    }
    F A[K][K], b[K];
#pragma unroll
    for (int r = 0; r < K; ++r) {
        b[r] = (F)bf[r];
#pragma unroll
        for (int c = 0; c < K; ++c) A[r][c] = (F)Af[r][c];
    }
    F acc = 0;
    for (int rep = 0; rep < reps; ++rep) {
        F L[K][K], x[K], z[K];
#pragma unroll
        for (int j = 0; j < K; ++j) {
            F d = A[j][j] + (F)rep * (F)1e-9;
#pragma unroll
            for (int c = 0; c < j; ++c) d -= L[j][c] * L[j][c];
            const F inv = (F)1 / sqrt(d);
            L[j][j] = d * inv;
#pragma unroll
            for (int r = j + 1; r < K; ++r) {
                F s = A[r][j];
#pragma unroll
                for (int c = 0; c < j; ++c) s -= L[r][c] * L[j][c];
                L[r][j] = s * inv;
            }
        }
#pragma unroll
        for (int r = 0; r < K; ++r) {
            F s = b[r];
#pragma unroll
            for (int c = 0; c < r; ++c) s -= L[r][c] * z[c];
            z[r] = s / L[r][r];
        }
#pragma unroll
        for (int r = K - 1; r >= 0; --r) {
            F s = z[r];
#pragma unroll
            for (int c = r + 1; c < K; ++c) s -= L[c][r] * x[c];
            x[r] = s / L[r][r];
        }
        acc += x[0] + x[K - 1];
    }
    if (acc == (F)-12345.678) g_solve_sink = (double)acc;  // never taken; keeps the work
}

template <typename F>
cudaError_t launch_k(int K, int64_t systems, int reps, cudaStream_t s) {
    const int64_t blocks = (systems + 255) / 256;
    switch (K) {
        case 4: solve_kernel<F, 4><<<(unsigned)blocks, 256, 0, s>>>(systems, reps); break;
        case 6: solve_kernel<F, 6><<<(unsigned)blocks, 256, 0, s>>>(systems, reps); break;
        default: solve_kernel<F, 8><<<(unsigned)blocks, 256, 0, s>>>(systems, reps); break;
    }
    return cudaGetLastError();
}

}  // namespace
}  // namespace bfm

using namespace bfm;

extern "C" bfm_status bfm_solve_rate(int K, int64_t systems, int fp64, void* stream, float* ms_out) {
    if (!ms_out || systems <= 0 || systems > ((int64_t)1 << 31) || (K != 4 && K != 6 && K != 8)) {
        set_error("bfm_solve_rate: K must be 4, 6 or 8, systems in 1..2^31, ms_out non-NULL");
        return BFM_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t ev[4] = {};
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < 4 && e == cudaSuccess; ++i) e = cudaEventCreate(&ev[i]);
    auto run = [&](int reps) { return fp64 ? launch_k<double>(K, systems, reps, s) : launch_k<float>(K, systems, reps, s); };
    // warm-up; then the same launch without solves and with two solves per system (beta0
    // and the refinement delta of Eq. 6): the difference is the cost of the two solves
    if (e == cudaSuccess) e = run(2);
    if (e == cudaSuccess) e = cudaEventRecord(ev[0], s);
    if (e == cudaSuccess) e = run(0);
    if (e == cudaSuccess) e = cudaEventRecord(ev[1], s);
    if (e == cudaSuccess) e = cudaEventRecord(ev[2], s);
    if (e == cudaSuccess) e = run(2);
    if (e == cudaSuccess) e = cudaEventRecord(ev[3], s);
    if (e == cudaSuccess) e = cudaEventSynchronize(ev[3]);
    float t0 = 0.f, t2 = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t0, ev[0], ev[1]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t2, ev[2], ev[3]);
    *ms_out = t2 - t0;
    for (int i = 0; i < 4; ++i)
        if (ev[i]) cudaEventDestroy(ev[i]);
    if (e != cudaSuccess) return cuda_fail(e, "bfm_solve_rate");
    return BFM_OK;
}
