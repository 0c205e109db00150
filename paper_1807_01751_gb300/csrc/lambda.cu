// Critical value lambda(alpha, h, N/n) of the boundary (Eq. 4) by simulation.
//
// The paper obtains lambda "by simulation" of the limiting MOSUM process
// (Section 2.3; the one printed value, 2.39, is for alpha = 0.05, h/n = 0.5,
// N/n = 2 in Section 4.3).  Here every thread simulates one path: a Brownian
// motion W on a grid of G steps per unit time up to T = N/n, Gaussian
// increments of variance 1/G, and the statistic
//     sup_{t in [1, T]} |W(t) - W(t - h) - h W(1)| / sqrt(log+ t)
// over the grid points t = i/G, i = G..T*G.  lambda is the (1 - alpha)
// empirical quantile over the paths.
//
// Random numbers: per path a SplitMix64 stream (Steele, Lea and Flood, 2014)
// started from (seed, path), two 53-bit uniforms per normal, Box-Muller
// (sqrt(-2 ln u1) cos(2 pi u2), u1 in (0, 1]).  The stream advances by a
// fixed increment per draw, so the lagged value W(t - h) is rebuilt by a
// second cursor over the same stream instead of being stored.  FP64
// throughout (the work is small: one thread per path).
#include <algorithm>
#include <cmath>
#include <vector>

#include "bfm_internal.cuh"

namespace bfm {
namespace {

constexpr uint64_t kGolden = 0x9E3779B97F4A7C15ull;  // SplitMix64 increment

__device__ __forceinline__ uint64_t splitmix_next(uint64_t& state) {
    uint64_t z = (state += kGolden);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ double box_muller(uint64_t& state) {
    const double two_pow_m53 = 1.0 / 9007199254740992.0;
    const double u1 = ((double)(splitmix_next(state) >> 11) + 1.0) * two_pow_m53;
    const double u2 = (double)(splitmix_next(state) >> 11) * two_pow_m53;
    return sqrt(-2.0 * log(u1)) * cos(6.283185307179586476925286766559 * u2);
}

// log+(x): 1 for x <= e, log x above (Eq. 4)
__device__ __forceinline__ double log_plus(double x) {
    return x <= 2.718281828459045235360287 ? 1.0 : log(x);
}

__global__ void lambda_paths(double h, int G, int nsteps, int ih, int reps, uint64_t seed, double* stats) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= reps) return;
    // stream of path r (one discarded draw after seeding)
    uint64_t s0 = seed * 0xA0761D6478BD642Full + (uint64_t)r * 0xE7037ED1A0B428DBull + 1ull;
    splitmix_next(s0);
    const double sd = 1.0 / sqrt((double)G);
    uint64_t lead = s0, lag = s0;
    double W = 0.0, Wlag = 0.0;
    for (int i = 1; i <= G; ++i) W += sd * box_muller(lead);  // W(1)
    const double w1 = W;
    for (int j = 1; j <= G - ih; ++j) Wlag += sd * box_muller(lag);  // W(1 - h)
    double best = 0.0;
    for (int i = G;; ++i) {
        const double z = W - Wlag - h * w1;
        const double v = fabs(z) / sqrt(log_plus((double)i / (double)G));
        best = v > best ? v : best;
        if (i == nsteps) break;
        W += sd * box_muller(lead);
        Wlag += sd * box_muller(lag);
    }
    stats[r] = best;
}

}  // namespace
}  // namespace bfm

using namespace bfm;

extern "C" bfm_status bfm_lambda(double alpha, double h, double T, int G, int reps, uint64_t seed,
                                 double* lambda_out, double* stats_host, void* stream) {
    if (!(alpha > 0.0 && alpha < 1.0) || !(h > 0.0 && h <= 1.0) || !(T > 1.0) || G < 1 || reps < 1 ||
        !lambda_out) {
        set_error("bfm_lambda: needs 0 < alpha < 1, 0 < h <= 1, T > 1, G >= 1, reps >= 1 and lambda_out");
        return BFM_EINVAL;
    }
    const int nsteps = (int)std::llround(T * (double)G);
    const int ih = (int)std::llround(h * (double)G);
    if (ih < 1 || nsteps < G) {
        set_error("bfm_lambda: h * G rounds to 0 or T * G to fewer than G steps");
        return BFM_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    double* d_stats = nullptr;
    cudaError_t e = cudaMallocAsync(&d_stats, sizeof(double) * (size_t)reps, st);
    if (e != cudaSuccess) return cuda_fail(e, "bfm_lambda: cudaMallocAsync");
    const int block = 128;
    lambda_paths<<<(reps + block - 1) / block, block, 0, st>>>(h, G, nsteps, ih, reps, seed, d_stats);
    e = cudaGetLastError();
    std::vector<double> stats((size_t)reps);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(stats.data(), d_stats, sizeof(double) * (size_t)reps, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaFreeAsync(d_stats, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "bfm_lambda: simulation");
    if (stats_host) std::copy(stats.begin(), stats.end(), stats_host);
    // (1 - alpha) empirical quantile: the ceil((1 - alpha) reps)-th smallest
    long q = (long)std::ceil((1.0 - alpha) * (double)reps) - 1;
    q = q < 0 ? 0 : (q >= reps ? reps - 1 : q);
    std::nth_element(stats.begin(), stats.begin() + q, stats.end());
    *lambda_out = stats[(size_t)q];
    return BFM_OK;
}
