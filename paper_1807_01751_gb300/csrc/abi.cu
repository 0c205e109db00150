// C ABI of libbfm: argument checks, the design cache, dispatch to the
// kernels, and the host-buffer entry point (chunked copy/compute overlap).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <cuda_fp16.h>

#include "bfm_internal.cuh"

namespace bfm {

namespace {
thread_local std::string t_last_error;

std::mutex g_cache_mu;
std::vector<bfm_design_s*> g_cache;

constexpr int kMaxDates = 1792;

uint64_t fnv1a(const void* data, size_t n, uint64_t h = 1469598103934665603ull) {
    const unsigned char* b = static_cast<const unsigned char*>(data);
    for (size_t i = 0; i < n; ++i) {
        h ^= b[i];
        h *= 1099511628211ull;
    }
    return h;
}

// Per-date basis rows (layout of bfm::Basis) in double.
void basis_rows(const bfm_design_s& d, std::vector<double>& rows) {
    const int k = d.k, K = d.K, NB = d.NB;
    auto S = [&](int j) { return j <= k ? 2 + 2 * (j - 1) : K + 1 + 2 * (j - k - 1); };
    auto TS = [&](int j) { return K + 1 + 2 * k + 2 * (j - 1); };
    rows.assign((size_t)d.N * NB, 0.0);
    const double two_pi = 6.283185307179586476925286766559;
    for (int t = 0; t < d.N; ++t) {
        double* r = rows.data() + (size_t)t * NB;
        const double tp = (d.dates[t] - d.c) / d.s;
        r[0] = 1.0;
        r[1] = tp;
        r[K] = tp * tp;
        for (int j = 1; j <= 2 * k; ++j) {
            const double a = two_pi * (double)j * d.dates[t] / d.f;
            const double sj = std::sin(a), cj = std::cos(a);
            r[S(j)] = sj;
            r[S(j) + 1] = cj;
            if (j <= k) {
                r[TS(j)] = tp * sj;
                r[TS(j) + 1] = tp * cj;
            }
        }
    }
}

// Tensor-core B tables: the basis value (row r, date t) split as fp16 hi + lo.
// Table A holds rows 0..15 for all npad dates, table B rows 16..31 for the
// first nhpad dates; in both, (row r, date t) sits at byte
// (t/8)*256 + ((r%16)/8)*128 + (r%8)*16 + (t%8)*2.  Order: A_hi, A_lo, B_hi, B_lo.
void tc_tables(const bfm_design_s& d, const std::vector<double>& rows, int npad, int nhpad,
               std::vector<unsigned char>& out) {
    const size_t a_one = (size_t)(npad / 8) * 256, b_one = (size_t)(nhpad / 8) * 256;
    out.assign(2 * a_one + 2 * b_one, 0);
    const int nbr = 3 + 6 * d.k;
    for (int t = 0; t < d.N; ++t)
        for (int r = 0; r < nbr; ++r) {
            const bool in_a = r < 16;
            if (!in_a && t >= nhpad) continue;
            const double v = rows[(size_t)t * d.NB + r];
            const __half hi = __double2half(v);
            const __half lo = __double2half(v - (double)__half2float(hi));
            const int rr = r % 16;
            const size_t o = (size_t)(t / 8) * 256 + (size_t)(rr / 8) * 128 + (size_t)(rr % 8) * 16 + (size_t)(t % 8) * 2;
            unsigned char* base = in_a ? out.data() : out.data() + 2 * a_one;
            const size_t one = in_a ? a_one : b_one;
            std::memcpy(base + o, &hi, 2);
            std::memcpy(base + one + o, &lo, 2);
        }
}

bool valid_common(bfm_design_t d, int dtype, int64_t m, int n_hist, double h_frac, double lambda, const char* fn) {
    char buf[256];
    if (!d) {
        snprintf(buf, sizeof buf, "%s: design handle is NULL", fn);
        set_error(buf);
        return false;
    }
    if (dtype != BFM_F32 && dtype != BFM_I16) {
        snprintf(buf, sizeof buf, "%s: dtype %d is not BFM_F32 or BFM_I16", fn, dtype);
        set_error(buf);
        return false;
    }
    if (m < 0) {
        snprintf(buf, sizeof buf, "%s: m = %lld < 0", fn, (long long)m);
        set_error(buf);
        return false;
    }
    if (!(n_hist >= 1 && n_hist < d->N)) {
        snprintf(buf, sizeof buf, "%s: n_hist = %d outside 1 <= n_hist < N = %d", fn, n_hist, d->N);
        set_error(buf);
        return false;
    }
    if (!(h_frac > 0.0 && h_frac <= 1.0)) {
        snprintf(buf, sizeof buf, "%s: h_frac = %g outside (0, 1]", fn, h_frac);
        set_error(buf);
        return false;
    }
    if (!(lambda > 0.0) || !std::isfinite(lambda)) {
        snprintf(buf, sizeof buf, "%s: lambda = %g must be positive and finite", fn, lambda);
        set_error(buf);
        return false;
    }
    return true;
}

// Internal streams/events for bfm_monitor_host, one set per device.
struct HostPipe {
    int device = -1;
    cudaStream_t h2d = nullptr, d2h = nullptr;
    cudaEvent_t start = nullptr;
    cudaEvent_t h2d_done[2] = {}, comp_done[2] = {}, d2h_done[2] = {};
};
std::mutex g_pipe_mu;
std::vector<HostPipe*> g_pipes;

HostPipe* get_pipe(int dev, bfm_status* st) {
    for (auto* p : g_pipes)
        if (p->device == dev) return p;
    auto* p = new HostPipe;
    p->device = dev;
    cudaError_t e = cudaStreamCreateWithFlags(&p->h2d, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->d2h, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->start, cudaEventDisableTiming);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
        e = cudaEventCreateWithFlags(&p->h2d_done[i], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->comp_done[i], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->d2h_done[i], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        *st = cuda_fail(e, "bfm_monitor_host: creating internal streams");
        return nullptr;
    }
    g_pipes.push_back(p);
    return p;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct SlotLayout {
    size_t y, mask, brk, mean, sigma, beta, status, total;
};

SlotLayout slot_layout(int N, int K, int dtype, int64_t chunk, bool with_mask) {
    SlotLayout L{};
    const size_t elt = dtype == BFM_F32 ? 4 : 2;
    size_t o = 0;
    L.y = o;
    o = align256(o + (size_t)N * chunk * elt);
    L.mask = o;
    if (with_mask) o = align256(o + (size_t)N * ((chunk + 31) / 32) * 4);
    L.brk = o;
    o = align256(o + (size_t)chunk * 4);
    L.mean = o;
    o = align256(o + (size_t)chunk * 4);
    L.sigma = o;
    o = align256(o + (size_t)chunk * 4);
    L.beta = o;
    o = align256(o + (size_t)chunk * 4 * K);
    L.status = o;
    o = align256(o + (size_t)chunk);
    L.total = o;
    return L;
}

}  // namespace

void set_error(const std::string& msg) { t_last_error = msg; }

bfm_status cuda_fail(cudaError_t e, const char* what) {
    set_error(std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
    return e == cudaErrorMemoryAllocation ? BFM_ENOMEM : BFM_ECUDA;
}

int auto_form(const bfm_design_s* d, int dtype, int n_hist, double h_frac, const void* Y, int64_t m) {
    if (hybrid_supported(d, dtype, n_hist, h_frac, Y, m)) return BFM_ALGO_HYBRID;
    if (stream_supported(d, dtype, n_hist, h_frac, Y, m)) return BFM_ALGO_STREAM;
    if (mma_supported(d, dtype, n_hist, h_frac, Y, m, nullptr)) return BFM_ALGO_MMA;
    return BFM_ALGO_SIMT;
}

}  // namespace bfm

using namespace bfm;

extern "C" {

const char* bfm_version(void) { return "bfm 0.1.0 sm_103a"; }

const char* bfm_last_error(void) { return t_last_error.c_str(); }

int bfm_max_dates(void) { return kMaxDates; }

bfm_status bfm_design_create(const double* dates, int N, int k_harm, double f, bfm_design_t* out) {
    if (!out) {
        set_error("bfm_design_create: out is NULL");
        return BFM_EINVAL;
    }
    *out = nullptr;
    if (!dates) {
        set_error("bfm_design_create: dates is NULL");
        return BFM_EINVAL;
    }
    if (N < 2 || N > kMaxDates) {
        set_error("bfm_design_create: N = " + std::to_string(N) + " outside 2.." + std::to_string(kMaxDates));
        return N < 2 ? BFM_EINVAL : BFM_EUNSUPPORTED;
    }
    if (k_harm < 1 || k_harm > 3) {
        set_error("bfm_design_create: k = " + std::to_string(k_harm) + " outside 1..3");
        return BFM_EINVAL;
    }
    if (!(f > 0.0) || !std::isfinite(f)) {
        set_error("bfm_design_create: f must be positive and finite");
        return BFM_EINVAL;
    }
    for (int i = 0; i < N; ++i) {
        if (!std::isfinite(dates[i]) || (i > 0 && !(dates[i] > dates[i - 1]))) {
            set_error("bfm_design_create: dates must be finite and strictly increasing (index " + std::to_string(i) +
                      ")");
            return BFM_EINVAL;
        }
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "bfm_design_create: cudaGetDevice");
    uint64_t key = fnv1a(dates, sizeof(double) * (size_t)N);
    key = fnv1a(&k_harm, sizeof k_harm, key);
    key = fnv1a(&f, sizeof f, key);
    key = fnv1a(&dev, sizeof dev, key);
    std::lock_guard<std::mutex> lk(g_cache_mu);
    for (auto* d : g_cache) {
        if (d->key == key && d->N == N && d->k == k_harm && d->f == f && d->device == dev &&
            std::memcmp(d->dates.data(), dates, sizeof(double) * (size_t)N) == 0) {
            ++d->refcount;
            *out = d;
            return BFM_OK;
        }
    }
    auto* d = new bfm_design_s;
    d->N = N;
    d->k = k_harm;
    d->K = 2 + 2 * k_harm;
    d->f = f;
    d->dates.assign(dates, dates + N);
    d->c = 0.5 * (dates[0] + dates[N - 1]);
    d->s = 0.5 * (dates[N - 1] - dates[0]);
    if (!(d->s > 0.0)) d->s = 1.0;
    d->NB = basis_stride(k_harm);
    d->device = dev;
    d->key = key;
    d->refcount = 1;
    std::vector<double> rowsd;
    basis_rows(*d, rowsd);
    std::vector<float> rows(rowsd.begin(), rowsd.end());
    e = cudaMalloc(&d->d_basis, rows.size() * sizeof(float));
    if (e != cudaSuccess) {
        delete d;
        return cuda_fail(e, "bfm_design_create: cudaMalloc");
    }
    e = cudaMemcpy(d->d_basis, rows.data(), rows.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        const int npad = (N + 31) / 32 * 32;  // whole 32-date chunks
        std::vector<unsigned char> tab;
        tc_tables(*d, rowsd, npad, npad, tab);  // table B covers every possible history length
        e = cudaMalloc(&d->d_phi_tc, tab.size());
        if (e == cudaSuccess) e = cudaMemcpy(d->d_phi_tc, tab.data(), tab.size(), cudaMemcpyHostToDevice);
        d->npad_tc = npad;
    }
    if (e == cudaSuccess) {
        std::vector<unsigned char> tab;
        hybrid_tables(*d, rowsd, tab);
        e = cudaMalloc(&d->d_hyb, tab.size());
        if (e == cudaSuccess) e = cudaMemcpy(d->d_hyb, tab.data(), tab.size(), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) {
        e = cudaMalloc(&d->d_dates, sizeof(double) * (size_t)N);
        if (e == cudaSuccess) e = cudaMemcpy(d->d_dates, dates, sizeof(double) * (size_t)N, cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        cudaFree(d->d_basis);
        if (d->d_phi_tc) cudaFree(d->d_phi_tc);
        if (d->d_hyb) cudaFree(d->d_hyb);
        if (d->d_dates) cudaFree(d->d_dates);
        delete d;
        return cuda_fail(e, "bfm_design_create: device tables");
    }
    g_cache.push_back(d);
    *out = d;
    return BFM_OK;
}

bfm_status bfm_design_destroy(bfm_design_t d) {
    if (!d) {
        set_error("bfm_design_destroy: NULL handle");
        return BFM_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g_cache_mu);
    for (size_t i = 0; i < g_cache.size(); ++i) {
        if (g_cache[i] == d) {
            if (--d->refcount == 0) {
                g_cache.erase(g_cache.begin() + (long)i);
                int cur = 0;
                cudaGetDevice(&cur);
                if (cur != d->device) cudaSetDevice(d->device);
                cudaFree(d->d_basis);
                if (d->d_phi_tc) cudaFree(d->d_phi_tc);
                if (d->d_hyb) cudaFree(d->d_hyb);
                if (d->d_dates) cudaFree(d->d_dates);
                for (auto& c : d->complete) cudaFree(c.d_tab);
                if (cur != d->device) cudaSetDevice(cur);
                delete d;
            }
            return BFM_OK;
        }
    }
    set_error("bfm_design_destroy: unknown handle");
    return BFM_EINVAL;
}

int bfm_design_K(bfm_design_t d) { return d ? d->K : 0; }

int bfm_design_N(bfm_design_t d) { return d ? d->N : 0; }

int bfm_algo_auto(bfm_design_t d, int dtype, int n_hist, double h_frac, const void* Y, int64_t m) {
    if (!d || (dtype != BFM_F32 && dtype != BFM_I16) || !(n_hist >= 1 && n_hist < d->N)) return BFM_ALGO_SIMT;
    return auto_form(d, dtype, n_hist, h_frac, Y, m);
}

bfm_status bfm_monitor_ext(bfm_design_t d, const void* Y, int dtype, const uint32_t* mask_bits, int64_t m,
                           int n_hist, double h_frac, double lambda, int32_t* break_idx, float* mean_mosum,
                           float* sigma, float* beta, uint8_t* status, float* max_mosum, int algo, void* stream) {
    if (!valid_common(d, dtype, m, n_hist, h_frac, lambda, "bfm_monitor")) return BFM_EINVAL;
    if (m == 0) return BFM_OK;
    if (!Y || !break_idx || !mean_mosum || !sigma || !beta || !status) {
        set_error("bfm_monitor: Y and all five outputs must be non-NULL device pointers");
        return BFM_EINVAL;
    }
    if (m > ((int64_t)1 << 31) - 64) {
        set_error("bfm_monitor: m too large for one call (split the pixel range)");
        return BFM_EUNSUPPORTED;
    }
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != d->device) {
        set_error("bfm_monitor: the design belongs to another device");
        return BFM_EINVAL;
    }
    if (algo != BFM_ALGO_AUTO && algo != BFM_ALGO_SIMT && algo != BFM_ALGO_MMA && algo != BFM_ALGO_COMPLETE &&
        algo != BFM_ALGO_STREAM && algo != BFM_ALGO_HYBRID) {
        set_error("bfm_monitor: unknown algo");
        return BFM_EINVAL;
    }
    if (algo == BFM_ALGO_HYBRID)
        return launch_hybrid(d, dtype, Y, mask_bits, m, n_hist, h_frac, lambda, break_idx, mean_mosum, sigma, beta,
                             status, (cudaStream_t)stream, max_mosum);
    if (algo == BFM_ALGO_STREAM)
        return launch_stream(d, dtype, Y, mask_bits, m, n_hist, h_frac, lambda, break_idx, mean_mosum, sigma, beta,
                             status, (cudaStream_t)stream, max_mosum);
    if (algo == BFM_ALGO_COMPLETE)
        return launch_complete(d, dtype, Y, mask_bits, m, n_hist, h_frac, lambda, break_idx, mean_mosum, sigma, beta,
                               status, (cudaStream_t)stream, max_mosum);
    const bool mma_ok = mma_supported(d, dtype, n_hist, h_frac, Y, m, nullptr);
    if (algo == BFM_ALGO_MMA && !mma_ok) {
        set_error("bfm_monitor: the tensor-core form needs basis tables and a MOSUM ring (bandwidth + 17 prefix sums per pixel) that fits shared memory, and Y with a 16-byte aligned base, m >= 128 and rows of a multiple of 16 bytes");
        return BFM_EUNSUPPORTED;
    }
    if (algo == BFM_ALGO_AUTO && hybrid_supported(d, dtype, n_hist, h_frac, Y, m))
        return launch_hybrid(d, dtype, Y, mask_bits, m, n_hist, h_frac, lambda, break_idx, mean_mosum, sigma, beta,
                             status, (cudaStream_t)stream, max_mosum);
    if (algo == BFM_ALGO_AUTO && stream_supported(d, dtype, n_hist, h_frac, Y, m))
        return launch_stream(d, dtype, Y, mask_bits, m, n_hist, h_frac, lambda, break_idx, mean_mosum, sigma, beta,
                             status, (cudaStream_t)stream, max_mosum);
    if (algo == BFM_ALGO_MMA || (algo == BFM_ALGO_AUTO && mma_ok))
        return launch_mma(d, dtype, Y, mask_bits, m, n_hist, h_frac, lambda, break_idx, mean_mosum, sigma, beta, status,
                          (cudaStream_t)stream, max_mosum);
    return launch_simt(d, Y, dtype, mask_bits, m, n_hist, h_frac, lambda, break_idx, mean_mosum, sigma, beta, status,
                       (cudaStream_t)stream, max_mosum);
}

bfm_status bfm_monitor_ex(bfm_design_t d, const void* Y, int dtype, const uint32_t* mask_bits, int64_t m, int n_hist,
                          double h_frac, double lambda, int32_t* break_idx, float* mean_mosum, float* sigma,
                          float* beta, uint8_t* status, int algo, void* stream) {
    return bfm_monitor_ext(d, Y, dtype, mask_bits, m, n_hist, h_frac, lambda, break_idx, mean_mosum, sigma, beta,
                           status, nullptr, algo, stream);
}

bfm_status bfm_monitor(bfm_design_t d, const void* Y, int dtype, const uint32_t* mask_bits, int64_t m, int n_hist,
                       double h_frac, double lambda, int32_t* break_idx, float* mean_mosum, float* sigma, float* beta,
                       uint8_t* status, void* stream) {
    return bfm_monitor_ex(d, Y, dtype, mask_bits, m, n_hist, h_frac, lambda, break_idx, mean_mosum, sigma, beta,
                          status, BFM_ALGO_AUTO, stream);
}

size_t bfm_monitor_host_workspace(bfm_design_t d, int dtype, int64_t chunk_px, int with_mask) {
    if (!d || chunk_px <= 0 || (dtype != BFM_F32 && dtype != BFM_I16)) return 0;
    int64_t chunk = (chunk_px + 31) / 32 * 32;
    return 2 * slot_layout(d->N, d->K, dtype, chunk, with_mask != 0).total;
}

bfm_status bfm_monitor_host(bfm_design_t d, const void* Y_host, int dtype, const uint32_t* mask_host, int64_t m,
                            int n_hist, double h_frac, double lambda, int32_t* break_idx, float* mean_mosum,
                            float* sigma, float* beta, uint8_t* status, void* workspace, size_t workspace_bytes,
                            int64_t chunk_px, void* stream) {
    if (!valid_common(d, dtype, m, n_hist, h_frac, lambda, "bfm_monitor_host")) return BFM_EINVAL;
    if (m == 0) return BFM_OK;
    if (!Y_host || !break_idx || !mean_mosum || !sigma || !beta || !status || !workspace || chunk_px <= 0) {
        set_error("bfm_monitor_host: NULL buffer or chunk_px <= 0");
        return BFM_EINVAL;
    }
    const int64_t chunk = (chunk_px + 31) / 32 * 32;
    const bool with_mask = mask_host != nullptr;
    const SlotLayout L = slot_layout(d->N, d->K, dtype, chunk, with_mask);
    if (workspace_bytes < 2 * L.total || ((uintptr_t)workspace & 255) != 0) {
        set_error("bfm_monitor_host: workspace smaller than bfm_monitor_host_workspace() or not 256-byte aligned");
        return BFM_EINVAL;
    }
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != d->device) {
        set_error("bfm_monitor_host: the design belongs to another device");
        return BFM_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g_pipe_mu);
    bfm_status st = BFM_OK;
    HostPipe* hp = get_pipe(dev, &st);
    if (!hp) return st;
    cudaStream_t cs = (cudaStream_t)stream;
    const size_t elt = dtype == BFM_F32 ? 4 : 2;
    const int N = d->N, K = d->K;
    const int64_t words = (m + 31) / 32;
    unsigned char* ws = static_cast<unsigned char*>(workspace);
    cudaError_t e;
#define BFM_CK(x, what)                                  \
    do {                                                 \
        e = (x);                                         \
        if (e != cudaSuccess) return cuda_fail(e, what); \
    } while (0)
    // earlier work on the caller's stream may still use the workspace
    BFM_CK(cudaEventRecord(hp->start, cs), "bfm_monitor_host: event");
    BFM_CK(cudaStreamWaitEvent(hp->h2d, hp->start, 0), "bfm_monitor_host: wait");
    BFM_CK(cudaStreamWaitEvent(hp->d2h, hp->start, 0), "bfm_monitor_host: wait");
    const int64_t nchunks = (m + chunk - 1) / chunk;
    for (int64_t ci = 0; ci < nchunks; ++ci) {
        const int s = (int)(ci & 1);
        unsigned char* base = ws + (size_t)s * L.total;
        const int64_t c0 = ci * chunk;
        const int64_t mc = (m - c0 < chunk) ? (m - c0) : chunk;
        if (ci >= 2) BFM_CK(cudaStreamWaitEvent(hp->h2d, hp->d2h_done[s], 0), "bfm_monitor_host: wait");
        BFM_CK(cudaMemcpy2DAsync(base + L.y, (size_t)mc * elt, static_cast<const unsigned char*>(Y_host) + c0 * elt,
                                 (size_t)m * elt, (size_t)mc * elt, (size_t)N, cudaMemcpyHostToDevice, hp->h2d),
               "bfm_monitor_host: H2D Y");
        if (with_mask) {
            const int64_t wc = (mc + 31) / 32;
            BFM_CK(cudaMemcpy2DAsync(base + L.mask, (size_t)wc * 4, mask_host + c0 / 32, (size_t)words * 4,
                                     (size_t)wc * 4, (size_t)N, cudaMemcpyHostToDevice, hp->h2d),
                   "bfm_monitor_host: H2D mask");
        }
        BFM_CK(cudaEventRecord(hp->h2d_done[s], hp->h2d), "bfm_monitor_host: event");
        BFM_CK(cudaStreamWaitEvent(cs, hp->h2d_done[s], 0), "bfm_monitor_host: wait");
        {
            // the form BFM_ALGO_AUTO picks for these parameters
            const uint32_t* mk = with_mask ? reinterpret_cast<const uint32_t*>(base + L.mask) : nullptr;
            int32_t* ob = reinterpret_cast<int32_t*>(base + L.brk);
            float* om = reinterpret_cast<float*>(base + L.mean);
            float* os = reinterpret_cast<float*>(base + L.sigma);
            float* obeta = reinterpret_cast<float*>(base + L.beta);
            uint8_t* ost = reinterpret_cast<uint8_t*>(base + L.status);
            const int form = auto_form(d, dtype, n_hist, h_frac, base + L.y, mc);
            st = form == BFM_ALGO_HYBRID
                     ? launch_hybrid(d, dtype, base + L.y, mk, mc, n_hist, h_frac, lambda, ob, om, os, obeta, ost, cs,
                                     nullptr)
                 : form == BFM_ALGO_STREAM
                     ? launch_stream(d, dtype, base + L.y, mk, mc, n_hist, h_frac, lambda, ob, om, os, obeta, ost, cs,
                                     nullptr)
                 : form == BFM_ALGO_MMA
                     ? launch_mma(d, dtype, base + L.y, mk, mc, n_hist, h_frac, lambda, ob, om, os, obeta, ost, cs)
                     : launch_simt(d, base + L.y, dtype, mk, mc, n_hist, h_frac, lambda, ob, om, os, obeta, ost, cs);
        }
        if (st != BFM_OK) return st;
        BFM_CK(cudaEventRecord(hp->comp_done[s], cs), "bfm_monitor_host: event");
        BFM_CK(cudaStreamWaitEvent(hp->d2h, hp->comp_done[s], 0), "bfm_monitor_host: wait");
        BFM_CK(cudaMemcpyAsync(break_idx + c0, base + L.brk, (size_t)mc * 4, cudaMemcpyDeviceToHost, hp->d2h),
               "bfm_monitor_host: D2H");
        BFM_CK(cudaMemcpyAsync(mean_mosum + c0, base + L.mean, (size_t)mc * 4, cudaMemcpyDeviceToHost, hp->d2h),
               "bfm_monitor_host: D2H");
        BFM_CK(cudaMemcpyAsync(sigma + c0, base + L.sigma, (size_t)mc * 4, cudaMemcpyDeviceToHost, hp->d2h),
               "bfm_monitor_host: D2H");
        BFM_CK(cudaMemcpyAsync(status + c0, base + L.status, (size_t)mc, cudaMemcpyDeviceToHost, hp->d2h),
               "bfm_monitor_host: D2H");
        BFM_CK(cudaMemcpy2DAsync(beta + c0, (size_t)m * 4, base + L.beta, (size_t)mc * 4, (size_t)mc * 4, (size_t)K,
                                 cudaMemcpyDeviceToHost, hp->d2h),
               "bfm_monitor_host: D2H beta");
        BFM_CK(cudaEventRecord(hp->d2h_done[s], hp->d2h), "bfm_monitor_host: event");
    }
    // the caller's stream completes after the last copies out
    for (int64_t ci = (nchunks > 2 ? nchunks - 2 : 0); ci < nchunks; ++ci)
        BFM_CK(cudaStreamWaitEvent(cs, hp->d2h_done[ci & 1], 0), "bfm_monitor_host: wait");
#undef BFM_CK
    return BFM_OK;
}

bfm_status bfm_stage_wait_limit(uint64_t consumer_wait_ns) {
    set_stage_wait_ns(consumer_wait_ns);
    return BFM_OK;
}

bfm_status bfm_device_errors(void* stream, uint32_t* bits) {
    if (!bits) {
        set_error("bfm_device_errors: bits is NULL");
        return BFM_EINVAL;
    }
    unsigned int v = 0, v2 = 0, v3 = 0, v4 = 0, v5 = 0;
    cudaError_t e = simt_read_clear_errors((cudaStream_t)stream, &v);
    if (e == cudaSuccess) e = mma_read_clear_errors((cudaStream_t)stream, &v2);
    if (e == cudaSuccess) e = complete_read_clear_errors((cudaStream_t)stream, &v3);
    if (e == cudaSuccess) e = stream_read_clear_errors((cudaStream_t)stream, &v4);
    if (e == cudaSuccess) e = hybrid_read_clear_errors((cudaStream_t)stream, &v5);
    if (e != cudaSuccess) return cuda_fail(e, "bfm_device_errors");
    v |= v2 | v3 | v4 | v5;
    *bits = v;
    return BFM_OK;
}

}  // extern "C"
