// Serving loop: continuous admission of scene tiles under an HBM budget.
//
// A server owns one device arena of `budget` bytes (a single cudaMalloc at
// creation) and `slots` CUDA streams.  Requests enter a FIFO; a scheduler
// thread admits the oldest request as soon as a slot is idle and the arena
// has room for its buffers (input copy if the tile is on the host, and the
// five outputs), enqueues on the slot's stream the host->device copy and the
// per-pixel path, and a host callback that stamps completion.  Requests in
// different slots run concurrently on the GPU; a request that arrives while
// others run is admitted the moment a slot and memory free up.  Results stay
// in the arena (device-resident) until the client releases them.  Designs are
// shared through the library's design cache (one per date set).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <memory>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "bfm_internal.cuh"

namespace bfm {

namespace {

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

int64_t now_ns() {
    using namespace std::chrono;
    return duration_cast<nanoseconds>(steady_clock::now().time_since_epoch()).count();
}

// First-fit allocator over [0, size) with 256-byte granules.
class Arena {
  public:
    void reset(size_t size) {
        size_ = size;
        free_.clear();
        free_[0] = size;
    }
    bool alloc(size_t bytes, size_t* off) {
        bytes = (bytes + 255) & ~(size_t)255;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes, noff = it->first + bytes;
                free_.erase(it);
                if (rest) free_[noff] = rest;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        bytes = (bytes + 255) & ~(size_t)255;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t size() const { return size_; }

  private:
    size_t size_ = 0;
    std::map<size_t, size_t> free_;
};

enum { ST_PENDING = 0, ST_RUNNING = 1, ST_DONE = 2, ST_FAILED = 3, ST_CANCELLED = 4 };

struct Req {
    uint64_t ticket = 0;
    bfm_serve_request r{};
    int K = 0;
    size_t bytes = 0, off = 0;
    bool has_mem = false;
    bool accounted = false;             // completion counted in the statistics
    std::atomic<int> state{ST_PENDING};  // DONE is stored by the completion callback
    int slot = -1;
    double t_arrive = 0, t_start = 0;
    std::atomic<int64_t> t_done_ns{0};
    bfm_status err = BFM_OK;
    // device buffers inside the arena
    void* y = nullptr;
    int32_t* brk = nullptr;
    float* mean = nullptr;
    float* sigma = nullptr;
    float* beta = nullptr;
    uint8_t* status = nullptr;
    struct bfm_server_s* srv = nullptr;
};

}  // namespace
}  // namespace bfm

struct bfm_server_s {
    int device = -1;
    unsigned char* arena = nullptr;
    bfm::Arena alloc;
    std::vector<cudaStream_t> streams;
    std::unique_ptr<std::atomic<int>[]> slot_busy;  // cleared by the completion callback
    int nslots = 0;
    std::thread worker;
    std::mutex mu;
    std::condition_variable cv, done_cv;
    bool stop = false;
    std::deque<bfm::Req*> pending;
    std::vector<bfm::Req*> running;
    std::map<uint64_t, bfm::Req*> reqs;
    uint64_t next_ticket = 1;
    std::vector<double> latencies;
    int64_t completed = 0, pixels = 0;
    double first_arrive = -1, last_done = 0;
};

namespace bfm {
namespace {

size_t req_bytes(const bfm_serve_request& r, int K) {
    const size_t elt = r.dtype == BFM_F32 ? 4 : 2;
    auto a = [](size_t x) { return (x + 255) & ~(size_t)255; };
    size_t b = a((size_t)r.m * (4 + 4 + 4 + 1)) + a((size_t)r.m * 4 * K) + 1024;
    if (r.y_on_host) b += a((size_t)bfm_design_N(r.design) * r.m * elt);
    return b;
}

// Host callback at the end of a request's stream work.  It runs on a driver
// thread and must neither call CUDA nor block: it only publishes atomics and
// wakes the scheduler; the bookkeeping happens in the scheduler thread.
void CUDART_CB on_done(void* p) {
    Req* q = static_cast<Req*>(p);
    bfm_server_s* s = q->srv;
    const int slot = q->slot;
    q->t_done_ns.store(now_ns());
    s->slot_busy[slot].store(0);
    q->state.store(ST_DONE);  // last access to q: a client may release it from now on
    s->cv.notify_all();
    s->done_cv.notify_all();
}

double done_ms(const Req* q) { return (double)q->t_done_ns.load() * 1e-6; }

// With the lock held: move finished requests out of `running` into the statistics.
void account(bfm_server_s* s) {
    for (size_t i = 0; i < s->running.size();) {
        Req* q = s->running[i];
        const int st = q->state.load();
        if (st == ST_DONE || st == ST_FAILED) {
            if (st == ST_DONE && !q->accounted) {
                const double td = done_ms(q);
                s->latencies.push_back(td - q->t_arrive);
                s->completed += 1;
                s->pixels += q->r.m;
                s->last_done = std::max(s->last_done, td);
            }
            q->accounted = true;
            s->running[i] = s->running.back();
            s->running.pop_back();
        } else {
            ++i;
        }
    }
}

// Called WITHOUT the lock (CUDA calls only): enqueues the admitted request on
// its slot's stream.  The request cannot be released while RUNNING.
void start(bfm_server_s* s, Req* q, int slot) {
    const bfm_serve_request& r = q->r;
    unsigned char* base = s->arena + q->off;
    auto a = [](size_t x) { return (x + 255) & ~(size_t)255; };
    size_t o = 0;
    q->brk = reinterpret_cast<int32_t*>(base + o);
    o += a((size_t)r.m * 4);
    q->mean = reinterpret_cast<float*>(base + o);
    o += a((size_t)r.m * 4);
    q->sigma = reinterpret_cast<float*>(base + o);
    o += a((size_t)r.m * 4);
    q->status = reinterpret_cast<uint8_t*>(base + o);
    o += a((size_t)r.m);
    q->beta = reinterpret_cast<float*>(base + o);
    o += a((size_t)r.m * 4 * q->K);
    const void* Y = r.Y;
    cudaStream_t st = s->streams[slot];
    cudaError_t e = cudaSuccess;
    if (r.y_on_host) {
        const size_t elt = r.dtype == BFM_F32 ? 4 : 2;
        q->y = base + o;
        e = cudaMemcpyAsync(q->y, r.Y, (size_t)bfm_design_N(r.design) * r.m * elt, cudaMemcpyHostToDevice, st);
        Y = q->y;
    }
    bfm_status bs = BFM_OK;
    if (e != cudaSuccess) {
        bs = cuda_fail(e, "serve: H2D");
    } else if (r.m > 0) {
        int algo = r.algo;
        if (algo == BFM_ALGO_AUTO) {
            algo = auto_form(r.design, r.dtype, r.n_hist, r.h_frac, Y, r.m);
        } else if (algo == BFM_ALGO_MMA) {
            const bool ok = mma_supported(r.design, r.dtype, r.n_hist, r.h_frac, Y, r.m, nullptr);
            algo = ok ? BFM_ALGO_MMA : BFM_ALGO_SIMT;
        }
        bs = algo == BFM_ALGO_HYBRID
                 ? launch_hybrid(r.design, r.dtype, Y, r.mask_bits, r.m, r.n_hist, r.h_frac, r.lambda, q->brk, q->mean,
                                 q->sigma, q->beta, q->status, st, nullptr)
             : algo == BFM_ALGO_STREAM
                 ? launch_stream(r.design, r.dtype, Y, r.mask_bits, r.m, r.n_hist, r.h_frac, r.lambda, q->brk, q->mean,
                                 q->sigma, q->beta, q->status, st, nullptr)
             : algo == BFM_ALGO_COMPLETE
                 ? launch_complete(r.design, r.dtype, Y, r.mask_bits, r.m, r.n_hist, r.h_frac, r.lambda, q->brk,
                                   q->mean, q->sigma, q->beta, q->status, st, nullptr)
             : algo == BFM_ALGO_MMA
                 ? launch_mma(r.design, r.dtype, Y, r.mask_bits, r.m, r.n_hist, r.h_frac, r.lambda, q->brk, q->mean, q->sigma,
                              q->beta, q->status, st)
                 : launch_simt(r.design, Y, r.dtype, r.mask_bits, r.m, r.n_hist, r.h_frac, r.lambda, q->brk, q->mean,
                               q->sigma, q->beta, q->status, st);
    }
    if (bs == BFM_OK) e = cudaLaunchHostFunc(st, on_done, q);
    if (bs != BFM_OK || e != cudaSuccess) {
        q->err = bs != BFM_OK ? bs : BFM_ECUDA;
        q->state.store(ST_FAILED);
        s->slot_busy[slot].store(0);
    }
}

void worker_loop(bfm_server_s* s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (!s->stop) {
        account(s);
        // admit in arrival order while a slot is idle and memory allows
        std::vector<std::pair<Req*, int>> to_start;
        while (!s->pending.empty()) {
            Req* q = s->pending.front();
            if (q->state.load() == ST_CANCELLED) {
                s->pending.pop_front();
                continue;
            }
            int slot = -1;
            for (int i = 0; i < s->nslots; ++i)
                if (s->slot_busy[i].load() == 0) {
                    slot = i;
                    break;
                }
            if (slot < 0) break;
            size_t off = 0;
            if (!s->alloc.alloc(q->bytes, &off)) break;  // FIFO: wait for memory
            q->off = off;
            q->has_mem = true;
            q->slot = slot;
            q->t_start = now_ms();
            q->state.store(ST_RUNNING);
            s->slot_busy[slot].store(1);
            s->pending.pop_front();
            s->running.push_back(q);
            to_start.emplace_back(q, slot);
        }
        if (!to_start.empty()) {
            lk.unlock();  // no CUDA call is made while the lock is held
            for (auto& qs : to_start) start(s, qs.first, qs.second);
            lk.lock();
            continue;
        }
        s->cv.wait_for(lk, std::chrono::milliseconds(2));
    }
}

}  // namespace
}  // namespace bfm

using namespace bfm;

extern "C" {

bfm_status bfm_serve_create(size_t hbm_budget, int slots, bfm_server_t* out) {
    if (!out || hbm_budget < 4096 || slots < 1 || slots > 64) {
        set_error("bfm_serve_create: out NULL, budget below 4 KB or slots outside 1..64");
        return BFM_EINVAL;
    }
    *out = nullptr;
    auto* s = new bfm_server_s;
    cudaGetDevice(&s->device);
    cudaError_t e = cudaMalloc(&s->arena, hbm_budget);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete s;
        set_error("bfm_serve_create: cannot reserve the HBM budget (" + std::to_string(hbm_budget) +
                  " bytes): " + cudaGetErrorString(e));
        return BFM_ENOMEM;
    }
    s->alloc.reset(hbm_budget);
    s->streams.resize(slots);
    s->nslots = slots;
    s->slot_busy.reset(new std::atomic<int>[slots]);
    for (int i = 0; i < slots; ++i) s->slot_busy[i].store(0);
    for (auto& st : s->streams) cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    s->worker = std::thread(worker_loop, s);
    *out = s;
    return BFM_OK;
}

bfm_status bfm_serve_submit(bfm_server_t s, const bfm_serve_request* r, uint64_t* ticket) {
    if (!s || !r || !r->design || !ticket) {
        set_error("bfm_serve_submit: NULL server, request, design or ticket");
        return BFM_EINVAL;
    }
    const bfm_design_s* d = r->design;
    if ((r->dtype != BFM_F32 && r->dtype != BFM_I16) || r->m < 0 || !(r->n_hist >= 1 && r->n_hist < d->N) ||
        !(r->h_frac > 0.0 && r->h_frac <= 1.0) || !(r->lambda > 0.0) || (r->m > 0 && !r->Y) ||
        !(r->algo >= BFM_ALGO_AUTO && r->algo <= BFM_ALGO_HYBRID)) {
        set_error("bfm_serve_submit: bad dtype, m, n_hist, h_frac, lambda, algo or NULL Y");
        return BFM_EINVAL;
    }
    auto* q = new Req;
    q->r = *r;
    q->K = d->K;
    q->bytes = req_bytes(*r, d->K);
    q->srv = s;
    std::lock_guard<std::mutex> lk(s->mu);
    if (q->bytes > s->alloc.size()) {
        delete q;
        set_error("bfm_serve_submit: the request needs more device memory than the whole budget");
        return BFM_EBUSY;
    }
    q->ticket = s->next_ticket++;
    q->t_arrive = now_ms();
    if (s->first_arrive < 0) s->first_arrive = q->t_arrive;
    s->reqs[q->ticket] = q;
    s->pending.push_back(q);
    *ticket = q->ticket;
    s->cv.notify_all();
    return BFM_OK;
}

bfm_status bfm_serve_poll(bfm_server_t s, uint64_t ticket, int* state, double* latency_ms) {
    if (!s || !state) {
        set_error("bfm_serve_poll: NULL server or state");
        return BFM_EINVAL;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) {
        set_error("bfm_serve_poll: unknown ticket");
        return BFM_EINVAL;
    }
    const int st = it->second->state.load();
    *state = st;
    if (latency_ms) *latency_ms = st == ST_DONE ? done_ms(it->second) - it->second->t_arrive : -1.0;
    return st == ST_FAILED ? it->second->err : BFM_OK;
}

bfm_status bfm_serve_result(bfm_server_t s, uint64_t ticket, int32_t** break_idx, float** mean_mosum, float** sigma,
                            float** beta, uint8_t** status) {
    if (!s) {
        set_error("bfm_serve_result: NULL server");
        return BFM_EINVAL;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end() || it->second->state.load() != ST_DONE) {
        set_error("bfm_serve_result: unknown ticket or request not done");
        return BFM_EINVAL;
    }
    Req* q = it->second;
    if (break_idx) *break_idx = q->brk;
    if (mean_mosum) *mean_mosum = q->mean;
    if (sigma) *sigma = q->sigma;
    if (beta) *beta = q->beta;
    if (status) *status = q->status;
    return BFM_OK;
}

bfm_status bfm_serve_release(bfm_server_t s, uint64_t ticket) {
    if (!s) {
        set_error("bfm_serve_release: NULL server");
        return BFM_EINVAL;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) {
        set_error("bfm_serve_release: unknown ticket");
        return BFM_EINVAL;
    }
    Req* q = it->second;
    const int st = q->state.load();
    if (st == ST_RUNNING || st == ST_PENDING) {
        set_error("bfm_serve_release: request still pending or running (cancel or wait first)");
        return BFM_EBUSY;
    }
    account(s);  // make sure the worker's bookkeeping no longer refers to it
    if (q->has_mem) s->alloc.release(q->off, q->bytes);
    s->reqs.erase(it);
    delete q;
    s->cv.notify_all();
    return BFM_OK;
}

bfm_status bfm_serve_cancel(bfm_server_t s, uint64_t ticket) {
    if (!s) {
        set_error("bfm_serve_cancel: NULL server");
        return BFM_EINVAL;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) {
        set_error("bfm_serve_cancel: unknown ticket");
        return BFM_EINVAL;
    }
    int expect = ST_PENDING;
    if (!it->second->state.compare_exchange_strong(expect, ST_CANCELLED)) {
        set_error("bfm_serve_cancel: request already admitted");
        return BFM_EBUSY;
    }
    s->cv.notify_all();
    return BFM_OK;
}

bfm_status bfm_serve_wait_all(bfm_server_t s, double timeout_s) {
    if (!s) {
        set_error("bfm_serve_wait_all: NULL server");
        return BFM_EINVAL;
    }
    std::unique_lock<std::mutex> lk(s->mu);
    auto busy = [&] {
        for (auto& kv : s->reqs) {
            const int st = kv.second->state.load();
            if (st == ST_PENDING || st == ST_RUNNING) return true;
        }
        return false;
    };
    const auto until = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
    while (busy()) {
        if (std::chrono::steady_clock::now() >= until) {
            set_error("bfm_serve_wait_all: timed out");
            return BFM_ETIMEOUT;
        }
        s->done_cv.wait_for(lk, std::chrono::milliseconds(2));
    }
    account(s);
    return BFM_OK;
}

bfm_status bfm_serve_stats(bfm_server_t s, double* p50_ms, double* p99_ms, int64_t* completed, int64_t* pixels,
                           double* span_ms) {
    if (!s) {
        set_error("bfm_serve_stats: NULL server");
        return BFM_EINVAL;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    account(s);
    std::vector<double> v = s->latencies;
    std::sort(v.begin(), v.end());
    auto q = [&](double f) { return v.empty() ? 0.0 : v[std::min(v.size() - 1, (size_t)(f * (double)v.size()))]; };
    if (p50_ms) *p50_ms = q(0.5);
    if (p99_ms) *p99_ms = q(0.99);
    if (completed) *completed = s->completed;
    if (pixels) *pixels = s->pixels;
    if (span_ms) *span_ms = s->first_arrive < 0 ? 0.0 : s->last_done - s->first_arrive;
    return BFM_OK;
}

bfm_status bfm_serve_destroy(bfm_server_t s) {
    if (!s) {
        set_error("bfm_serve_destroy: NULL server");
        return BFM_EINVAL;
    }
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->cv.notify_all();
    }
    s->worker.join();
    for (auto st : s->streams) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    for (auto& kv : s->reqs) delete kv.second;
    cudaFree(s->arena);
    delete s;
    return BFM_OK;
}

}  // extern "C"
