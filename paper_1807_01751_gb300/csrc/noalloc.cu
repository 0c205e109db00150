// Batched launch without any allocation (bfm_batch_run_static).
//
// Some callers cannot allocate device memory at the moment they want to run
// a batch: a serving process whose whole device memory is pre-reserved by
// its own pool allocator (a cudaMalloc outside the pool may fail, or steal
// memory the pool already promised to someone else), and latency-critical
// loops where cudaMalloc/cudaFree would synchronise the device and stall
// every other stream.  For them this entry point keeps everything the
// persistent kernel needs beyond the caller's inputs and outputs -- the tile
// table, the tensor maps and the work counter -- in one fixed array that is
// part of the library's device image.  A small kernel, given the table as its
// argument, writes it there ahead of the persistent kernel.
#include <cuda.h>

#include <cstring>
#include <mutex>

#include "bfm_internal.cuh"

namespace bfm {

bool make_tensor_map(CUtensorMap* tm, const void* Y, int dtype, int64_t m, int N, int box_rows);
size_t simt_smem_bytes(int N, int k, int dtype, int* box_rows, int* nbox);
bfm_status batch_launch_kernel(const void* tiles, const void* tmaps, int ntiles, int64_t total_blocks,
                               unsigned long long* counter, int grab, int grid, size_t smem, cudaStream_t s,
                               cudaGraph_t graph, const cudaGraphNode_t* dep, cudaGraphNode_t* node_out);

namespace {

constexpr int kStaticMaxTiles = BFM_STATIC_MAX_TILES;
// layout: [tensor maps (128 B each)] [tile table] [work counter]
constexpr size_t kMapsBytes = sizeof(CUtensorMap) * kStaticMaxTiles;
constexpr size_t kTilesOff = kMapsBytes;
constexpr size_t kTilesBytes = ((sizeof(BatchTileDesc) * kStaticMaxTiles + 255) / 256) * 256;
constexpr size_t kCounterOff = kTilesOff + kTilesBytes;
constexpr size_t kScratchBytes = kCounterOff + 256;

// The scratch: every device that loads the library holds it until exit.
static __device__ __align__(256) unsigned char g_static_scratch[kScratchBytes];

// The tile table and tensor maps of one call, passed by value as the argument
// of the kernel that writes them into the scratch: the launch copies them, so
// nothing of the call refers to host memory once it returns, and the host does
// not wait for earlier work in the stream (a copy from pageable host memory
// would).
struct StaticTable {
    uint4 w[kCounterOff / 16];
};
static_assert(kCounterOff % 16 == 0, "table size must be a multiple of 16 bytes");
static_assert(sizeof(StaticTable) <= 32000, "the table must fit the kernel argument space");

// Device code names the scratch directly; it overwrites the table and clears
// the work counter, which the previous call left behind.
__global__ void fill_static_table(const __grid_constant__ StaticTable t) {
    uint4* dst = reinterpret_cast<uint4*>(g_static_scratch);
    for (int i = threadIdx.x; i < (int)(kCounterOff / 16); i += blockDim.x) dst[i] = t.w[i];
    if (threadIdx.x == 0) *reinterpret_cast<unsigned long long*>(g_static_scratch + kCounterOff) = 0ull;
}

std::mutex g_mu;
unsigned char* g_scratch_ptr[64] = {};  // device address of g_static_scratch, per device

}  // namespace
}  // namespace bfm

using namespace bfm;

extern "C" bfm_status bfm_batch_run_static(const bfm_tile_spec* tiles, int ntiles, void* stream) {
    if (ntiles < 0 || (ntiles > 0 && !tiles)) {
        set_error("bfm_batch_run_static: tiles is NULL or ntiles < 0");
        return BFM_EINVAL;
    }
    if (ntiles > kStaticMaxTiles) {
        set_error("bfm_batch_run_static: " + std::to_string(ntiles) + " tiles exceed the fixed maximum of " +
                  std::to_string(kStaticMaxTiles) + " (BFM_STATIC_MAX_TILES); split the batch");
        return BFM_EINVAL;
    }
    if (ntiles == 0) return BFM_OK;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "bfm_batch_run_static: cudaGetDevice");
    if (dev < 0 || dev >= 64) {
        set_error("bfm_batch_run_static: device ordinal above 63");
        return BFM_EUNSUPPORTED;
    }
    unsigned char* base = nullptr;
    {
        // first call on this device: look up the scratch array's device address
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_scratch_ptr[dev]) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_static_scratch);
            if (e != cudaSuccess) return cuda_fail(e, "bfm_batch_run_static: cudaGetSymbolAddress");
            g_scratch_ptr[dev] = static_cast<unsigned char*>(p);
        }
        base = g_scratch_ptr[dev];
    }
    // Build the tile table and tensor maps in fixed host arrays (no heap use).
    alignas(64) unsigned char host[kCounterOff];
    std::memset(host, 0, sizeof host);
    CUtensorMap* maps = reinterpret_cast<CUtensorMap*>(host);
    BatchTileDesc* descs = reinterpret_cast<BatchTileDesc*>(host + kTilesOff);
    int64_t total = 0;
    size_t smem = 0;
    for (int i = 0; i < ntiles; ++i) {
        const bfm_tile_spec& s = tiles[i];
        const bfm_design_s* d = s.design;
        if (!d || (s.dtype != BFM_F32 && s.dtype != BFM_I16) || s.m < 0 || !(s.n_hist >= 1 && s.n_hist < d->N) ||
            !(s.h_frac > 0.0 && s.h_frac <= 1.0) || !(s.lambda > 0.0) ||
            (s.m > 0 && (!s.Y || !s.break_idx || !s.mean_mosum || !s.sigma || !s.beta || !s.status))) {
            set_error("bfm_batch_run_static: tile " + std::to_string(i) +
                      ": bad design, dtype, m, n_hist, h_frac, lambda or NULL buffer");
            return BFM_EINVAL;
        }
        if (d->device != dev) {
            set_error("bfm_batch_run_static: tile " + std::to_string(i) + ": design belongs to another device");
            return BFM_EINVAL;
        }
        int br = 0, nb = 0;
        const size_t sm = simt_smem_bytes(d->N, d->k, s.dtype, &br, &nb);
        if (sm == 0 || sm > 227 * 1024 - 256) {
            set_error("bfm_batch_run_static: tile " + std::to_string(i) + ": series does not fit one on-chip tile");
            return BFM_EUNSUPPORTED;
        }
        BatchTileDesc& t = descs[i];
        MonitorParams& P = t.P;
        P.Y = s.Y;
        P.mask = s.mask_bits;
        P.m = s.m;
        P.mask_words = (s.m + 31) / 32;
        P.N = d->N;
        P.n_hist = s.n_hist;
        P.basis = d->d_basis;
        P.h_frac = s.h_frac;
        P.lambda = (float)s.lambda;
        P.c_over_s = (float)(d->c / d->s);
        P.inv_s = (float)(1.0 / d->s);
        P.box_rows = br;
        P.nbox = nb;
        P.brk = s.break_idx;
        P.mean = s.mean_mosum;
        P.sigma = s.sigma;
        P.beta = s.beta;
        P.status = s.status;
        t.block0 = total;
        t.kh = d->k;
        t.dtype = s.dtype;
        t.has_mask = s.mask_bits != nullptr;
        t.has_tma = s.m >= 32 && make_tensor_map(&maps[i], s.Y, s.dtype, s.m, d->N, br);
        total += (s.m + 31) / 32;
        if (sm > smem) smem = sm;
    }
    if (total == 0) return BFM_OK;
    cudaStream_t st = (cudaStream_t)stream;
    // The array keeps the previous call's contents: overwrite the table and
    // clear the work counter, in stream order before the kernel.
    StaticTable table;
    std::memcpy(&table, host, sizeof table);
    fill_static_table<<<1, 256, 0, st>>>(table);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "bfm_batch_run_static: filling the static scratch");
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int per = (int)((228 * 1024) / (smem + 1024));
    per = per < 1 ? 1 : (per > 8 ? 8 : per);
    return batch_launch_kernel(base + kTilesOff, base, ntiles, total,
                               reinterpret_cast<unsigned long long*>(base + kCounterOff), 2, sms * per, smem, st,
                               nullptr, nullptr, nullptr);
}
