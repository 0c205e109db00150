// Batched persistent launch: many scene tiles of uneven pixel counts, series
// lengths, harmonics and storage types in one CUDA-graph replay.
//
// Each tile takes the first form of hybrid, tensor-core, CUDA-core that
// applies (bfm_batch_set_forms narrows the choice).  Hybrid tiles are grouped
// by kernel variant (k, storage, mask) and a shared-memory layout that holds
// the group's largest tables and ring; per group one persistent kernel (one
// CTA per SM) takes 512-pixel blocks in a fixed order and finds the owning
// tile by binary search (hybrid.cu).  Each tensor-core tile is one kernel node,
// the kernel a single call launches over the tile's own 128-pixel blocks.  The
// CUDA-core tiles go to one persistent kernel whose CTAs take 32-pixel blocks
// from a device counter, `grab` at a time.  The counter reset (one memset
// node), the hybrid kernels (a chain after it) and, after them in parallel
// branches, the tensor-core tile nodes and the CUDA-core kernel form one
// graph, instantiated once and replayed.  An autotuner times (CTAs per SM,
// grab) for the CUDA-core kernel on the batch itself and caches the best pair
// per batch signature.
#include <cuda.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "bfm_internal.cuh"
#include "ptx.cuh"
#include "simt_seg.cuh"

namespace bfm {

// implemented in monitor_simt.cu
bool make_tensor_map(CUtensorMap* tm, const void* Y, int dtype, int64_t m, int N, int box_rows);
size_t simt_smem_bytes(int N, int k, int dtype, int* box_rows, int* nbox);
bfm_status batch_launch_kernel(const void* tiles, const void* tmaps, int ntiles, int64_t total_blocks,
                               unsigned long long* counter, int grab, int grid, size_t smem, cudaStream_t s,
                               cudaGraph_t graph_or_null, const cudaGraphNode_t* dep, cudaGraphNode_t* node_out);

}  // namespace bfm

struct bfm_batch_s {
    // CUDA-core tiles
    std::vector<bfm::BatchTileDesc> tiles;
    std::vector<CUtensorMap> tmaps;
    int64_t total_blocks = 0;
    size_t smem = 0;
    // tensor-core tiles: one kernel node each (arguments and dynamic shared memory)
    std::vector<std::pair<bfm::MmaBatchTile, size_t>> mtiles;
    // hybrid tiles, per group = kernel variant x shared-memory layout
    std::vector<bfm::HybGroup*> hgroups;
    int ntiles_all = 0;
    int forms = BFM_ALGO_AUTO;  // the forms tiles may take (bfm_batch_set_forms)
    std::vector<int> tile_form;  // per tile id: the form it takes
    std::vector<bfm_design_t> designs;  // references held until destroy
    // device copies
    void* d_tiles = nullptr;
    void* d_tmaps = nullptr;
    unsigned long long* d_counter = nullptr;  // the CUDA-core kernel's work counter
    bool dirty = true;
    // launch configuration
    int ctas_per_sm = 0;  // 0 = not tuned yet (use the occupancy maximum)
    int grab = 2;
    // graph
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int graph_grid = 0, graph_grab = 0;
    int device = -1;
};

namespace bfm {
namespace {

std::mutex g_tune_mu;
std::map<std::string, std::pair<int, int>> g_tune_cache;  // signature -> (ctas_per_sm, grab)

std::string signature(const bfm_batch_s* b) {
    // tiles of equal (N, K, dtype) and similar size behave alike: key on the multiset
    std::vector<std::string> parts;
    for (auto& t : b->tiles) {
        int64_t mb = 1;
        while (mb < t.P.m) mb <<= 1;
        parts.push_back(std::to_string(t.P.N) + ":" + std::to_string(t.kh) + ":" + std::to_string(t.dtype) + ":" +
                        std::to_string(mb));
    }
    std::sort(parts.begin(), parts.end());
    std::string s;
    for (auto& p : parts) s += p + ",";
    return s;
}

void free_dev(bfm_batch_s* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    if (b->d_tiles) cudaFree(b->d_tiles);
    if (b->d_tmaps) cudaFree(b->d_tmaps);
    if (b->d_counter) cudaFree(b->d_counter);
    b->d_tiles = b->d_tmaps = nullptr;
    b->d_counter = nullptr;
}

bfm_status upload(bfm_batch_s* b) {
    if (!b->dirty) return BFM_OK;
    free_dev(b);
    cudaError_t e = cudaSuccess;
    for (auto* g : b->hgroups) {
        const bfm_status st = hyb_group_upload(g);
        if (st != BFM_OK) return st;
    }
    if (!b->tiles.empty()) e = cudaMalloc(&b->d_tiles, sizeof(BatchTileDesc) * b->tiles.size());
    if (e == cudaSuccess && !b->tmaps.empty()) e = cudaMalloc(&b->d_tmaps, sizeof(CUtensorMap) * b->tmaps.size());
    if (e == cudaSuccess) e = cudaMalloc(&b->d_counter, sizeof(unsigned long long));
    if (e == cudaSuccess && !b->tiles.empty())
        e = cudaMemcpy(b->d_tiles, b->tiles.data(), sizeof(BatchTileDesc) * b->tiles.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !b->tmaps.empty())
        e = cudaMemcpy(b->d_tmaps, b->tmaps.data(), sizeof(CUtensorMap) * b->tmaps.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "bfm_batch: uploading tile descriptors");
    b->dirty = false;
    return BFM_OK;
}

int sm_count(int dev) {
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

int max_ctas_per_sm(size_t smem) {
    // shared memory bound (228 KB per SM, 1 KB reserved per CTA), at most 8
    const size_t per = smem + 1024;
    int n = (int)((228 * 1024) / per);
    return std::max(1, std::min(n, 8));
}

bfm_status build_graph(bfm_batch_s* b, int grid, int grab) {
    if (b->exec && b->graph_grid == grid && b->graph_grab == grab) return BFM_OK;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    cudaError_t e = cudaGraphCreate(&b->graph, 0);
    if (e != cudaSuccess) return cuda_fail(e, "bfm_batch: cudaGraphCreate");
    cudaGraphNode_t memset_node, kernel_node;
    cudaMemsetParams mp{};
    mp.dst = b->d_counter;
    mp.value = 0;
    mp.elementSize = 4;
    mp.width = 2;  // the CUDA-core kernel's 64-bit work counter
    mp.height = 1;
    mp.pitch = 0;
    e = cudaGraphAddMemsetNode(&memset_node, b->graph, nullptr, 0, &mp);
    if (e != cudaSuccess) return cuda_fail(e, "bfm_batch: memset node");
    bfm_status st = BFM_OK;
    // the hybrid groups: a chain after the memset (their CTAs take work blocks in a fixed
    // order and so should find every SM free)
    cudaGraphNode_t prev = memset_node;
    for (auto* g : b->hgroups) {
        cudaGraphNode_t node;
        st = hyb_group_node(g, b->graph, &prev, &node);
        if (st != BFM_OK) return st;
        prev = node;
    }
    // after them, in parallel branches: one node per tensor-core tile (the kernel a single
    // call launches, over the tile's own blocks) and the persistent CUDA-core kernel
    for (auto& mt : b->mtiles) {
        cudaGraphNode_t node;
        st = mma_tile_node(mt.first, mt.second, b->graph, &prev, &node);
        if (st != BFM_OK) return st;
    }
    if (!b->tiles.empty() && b->total_blocks > 0) {
        st = batch_launch_kernel(b->d_tiles, b->d_tmaps, (int)b->tiles.size(), b->total_blocks, b->d_counter, grab,
                                 grid, b->smem, nullptr, b->graph, &prev, &kernel_node);
        if (st != BFM_OK) return st;
    }
    e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    if (e != cudaSuccess) return cuda_fail(e, "bfm_batch: graph instantiate");
    b->graph_grid = grid;
    b->graph_grab = grab;
    return BFM_OK;
}

bfm_status run_cfg(bfm_batch_s* b, int ctas_per_sm, int grab, cudaStream_t s) {
    bfm_status st = upload(b);
    if (st != BFM_OK) return st;
    const int grid = sm_count(b->device) * ctas_per_sm;
    st = build_graph(b, grid, grab);
    if (st != BFM_OK) return st;
    cudaError_t e = cudaGraphLaunch(b->exec, s);
    if (e != cudaSuccess) return cuda_fail(e, "bfm_batch: cudaGraphLaunch");
    return BFM_OK;
}

}  // namespace
}  // namespace bfm

using namespace bfm;

extern "C" {

bfm_status bfm_batch_create(bfm_batch_t* out) {
    if (!out) {
        set_error("bfm_batch_create: out is NULL");
        return BFM_EINVAL;
    }
    auto* b = new bfm_batch_s;
    cudaGetDevice(&b->device);
    *out = b;
    return BFM_OK;
}

bfm_status bfm_batch_destroy(bfm_batch_t b) {
    if (!b) {
        set_error("bfm_batch_destroy: NULL handle");
        return BFM_EINVAL;
    }
    free_dev(b);
    for (auto* g : b->hgroups) hyb_group_destroy(g);
    for (auto d : b->designs) bfm_design_destroy(d);
    delete b;
    return BFM_OK;
}

bfm_status bfm_batch_add(bfm_batch_t b, bfm_design_t d, const void* Y, int dtype, const uint32_t* mask_bits,
                         int64_t m, int n_hist, double h_frac, double lambda, int32_t* break_idx, float* mean_mosum,
                         float* sigma, float* beta, uint8_t* status, int* tile_id) {
    if (!b || !d) {
        set_error("bfm_batch_add: NULL batch or design");
        return BFM_EINVAL;
    }
    if (dtype != BFM_F32 && dtype != BFM_I16) {
        set_error("bfm_batch_add: dtype must be BFM_F32 or BFM_I16");
        return BFM_EINVAL;
    }
    if (m < 0 || !(n_hist >= 1 && n_hist < d->N) || !(h_frac > 0.0 && h_frac <= 1.0) || !(lambda > 0.0)) {
        set_error("bfm_batch_add: m < 0, n_hist outside [1, N), h_frac outside (0, 1] or lambda <= 0");
        return BFM_EINVAL;
    }
    if (m > 0 && (!Y || !break_idx || !mean_mosum || !sigma || !beta || !status)) {
        set_error("bfm_batch_add: Y and all outputs must be non-NULL device pointers");
        return BFM_EINVAL;
    }
    // keep the design alive while the batch may run
    auto hold = [&](int form) {
        bfm_design_t dd = nullptr;
        bfm_design_create(d->dates.data(), d->N, d->k, d->f, &dd);
        b->designs.push_back(dd);
        b->dirty = true;
        b->tile_form.push_back(form);
        if (tile_id) *tile_id = b->ntiles_all;
        ++b->ntiles_all;
        return BFM_OK;
    };
    const bool hyb_ok = b->forms == BFM_ALGO_AUTO || b->forms == BFM_ALGO_HYBRID;
    const bool mma_ok = b->forms == BFM_ALGO_AUTO || b->forms == BFM_ALGO_MMA;
    if (hyb_ok && m > 0 && hybrid_supported(d, dtype, n_hist, h_frac, Y, m)) {
        // the hybrid form: the first group of this variant whose layout still fits, else a new one
        const bool hm = mask_bits != nullptr;
        for (auto* g : b->hgroups) {
            if (!hyb_group_variant(g, d->k, dtype, hm)) continue;
            const int r = hyb_group_add(g, d, Y, mask_bits, m, n_hist, h_frac, lambda, break_idx, mean_mosum, sigma,
                                        beta, status);
            if (r < 0) return BFM_EUNSUPPORTED;
            if (r > 0) return hold(BFM_ALGO_HYBRID);
        }
        HybGroup* g = hyb_group_create(d->k, dtype, hm);
        const int r = hyb_group_add(g, d, Y, mask_bits, m, n_hist, h_frac, lambda, break_idx, mean_mosum, sigma, beta,
                                    status);
        if (r <= 0) {
            hyb_group_destroy(g);
            if (r == 0) set_error("bfm_batch_add: the tile does not fit the hybrid form's shared memory");
            return BFM_EUNSUPPORTED;
        }
        b->hgroups.push_back(g);
        return hold(BFM_ALGO_HYBRID);
    }
    if (mma_ok && m > 0 && mma_supported(d, dtype, n_hist, h_frac, Y, m, nullptr)) {
        // the tensor-core form, as bfm_monitor's AUTO would take it
        MmaBatchTile mt;
        size_t msm = 0;
        if (!mma_fill_tile(d, dtype, Y, mask_bits, m, n_hist, h_frac, lambda, break_idx, mean_mosum, sigma, beta,
                           status, &mt, &msm))
            return BFM_EUNSUPPORTED;
        b->mtiles.emplace_back(mt, msm);
        return hold(BFM_ALGO_MMA);
    }
    int br = 0, nb = 0;
    const size_t smem = simt_smem_bytes(d->N, d->k, dtype, &br, &nb);
    if (smem == 0 || smem > 227 * 1024 - 256) {
        set_error("bfm_batch_add: the series does not fit one on-chip tile");
        return BFM_EUNSUPPORTED;
    }
    BatchTileDesc t{};
    MonitorParams& P = t.P;
    P.Y = Y;
    P.mask = mask_bits;
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
    P.brk = break_idx;
    P.mean = mean_mosum;
    P.sigma = sigma;
    P.beta = beta;
    P.status = status;
    t.block0 = b->total_blocks;
    t.kh = d->k;
    t.dtype = dtype;
    t.has_mask = mask_bits != nullptr;
    CUtensorMap tm;
    std::memset(&tm, 0, sizeof tm);
    t.has_tma = m >= 32 && make_tensor_map(&tm, Y, dtype, m, d->N, br);
    b->tiles.push_back(t);
    b->tmaps.push_back(tm);
    b->total_blocks += (m + 31) / 32;
    b->smem = std::max(b->smem, smem);
    return hold(BFM_ALGO_SIMT);
}

bfm_status bfm_batch_run(bfm_batch_t b, void* stream) {
    if (!b) {
        set_error("bfm_batch_run: NULL batch");
        return BFM_EINVAL;
    }
    if (b->ntiles_all == 0) return BFM_OK;
    int cps = b->ctas_per_sm;
    if (cps == 0) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(signature(b));
        if (it != g_tune_cache.end()) {
            cps = it->second.first;
            b->grab = it->second.second;
        } else {
            cps = b->tiles.empty() ? 1 : max_ctas_per_sm(b->smem);
        }
    }
    return run_cfg(b, cps, b->grab, (cudaStream_t)stream);
}

bfm_status bfm_batch_autotune(bfm_batch_t b, void* stream, int* ctas_per_sm, int* grab, float* best_ms) {
    if (!b) {
        set_error("bfm_batch_autotune: NULL batch");
        return BFM_EINVAL;
    }
    if (b->ntiles_all == 0) return BFM_OK;
    cudaStream_t s = (cudaStream_t)stream;
    // only the CUDA-core kernel has choices; without CUDA-core tiles one pair is timed
    const int maxc = b->tiles.empty() ? 1 : max_ctas_per_sm(b->smem);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    int bc = maxc, bg = 2;
    const int ng = b->tiles.empty() ? 1 : 4;
    for (int c = 1; c <= maxc; ++c)
        for (int gi = 0; gi < ng; ++gi) {
            const int g = 1 << gi;
            bfm_status st = run_cfg(b, c, g, s);  // warm-up (and graph build)
            if (st != BFM_OK) {
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                return st;
            }
            cudaEventRecord(e0, s);
            for (int r = 0; r < 3; ++r) run_cfg(b, c, g, s);
            cudaEventRecord(e1, s);
            cudaError_t e = cudaEventSynchronize(e1);
            if (e != cudaSuccess) {
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                return cuda_fail(e, "bfm_batch_autotune");
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            ms /= 3.f;
            if (ms < best) {
                best = ms;
                bc = c;
                bg = g;
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->ctas_per_sm = bc;
    b->grab = bg;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[signature(b)] = {bc, bg};
    }
    if (ctas_per_sm) *ctas_per_sm = bc;
    if (grab) *grab = bg;
    if (best_ms) *best_ms = best;
    return BFM_OK;
}

bfm_status bfm_batch_set_config(bfm_batch_t b, int ctas_per_sm, int grab) {
    if (!b || ctas_per_sm < 0 || ctas_per_sm > 8 || grab < 1 || grab > 64) {
        set_error("bfm_batch_set_config: NULL batch, ctas_per_sm outside 0..8 or grab outside 1..64");
        return BFM_EINVAL;
    }
    b->ctas_per_sm = ctas_per_sm;
    b->grab = grab;
    return BFM_OK;
}

int bfm_batch_tiles(bfm_batch_t b) { return b ? b->ntiles_all : 0; }

int bfm_batch_form(bfm_design_t d, int dtype, int n_hist, double h_frac, const void* Y, int64_t m) {
    if (!d || (dtype != BFM_F32 && dtype != BFM_I16) || !(n_hist >= 1 && n_hist < d->N)) return BFM_ALGO_SIMT;
    if (m > 0 && hybrid_supported(d, dtype, n_hist, h_frac, Y, m)) return BFM_ALGO_HYBRID;
    return m > 0 && mma_supported(d, dtype, n_hist, h_frac, Y, m, nullptr) ? BFM_ALGO_MMA : BFM_ALGO_SIMT;
}

bfm_status bfm_batch_set_forms(bfm_batch_t b, int algo) {
    if (!b) {
        set_error("bfm_batch_set_forms: NULL batch");
        return BFM_EINVAL;
    }
    if (algo != BFM_ALGO_AUTO && algo != BFM_ALGO_HYBRID && algo != BFM_ALGO_MMA && algo != BFM_ALGO_SIMT) {
        set_error("bfm_batch_set_forms: algo must be BFM_ALGO_AUTO, BFM_ALGO_HYBRID, BFM_ALGO_MMA or BFM_ALGO_SIMT");
        return BFM_EINVAL;
    }
    if (b->ntiles_all > 0) {
        set_error("bfm_batch_set_forms: tiles were already added");
        return BFM_EINVAL;
    }
    b->forms = algo;
    return BFM_OK;
}

int bfm_batch_tile_form(bfm_batch_t b, int tile_id) {
    if (!b || tile_id < 0 || tile_id >= (int)b->tile_form.size()) return -1;
    return b->tile_form[(size_t)tile_id];
}

}  // extern "C"
