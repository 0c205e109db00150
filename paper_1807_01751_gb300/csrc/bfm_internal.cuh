// Internal declarations of libbfm (not part of the public ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>
#include <vector>

#include "../../include/bfm.h"

namespace bfm {

// ---------------------------------------------------------------------------
// Per-date basis row.
//
// The normal equations of Eq. 6 need, per pixel, G = sum_t m_t x_t x_t' with
// x_t the Eq. 2 regressors.  Products of harmonics reduce to single harmonics
// (sin a sin b = [cos(a-b) - cos(a+b)]/2 and the like), so G is a linear
// function of the masked sums of only 3 + 6k functions of t:
//   x_t itself               (1, t', s_1, c_1, ..., s_k, c_k)        K = 2 + 2k
//   t'^2
//   s_j, c_j for j = k+1..2k (the sum frequencies)
//   t' s_j, t' c_j for j = 1..k
// where s_j = sin(2 pi j t / f), c_j = cos(2 pi j t / f) and t' = (t - c)/s
// is the centred and scaled trend.  A basis row holds these values for one
// date, x_t first, padded to a multiple of 4 floats.
// ---------------------------------------------------------------------------
template <int KH>
struct Basis {
    static constexpr int K = 2 + 2 * KH;
    static constexpr int NBR = 3 + 6 * KH;       // live entries
    static constexpr int NB = (NBR + 3) & ~3;    // row stride (floats)
    static constexpr int TT = K;                 // t'^2
    __host__ __device__ static constexpr int S(int j) { return j <= KH ? 2 + 2 * (j - 1) : K + 1 + 2 * (j - KH - 1); }
    __host__ __device__ static constexpr int C(int j) { return S(j) + 1; }
    __host__ __device__ static constexpr int TS(int j) { return K + 1 + 2 * KH + 2 * (j - 1); }
    __host__ __device__ static constexpr int TC(int j) { return TS(j) + 1; }
};

inline int basis_stride(int kh) {
    return kh == 1 ? Basis<1>::NB : kh == 2 ? Basis<2>::NB : Basis<3>::NB;
}

// ---------------------------------------------------------------------------
// Kernel arguments
// ---------------------------------------------------------------------------
struct MonitorParams {
    const void* Y;            // [N][m] time-major
    const uint32_t* mask;     // [N][mask_words] or null
    int64_t m;
    int64_t mask_words;       // ceil(m/32)
    int N;
    int n_hist;
    const float* basis;       // [N][NB]
    double h_frac;
    float lambda;
    float c_over_s;           // trend centring, to map beta back to raw t
    float inv_s;
    int box_rows;             // TMA box height (dates per box)
    int nbox;                 // boxes per tile (nbox * box_rows >= N)
    int32_t* brk;
    float* mean;
    float* sigma;
    float* beta;              // [K][m]
    uint8_t* status;
    float* maxmo;             // nullable: MO of largest magnitude per pixel
};

// One tile of a batched launch (device-side descriptor).
struct BatchTileDesc {
    MonitorParams P;
    int64_t block0;  // first 32-pixel work block of this tile
    int kh, dtype, has_tma, has_mask;
};

// Parameters of one tile for the tensor-core form (monitor_mma.cu).
struct MmaParams {
    const void* Y;
    const uint32_t* mask;
    int64_t m, mask_words;
    int N, n_hist, npad, nhpad;  // npad = N padded to 32, nhpad = n_hist padded to 32
    int stages;                   // Y blocks in flight
    int region_bytes;             // table B + A buffers, later the MOSUM ring
    int vb_extra;                 // bytes of a separate valid-byte area (0: it overlays the delta planes)
    const uint4* phi;             // A_hi, A_lo, B_hi, B_lo (abi.cu tc_tables), each npad dates long
    double h_frac;
    float lambda, c_over_s, inv_s;
    int ring;
    int32_t* brk;
    float* mean;
    float* sigma;
    float* beta;
    uint8_t* status;
    float* maxmo;  // nullable: MO of largest magnitude per pixel
};

// One tile of a batched tensor-core launch: the arguments of its kernel node.
struct MmaBatchTile {
    CUtensorMap tm;  // 64-byte aligned type
    MmaParams P;
    int kh, dtype, has_mask;
};

// Fill one batch tile for the tensor-core form (false with a message when the
// form does not take it); *smem receives the tile's dynamic shared memory.
bool mma_fill_tile(const bfm_design_s* d, int dtype, const void* Y, const uint32_t* mask, int64_t m, int n_hist,
                   double h_frac, double lambda, int32_t* brk, float* mean, float* sigma, float* beta,
                   uint8_t* status, MmaBatchTile* out, size_t* smem);
// Kernel variant (0..11) of a tile: harmonics k, storage type, explicit mask.
int mma_variant(int k, int dtype, bool has_mask);
// Add the single-tile tensor-core kernel of tile t (its own grid of 128-pixel
// blocks, as bfm_monitor launches it) to `graph` after `dep` (nullable).
bfm_status mma_tile_node(const MmaBatchTile& t, size_t smem, cudaGraph_t graph, const cudaGraphNode_t* dep,
                         cudaGraphNode_t* node_out);

// Each kernel translation unit keeps its own device error word (bit 0: a
// tile-load wait gave up); these read and clear it, synchronising `s`.
cudaError_t simt_read_clear_errors(cudaStream_t s, unsigned int* bits);

}  // namespace bfm

// ---------------------------------------------------------------------------
// Public design handle
// ---------------------------------------------------------------------------
// Shared table of the complete-series form for one history length
// (complete.cu): M' [n_hist][K] then X [N][K] in float, and the status every
// pixel gets from the shared design (OK, INSUFFICIENT_HISTORY or SINGULAR).
struct CompleteTab {
    int n_hist;
    int status;
    float* d_tab;
};

struct bfm_design_s {
    int N = 0, k = 0, K = 0;
    double f = 0.0;
    std::vector<double> dates;
    double c = 0.0, s = 1.0;  // trend centring/scaling
    int NB = 0;               // basis row stride (floats)
    float* d_basis = nullptr; // device [N][NB]
    double* d_dates = nullptr; // device [N]: the date values (bfm_trace)
    std::mutex complete_mu;            // guards `complete`
    std::vector<CompleteTab> complete; // built on first use per n_hist, freed with the design
    // Tensor-core B operands: the basis table as fp16 hi and lo parts in the
    // no-swizzle core-matrix layout (see abi.cu tc_tables); nullptr when N
    // exceeds the tensor-core limit.
    void* d_phi_tc = nullptr;
    int npad_tc = 0;
    // Hybrid-form tables (hybrid.cu hybrid_tables): Gram hi/lo, tf32 regressors,
    // fitted-value regressors hi/lo.
    void* d_hyb = nullptr;
    int device = -1;
    int refcount = 0;
    uint64_t key = 0;
};

namespace bfm {

void set_error(const std::string& msg);
bfm_status cuda_fail(cudaError_t e, const char* what);

// Launch the CUDA-core (SIMT) kernel for one tile set on `stream`.
bfm_status launch_simt(const bfm_design_s* d, const void* Y, int dtype, const uint32_t* mask, int64_t m,
                       int n_hist, double h_frac, double lambda, int32_t* brk, float* mean, float* sigma,
                       float* beta, uint8_t* status, cudaStream_t stream, float* maxmo = nullptr);

// Tensor-core form: limits and launch.
// Basis tables of the tensor-core form (abi.cu tc_tables): table A = basis
// rows 0..15, table B = rows 16..31, each as fp16 hi then lo, over npad dates.
// True when the tensor-core form takes these parameters and this Y (a TMA-describable layout).
bool mma_supported(const bfm_design_s* d, int dtype, int n_hist, double h_frac, const void* Y, int64_t m,
                   size_t* smem_out);
bfm_status launch_mma(const bfm_design_s* d, int dtype, const void* Y, const uint32_t* mask, int64_t m,
                      int n_hist, double h_frac, double lambda, int32_t* brk, float* mean, float* sigma,
                      float* beta, uint8_t* status, cudaStream_t stream, float* maxmo = nullptr);
cudaError_t mma_read_clear_errors(cudaStream_t s, unsigned int* bits);

// Complete-series form (complete.cu): shared pseudo-inverse, one thread per pixel.
size_t complete_smem_bytes(int N, int n, int K, int h, bool staged);
cudaError_t complete_read_clear_errors(cudaStream_t s, unsigned int* bits);

// Streaming CUDA-core form (stream.cu).
bool stream_supported(const bfm_design_s* d, int dtype, int n_hist, double h_frac, const void* Y, int64_t m);
bfm_status launch_stream(const bfm_design_s* d, int dtype, const void* Y, const uint32_t* mask, int64_t m,
                         int n_hist, double h_frac, double lambda, int32_t* brk, float* mean, float* sigma,
                         float* beta, uint8_t* status, cudaStream_t stream, float* maxmo);
cudaError_t stream_read_clear_errors(cudaStream_t s, unsigned int* bits);
// Hybrid form (hybrid.cu): tensor-core contractions, one thread per pixel for the scans.
void hybrid_tables(const bfm_design_s& d, const std::vector<double>& rows, std::vector<unsigned char>& out);
bool hybrid_supported(const bfm_design_s* d, int dtype, int n_hist, double h_frac, const void* Y, int64_t m);
bfm_status launch_hybrid(const bfm_design_s* d, int dtype, const void* Y, const uint32_t* mask, int64_t m,
                         int n_hist, double h_frac, double lambda, int32_t* brk, float* mean, float* sigma,
                         float* beta, uint8_t* status, cudaStream_t stream, float* maxmo);
cudaError_t hybrid_read_clear_errors(cudaStream_t s, unsigned int* bits);
// Batched hybrid launch (bfm_batch): a group holds tiles of one kernel variant
// (k, storage, mask) whose tables and rings fit one shared-memory layout, run
// by one persistent kernel over 512-pixel work blocks.
struct HybGroup;
HybGroup* hyb_group_create(int k, int dtype, bool has_mask);
void hyb_group_destroy(HybGroup* g);
bool hyb_group_variant(const HybGroup* g, int k, int dtype, bool has_mask);
// 1: appended; 0: the group's layout would no longer fit (nothing changed);
// -1: the hybrid form does not take the tile (message set).
int hyb_group_add(HybGroup* g, const bfm_design_s* d, const void* Y, const uint32_t* mask, int64_t m, int n_hist,
                  double h_frac, double lambda, int32_t* brk, float* mean, float* sigma, float* beta,
                  uint8_t* status);
bfm_status hyb_group_upload(HybGroup* g);  // device tile table (again after adds)
bfm_status hyb_group_node(HybGroup* g, cudaGraph_t graph, const cudaGraphNode_t* dep, cudaGraphNode_t* node);
int64_t hyb_group_blocks(const HybGroup* g);

// Bound of the staged forms' consumer-side stage waits (bfm_stage_wait_limit).
uint64_t stage_wait_ns();
void set_stage_wait_ns(uint64_t ns);

// The form BFM_ALGO_AUTO takes for a single call, the host-buffer entry and
// the server: the hybrid form where it applies, else the streaming form, else
// the tensor-core form, else the CUDA-core form.
int auto_form(const bfm_design_s* d, int dtype, int n_hist, double h_frac, const void* Y, int64_t m);
bfm_status launch_complete(bfm_design_s* d, int dtype, const void* Y, const uint32_t* mask, int64_t m, int n_hist,
                           double h_frac, double lambda, int32_t* brk, float* mean, float* sigma, float* beta,
                           uint8_t* status, cudaStream_t stream, float* maxmo);

// Shared-memory bytes the SIMT kernel needs for N dates, k harmonics and a dtype (0 if too large).
size_t simt_smem_bytes(int N, int k, int dtype, int* box_rows, int* nbox);

}  // namespace bfm
