// Internal declarations of the sm_103a implementation behind include/latentam.h.
#pragma once

#include <cuda_runtime.h>

#include <functional>
#include <stdint.h>

#include "latentam.h"

namespace lat {

// Constants of the splat footprint (readings listed in latentam.h).
constexpr int kTile = LATENTAM_TILE;
constexpr int kTilePixels = kTile * kTile;
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kAlphaMax = 0.99f;
constexpr float kTMin = 1e-4f;
constexpr float kDilation = 0.3f;

struct CamParams {
    float R[9];
    float t[3];
    float fx, fy, cx, cy, z_near;
    int W, H, tiles_x, tiles_y;
    // launch order of the per-tile kernels (block b renders tile tile_order[b]); null: b itself
    const int32_t* tile_order;
};

inline CamParams cam_params(const latentam_camera& c) {
    CamParams p;
    for (int i = 0; i < 9; ++i) p.R[i] = c.R[i];
    for (int i = 0; i < 3; ++i) p.t[i] = c.t[i];
    p.fx = c.fx;
    p.fy = c.fy;
    p.cx = c.cx;
    p.cy = c.cy;
    p.z_near = c.z_near;
    p.W = c.width;
    p.H = c.height;
    p.tiles_x = (c.width + kTile - 1) / kTile;
    p.tiles_y = (c.height + kTile - 1) / kTile;
    p.tile_order = nullptr;
    return p;
}

// Workspace slots owned by the context.
enum Slot : int {
    WS_SORT_K0 = 0,
    WS_SORT_K1,
    WS_SORT_V0,
    WS_SORT_V1,
    WS_SORT_HIST,
    WS_SCAN_SUMS,
    WS_OFFSETS,
    WS_COUNTERS,
    WS_DEC_A,      // n x M attention (FP32 form) / bf16 copies (tensor form)
    WS_DEC_DF,     // n x D Fhat, then dFhat
    WS_DEC_DS,     // n x M softmax-input gradient
    WS_DEC_ROW,    // n x 4 per-pixel coefficients
    WS_DEC_PART,   // split-K partial sums of dK / dV
    WS_DEC_AUX,    // transposed / converted operands of the tensor-core path
    WS_DEC_AUX2,
    WS_DEC_AUX3,
    WS_LOSS,       // double accumulators
    WS_STEP_PROJ,  // latentam_step's own projection, bins, images and gradients
    WS_STEP_PAIRS,
    WS_STEP_IMG,
    WS_STEP_GRAD,
    WS_PAPER,      // keys, norms, Gram matrix, scaled queries and gradients of the W/D form
    WS_MASKS,      // mask-pooling plan, pooled queries and their gradients
    WS_KMEANS,     // streaming K-means scratch
    WS_FULL_IMG,   // images and gradients of the full Stage I backward
    WS_FULL_AUX,   // SSIM maps and loss sums
    WS_TILE_ORDER, // launch order of the per-tile render kernels (per frame)
    WS_NUM_SLOTS
};

}  // namespace lat

namespace lat {
constexpr int kProfPairs = 256;  // event pairs per stage before folding
struct GraphCache;  // api.cu
struct StageProfile {
    cudaEvent_t ev[2 * kProfPairs];
    int created;
    int used;
    double acc_ms;
    int64_t count;
};
}  // namespace lat

struct latentam_ctx {
    int device;
    int num_sms;
    int cc_major, cc_minor;
    void* slot_ptr[lat::WS_NUM_SLOTS];
    size_t slot_bytes[lat::WS_NUM_SLOTS];
    int profiling;
    lat::StageProfile prof[LATENTAM_NUM_STAGES];
    // per-frame buffers of the batched step: [2k] projection + tile ranges, [2k+1] pairs,
    // [2 LATENTAM_MAX_BATCH + 6k + j] the scratch of binning slot k (j: scan sums, sort keys 0 / 1,
    // sort values, long-list merge buffers, radix counters)
    void* frame_ptr[8 * LATENTAM_MAX_BATCH];
    size_t frame_bytes[8 * LATENTAM_MAX_BATCH];
    // streams on which the keyframes of a batch are binned concurrently, created on first use
    cudaStream_t bin_streams[8];
    cudaEvent_t bin_events[9];  // [0] fork, [1 + i] join of stream i
    cudaEvent_t iter_events[2];  // fork and join of the render backward branch of an iteration
    int bin_streams_ready;
    // set by a step around its decode: called by the tensor-core decode on its stream once dQ is
    // final, before the pixel reductions of dV and dK (the step forks its render backward there);
    // after_dq_called reports whether it ran
    const std::function<latentam_status(cudaStream_t)>* after_dq;
    int after_dq_called;
    // CUDA graphs of the step's iteration (see latentam_graphs_enable)
    int use_graphs;
    uint64_t ws_generation;  // bumped whenever a workspace buffer moves
    cudaStream_t cap_stream;
    int* step_dev;
    lat::GraphCache* graphs;
    lat::GraphCache* sort_graphs;  // the binning before and after its host read (see cached_launch)
    uint32_t* host_counts;         // pinned: [4..5] the device flags read with a step's loss, [8 + 4 k ..] the
                                   // counts of binning slot k read back by the host
    // autotuned split factors of the pixel reductions (see latentam_autotune_enable)
    int autotune;
    struct TuneEntry {
        int64_t n;
        int M, D, which, shape, z;
        float ms;  // the chosen candidate's measured time
    } tune[32];
    int tune_used, tune_next;
    // device address of the allocation-free decode's static scratch (resolved at creation)
    void* noalloc_scratch;
    // sticky device flags, cleared when a synchronising call reports them:
    // [0] a bounded wait of a tensor-core kernel gave up, [1] a non-finite gradient met Adam
    int* dev_flags;
    // test hook (latentam_test_wait_timeout): the next binning's look-back stalls once
    int test_stall_sort;
};

namespace lat {

// Error reporting (thread-local message, see latentam_last_error).
void set_error(const char* fmt, ...);
latentam_status cuda_error(cudaError_t e, const char* what);

// Workspace slot of at least `bytes` bytes (grows by synchronising the device and
// reallocating; contents are not preserved).  Returns NULL and sets the error on failure.
void* ws(latentam_ctx* ctx, Slot s, size_t bytes);

// Stage timer: records an event pair on `st` around its scope when profiling is enabled.
int prof_begin(latentam_ctx* ctx, int stage, cudaStream_t st);
void prof_end(latentam_ctx* ctx, int stage, int idx, cudaStream_t st);
struct StageTimer {
    latentam_ctx* ctx;
    int stage;
    cudaStream_t st;
    int idx;
    StageTimer(latentam_ctx* c, int s, cudaStream_t stream) : ctx(c), stage(s), st(stream), idx(-1) {
        if (c && c->profiling) idx = prof_begin(c, s, stream);
    }
    ~StageTimer() {
        if (idx >= 0) prof_end(ctx, stage, idx, st);
    }
};

// Called after every kernel launch: counts it and turns a launch error into a status.
void count_launch();
#define LAT_CHECK_LAUNCH(what)                                          \
    do {                                                                \
        ::lat::count_launch();                                          \
        cudaError_t e_ = cudaGetLastError();                            \
        if (e_ != cudaSuccess) return ::lat::cuda_error(e_, what);      \
    } while (0)

#define LAT_TRY(expr)                                 \
    do {                                              \
        latentam_status s_ = (expr);                  \
        if (s_ != LATENTAM_OK) return s_;             \
    } while (0)

// ---- launchers (each .cu file implements its own) ----------------------------------

latentam_status launch_project(const latentam_gaussians& g, const CamParams& cam,
                               const latentam_projected& out, cudaStream_t st);

// Exclusive scan of n uint32 values; *total_dev (device, nullable) receives the sum.  sums: the
// block-sum scratch (scan_scratch_words(n) words), the context's workspace when null.
latentam_status scan_exclusive_u32(latentam_ctx* ctx, const uint32_t* in, uint32_t* out, int64_t n,
                                   uint32_t* total_dev, cudaStream_t st,
                                   uint32_t* sums = nullptr);
// Stable LSD radix sort of n (key, value) pairs on key bits [0, bits), bits <= 32, n < 2^30.
// keys[0]/vals[0] hold the input (vals_iota: value = index, vals[0] is then only scratch);
// keys[1]/vals[1] are scratch.  *result receives the index of the buffer pair holding the
// sorted output.  *err (device) is set if a bounded cross-block wait gave up.  counters: the
// digit-count, ticket and look-back scratch (radix_scratch_words(n, bits) words), the context's
// workspace when null.
latentam_status radix_sort_pairs(latentam_ctx* ctx, uint32_t* const keys[2], uint32_t* const vals[2], bool vals_iota,
                                 int64_t n, int bits, int* result, uint32_t* err, cudaStream_t st,
                                 uint32_t* counters = nullptr);
// 32-bit words of the scratch of scan_exclusive_u32 over n items and of radix_sort_pairs over n
// keys of `bits` bits (the buffers the optional `sums` / `counters` arguments must hold).
size_t scan_scratch_words(int64_t n);
size_t radix_scratch_words(int64_t n, int bits);
latentam_status bin_and_sort(latentam_ctx* ctx, int32_t n, const latentam_projected& proj,
                             const CamParams& cam, latentam_bins* bins, cudaStream_t st);
// The two halves of bin_and_sort, for several keyframes binned with one host synchronisation:
// bin_count enqueues the pair count of binning slot `slot` (0 .. LATENTAM_MAX_BATCH - 1) into
// its pinned host words, the offsets into off[n + 1]; once the stream has been synchronised,
// bin_finish reads them and enqueues the pairs, their sort and the ranges (LATENTAM_ERR_CAPACITY
// when bins->capacity is short: bin_finish may then be called again with a larger buffer).
latentam_status bin_count(latentam_ctx* ctx, int32_t n, const latentam_projected& proj, const CamParams& cam,
                          latentam_bins* bins, uint32_t* off, int slot, cudaStream_t st);
latentam_status bin_finish(latentam_ctx* ctx, int32_t n, const latentam_projected& proj, const CamParams& cam,
                           latentam_bins* bins, const uint32_t* off, int slot, cudaStream_t st);

// The tiles of a binned frame in decreasing order of list length (power-of-two classes), into
// order[tiles]: the per-tile kernels start the longest tiles first.
latentam_status launch_tile_order(const CamParams& cam, const latentam_bins& bins, int32_t* order, cudaStream_t st);
latentam_status launch_render_fwd(const CamParams& cam, const latentam_projected& proj,
                                  const latentam_bins& bins, const float* f, int d, float* Q,
                                  float* T_final, int32_t* n_contrib, cudaStream_t st);
// df = (accumulate ? df : 0) + sum_p w_ip dQ_p.
latentam_status launch_render_bwd(const CamParams& cam, const latentam_projected& proj,
                                  const latentam_bins& bins, const int32_t* n_contrib,
                                  const float* dQ, int d, float* df, int32_t n, cudaStream_t st,
                                  bool accumulate = false);
// One tile of one frame: its list range, the frame's buffers and image size.
struct TileJob {
    int tile, tiles_x, W, H;
    const int2* ranges;
    const int32_t* pair_ids;
    const float2* xy;
    const float4* conic_opac;
    const float4* f;
    float4* Q;
    float* T_final;
    int32_t* n_contrib;
    const float4* dQ;
    float* df;
};

// The frames of a batch (one launch renders the tiles of all of them).
struct BatchJobs {
    TileJob fr[LATENTAM_MAX_BATCH];  // tile unused
    int n;
};

// Longest tiles first over every frame of jobs (entries (frame << 20) | tile, Σ tiles of all frames).
latentam_status launch_batch_order(const BatchJobs& jobs, int32_t* order, cudaStream_t st);
// Persistent render forward / backward over the `total` entries of order (atomic work ticket
// *counter, reset by the launch); the backward adds into each frame's df.
latentam_status launch_render_fwd_batch(const BatchJobs& jobs, int d, const int32_t* order, int total, int* counter,
                                        cudaStream_t st);
latentam_status launch_render_bwd_batch(const BatchJobs& jobs, int d, const int32_t* order, int total, int* counter,
                                        cudaStream_t st);
// Queries, colours and depth blended together (Q, C n x 3, Z, T_final, n_contrib).
latentam_status launch_render_full(const CamParams& cam, const latentam_projected& proj, const latentam_bins& bins,
                                   const float* f, int d, const float* colours, float* Q, float* C, float* Z,
                                   float* T_final, int32_t* n_contrib, cudaStream_t st);
// df, dcol (n x 3) and dgeo (n x 8: d mean2d x, y, d conic a, b, c, d opacity, d depth, -), zeroed
// first, from the image gradients dQ, dC, dZ and the rendered Q, C, Z.
latentam_status launch_render_bwd_full(const CamParams& cam, const latentam_projected& proj,
                                       const latentam_bins& bins, const float* f, int d, const float* colours,
                                       const int32_t* n_contrib, const float* Q, const float* C, const float* Z,
                                       const float* dQ, const float* dC, const float* dZ, float* df, float* dcol,
                                       float* dgeo, int32_t n, cudaStream_t st);
// L_rgb and L_d with their image gradients; parts[5..9] (parts[3] must hold lambda_f L_f).
latentam_status launch_image_loss(latentam_ctx* ctx, const float* C, const float* Z, const float* image,
                                  const float* depth_obs, int W, int H, const latentam_image_cfg& cfg,
                                  double* parts, float* dC, float* dZ, cudaStream_t st);
latentam_status launch_project_bwd(const latentam_gaussians& g, const CamParams& cam, const float* dgeo,
                                   float* dmean, float* dquat, float* dscale, float* dopac, cudaStream_t st);
// Runs fn(stream) eagerly the first time a key is seen, captures it into a CUDA graph (on
// the context's capture stream) the second time and replays the graph on `st` from then on,
// while graphs are enabled and stage timing is off.  The key must name every pointer, size and
// workspace generation the launches depend on.
latentam_status cached_launch(latentam_ctx* ctx, const uint64_t* key, int n, cudaStream_t st,
                              const std::function<latentam_status(cudaStream_t)>& fn);
// Per-frame buffer `idx` of at least `bytes` (grows like ws()).
void* frame_ws(latentam_ctx* ctx, int idx, size_t bytes);

struct DecodeArgs {
    const float* Q;
    int64_t n;
    int d;
    const float* K;
    const float* V;
    const float* V0;
    int M, D;
    float c;                 // logit scale
    const void* F;
    latentam_dtype F_dtype;
    const uint8_t* mask;
    latentam_loss_cfg cfg;
    double* loss_parts;
    float* dQ;
    float* dK;
    float* dV;
};

latentam_status decode_fwd_f32(latentam_ctx* ctx, const float* Q, int64_t n, int d, const float* K,
                               const float* V, int M, int D, float c, float* F_hat, float* row_stats,
                               cudaStream_t st);
latentam_status decode_loss_bwd_f32(latentam_ctx* ctx, const DecodeArgs& a, cudaStream_t st);
// fp8: the value contraction (softmax weights times V) on E4M3 operands
latentam_status decode_loss_bwd_bf16(latentam_ctx* ctx, const DecodeArgs& a, cudaStream_t st, bool fp8 = false);
// FP32 decode + loss + backward with all scratch in a static device array (no allocation).
latentam_status decode_loss_bwd_f32_noalloc(latentam_ctx* ctx, const DecodeArgs& a, cudaStream_t st);
// Resolves the device address of that array into ctx->noalloc_scratch (the context's device
// current); called once when the context is created.
latentam_status decode_noalloc_setup(latentam_ctx* ctx);
latentam_status decode_fwd_bf16(latentam_ctx* ctx, const float* Q, int64_t n, int d, const float* K,
                                const float* V, int M, int D, float c, float* F_hat, float* row_stats,
                                cudaStream_t st, bool fp8 = false);
// The FP32 form on the tensor cores: every FP32 operand as a hi / lo pair of BF16 terms and every
// product as three MMAs (hi hi + hi lo + lo hi), FP32 accumulation; supported for M, D <= 1024.
bool decode_split_supported(int d, int M, int D);
latentam_status decode_loss_bwd_split(latentam_ctx* ctx, const DecodeArgs& a, cudaStream_t st);
latentam_status decode_fwd_split(latentam_ctx* ctx, const float* Q, int64_t n, int d, const float* K,
                                 const float* V, int M, int D, float c, float* F_hat, float* row_stats,
                                 cudaStream_t st);

// The paper's W / D / tau form of the decode, computed through the free-key decode.
struct PaperArgs {
    const float* Q;  // n x ds
    int64_t n;
    int ds;
    const float* W;  // ds x df
    const float* D;  // M x df
    int M, df;
};
struct PaperBuffers {
    float *K, *nrm, *G, *Qp, *r, *dQp, *dK, *dV, *Cm;
};
// keys K, norms, G = W W^T, scaled queries Q' and 1/|q W|
latentam_status paper_prepare(latentam_ctx* ctx, const PaperArgs& a, const PaperBuffers& b, cudaStream_t st);
// dQ, dW, dD (each nullable) from the free-key gradients dQ' (b.dQp), dK (b.dK), dV (b.dV)
latentam_status paper_chain(latentam_ctx* ctx, const PaperArgs& a, const PaperBuffers& b, float* dQ, float* dW,
                            float* dD, cudaStream_t st);

// C = scale A B^T on the FP32 tiled GEMM: A (m x k) and B (n x k) row-major with row stride k,
// C row stride ldc.  k and ldc multiples of 4, pointers 16-byte aligned, C rows padded to a
// multiple of 4 columns (the tile stores float4).
latentam_status sgemm_abt(const float* A, int64_t m, const float* B, int64_t n, int64_t k, float* C, int64_t ldc,
                          float scale, cudaStream_t st);

// Streaming K-means update of the dictionary (see latentam_stream_kmeans).
struct KMeansArgs {
    const float* F;          // n x D embeddings of the new keyframe
    int64_t n;
    int D;
    const uint8_t* valid;    // n flags, nullable
    const int32_t* init_idx; // k initial rows of the micro-clusters (device)
    int k;                   // micro-clusters, 1..32
    int iters_local, iters_global;
    float* centres;          // K x D, in/out
    float* weights;          // K, in/out
    int K;
    float* micro_C;          // k x D out, nullable
    float* micro_W;          // k out, nullable
    int32_t* micro_assign;   // n out, nullable
    int32_t* point_assign;   // K + k out, nullable
};
latentam_status stream_kmeans(latentam_ctx* ctx, const KMeansArgs& a, cudaStream_t st);

// Mask pooling (SAM-based targets): the plan of one mask set over an image of npix pixels.
struct MaskPlan {
    const int32_t* offsets;  // S + 1 CSR offsets (device)
    const int32_t* pixels;   // n_entries pixel indices (device)
    int64_t n_entries;
    int32_t S;
    int64_t npix;
    int64_t max_chunks;      // capacity of part, in chunks
    int32_t* chunk_start;    // S + 1: first chunk of each mask, [S] = number of chunks
    int32_t* count;          // S: valid entries per mask
    float* part;             // max_chunks x d chunk partial sums
};
int64_t mask_max_chunks(int32_t S, int64_t E);
size_t mask_plan_bytes(int32_t S, int64_t E, int d);
void mask_plan_carve(void* base, const int32_t* offsets, const int32_t* pixels, int64_t E, int32_t S, int64_t npix,
                     int d, MaskPlan* p);
latentam_status launch_mask_plan(const MaskPlan& p, cudaStream_t st);
// Qm (S x d) = per-mask mean of the valid rows of Q (npix x d)
latentam_status launch_pool_fwd(const MaskPlan& p, const float* Q, int d, float* Qm, cudaStream_t st);
// dQ (npix x d) = 0, then += dQm_m / count_m over the valid entries of every mask
latentam_status launch_pool_bwd(const MaskPlan& p, const float* dQm, int d, float* dQ, cudaStream_t st);

struct AdamTensor {
    float* p;
    const float* g;
    float* m;
    float* v;
    int64_t n;
    float lr;
};
// step_dev (nullable): read the step from device memory instead of `step` (graph replays).
latentam_status launch_adam(latentam_ctx* ctx, const AdamTensor* t, int count, float beta1, float beta2,
                            float eps, int step, cudaStream_t st, const int* step_dev = nullptr);
latentam_status launch_step_set(int* step_dev, int value, cudaStream_t st);
latentam_status launch_step_advance(int* step_dev, cudaStream_t st);

}  // namespace lat
