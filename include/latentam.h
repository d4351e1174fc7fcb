/*
 * latentam.h — C ABI of the GB300 (sm_103a) implementation of LatentAM's per-keyframe
 * latent-feature optimisation step (arxiv 2602.12314, Sec. III-B and III-C, Algorithm 1
 * Stage I/II):
 *
 *   query splatting   Q = R_f(G, T)                 Eq. (alpha_blending), Eq. (render_query)
 *   dictionary decode Fhat = softmax(c Q K^T) V     Eq. (dict_recon)
 *   feature objective lambda_f L_f                  Eq. (feat_loss), Eq. (full_obj)
 *   backward to the queries f and the dictionary (K, V), then an Adam update.
 *
 * Conventions shared by every call
 *  - Every tensor argument is a DEVICE pointer owned by the caller, row-major and
 *    contiguous, 16-byte aligned (float4 access); the library never frees it.  Pointer
 *    members of the structs below follow the same rule.  Host pointers are marked "host".
 *  - The library owns only the context: a growable device workspace (sort buffers,
 *    decode intermediates, loss accumulators, the tile launch order of the render calls).
 *    A context belongs to one device and must not be used by two host threads at once; its
 *    calls share the workspace, so calls that overlap on the GPU (enqueued on different
 *    streams without an ordering event) race on it: enqueue a context's calls on one stream
 *    or order the streams.
 *  - All work is enqueued on `stream` (a cudaStream_t; NULL = the legacy default stream)
 *    and returns without waiting, except where a call says it synchronises.  The steps run
 *    some of it on the context's own side streams (the keyframes of a batch binned at once;
 *    the render backward of an iteration beside the decode's pixel reductions), each branch
 *    forked from `stream` after the work enqueued on it before the call and joined back into
 *    it before the call returns: ordered for the caller as if all of it ran on `stream`.
 *  - Gradients are OVERWRITTEN, never accumulated; callers zero nothing.
 *  - Shapes outside the supported set return LATENTAM_ERR_UNSUPPORTED_SHAPE; there is no
 *    slow or CPU fallback.  On any error nothing is guaranteed about the outputs.
 *    latentam_last_error() returns a message for the calling host thread.
 *  - Supported: query dimension d in {16, 32, 64}; dictionary size M a multiple of 32 in
 *    [32, 1024]; value dimension D a multiple of 128 in [128, 2048]; image sides
 *    1..16384; N < 2^31 Gaussians; pair count < 2^31.
 *
 * Readings of the paper where it is silent (shared with the test oracle, stated here
 * because they define the results):
 *  - footprint (the 3DGS renderer Sec. III-A cites): EWA projection with a 0.3 px^2
 *    dilation, alpha = min(0.99, o exp(-d^T Sigma'^-1 d / 2)), contributions with
 *    alpha < 1/255 skipped, blending stops before a contribution that would take the
 *    transmittance below 1e-4; pixel centres at integer coordinates; 16x16 tiles; a
 *    Gaussian's tile rectangle is the axis-aligned box of its alpha >= 1/255 ellipse.
 *  - front-to-back order: the camera depth of the mean, evaluated in binary32 with every
 *    operation rounded as ((R20 x + R21 y) + R22 z) + t2 (no fused multiply-add), ascending;
 *    ties by index; the near-plane test compares that key with z_near.
 *  - Gaussians with depth <= z_near or opacity < 1/255 are culled; an uncovered pixel
 *    renders Q_p = 0.
 *  - decode with free keys K (M x d) and values V (M x D), logit scale c (1/sqrt(d) by
 *    default); the paper's W/D/tau form is the special case K = W D^T / |D|, V = D.
 *  - loss: lambda_f [lambda_cos mean_valid(1 - cos_p) + lambda_2 mean_{valid x D}(Fhat - F)^2
 *    + lambda_D sum_j ReLU(|V_j - V0_j| - delta)], cos_p = <Fhat_p, F_p> /
 *    max(|Fhat_p| |F_p|, 1e-8); the trust region acts on the value rows only.
 */
#ifndef LATENTAM_H
#define LATENTAM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define LATENTAM_API __attribute__((visibility("default")))
#else
#define LATENTAM_API
#endif

#define LATENTAM_TILE 16
#define LATENTAM_ABI_VERSION 3

typedef int32_t latentam_status;
#define LATENTAM_OK 0
#define LATENTAM_ERR_INVALID_ARG (-1)       /* null/misaligned pointer, bad count or config */
#define LATENTAM_ERR_UNSUPPORTED_SHAPE (-2) /* d, M, D or image size outside the supported set */
#define LATENTAM_ERR_OUT_OF_MEMORY (-3)     /* workspace allocation failed */
#define LATENTAM_ERR_CUDA (-4)              /* a CUDA runtime call or launch failed */
#define LATENTAM_ERR_CAPACITY (-5)          /* caller buffer too small; required size reported */
#define LATENTAM_ERR_TIMEOUT (-6)           /* a bounded device-side wait gave up */
#define LATENTAM_ERR_NOT_FINITE (-7)        /* a step's loss or a gradient fed to Adam was not finite */

typedef int32_t latentam_precision;
#define LATENTAM_PREC_FP32 0 /* FP32 form: where M <= 1024 and D <= 1024, the decode contractions on
                                tcgen05 tensor cores with every FP32 operand split into two BF16 terms
                                x = hi + lo (hi = bf16(x), lo = bf16(x - hi): x within 2^-16 |x|) and
                                every product taken as three MMAs a_hi b_hi + a_hi b_lo + a_lo b_hi
                                with FP32 accumulation (the dropped a_lo b_lo is below 2^-16 |a b|);
                                softmax, loss and the a_p/b_p coefficients in FP32, frame sums in
                                FP64; larger dictionaries run the LATENTAM_PREC_FP32_FMA kernels */
#define LATENTAM_PREC_BF16 1 /* decode contractions on tcgen05 tensor cores: BF16 operands, FP32 accumulation;
                                 M <= 1024 and D <= 1024 (else LATENTAM_ERR_UNSUPPORTED_SHAPE) */
#define LATENTAM_PREC_FP8 2  /* the BF16 form with the value contraction Fhat = A V on E4M3 operands
                                (kind::f8f6f4): attention rows scaled per pixel by 448 l_p (l_p the
                                softmax denominator: the row maximum of A is 1 / l_p), V scaled per
                                feature by 448 / max_j |V_jc|, FP32 accumulation, scales undone in
                                the epilogue; same shape limits as BF16 */
#define LATENTAM_PREC_FP32_FMA 3 /* every decode contraction in FP32 on the FMA pipes (CUDA cores) */

typedef int32_t latentam_dtype;
#define LATENTAM_DTYPE_F32 0
#define LATENTAM_DTYPE_BF16 1

typedef struct CUstream_st* latentam_stream; /* cudaStream_t */
typedef struct latentam_ctx latentam_ctx;

/* Pinhole camera (host struct).  p_cam = R p_world + t with R row-major; camera x right,
 * y down, z forward; pixel (x, y) = x + y * width. */
typedef struct {
    float R[9];
    float t[3];
    float fx, fy, cx, cy;
    float z_near;
    int32_t width, height;
} latentam_camera;

/* Gaussian primitives G_i = {p_i, q_i, s_i, alpha_i} of Eq. (gs_repr_basic) (colour unused). */
typedef struct {
    int32_t n;               /* N */
    const float* means;      /* N x 3 world positions p_i */
    const float* quats;      /* N x 4 orientations q_i = (w, x, y, z); normalised internally */
    const float* scales;     /* N x 3 linear scales s_i */
    const float* opacities;  /* N opacities alpha_i in [0, 1] */
} latentam_gaussians;

/* Per-Gaussian projection, written by latentam_project (caller-owned, N entries each). */
typedef struct {
    float* xy;              /* N x 2 pixel-space mean */
    float* conic_opacity;   /* N x 4: (Sigma'^-1)_00, (Sigma'^-1)_01, (Sigma'^-1)_11, opacity */
    float* depth;           /* N camera depth (binary32 sort key, see readings) */
    int32_t* rect;          /* N x 4 tile rectangle x0, y0, x1, y1 (half-open; all 0 if culled/off-screen) */
    int32_t* tiles_touched; /* N number of tiles in rect */
} latentam_projected;

/* (tile, Gaussian) pairs grouped by tile, each group front to back. */
typedef struct {
    int32_t* pair_ids;      /* capacity entries: Gaussian index of each pair */
    int64_t capacity;       /* length of pair_ids */
    int32_t* tile_ranges;   /* num_tiles x 2: [start, end) of each tile's pairs */
    int64_t num_pairs;      /* out: number of pairs P (also on CAPACITY errors) */
} latentam_bins;

/* Weights of Eq. (feat_loss) and lambda_f of Eq. (full_obj); Sec. IV-A values:
 * lambda_f 5, lambda_cos 0.5, lambda_2 0.5, lambda_D 0.2, delta 0.1. */
typedef struct {
    float lambda_f, lambda_cos, lambda_2, lambda_D, delta;
    float logit_scale; /* c of the decode; <= 0 selects 1/sqrt(d) */
} latentam_loss_cfg;

/* Adam: m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2; p -= lr mhat / (sqrt(vhat) + eps),
 * with bias corrections 1 - b^step.  Sec. IV-A gives lr = 0.01 for the dictionary. */
typedef struct {
    float lr_f, lr_dict, beta1, beta2, eps;
    int32_t step; /* step number of the NEXT update (1 for the first) */
} latentam_adam_cfg;

/* loss_parts layout (device doubles, written by the loss calls):
 * [0] mean over valid pixels of (1 - cos_p)   [1] mean over valid pixels x D of (Fhat - F)^2
 * [2] sum_j ReLU(|V_j - V0_j| - delta)         [3] total lambda_f L_f
 * [4] number of valid pixels |Omega| */
#define LATENTAM_LOSS_PARTS 5

/* ---- context ---------------------------------------------------------------------- */

/* Create a context bound to CUDA device `device` (made current on each call).  Returns
 * INVALID_ARG if out is NULL, CUDA if the device is absent or not sm_103. */
LATENTAM_API latentam_status latentam_ctx_create(int32_t device, latentam_ctx** out);
/* Synchronise the device and free the workspace.  NULL is accepted. */
LATENTAM_API latentam_status latentam_ctx_destroy(latentam_ctx* ctx);
/* Message describing the last error on the calling host thread ("" if none). */
LATENTAM_API const char* latentam_last_error(void);
/* ABI version (LATENTAM_ABI_VERSION). */
LATENTAM_API int32_t latentam_version(void);
/* Number of kernels this library has launched in this process (all contexts). */
LATENTAM_API int64_t latentam_launch_count(void);
/* Number of 16x16 tiles of the camera's image, ceil(W/16) * ceil(H/16). */
LATENTAM_API int32_t latentam_num_tiles(const latentam_camera* cam);

/* ---- stage timers -------------------------------------------------------------------- */

/* CUDA-event timers around each stage of the step, on the stream it runs on.  While
 * enabled every call records an event pair per stage (no effect on results; do not enable
 * during stream capture).  latentam_profile_read synchronises the device, writes the
 * accumulated milliseconds and launch-group counts of the LATENTAM_NUM_STAGES stages into
 * ms / counts (host arrays, nullable) and clears them when reset != 0. */
#define LATENTAM_STAGE_PROJECT 0
#define LATENTAM_STAGE_SORT 1
#define LATENTAM_STAGE_RENDER_FWD 2
#define LATENTAM_STAGE_DECODE 3     /* decode + loss + decode backward (all its kernels) */
#define LATENTAM_STAGE_RENDER_BWD 4
#define LATENTAM_STAGE_ADAM 5
#define LATENTAM_NUM_STAGES 6
LATENTAM_API latentam_status latentam_profile_enable(latentam_ctx* ctx, int32_t enable);
LATENTAM_API latentam_status latentam_profile_read(latentam_ctx* ctx, double* ms, int64_t* counts, int32_t reset);

/* CUDA graphs of the step (on by default).  latentam_step captures one Stage-I iteration
 * (learn_f != 0: render, decode + loss + backward, render backward, Adam) into a CUDA graph
 * the second time it sees a configuration (the same buffers, shapes, pair count, scalars and
 * workspace), instantiates it on a stream of the context, and from then on launches each
 * iteration as one graph on the caller's stream; the Adam step then lives in a device counter
 * (set from adam->step before the replays; adam->step is advanced on the host as before).  Up
 * to four configurations are kept.  With profiling enabled, or learn_f == 0, the iterations run
 * as plain launches.  Disabling drops the instantiated graphs (synchronises the device). */
LATENTAM_API latentam_status latentam_graphs_enable(latentam_ctx* ctx, int32_t enable);

/* Test hook for the failure paths of the bounded device waits (no GPU fault is involved).
 * which = 0: the next binning's radix sort makes the look-back of one 1024-key block poll a
 * word that nothing writes, with a short limit (4096 polls), so that the wait gives up: that
 * binning leaves its tiles empty and the NEXT binning returns LATENTAM_ERR_TIMEOUT.
 * which = 1: raises the flag a tensor-core kernel's bounded wait raises when it gives up, so
 * that the next synchronising call (binning, or a step reading its loss) reports it.
 * INVALID_ARG for other values. */
LATENTAM_API latentam_status latentam_test_wait_timeout(latentam_ctx* ctx, int32_t which);

/* Autotuning of the tensor-core decode (on by default): the first time a context meets a shape
 * (pixel count, M, D) outside stream capture, the launch shape of each GEMM reduction over
 * pixels (dV = A^T dFhat always; dK = c dS^T Q only where it is a GEMM of its own, M > 512 or
 * no dQ requested: otherwise the dA -> dS kernel computes it per 128-pixel tile and a fixed
 * reduction sums the tiles in order) is chosen by timing its candidates with CUDA
 * events on the caller's stream (this synchronises that stream once): for dV the CTA tile
 * (256 atoms x 256 features, the pixel block read once for both 128-atom halves, or 128 x 256
 * on twice the CTAs), for both the pixel split (the one-wave split of that tile, half and twice
 * it); each candidate is timed together with the reduction of its partial sums.  The fastest
 * is kept for the context's lifetime (32 shapes).  Results differ between
 * candidates only by FP32 summation order.  Disabling clears the choices and uses the first
 * tile shape with its one-wave split. */
LATENTAM_API latentam_status latentam_autotune_enable(latentam_ctx* ctx, int32_t enable);

/* One choice of the autotuner. */
typedef struct latentam_tune_choice {
    int64_t n;          /* pixels of the decode */
    int32_t M, D;       /* dictionary atoms and feature width */
    int32_t reduction;  /* 5: dV, 6: dK; plus 16 in the FP32 (split-BF16) form */
    int32_t tile;       /* dV: 0 = 256 x 256 per CTA, 1 = 128 x 256; dK: 0 (128 x 64) */
    int32_t split;      /* pixel split: CTAs along the pixel axis per output tile */
    float ms;           /* measured time of the chosen candidate */
} latentam_tune_choice;

/* The choices the context holds: *count receives their number; when out is not NULL and
 * 0 <= i < *count, *out receives choice i (oldest first while fewer than 32 are held).
 * INVALID_ARG when out is not NULL and i is out of range. */
LATENTAM_API latentam_status latentam_autotune_query(latentam_ctx* ctx, int32_t i, latentam_tune_choice* out,
                                                     int32_t* count);

/* ---- splatting (Sec. III-A, Eq. alpha_blending; Sec. III-B, Eq. render_query) ------- */

/* Project every Gaussian: EWA screen-space covariance, conic, opacity, depth key and
 * the tile rectangle of its alpha >= 1/255 footprint.  One thread per Gaussian. */
LATENTAM_API latentam_status latentam_project(latentam_ctx* ctx, const latentam_gaussians* g,
                                 const latentam_camera* cam, const latentam_projected* out,
                                 latentam_stream stream);

/* Bin and sort: emit one (tile, Gaussian) pair per covered tile in Gaussian index order,
 * stable radix sort of the pairs by tile, per-tile ranges, then each tile's list sorted by
 * (binary32 depth key, index): the front-to-back order, ties in index order.
 * SYNCHRONISES `stream` once to read the pair count P into bins->num_pairs; if
 * P > bins->capacity returns LATENTAM_ERR_CAPACITY and writes no pairs (retry with a larger
 * buffer).  Returns LATENTAM_ERR_TIMEOUT if a bounded wait of an EARLIER call's sort gave up
 * (that call's tiles were left empty), or if a bounded wait of a tensor-core decode kernel
 * gave up since the last report (that call's loss was NaN); the flag is cleared when reported. */
LATENTAM_API latentam_status latentam_sort(latentam_ctx* ctx, int32_t n, const latentam_projected* proj,
                              const latentam_camera* cam, latentam_bins* bins,
                              latentam_stream stream);

/* Front-to-back blend of the d-dimensional queries f (N x d) of each tile's Gaussians:
 * Q (H*W x d), final transmittance T_final (H*W) and number of contributions n_contrib
 * (H*W).  One 16x16-pixel CTA per tile, Gaussians staged through shared memory. */
LATENTAM_API latentam_status latentam_render_fwd(latentam_ctx* ctx, int32_t n, const latentam_projected* proj,
                                    const latentam_camera* cam, const latentam_bins* bins,
                                    const float* f, int32_t d, float* Q, float* T_final,
                                    int32_t* n_contrib, latentam_stream stream);

/* Gradient of the blend with respect to the queries: df_i = sum_p w_ip dQ_p with the
 * blend weights w_ip = alpha_ip T_ip recomputed front to back (no division) into shared
 * memory per tile and batch, summed over the tile's pixels, one atomic add per Gaussian,
 * channel and tile.  n_contrib is the output of latentam_render_fwd for the same inputs.
 * df is N x d (overwritten). */
LATENTAM_API latentam_status latentam_render_bwd(latentam_ctx* ctx, int32_t n, const latentam_projected* proj,
                                    const latentam_camera* cam, const latentam_bins* bins,
                                    const int32_t* n_contrib, const float* dQ, int32_t d,
                                    float* df, latentam_stream stream);

/* ---- dictionary decode (Sec. III-B, Eq. dict_recon) --------------------------------- */

/* Fhat = softmax_rows(c Q K^T) V for Q (n x d), K (M x d), V (M x D).  F_hat (n x D) and
 * row_stats (n x 2: row maximum of the logits, softmax denominator) may each be NULL. */
LATENTAM_API latentam_status latentam_decode_fwd(latentam_ctx* ctx, const float* Q, int64_t n, int32_t d,
                                    const float* K, const float* V, int32_t M, int32_t D,
                                    float logit_scale, latentam_precision prec, float* F_hat,
                                    float* row_stats, latentam_stream stream);

/* Feature objective and its gradients in one pass: decode, lambda_f L_f against the
 * target F (n x D, dtype F_dtype) on the pixels with mask != 0 (NULL mask = all), then
 * dQ (n x d), dK (M x d), dV (M x D, including the trust-region subgradient against V0).
 * loss_parts: device doubles (LATENTAM_LOSS_PARTS).  Any of dQ/dK/dV may be NULL. */
LATENTAM_API latentam_status latentam_decode_loss_bwd(latentam_ctx* ctx, const float* Q, int64_t n, int32_t d,
                                         const float* K, const float* V, const float* V0,
                                         int32_t M, int32_t D, const void* F,
                                         latentam_dtype F_dtype, const uint8_t* mask,
                                         const latentam_loss_cfg* cfg, latentam_precision prec,
                                         double* loss_parts, float* dQ, float* dK, float* dV,
                                         latentam_stream stream);

/* ---- the paper's cosine / temperature form of the decode (Sec. III-B, Eq. dict_recon) -------
 *
 * Queries Q (n x ds) are projected by W (ds x df); each projection u_p = q_p W is compared with
 * every atom of the dictionary D (M x df) by cosine similarity after l2 normalisation (norms
 * floored at 1e-12), divided by the temperature tau (> 0, no default: the paper defers to the
 * work it follows), and Fhat = softmax_rows(cos / tau) D.  Computed exactly through the
 * free-key decode with keys k_j = W D_j^T / |D_j|, queries q_p / |q_p W| and logit scale
 * 1 / tau, so the n x df product Q W is never formed.  Shapes and precisions as for the
 * free-key calls (ds plays the role of d, df of D, M <= 1024 / df <= 1024 in BF16).  Q, W, D,
 * D0, F and the gradient buffers must be 16-byte aligned. */
LATENTAM_API latentam_status latentam_decode_fwd_paper(latentam_ctx* ctx, const float* Q, int64_t n, int32_t ds,
                                          const float* W, const float* D, int32_t M, int32_t df, float tau,
                                          latentam_precision prec, float* F_hat, float* row_stats,
                                          latentam_stream stream);

/* lambda_f L_f of the cosine form against the target F (n x df) on the pixels with
 * mask != 0, with the trust region on the atoms D against D0 (cfg->logit_scale is not used:
 * tau is), and the gradients dQ (n x ds), dW (ds x df), dD (M x df), each nullable and
 * overwritten.  loss_parts: device doubles (LATENTAM_LOSS_PARTS). */
LATENTAM_API latentam_status latentam_decode_loss_bwd_paper(latentam_ctx* ctx, const float* Q, int64_t n, int32_t ds,
                                               const float* W, const float* D, const float* D0, int32_t M,
                                               int32_t df, float tau, const void* F, latentam_dtype F_dtype,
                                               const uint8_t* mask, const latentam_loss_cfg* cfg,
                                               latentam_precision prec, double* loss_parts, float* dQ,
                                               float* dW, float* dD, latentam_stream stream);

/* Allocation-free form of latentam_decode_loss_bwd (FP32 only).  The paper has no
 * counterpart: this entry point exists for callers that cannot allocate device memory while
 * the step runs, e.g. a real-time mapping loop whose device memory is carved up once at
 * start-up by another runtime's allocator, or a caller that cannot accept the device-wide
 * synchronisation that cudaMalloc/cudaFree may imply.  It calls no allocation routine.
 * Its scratch (attention, dFhat, dS, per-pixel coefficients, split-K partial sums, loss
 * accumulators) lives in one static 16 MiB device array inside the library.  Creating a
 * context loads the library's device code on that device, which commits the array there, and
 * resolves its device address (latentam_ctx_create, with the device current); the array then
 * stays committed until the process exits, and the call itself neither allocates nor
 * resolves anything.  The address belongs to the CUDA context it was resolved in: after a
 * cudaDeviceReset create a new latentam context.  A call whose scratch would not fit returns
 * LATENTAM_ERR_UNSUPPORTED_SHAPE with the required size in latentam_last_error().  The
 * scratch is 4 n (2M + D) bytes (attention, dFhat, dS) + 16 n (coefficients) + 4 M (D + d) s
 * bytes of split partial sums, where the split count s grows with the SM count up to
 * min(2 SMs / tiles, n / 256); for example n <= 2048 rows fit at M = 256, D = 512, d = 32 on
 * any SM count, which covers mask-pooled targets.  All calls share the one array, which keeps
 * the last call's contents (the loss accumulators are cleared at the start of each call):
 * calls that overlap on the GPU (other streams or other host threads) race on it and must
 * be serialised by the caller.  Arguments, layouts and the other errors are those of
 * latentam_decode_loss_bwd. */
LATENTAM_API latentam_status latentam_decode_loss_bwd_noalloc(latentam_ctx* ctx, const float* Q, int64_t n,
                                                              int32_t d, const float* K, const float* V,
                                                              const float* V0, int32_t M, int32_t D, const void* F,
                                                              latentam_dtype F_dtype, const uint8_t* mask,
                                                              const latentam_loss_cfg* cfg, double* loss_parts,
                                                              float* dQ, float* dK, float* dV,
                                                              latentam_stream stream);

/* The whole backward of one keyframe: latentam_decode_loss_bwd on the rendered Q, then
 * latentam_render_bwd into df (skipped when df is NULL, as in Stage II where the
 * Gaussians are fixed).  dQ_scratch (H*W x d) receives the query-image gradient. */
LATENTAM_API latentam_status latentam_backward(latentam_ctx* ctx, int32_t n, const latentam_projected* proj,
                                  const latentam_camera* cam, const latentam_bins* bins,
                                  const int32_t* n_contrib, const float* Q, int32_t d,
                                  const float* K, const float* V, const float* V0, int32_t M,
                                  int32_t D, const void* F, latentam_dtype F_dtype,
                                  const uint8_t* mask, const latentam_loss_cfg* cfg,
                                  latentam_precision prec, double* loss_parts, float* dQ_scratch,
                                  float* df, float* dK, float* dV, latentam_stream stream);

/* ---- mask pooling (SAM-based targets) ------------------------------------------------ */

/* With SAM-based targets the decode's rows are the n valid masks instead of the pixels
 * (Sec. III-B, the passage after Eq. render_query), and the target of a mask is pooled over
 * its region.  Reading: the query of mask m is the mean of the rendered per-pixel queries over
 * the mask, Qm_m = (1/|m|) sum_{p in m} Q_p.
 *
 * Masks are CSR lists on the device: mask m owns entries [mask_offsets[m], mask_offsets[m+1])
 * of mask_pixels (pixel index y*W + x).  Offsets are clamped into [0, n_entries] and a
 * decreasing pair gives an empty mask; a pixel index outside [0, npix) is skipped and not
 * counted; masks may overlap and list a pixel several times; an empty mask pools to 0.
 * Q, Qm, dQm and dQ are row-major float32, 16-byte aligned; d in {16, 32, 64}; S >= 0;
 * 0 <= n_entries <= INT32_MAX.  All buffers are caller-owned device memory.  The result
 * does not depend on scheduling (fixed chunking and summation order). */
LATENTAM_API latentam_status latentam_pool_queries(latentam_ctx* ctx, const float* Q, int64_t npix, int32_t d,
                                                   const int32_t* mask_offsets, const int32_t* mask_pixels,
                                                   int64_t n_entries, int32_t S, float* Qm,
                                                   latentam_stream stream);
/* Backward of latentam_pool_queries: dQ (npix x d) is overwritten with
 * dQ_p = sum over the masks m listing p of dQm_m / |m| (zero for pixels in no mask).  Where
 * masks overlap the sum is taken with atomic adds (order-dependent in the last bits). */
LATENTAM_API latentam_status latentam_pool_queries_bwd(latentam_ctx* ctx, const float* dQm, int32_t S, int32_t d,
                                                       const int32_t* mask_offsets, const int32_t* mask_pixels,
                                                       int64_t n_entries, int64_t npix, float* dQ,
                                                       latentam_stream stream);

/* ---- dictionary initialisation from streaming data ------------------------------------ */

/* Streaming K-means update of the dictionary atoms (Algorithm 1, Eq. stream_kmeans_init,
 * Sec. III-C): D_t^(0) = StreamKMeans(F_t, D_{t-1}, K).
 *   1. local K-means: the valid rows of F (n x D, row-major float32; valid: n flags, NULL = all)
 *      are clustered into k_micro micro-clusters by iters_local Lloyd iterations started at the
 *      rows init_idx (device, k_micro int32; distinct valid rows; an index outside [0, n)
 *      starts its centre at the origin);
 *   2. merge: the occupied slots of the dictionary (weights > 0) and the non-empty
 *      micro-clusters (weight = row count) form weighted points; the empty slots, in slot
 *      order, start at the micro-centres, heaviest first (ties: lower micro index);
 *   3. re-cluster: iters_global weighted Lloyd iterations of the points against the occupied
 *      slots; a slot becomes the weighted mean of its points and its weight their total weight
 *      (a slot left without points keeps its centre with weight 0).
 * Squared Euclidean distances in float32 (|c|^2 - 2 <x, c>), ties to the lower index; fixed
 * iteration counts; deterministic summation order.  centres (K x D) and weights (K) are
 * updated in place; slots keep their identity.  micro_centres (k_micro x D), micro_weights
 * (k_micro) and micro_assign (n, -1 for invalid rows) receive the local clustering, and
 * point_assign (K + k_micro) the slot of each merged point in the last global iteration (points
 * in merge order: occupied slots, then non-empty micro-clusters; -1 past the last point), when
 * not NULL.  Limits: 1 <= k_micro <= min(32, n) (n >= 1), 1 <= K <= 8192, D % 4 == 0 and
 * D <= 1024, iteration counts >= 1; pointers 16-byte aligned; UNSUPPORTED_SHAPE otherwise. */
LATENTAM_API latentam_status latentam_stream_kmeans(latentam_ctx* ctx, const float* F, int64_t n, int32_t D,
                                                    const uint8_t* valid, const int32_t* init_idx, int32_t k_micro,
                                                    int32_t iters_local, int32_t iters_global, float* centres,
                                                    float* weights, int32_t K, float* micro_centres,
                                                    float* micro_weights, int32_t* micro_assign,
                                                    int32_t* point_assign, latentam_stream stream);

/* ---- voxel-hashed global map and the active local map (Sec. III-E) ----------------------- */

/* The global Gaussian map and its voxel hash, and the local map optimised around the camera.
 * Every Gaussian of the global store owns the table slot of the voxel floor(p / voxel_size) it
 * was inserted from (floor of the float32 quotient per axis); the slot of voxel (x, y, z) is
 * (x 73856093 ^ y 19349663 ^ z 83492791) mod 2^table_log2 on 64-bit two's-complement integers
 * (the spatial hash of Teschner et al.); the table stores no key, so two voxels with the same
 * slot collide and the later one counts as occupied; at most one Gaussian per slot.  The store,
 * the table and the local map live in device memory owned by the map. */
typedef struct latentam_map latentam_map;

/* The local map (device pointers owned by the map, valid until the next call that changes it):
 * count rows of means (x3), quats (x4), scales (x3), opacities, queries f (x d) and the Adam
 * moments of f (x d, zero for rows appended from the store), and gidx, each row's index in the
 * global store (-1: not in the store). */
typedef struct {
    float *means, *quats, *scales, *opacities, *f, *m_f, *v_f;
    int32_t* gidx;
    int64_t count;
} latentam_map_local;

/* The global store (device pointers owned by the map): count rows in index order, and the slot
 * table of table_size entries (-1 = empty). */
typedef struct {
    const float *means, *quats, *scales, *opacities, *f;
    const int32_t* table;
    int64_t count, table_size;
} latentam_map_global;

/* An empty map for queries of dimension d (1..256) with 2^table_log2 slots (4..30), voxel
 * edge voxel_size (> 0; 0.01 m in the paper) and room for `capacity` Gaussians (grown on
 * demand).  host_store != 0 keeps the store's rows in pinned host memory, which the kernels
 * read and write in place through unified addressing (the slot table and the local map stay
 * in device memory); the global_view pointers are then host pointers.  INVALID_ARG,
 * OUT_OF_MEMORY. */
LATENTAM_API latentam_status latentam_map_create(latentam_ctx* ctx, int32_t d, int32_t table_log2, float voxel_size,
                                                 int64_t capacity, int32_t host_store, latentam_map** out);
/* Synchronises the device and frees the map.  NULL is accepted. */
LATENTAM_API latentam_status latentam_map_destroy(latentam_map* map);
/* Insert-if-free of g->n new Gaussians (device SoA, queries f n x d) in input order: a
 * Gaussian whose slot is empty takes the next index of the store and the slot, the others are
 * not inserted (the same result as inserting one at a time).  out_index (device, n, nullable)
 * receives each Gaussian's new index or -1; n_inserted (host, nullable) the count.
 * Synchronises the stream.  At most 2^24 Gaussians per call; the store holds up to 2^31 - 1. */
LATENTAM_API latentam_status latentam_map_insert(latentam_ctx* ctx, latentam_map* map, const latentam_gaussians* g,
                                                 const float* f, int32_t* out_index, int64_t* n_inserted,
                                                 latentam_stream stream);
/* Appends g->n Gaussians created during local mapping to the local map (gidx -1, zero
 * moments); the next synchronisation inserts them into the store if their slot is free. */
LATENTAM_API latentam_status latentam_map_add_local(latentam_ctx* ctx, latentam_map* map,
                                                    const latentam_gaussians* g, const float* f,
                                                    latentam_stream stream);
/* The two synchronisation steps around camera position centre (host, 3 floats) with the
 * active radius: Local -> Global (local Gaussians from the store overwrite their entries, new
 * ones are inserted if their slot is free), then Global -> Local (local Gaussians with
 * (dx*dx + dy*dy) + dz*dz > radius*radius in float32 are dropped, the kept ones keep their order
 * and moments, and the store's Gaussians inside the radius that are not local are appended in
 * index order).  local_out (host, nullable) receives the new local map.  Synchronises. */
LATENTAM_API latentam_status latentam_map_sync(latentam_ctx* ctx, latentam_map* map, const float* centre,
                                               float radius, latentam_map_local* local_out,
                                               latentam_stream stream);
/* The current local map / global store (no device work). */
LATENTAM_API latentam_status latentam_map_local_view(latentam_map* map, latentam_map_local* out);
LATENTAM_API latentam_status latentam_map_global_view(latentam_map* map, latentam_map_global* out);

/* ---- the full Stage I objective: geometry, colour and depth (Eq. full_obj) ------------- */

/* Weights of Eq. (full_obj) and Eq. (rgb_loss): lambda_rgb (1; the paper gives no value),
 * lambda_I1 = 0.2, lambda_I2 = 0.8, lambda_d = 0.1 (Sec. IV-A); lambda_f is the feature
 * loss's own weight (latentam_loss_cfg). */
typedef struct {
    float lambda_rgb, lambda_I1, lambda_I2, lambda_d;
} latentam_image_cfg;

/* Loss parts of latentam_backward_full (device doubles): [0..4] those of
 * latentam_decode_loss_bwd ([3] = lambda_f L_f), [5] mean |I_hat - I| over pixels and channels,
 * [6] 1 - mean SSIM (11 x 11 Gaussian window, sigma 1.5, zero padding, C1 = 0.01^2,
 * C2 = 0.03^2), [7] L_d = mean |Z_hat - Z| over pixels with an observed depth (Z > 0), [8] their
 * count, [9] the total lambda_rgb (lambda_I1 [5] + lambda_I2 [6]) + lambda_d [7] + [3]. */
#define LATENTAM_FULL_LOSS_PARTS 10

/* The gradients of the full Stage I objective of one keyframe with respect to every attribute
 * of every Gaussian and the dictionary: projection and binning, the render of the queries f,
 * the colours (n x 3, view-independent) and the camera depth with the same blend (Eq.
 * alpha_blending), the decode, the feature loss, L_rgb against `image` (H*W x 3 float32, row
 * y*W + x) and L_d against `depth` (H*W float32, 0 = not observed), then the backward through
 * the blend (queries, colours, depth channel, opacities, screen means, conics) and the EWA
 * projection (means, quaternions, scales).  Gradients are written (not accumulated): d_means
 * (n x 3), d_quats (n x 4; through the normalisation), d_scales (n x 3), d_opacities (n),
 * d_colours (n x 3), df (n x d), dK, dV; every one of them is required.  loss_parts: device,
 * LATENTAM_FULL_LOSS_PARTS doubles.  Synchronises once for the pair count. */
LATENTAM_API latentam_status latentam_backward_full(latentam_ctx* ctx, const latentam_gaussians* g,
                                                    const float* colours, const float* f, int32_t d,
                                                    const latentam_camera* cam, const float* K, const float* V,
                                                    const float* V0, int32_t M, int32_t D, const void* F,
                                                    latentam_dtype F_dtype, const uint8_t* mask,
                                                    const float* image, const float* depth,
                                                    const latentam_loss_cfg* cfg, const latentam_image_cfg* icfg,
                                                    latentam_precision prec, double* loss_parts, float* d_means,
                                                    float* d_quats, float* d_scales, float* d_opacities,
                                                    float* d_colours, float* df, float* dK, float* dV,
                                                    latentam_stream stream);

/* ---- optimiser ----------------------------------------------------------------------- */

/* One Adam update of `count` tensors in a single launch: params[i], grads[i], m[i], v[i]
 * are device arrays of sizes[i] floats (host arrays of pointers); lrs[i] (host) is the
 * learning rate of tensor i.  Step number and betas from cfg. */
LATENTAM_API latentam_status latentam_adam(latentam_ctx* ctx, int32_t count, float* const* params,
                              const float* const* grads, float* const* m, float* const* v,
                              const int64_t* sizes, const float* lrs,
                              const latentam_adam_cfg* cfg, latentam_stream stream);

/* ---- the step (Algorithm 1, optimisation stages) ------------------------------------- */

/* One keyframe's state for latentam_step.  With n_masks > 0 the step is mask-pooled (see
 * latentam_pool_queries): the rendered queries are pooled per mask before the decode, F holds
 * one target per mask (n_masks x D) and mask one loss-set flag per mask; the query gradient
 * flows back to the pixels through the pooling's adjoint.  n_masks == 0 (the zero-initialised
 * struct) is the per-pixel step. */
typedef struct {
    latentam_gaussians gaussians;
    latentam_camera camera;
    const void* F;          /* H*W x D target features (n_masks x D when mask-pooled) */
    latentam_dtype F_dtype;
    const uint8_t* mask;    /* loss-set flags per pixel (per mask when mask-pooled), NULL = all */
    const int32_t* mask_offsets;  /* device, n_masks + 1 CSR offsets (mask-pooled only) */
    const int32_t* mask_pixels;   /* device, n_mask_entries pixel indices (mask-pooled only) */
    int64_t n_mask_entries;
    int32_t n_masks;        /* 0 = per-pixel targets */
} latentam_frame;

/* Learnable state: queries f (N x d) and dictionary K (M x d), V (M x D), the trust-region
 * centre V0 (M x D), and the Adam moments of each (same shapes).  tau > 0 selects the paper's
 * own parameterisation (Sec. III-B, the decode of latentam_decode_loss_bwd_paper with
 * temperature tau): K then holds the projection W (d x D, moments likewise) and V the atoms
 * D (M x D); tau = 0 (the zero-initialised struct) is the free-key decode with logit scale
 * cfg->logit_scale. */
typedef struct {
    float* f;
    float* K;
    float* V;
    const float* V0;
    float *m_f, *v_f, *m_K, *v_K, *m_V, *v_V;
    int32_t d, M, D;
    float tau;
} latentam_params;

/* `iters` iterations of: render (Q from f) -> decode + loss -> backward -> Adam on
 * (f if learn_f, K, V).  Projection and binning run once (the geometry is fixed during
 * the step).  With learn_f == 0 (Stage II) Q is rendered once and f is left untouched.
 * adam->step is the step number of the first update; it is incremented per iteration in
 * the caller's struct.  loss_host (host, nullable, LATENTAM_LOSS_PARTS doubles) receives
 * the loss of the LAST iteration (evaluated before its update); passing it synchronises
 * the stream at the end and then reports the context's device flags: LATENTAM_ERR_TIMEOUT
 * if a bounded wait of a tensor-core decode kernel gave up since they were last reported
 * (that loss is NaN), LATENTAM_ERR_NOT_FINITE if the loss or any gradient entry fed to Adam
 * was not finite (the update has been applied: parameters may then hold non-finite values).
 * Also synchronises once for the pair count (latentam_sort). */
LATENTAM_API latentam_status latentam_step(latentam_ctx* ctx, const latentam_frame* frame,
                              latentam_params* params, const latentam_loss_cfg* cfg,
                              latentam_adam_cfg* adam, int32_t iters, int32_t learn_f,
                              latentam_precision prec, double* loss_host, latentam_stream stream);

/* ---- batched step (Algorithm 1: the new keyframe plus B history keyframes) -------------- */

#define LATENTAM_MAX_BATCH 32

/* One keyframe of a batch: its Gaussians and camera, and the queries it renders.  Frames that
 * view the same map pass the same f (and the same Gaussians, N and moments): their query
 * gradients are summed before the single Adam update of f.  The mask fields are those of
 * latentam_frame (mask-pooled targets, see latentam_pool_queries); the batch is mask-pooled
 * when any frame has n_masks > 0, and then every frame contributes its n_masks pooled rows
 * (possibly none). */
typedef struct {
    latentam_gaussians gaussians;
    latentam_camera camera;
    float* f;     /* N x d */
    float* m_f;   /* Adam moments of f */
    float* v_f;
    const int32_t* mask_offsets;  /* device, n_masks + 1 CSR offsets (mask-pooled only) */
    const int32_t* mask_pixels;   /* device, n_mask_entries pixel indices */
    int64_t n_mask_entries;
    int32_t n_masks;
} latentam_batch_frame;

/* The dictionary shared by every frame: keys K (M x d), values V (M x D), trust-region centre
 * V0 (M x D) and the Adam moments of K and V; tau as in latentam_params (K = W, d x D, when
 * tau > 0). */
typedef struct {
    float* K;
    float* V;
    const float* V0;
    float *m_K, *v_K, *m_V, *v_V;
    int32_t d, M, D;
    float tau;
} latentam_dictionary;

/* `iters` iterations over a batch of n_frames (1..LATENTAM_MAX_BATCH) keyframes that share the
 * dictionary: every frame is projected and binned once (one synchronisation per frame for its
 * pair count), then each iteration renders every frame into one stacked query image, decodes
 * all stacked pixels in one call, back-propagates to every frame and takes one Adam step on
 * (each distinct f if learn_f, K, V).  The objective pools the loss-set pixels of all frames
 * (one |Omega|) and adds the trust-region term once.  F (sum_k H_k W_k x D, dtype F_dtype) and
 * mask (sum_k H_k W_k, NULL = all) hold the frames' targets concatenated in frame order; in a
 * mask-pooled batch they hold one row and one flag per mask (sum_k n_masks_k rows), the pooled
 * queries of every frame are stacked in frame order and decoded in one call.
 * adam->step and loss_host behave as in latentam_step. */
LATENTAM_API latentam_status latentam_step_batch(latentam_ctx* ctx, const latentam_batch_frame* frames,
                                                 int32_t n_frames, const void* F, latentam_dtype F_dtype,
                                                 const uint8_t* mask, latentam_dictionary* dict,
                                                 const latentam_loss_cfg* cfg, latentam_adam_cfg* adam,
                                                 int32_t iters, int32_t learn_f, latentam_precision prec,
                                                 double* loss_host, latentam_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* LATENTAM_H */
