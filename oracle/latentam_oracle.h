/*
 * FP64 CPU oracle for the per-keyframe latent-feature optimisation step of LatentAM
 * (arxiv 2602.12314).  TEST INFRASTRUCTURE ONLY: it is called by the test suite, by the
 * smoke check and by the CPU-baseline leg of the benchmark, never by the product path.
 * It shares no code, header, table or constant generator with the CUDA library.
 *
 * Every function works in double precision on plain row-major arrays.  Readings of the
 * paper where it is silent (splat footprint, thresholds, loss normalisation, ...) are
 * listed next to each function in latentam_oracle.c.
 */
#ifndef LATENTAM_ORACLE_H
#define LATENTAM_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Pinhole camera: p_cam = R p_world + t (R row-major 3x3); x right, y down, z forward;
 * pixel (x, y) has its centre at integer coordinates. */
typedef struct {
    double R[9];
    double t[3];
    double fx, fy, cx, cy;
    double z_near;
    int32_t width, height;
} orc_camera;

/* Weights of the feature objective, Eq. (feat_loss) scaled by lambda_f of Eq. (full_obj),
 * and the logit scale c of the decode (1/sqrt(d) for free keys, 1/tau in the paper's
 * cosine form). */
typedef struct {
    double lambda_f, lambda_cos, lambda_2, lambda_D, delta;
    double logit_scale;
} orc_loss_cfg;

/* Per-Gaussian projection (Sec. III-A; EWA footprint of the 3DGS renderer it cites). */
void orc_project(int64_t N, const double* means, const double* quats, const double* scales,
                 const double* opacities, const orc_camera* cam,
                 double* xy, double* cov2d, double* conic, double* depth, double* extent,
                 int32_t* rect, int32_t* visible, int32_t* rect_ambiguous);

/* Untiled query rendering, Eq. (alpha_blending) with f_i in place of c_i = Eq. (render_query),
 * over the whole frame.  Q: (H*W, d); T_final, n_contrib, ambiguous: (H*W). */
int orc_render_frame(int64_t N, int d, const double* xy, const double* conic,
                     const double* opacities, const double* depth, const int32_t* visible,
                     const double* cov2d, const double* f, const orc_camera* cam,
                     double* Q, double* T_final, int32_t* n_contrib, uint8_t* ambiguous);

/* Backward of orc_render_frame with respect to the queries: df_i = sum_p w_ip dQ_p. */
int orc_render_frame_bwd(int64_t N, int d, const double* xy, const double* conic,
                         const double* opacities, const double* depth, const int32_t* visible,
                         const double* cov2d, const orc_camera* cam, const double* dQ, double* df);

/* Same blend for a list of pixels, each checked against all N Gaussians (brute force). */
void orc_render_pixels(int64_t N, int d, const double* xy, const double* conic,
                       const double* opacities, const double* depth, const int32_t* visible,
                       const double* f, int64_t n_pix, const int32_t* px, const int32_t* py,
                       double* Q, double* T_final, int32_t* n_contrib, uint8_t* ambiguous);

/* Per-tile lists (16x16 tiles) from the projected rectangles, each sorted by (depth, index).
 * With ids == NULL or capacity too small, only *num_pairs is written. */
int orc_tile_lists(int64_t N, const double* depth, const int32_t* visible, const int32_t* rect,
                   const orc_camera* cam, int64_t capacity, int64_t* num_pairs,
                   int64_t* tile_offsets, int32_t* ids);

/* Tiled blend over those lists (the second, independent path of the renderer). */
void orc_render_tiled(int d, const double* xy, const double* conic, const double* opacities,
                      const double* f, const orc_camera* cam, const int64_t* tile_offsets,
                      const int32_t* ids, double* Q, double* T_final, int32_t* n_contrib);

/* Dictionary decode, Eq. (dict_recon) with free keys: S = c Q K^T, A = softmax_rows(S), Fhat = A V. */
void orc_decode(int64_t n, int d, int M, int D, const double* Q, const double* K, const double* V,
                double c, double* S, double* A, double* Fhat);

/* Feature objective lambda_f * L_f, Eq. (feat_loss) and (full_obj).
 * parts = {mean_cos_term, mean_l2_term, tr_sum, total, n_valid}; cos_p (nullable): per pixel. */
void orc_loss(int64_t n, int M, int D, const double* Fhat, const double* F, const uint8_t* mask,
              const double* V, const double* V0, const orc_loss_cfg* cfg, double* parts,
              double* cos_p);

/* Exact gradients of orc_loss(orc_decode(Q, K, V)) with respect to Q, K and V. */
void orc_backward(int64_t n, int d, int M, int D, const double* Q, const double* K,
                  const double* V, const double* V0, const double* A, const double* Fhat,
                  const double* F, const uint8_t* mask, const orc_loss_cfg* cfg,
                  double* dQ, double* dK, double* dV);

/* One bias-corrected Adam step on len parameters (step = 1 for the first update). */
void orc_adam(int64_t len, double* param, const double* grad, double* m, double* v, int step,
              double lr, double beta1, double beta2, double eps);

#ifdef __cplusplus
}
#endif
#endif
