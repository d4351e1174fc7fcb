/*
 * FP64 CPU oracle of the per-keyframe latent-feature optimisation step of LatentAM
 * (arxiv 2602.12314): query splatting (Sec. III-A/III-B, Eq. alpha_blending and
 * Eq. render_query), dictionary decode (Eq. dict_recon), feature objective with the
 * trust-region term (Eq. feat_loss, weighted by lambda_f of Eq. full_obj), its exact
 * gradients, and the optimiser step.
 *
 * TEST INFRASTRUCTURE ONLY.  Plain, slow, obviously correct; called by tests, by the
 * smoke check and by the CPU-baseline leg of the benchmark, never by the product path.
 * It shares no code with the CUDA library.  OpenMP (when enabled) only splits loops over
 * independent outputs; every output element is summed in the order written here.
 *
 * Readings of the paper (it defers the splat footprint to the 3DGS renderer it cites
 * and leaves several constants open); each is applied identically everywhere below:
 *  R1 footprint: EWA projection, Sigma' = J W Sigma W^T J^T + 0.3 I (pixel^2 dilation);
 *     alpha = min(0.99, o exp(-1/2 d^T Sigma'^-1 d)); a contribution with alpha < 1/255
 *     (or a positive exponent) is skipped; blending stops before a contribution that
 *     would take the transmittance below 1e-4; near plane z = 0.2 (camera field).
 *  R2 pixel centres sit at integer coordinates (x, y).
 *  R3 front-to-back order: the camera-space depth of the mean evaluated in binary32, every
 *     product and sum rounded to binary32 in the order ((R20 x + R21 y) + R22 z) + t2, is
 *     the sort key, and the near-plane test compares it with the binary32 z_near; equal keys
 *     are ordered by Gaussian index.  The order is thereby an exact function
 *     of the inputs, identical for every implementation that evaluates the key the same way.
 *  R4 an uncovered pixel renders Q_p = 0 (no background query).
 *  R5 decode with free keys K (M x d) and values V (M x D): S = c Q K^T, row softmax
 *     with the row maximum subtracted, Fhat = A V.
 *  R6 loss: cos term = mean over valid pixels of (1 - cos_p), cos_p =
 *     <Fhat_p, F_p> / max(|Fhat_p| |F_p|, 1e-8); L2 term = mean over valid pixels x D
 *     elements; trust-region term summed over atoms; all times lambda_f.
 *  R7 trust region on the value rows only; subgradient 0 at |V_j - V0_j| = delta.
 *  R8 optimiser: Adam with bias correction.
 */
#include "latentam_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_TILE 16

static const double ALPHA_MIN = 1.0 / 255.0;
static const double ALPHA_MAX = 0.99;
static const double T_MIN = 1e-4;
static const double DILATION = 0.3;
/* Relative half-widths of the bands around the thresholds alpha = 1/255 and T = 1e-4
 * inside which a float32 evaluation may legitimately decide the other way (alpha carries
 * a few 1e-6 relative error from the exponent; T compounds (1 - alpha) factors whose
 * relative error reaches 1e-4 for alpha near 0.99).  Pixels with a candidate inside a
 * band are flagged "ambiguous" for the parity tests. */
static const double AMB_TOL = 5e-5;
static const double AMB_TOL_T = 1e-3;
/* Same idea for the tile rectangle edges (pixels). */
static const double RECT_TOL_PX = 1e-3;

/* Sort key of reading R3: the camera depth of the mean in binary32, every operation rounded
 * to binary32 in the order ((R20 x + R21 y) + R22 z) + t2 (this file is compiled without FMA
 * contraction).  The camera and the means are binary32 values held in doubles. */
static float depth_key32(const double* W, const double* p, double t2) {
    const float a = (float)W[6] * (float)p[0];
    const float b = (float)W[7] * (float)p[1];
    const float c = (float)W[8] * (float)p[2];
    const float ab = a + b;
    const float abc = ab + c;
    return abc + (float)t2;
}
/* The key as the lists use it: binary32 (depth[] from orc_project already holds binary32 values). */
static double depth_key(double z) { return (double)(float)z; }

/* ------------------------------------------------------------------------------------ */
/* Projection                                                                            */
/* ------------------------------------------------------------------------------------ */

/* Tiles [t0, t1) holding the pixel centres x in [lo, hi] of a row of npix pixels. */
static void tile_span(double lo, double hi, int npix, int* t0, int* t1) {
    double plo = ceil(lo), phi = floor(hi);
    if (plo < 0.0) plo = 0.0;
    if (phi > (double)(npix - 1)) phi = (double)(npix - 1);
    if (!(plo <= phi)) {
        *t0 = 0;
        *t1 = 0;
        return;
    }
    *t0 = (int)plo / ORC_TILE;
    *t1 = (int)phi / ORC_TILE + 1;
}

static void rect_of(double mx, double my, double ex, double ey, const orc_camera* cam, int r[4]) {
    int x0, x1, y0, y1;
    tile_span(mx - ex, mx + ex, cam->width, &x0, &x1);
    tile_span(my - ey, my + ey, cam->height, &y0, &y1);
    if (x0 == x1 || y0 == y1) {
        r[0] = r[1] = r[2] = r[3] = 0;
        return;
    }
    r[0] = x0;
    r[1] = y0;
    r[2] = x1;
    r[3] = y1;
}

void orc_project(int64_t N, const double* means, const double* quats, const double* scales,
                 const double* opacities, const orc_camera* cam,
                 double* xy, double* cov2d, double* conic, double* depth, double* extent,
                 int32_t* rect, int32_t* visible, int32_t* rect_ambiguous) {
    const double* W = cam->R;
    for (int64_t i = 0; i < N; ++i) {
        const double* p = means + 3 * i;
        double x = W[0] * p[0] + W[1] * p[1] + W[2] * p[2] + cam->t[0];
        double y = W[3] * p[0] + W[4] * p[1] + W[5] * p[2] + cam->t[1];
        double z = W[6] * p[0] + W[7] * p[1] + W[8] * p[2] + cam->t[2];
        double o = opacities[i];
        const float zk = depth_key32(W, p, cam->t[2]);
        depth[i] = (double)zk;
        visible[i] = 0;
        rect_ambiguous[i] = 0;
        for (int k = 0; k < 4; ++k) rect[4 * i + k] = 0;
        for (int k = 0; k < 3; ++k) cov2d[3 * i + k] = conic[3 * i + k] = 0.0;
        xy[2 * i] = xy[2 * i + 1] = extent[2 * i] = extent[2 * i + 1] = 0.0;
        if (!(zk > (float)cam->z_near) || o < ALPHA_MIN) continue;

        /* Rotation of the primitive from its unit quaternion q = (w, x, y, z). */
        const double* q = quats + 4 * i;
        double qn = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
        double qw = q[0] / qn, qx = q[1] / qn, qy = q[2] / qn, qz = q[3] / qn;
        double Rq[9] = {1 - 2 * (qy * qy + qz * qz), 2 * (qx * qy - qw * qz), 2 * (qx * qz + qw * qy),
                        2 * (qx * qy + qw * qz), 1 - 2 * (qx * qx + qz * qz), 2 * (qy * qz - qw * qx),
                        2 * (qx * qz - qw * qy), 2 * (qy * qz + qw * qx), 1 - 2 * (qx * qx + qy * qy)};
        /* Sigma = Rq S S^T Rq^T with S = diag(scale). */
        const double* s = scales + 3 * i;
        double Sig[9];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                double acc = 0.0;
                for (int k = 0; k < 3; ++k) acc += Rq[3 * a + k] * s[k] * s[k] * Rq[3 * b + k];
                Sig[3 * a + b] = acc;
            }
        /* Jacobian of the pinhole projection at the camera-space mean, times W. */
        double J[6] = {cam->fx / z, 0.0, -cam->fx * x / (z * z), 0.0, cam->fy / z, -cam->fy * y / (z * z)};
        double T[6];
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 3; ++b) {
                double acc = 0.0;
                for (int k = 0; k < 3; ++k) acc += J[3 * a + k] * W[3 * k + b];
                T[3 * a + b] = acc;
            }
        double C[4];
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) {
                double acc = 0.0;
                for (int k = 0; k < 3; ++k)
                    for (int l = 0; l < 3; ++l) acc += T[3 * a + k] * Sig[3 * k + l] * T[3 * b + l];
                C[2 * a + b] = acc;
            }
        double ca = C[0] + DILATION, cb = 0.5 * (C[1] + C[2]), cc = C[3] + DILATION;
        double det = ca * cc - cb * cb;
        if (!(det > 0.0)) continue;
        double mx = cam->fx * x / z + cam->cx;
        double my = cam->fy * y / z + cam->cy;
        /* Every pixel with alpha >= 1/255 satisfies d^T Sigma'^-1 d <= 2 ln(255 o), whose
         * axis-aligned extent is sqrt(2 ln(255 o) Sigma'_xx) and sqrt(... Sigma'_yy). */
        double mmax = 2.0 * log(255.0 * o);
        if (mmax < 0.0) mmax = 0.0;
        double ex = sqrt(mmax * ca), ey = sqrt(mmax * cc);
        xy[2 * i] = mx;
        xy[2 * i + 1] = my;
        cov2d[3 * i] = ca;
        cov2d[3 * i + 1] = cb;
        cov2d[3 * i + 2] = cc;
        conic[3 * i] = cc / det;
        conic[3 * i + 1] = -cb / det;
        conic[3 * i + 2] = ca / det;
        extent[2 * i] = ex;
        extent[2 * i + 1] = ey;
        int r[4];
        rect_of(mx, my, ex, ey, cam, r);
        for (int k = 0; k < 4; ++k) rect[4 * i + k] = r[k];
        visible[i] = 1;
        /* Would a float32 evaluation of the edges land in other tiles? */
        for (int sx = -1; sx <= 1; sx += 2)
            for (int sy = -1; sy <= 1; sy += 2) {
                int r2[4];
                rect_of(mx + sx * RECT_TOL_PX, my + sy * RECT_TOL_PX, ex + RECT_TOL_PX, ey + RECT_TOL_PX, cam, r2);
                int r3[4];
                rect_of(mx + sx * RECT_TOL_PX, my + sy * RECT_TOL_PX, ex > RECT_TOL_PX ? ex - RECT_TOL_PX : 0.0,
                        ey > RECT_TOL_PX ? ey - RECT_TOL_PX : 0.0, cam, r3);
                for (int k = 0; k < 4; ++k)
                    if (r2[k] != r[k] || r3[k] != r[k]) rect_ambiguous[i] = 1;
            }
    }
}

/* ------------------------------------------------------------------------------------ */
/* Blending                                                                              */
/* ------------------------------------------------------------------------------------ */

typedef struct {
    double depth;
    int32_t id;
    double alpha_raw; /* o exp(power) before the 0.99 clamp */
} cand_t;

static int cand_cmp(const void* a, const void* b) {
    const cand_t* x = (const cand_t*)a;
    const cand_t* y = (const cand_t*)b;
    if (x->depth < y->depth) return -1;
    if (x->depth > y->depth) return 1;
    return (x->id > y->id) - (x->id < y->id);
}

/* o exp(-1/2 d^T conic d) at pixel centre (px, py); *skip set when the exponent is positive. */
static double alpha_raw_at(const double* xy, const double* conic, double o, double px, double py, int* skip) {
    double dx = xy[0] - px, dy = xy[1] - py;
    double power = -0.5 * (conic[0] * dx * dx + conic[2] * dy * dy) - conic[1] * dx * dy;
    *skip = power > 0.0;
    return o * exp(power);
}

/* Is this candidate kept for the ambiguity bookkeeping (alpha near or above 1/255)? */
static int is_candidate(double a, int skip) { return !skip && a >= ALPHA_MIN * (1.0 - AMB_TOL); }

/* Front-to-back blend of one pixel over its candidates sorted by (depth, index).
 * Returns the number of contributions; if df != NULL accumulates w * dQ into df instead
 * of writing Q. */
static int blend_pixel(int d, const cand_t* c, int64_t nc, const double* f, double* Q, double* T_out,
                       uint8_t* amb, const double* dQ, double* df) {
    double T = 1.0;
    int n = 0;
    uint8_t a = 0;
    if (Q)
        for (int k = 0; k < d; ++k) Q[k] = 0.0;
    for (int64_t e = 0; e < nc; ++e) {
        if (fabs(c[e].alpha_raw * 255.0 - 1.0) < AMB_TOL) a = 1;
        if (c[e].alpha_raw < ALPHA_MIN) continue;
        double alpha = c[e].alpha_raw < ALPHA_MAX ? c[e].alpha_raw : ALPHA_MAX;
        double test_T = T * (1.0 - alpha);
        if (fabs(test_T / T_MIN - 1.0) < AMB_TOL_T) a = 1;
        if (test_T < T_MIN) break;
        double w = alpha * T;
        const double* fi = f ? f + (int64_t)c[e].id * d : NULL;
        if (Q)
            for (int k = 0; k < d; ++k) Q[k] += w * fi[k];
        if (df) {
            double* g = df + (int64_t)c[e].id * d;
            for (int k = 0; k < d; ++k) g[k] += w * dQ[k];
        }
        T = test_T;
        ++n;
    }
    if (T_out) *T_out = T;
    if (amb) *amb = a;
    return n;
}

typedef struct {
    int64_t* off; /* n_pix + 1 */
    cand_t* c;
} frame_lists;

/* Candidate lists of every pixel: all visible Gaussians whose alpha at the pixel is at
 * least 1/255 (slightly below, for the ambiguity flags), sorted by (depth, index).  Only
 * pixels inside each Gaussian's extent box are visited, which by the bound in
 * orc_project (widened to the lower candidate threshold) loses none of them. */
static int build_frame_lists(int64_t N, const double* xy, const double* conic, const double* opac,
                             const double* depth, const int32_t* visible, const double* cov2d,
                             const orc_camera* cam, frame_lists* out) {
    const int W = cam->width, H = cam->height;
    const int64_t n_pix = (int64_t)W * H;
    int64_t* cnt = (int64_t*)calloc((size_t)n_pix + 1, sizeof(int64_t));
    if (!cnt) return -1;
    for (int pass = 0; pass < 2; ++pass) {
        int64_t* pos = NULL;
        if (pass == 1) {
            pos = (int64_t*)malloc(sizeof(int64_t) * (size_t)n_pix);
            if (!pos) return -1;
            memcpy(pos, out->off, sizeof(int64_t) * (size_t)n_pix);
        }
#pragma omp parallel for schedule(dynamic, 256)
        for (int64_t g = 0; g < N; ++g) {
            if (!visible[g]) continue;
            double o = opac[g];
            double mm = 2.0 * log(255.0 * o / (1.0 - AMB_TOL));
            if (mm < 0.0) mm = 0.0;
            double ex = sqrt(mm * cov2d[3 * g]), ey = sqrt(mm * cov2d[3 * g + 2]);
            double mx = xy[2 * g], my = xy[2 * g + 1];
            double x0 = ceil(mx - ex), x1 = floor(mx + ex), y0 = ceil(my - ey), y1 = floor(my + ey);
            if (x0 < 0) x0 = 0;
            if (y0 < 0) y0 = 0;
            if (x1 > W - 1) x1 = W - 1;
            if (y1 > H - 1) y1 = H - 1;
            if (x0 > x1 || y0 > y1) continue;
            for (int y = (int)y0; y <= (int)y1; ++y)
                for (int x = (int)x0; x <= (int)x1; ++x) {
                    int skip;
                    double a = alpha_raw_at(xy + 2 * g, conic + 3 * g, o, (double)x, (double)y, &skip);
                    if (!is_candidate(a, skip)) continue;
                    int64_t p = (int64_t)y * W + x;
                    if (pass == 0) {
#pragma omp atomic
                        cnt[p]++;
                    } else {
                        int64_t at;
#pragma omp atomic capture
                        at = pos[p]++;
                        out->c[at].depth = depth_key(depth[g]);
                        out->c[at].id = (int32_t)g;
                        out->c[at].alpha_raw = a;
                    }
                }
        }
        if (pass == 0) {
            out->off = (int64_t*)malloc(sizeof(int64_t) * ((size_t)n_pix + 1));
            if (!out->off) return -1;
            int64_t run = 0;
            for (int64_t p = 0; p < n_pix; ++p) {
                out->off[p] = run;
                run += cnt[p];
            }
            out->off[n_pix] = run;
            out->c = (cand_t*)malloc(sizeof(cand_t) * (size_t)(run > 0 ? run : 1));
            if (!out->c) return -1;
        } else {
            free(pos);
        }
    }
    free(cnt);
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t p = 0; p < n_pix; ++p)
        qsort(out->c + out->off[p], (size_t)(out->off[p + 1] - out->off[p]), sizeof(cand_t), cand_cmp);
    return 0;
}

int orc_render_frame(int64_t N, int d, const double* xy, const double* conic,
                     const double* opacities, const double* depth, const int32_t* visible,
                     const double* cov2d, const double* f, const orc_camera* cam,
                     double* Q, double* T_final, int32_t* n_contrib, uint8_t* ambiguous) {
    frame_lists L = {0, 0};
    if (build_frame_lists(N, xy, conic, opacities, depth, visible, cov2d, cam, &L)) return -1;
    const int64_t n_pix = (int64_t)cam->width * cam->height;
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t p = 0; p < n_pix; ++p)
        n_contrib[p] = blend_pixel(d, L.c + L.off[p], L.off[p + 1] - L.off[p], f, Q + p * d, T_final + p,
                                   ambiguous + p, NULL, NULL);
    free(L.off);
    free(L.c);
    return 0;
}

int orc_render_frame_bwd(int64_t N, int d, const double* xy, const double* conic,
                         const double* opacities, const double* depth, const int32_t* visible,
                         const double* cov2d, const orc_camera* cam, const double* dQ, double* df) {
    frame_lists L = {0, 0};
    if (build_frame_lists(N, xy, conic, opacities, depth, visible, cov2d, cam, &L)) return -1;
    const int64_t n_pix = (int64_t)cam->width * cam->height;
    memset(df, 0, sizeof(double) * (size_t)N * d);
    for (int64_t p = 0; p < n_pix; ++p)
        blend_pixel(d, L.c + L.off[p], L.off[p + 1] - L.off[p], NULL, NULL, NULL, NULL, dQ + p * d, df);
    free(L.off);
    free(L.c);
    return 0;
}

void orc_render_pixels(int64_t N, int d, const double* xy, const double* conic,
                       const double* opacities, const double* depth, const int32_t* visible,
                       const double* f, int64_t n_pix, const int32_t* px, const int32_t* py,
                       double* Q, double* T_final, int32_t* n_contrib, uint8_t* ambiguous) {
#pragma omp parallel
    {
        int64_t cap = 1024;
        cand_t* c = (cand_t*)malloc(sizeof(cand_t) * (size_t)cap);
#pragma omp for schedule(dynamic, 4)
        for (int64_t k = 0; k < n_pix; ++k) {
            int64_t nc = 0;
            for (int64_t g = 0; g < N; ++g) {
                if (!visible[g]) continue;
                int skip;
                double a = alpha_raw_at(xy + 2 * g, conic + 3 * g, opacities[g], (double)px[k], (double)py[k], &skip);
                if (!is_candidate(a, skip)) continue;
                if (nc == cap) {
                    cap *= 2;
                    c = (cand_t*)realloc(c, sizeof(cand_t) * (size_t)cap);
                }
                c[nc].depth = depth_key(depth[g]);
                c[nc].id = (int32_t)g;
                c[nc].alpha_raw = a;
                ++nc;
            }
            qsort(c, (size_t)nc, sizeof(cand_t), cand_cmp);
            n_contrib[k] = blend_pixel(d, c, nc, f, Q + k * d, T_final + k, ambiguous + k, NULL, NULL);
        }
        free(c);
    }
}

/* ------------------------------------------------------------------------------------ */
/* Tiled path                                                                            */
/* ------------------------------------------------------------------------------------ */

typedef struct {
    double depth;
    int32_t id;
} tile_ent;

static int tile_ent_cmp(const void* a, const void* b) {
    const tile_ent* x = (const tile_ent*)a;
    const tile_ent* y = (const tile_ent*)b;
    if (x->depth < y->depth) return -1;
    if (x->depth > y->depth) return 1;
    return (x->id > y->id) - (x->id < y->id);
}

int orc_tile_lists(int64_t N, const double* depth, const int32_t* visible, const int32_t* rect,
                   const orc_camera* cam, int64_t capacity, int64_t* num_pairs,
                   int64_t* tile_offsets, int32_t* ids) {
    const int tx = (cam->width + ORC_TILE - 1) / ORC_TILE, ty = (cam->height + ORC_TILE - 1) / ORC_TILE;
    const int64_t nt = (int64_t)tx * ty;
    int64_t P = 0;
    for (int64_t g = 0; g < N; ++g)
        if (visible[g]) P += (int64_t)(rect[4 * g + 2] - rect[4 * g]) * (rect[4 * g + 3] - rect[4 * g + 1]);
    *num_pairs = P;
    if (!ids || capacity < P) return 0;
    int64_t* cnt = (int64_t*)calloc((size_t)nt, sizeof(int64_t));
    tile_ent* e = (tile_ent*)malloc(sizeof(tile_ent) * (size_t)(P > 0 ? P : 1));
    if (!cnt || !e) return -1;
    for (int64_t g = 0; g < N; ++g) {
        if (!visible[g]) continue;
        for (int y = rect[4 * g + 1]; y < rect[4 * g + 3]; ++y)
            for (int x = rect[4 * g]; x < rect[4 * g + 2]; ++x) cnt[(int64_t)y * tx + x]++;
    }
    int64_t run = 0;
    for (int64_t t = 0; t < nt; ++t) {
        tile_offsets[t] = run;
        run += cnt[t];
        cnt[t] = tile_offsets[t];
    }
    tile_offsets[nt] = run;
    for (int64_t g = 0; g < N; ++g) {
        if (!visible[g]) continue;
        for (int y = rect[4 * g + 1]; y < rect[4 * g + 3]; ++y)
            for (int x = rect[4 * g]; x < rect[4 * g + 2]; ++x) {
                int64_t at = cnt[(int64_t)y * tx + x]++;
                e[at].depth = depth_key(depth[g]);
                e[at].id = (int32_t)g;
            }
    }
    for (int64_t t = 0; t < nt; ++t)
        qsort(e + tile_offsets[t], (size_t)(tile_offsets[t + 1] - tile_offsets[t]), sizeof(tile_ent), tile_ent_cmp);
    for (int64_t k = 0; k < P; ++k) ids[k] = e[k].id;
    free(cnt);
    free(e);
    return 0;
}

void orc_render_tiled(int d, const double* xy, const double* conic, const double* opacities,
                      const double* f, const orc_camera* cam, const int64_t* tile_offsets,
                      const int32_t* ids, double* Q, double* T_final, int32_t* n_contrib) {
    const int W = cam->width, H = cam->height;
    const int tx = (W + ORC_TILE - 1) / ORC_TILE;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t p = 0; p < (int64_t)W * H; ++p) {
        int x = (int)(p % W), y = (int)(p / W);
        int64_t t = (int64_t)(y / ORC_TILE) * tx + x / ORC_TILE;
        double* q = Q + p * d;
        for (int k = 0; k < d; ++k) q[k] = 0.0;
        double T = 1.0;
        int n = 0;
        for (int64_t e = tile_offsets[t]; e < tile_offsets[t + 1]; ++e) {
            int32_t g = ids[e];
            int skip;
            double a = alpha_raw_at(xy + 2 * g, conic + 3 * g, opacities[g], (double)x, (double)y, &skip);
            if (skip || a < ALPHA_MIN) continue;
            double alpha = a < ALPHA_MAX ? a : ALPHA_MAX;
            double test_T = T * (1.0 - alpha);
            if (test_T < T_MIN) break;
            for (int k = 0; k < d; ++k) q[k] += alpha * T * f[(int64_t)g * d + k];
            T = test_T;
            ++n;
        }
        T_final[p] = T;
        n_contrib[p] = n;
    }
}

/* ------------------------------------------------------------------------------------ */
/* Decode, loss, gradients                                                               */
/* ------------------------------------------------------------------------------------ */

void orc_decode(int64_t n, int d, int M, int D, const double* Q, const double* K, const double* V,
                double c, double* S, double* A, double* Fhat) {
#pragma omp parallel
    {
        double* s = (double*)malloc(sizeof(double) * (size_t)M);
#pragma omp for schedule(static)
        for (int64_t p = 0; p < n; ++p) {
            const double* q = Q + p * d;
            for (int j = 0; j < M; ++j) {
                double acc = 0.0;
                for (int k = 0; k < d; ++k) acc += q[k] * K[(int64_t)j * d + k];
                s[j] = c * acc;
            }
            double mx = s[0];
            for (int j = 1; j < M; ++j)
                if (s[j] > mx) mx = s[j];
            double sum = 0.0;
            for (int j = 0; j < M; ++j) sum += exp(s[j] - mx);
            double* a = A + p * M;
            for (int j = 0; j < M; ++j) {
                a[j] = exp(s[j] - mx) / sum;
                if (S) S[p * M + j] = s[j];
            }
            double* fh = Fhat + p * D;
            for (int k = 0; k < D; ++k) fh[k] = 0.0;
            for (int j = 0; j < M; ++j) {
                const double* v = V + (int64_t)j * D;
                for (int k = 0; k < D; ++k) fh[k] += a[j] * v[k];
            }
        }
        free(s);
    }
}

static int64_t count_valid(int64_t n, const uint8_t* mask) {
    int64_t nv = 0;
    for (int64_t p = 0; p < n; ++p) nv += mask[p] != 0;
    return nv;
}

void orc_loss(int64_t n, int M, int D, const double* Fhat, const double* F, const uint8_t* mask,
              const double* V, const double* V0, const orc_loss_cfg* cfg, double* parts,
              double* cos_p) {
    int64_t nv = count_valid(n, mask);
    double sum_cos = 0.0, sum_l2 = 0.0;
    for (int64_t p = 0; p < n; ++p) {
        const double* a = Fhat + p * D;
        const double* b = F + p * D;
        double dot = 0.0, na = 0.0, nb = 0.0, e = 0.0;
        for (int k = 0; k < D; ++k) {
            dot += a[k] * b[k];
            na += a[k] * a[k];
            nb += b[k] * b[k];
            e += (a[k] - b[k]) * (a[k] - b[k]);
        }
        double den = sqrt(na) * sqrt(nb);
        double cs = dot / (den > 1e-8 ? den : 1e-8);
        if (cos_p) cos_p[p] = cs;
        if (!mask[p]) continue;
        sum_cos += 1.0 - cs;
        sum_l2 += e;
    }
    double tr = 0.0;
    for (int j = 0; j < M; ++j) {
        double s2 = 0.0;
        for (int k = 0; k < D; ++k) {
            double t = V[(int64_t)j * D + k] - V0[(int64_t)j * D + k];
            s2 += t * t;
        }
        double r = sqrt(s2) - cfg->delta;
        if (r > 0.0) tr += r;
    }
    double lcos = nv ? sum_cos / (double)nv : 0.0;
    double l2 = nv ? sum_l2 / ((double)nv * D) : 0.0;
    parts[0] = lcos;
    parts[1] = l2;
    parts[2] = tr;
    parts[3] = cfg->lambda_f * (cfg->lambda_cos * lcos + cfg->lambda_2 * l2 + cfg->lambda_D * tr);
    parts[4] = (double)nv;
}

void orc_backward(int64_t n, int d, int M, int D, const double* Q, const double* K,
                  const double* V, const double* V0, const double* A, const double* Fhat,
                  const double* F, const uint8_t* mask, const orc_loss_cfg* cfg,
                  double* dQ, double* dK, double* dV) {
    const double c = cfg->logit_scale;
    int64_t nv = count_valid(n, mask);
    double* dF = (double*)calloc((size_t)n * D, sizeof(double));
    double* dS = (double*)calloc((size_t)n * M, sizeof(double));
    /* dL/dFhat_p for p in the loss set (zero elsewhere). */
    if (nv > 0) {
        const double scale = cfg->lambda_f / (double)nv;
#pragma omp parallel for schedule(static)
        for (int64_t p = 0; p < n; ++p) {
            if (!mask[p]) continue;
            const double* a = Fhat + p * D;
            const double* b = F + p * D;
            double dot = 0.0, na = 0.0, nb = 0.0;
            for (int k = 0; k < D; ++k) {
                dot += a[k] * b[k];
                na += a[k] * a[k];
                nb += b[k] * b[k];
            }
            double nha = sqrt(na), nhb = sqrt(nb);
            double den = nha * nhb;
            for (int k = 0; k < D; ++k) {
                double dcos = den > 1e-8 ? b[k] / den - (dot / den) * a[k] / na : b[k] / 1e-8;
                dF[p * D + k] = scale * (-cfg->lambda_cos * dcos + (2.0 * cfg->lambda_2 / D) * (a[k] - b[k]));
            }
        }
    }
    /* Through Fhat = A V and the row softmax. */
#pragma omp parallel
    {
        double* dA = (double*)malloc(sizeof(double) * (size_t)M);
#pragma omp for schedule(static)
        for (int64_t p = 0; p < n; ++p) {
            const double* g = dF + p * D;
            const double* a = A + p * M;
            double rowdot = 0.0;
            for (int j = 0; j < M; ++j) {
                double acc = 0.0;
                for (int k = 0; k < D; ++k) acc += g[k] * V[(int64_t)j * D + k];
                dA[j] = acc;
                rowdot += a[j] * acc;
            }
            for (int j = 0; j < M; ++j) dS[p * M + j] = a[j] * (dA[j] - rowdot);
            for (int k = 0; k < d; ++k) {
                double acc = 0.0;
                for (int j = 0; j < M; ++j) acc += dS[p * M + j] * K[(int64_t)j * d + k];
                dQ[p * d + k] = c * acc;
            }
        }
        free(dA);
    }
    /* dK = c dS^T Q and dV = A^T dFhat, summed over pixels in ascending order; each
     * thread owns a band of atoms (dK) and a band of value columns (dV). */
    memset(dK, 0, sizeof(double) * (size_t)M * d);
    memset(dV, 0, sizeof(double) * (size_t)M * D);
#pragma omp parallel
    {
        int nth = 1, tid = 0;
#ifdef _OPENMP
        nth = omp_get_num_threads();
        tid = omp_get_thread_num();
#endif
        int j0 = (int)((int64_t)M * tid / nth), j1 = (int)((int64_t)M * (tid + 1) / nth);
        int k0 = (int)((int64_t)D * tid / nth), k1 = (int)((int64_t)D * (tid + 1) / nth);
        for (int64_t p = 0; p < n; ++p) {
            const double* q = Q + p * d;
            for (int j = j0; j < j1; ++j) {
                double s = dS[p * M + j];
                double* out = dK + (int64_t)j * d;
                for (int k = 0; k < d; ++k) out[k] += s * q[k];
            }
            const double* a = A + p * M;
            const double* g = dF + p * D;
            for (int j = 0; j < M; ++j) {
                double aj = a[j];
                double* out = dV + (int64_t)j * D;
                for (int k = k0; k < k1; ++k) out[k] += aj * g[k];
            }
        }
    }
    for (int64_t e = 0; e < (int64_t)M * d; ++e) dK[e] *= c;
    for (int j = 0; j < M; ++j) {
        double s2 = 0.0;
        for (int k = 0; k < D; ++k) {
            double t = V[(int64_t)j * D + k] - V0[(int64_t)j * D + k];
            s2 += t * t;
        }
        double nrm = sqrt(s2);
        if (nrm > cfg->delta) {
            double w = cfg->lambda_f * cfg->lambda_D / nrm;
            for (int k = 0; k < D; ++k) dV[(int64_t)j * D + k] += w * (V[(int64_t)j * D + k] - V0[(int64_t)j * D + k]);
        }
    }
    free(dF);
    free(dS);
}

void orc_adam(int64_t len, double* param, const double* grad, double* m, double* v, int step,
              double lr, double beta1, double beta2, double eps) {
    double bc1 = 1.0 - pow(beta1, step), bc2 = 1.0 - pow(beta2, step);
    for (int64_t i = 0; i < len; ++i) {
        m[i] = beta1 * m[i] + (1.0 - beta1) * grad[i];
        v[i] = beta2 * v[i] + (1.0 - beta2) * grad[i] * grad[i];
        double mh = m[i] / bc1, vh = v[i] / bc2;
        param[i] -= lr * mh / (sqrt(vh) + eps);
    }
}
