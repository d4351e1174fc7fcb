// Photometric and depth losses of the full Stage I objective (Eq. rgb_loss, Eq. depth_loss,
// Eq. full_obj) with their image gradients, and the backward of the EWA projection from the
// screen-space gradients to the Gaussians' means, orientations and scales.
//
// L_rgb = lambda_I1 mean|I_hat - I| + lambda_I2 (1 - mean SSIM(I_hat, I)): SSIM per channel with
// an 11 x 11 Gaussian window (sigma 1.5, zero padding, C1 = 0.01^2, C2 = 0.03^2), evaluated by
// separable blurs.  With m = blur(x), e_xx = blur(x^2), e_xy = blur(x y) the gradient is
//   dL_ssim/dx = -(1/N) (blur(ds/dm) + 2 x blur(ds/de_xx) + y blur(ds/de_xy)),
// the blur being its own adjoint (a symmetric window, zero outside the image).
// L_d = mean over pixels with an observed depth of |Z_hat - Z|.
#include <math.h>

#include "internal.cuh"

namespace lat {
namespace {

constexpr int kWin = 11, kHalf = 5;
__constant__ float c_win[kWin];
constexpr float kC1 = 0.01f * 0.01f, kC2 = 0.03f * 0.03f;

__device__ __forceinline__ double block_sum_d(double v, double* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[k];
    __syncthreads();
    return s;
}

// Horizontal pass of the five moments of each channel: out[(k * 3 + ch) * n + p], k = x, y,
// x^2, y^2, x y.  x = rendered image, y = observed image (both n x 3 interleaved).
__global__ void ssim_moments_h(const float* __restrict__ X, const float* __restrict__ Y, int W, int H,
                               float* __restrict__ out) {
    const int64_t n = (int64_t)W * H;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 3 * n) return;
    const int ch = (int)(i / n);
    const int64_t p = i % n;
    const int py = (int)(p / W), px = (int)(p % W);
    float s[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    for (int k = -kHalf; k <= kHalf; ++k) {
        const int x = px + k;
        if (x < 0 || x >= W) continue;
        const int64_t q = (int64_t)py * W + x;
        const float a = X[3 * q + ch], b = Y[3 * q + ch], w = c_win[k + kHalf];
        s[0] += w * a;
        s[1] += w * b;
        s[2] += w * a * a;
        s[3] += w * b * b;
        s[4] += w * a * b;
    }
#pragma unroll
    for (int k = 0; k < 5; ++k) out[((int64_t)k * 3 + ch) * n + p] = s[k];
}

// Vertical pass, the SSIM map and the partial derivatives ds/dm_x, ds/de_xx, ds/de_xy
// (written to dpart[(k * 3 + ch) * n + p]); acc[1] += sum of SSIM values.
__global__ void __launch_bounds__(256) ssim_map_v(const float* __restrict__ hm, int W, int H,
                                                  float* __restrict__ dpart, double* __restrict__ acc) {
    __shared__ double red[8];
    const int64_t n = (int64_t)W * H;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double ssim = 0.0;
    if (i < 3 * n) {
        const int ch = (int)(i / n);
        const int64_t p = i % n;
        const int py = (int)(p / W), px = (int)(p % W);
        float m[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
        for (int k = -kHalf; k <= kHalf; ++k) {
            const int y = py + k;
            if (y < 0 || y >= H) continue;
            const int64_t q = (int64_t)y * W + px;
            const float w = c_win[k + kHalf];
#pragma unroll
            for (int j = 0; j < 5; ++j) m[j] += w * hm[((int64_t)j * 3 + ch) * n + q];
        }
        const float mx = m[0], my = m[1];
        const float sxx = m[2] - mx * mx, syy = m[3] - my * my, sxy = m[4] - mx * my;
        const float A1 = 2.0f * mx * my + kC1, A2 = 2.0f * sxy + kC2;
        const float B1 = mx * mx + my * my + kC1, B2 = sxx + syy + kC2;
        const float s = (A1 * A2) / (B1 * B2);
        ssim = s;
        // s as a function of m_x, e_xx, e_xy (with sxx = e_xx - m_x^2, sxy = e_xy - m_x m_y)
        const float ds_dmx = (2.0f * my * A2 - 2.0f * my * A1) / (B1 * B2) - s * (2.0f * mx / B1 - 2.0f * mx / B2);
        const float ds_dexx = -s / B2;
        const float ds_dexy = 2.0f * A1 / (B1 * B2);
        dpart[((int64_t)0 * 3 + ch) * n + p] = ds_dmx;
        dpart[((int64_t)1 * 3 + ch) * n + p] = ds_dexx;
        dpart[((int64_t)2 * 3 + ch) * n + p] = ds_dexy;
    }
    const double b = block_sum_d(ssim, red);
    if (threadIdx.x == 0) atomicAdd(&acc[1], b);
}

// Horizontal blur of the three partial-derivative maps.
__global__ void ssim_partials_h(const float* __restrict__ dpart, int W, int H, float* __restrict__ out) {
    const int64_t n = (int64_t)W * H;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 9 * n) return;
    const int64_t plane = i / n, p = i % n;
    const int py = (int)(p / W), px = (int)(p % W);
    float s = 0.f;
    for (int k = -kHalf; k <= kHalf; ++k) {
        const int x = px + k;
        if (x < 0 || x >= W) continue;
        s += c_win[k + kHalf] * dpart[plane * n + (int64_t)py * W + x];
    }
    out[i] = s;
}

// Vertical blur of the partials and the image gradient dC = lambda_rgb (lambda_I1 dL1 +
// lambda_I2 dL_ssim); acc[0] += sum |x - y|.
__global__ void __launch_bounds__(256) rgb_grad(const float* __restrict__ X, const float* __restrict__ Y,
                                                const float* __restrict__ hpart, int W, int H,
                                                latentam_image_cfg cfg, float* __restrict__ dC,
                                                double* __restrict__ acc) {
    __shared__ double red[8];
    const int64_t n = (int64_t)W * H;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double l1 = 0.0;
    if (i < 3 * n) {
        const int ch = (int)(i / n);
        const int64_t p = i % n;
        const int py = (int)(p / W), px = (int)(p % W);
        float b[3] = {0.f, 0.f, 0.f};
        for (int k = -kHalf; k <= kHalf; ++k) {
            const int y = py + k;
            if (y < 0 || y >= H) continue;
            const float w = c_win[k + kHalf];
            const int64_t q = (int64_t)y * W + px;
#pragma unroll
            for (int j = 0; j < 3; ++j) b[j] += w * hpart[((int64_t)j * 3 + ch) * n + q];
        }
        const float x = X[3 * p + ch], y = Y[3 * p + ch];
        const float inv = 1.0f / (3.0f * (float)n);
        const float d_ssim = -inv * (b[0] + 2.0f * x * b[1] + y * b[2]);
        const float diff = x - y;
        const float d_l1 = inv * (diff > 0.f ? 1.f : (diff < 0.f ? -1.f : 0.f));
        l1 = fabs((double)diff);
        dC[3 * p + ch] = cfg.lambda_rgb * (cfg.lambda_I1 * d_l1 + cfg.lambda_I2 * d_ssim);
    }
    const double s = block_sum_d(l1, red);
    if (threadIdx.x == 0) atomicAdd(&acc[0], s);
}

// acc[2] += sum over valid pixels of |Z_hat - Z|, acc[3] += their count.
__global__ void __launch_bounds__(256) depth_sums(const float* __restrict__ Zh, const float* __restrict__ Zo,
                                                  int64_t n, double* __restrict__ acc) {
    __shared__ double red[8];
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double e = 0.0, c = 0.0;
    if (p < n && Zo[p] > 0.f) {
        e = fabs((double)Zh[p] - (double)Zo[p]);
        c = 1.0;
    }
    const double se = block_sum_d(e, red);
    const double sc = block_sum_d(c, red);
    if (threadIdx.x == 0) {
        atomicAdd(&acc[2], se);
        atomicAdd(&acc[3], sc);
    }
}

__global__ void depth_grad(const float* __restrict__ Zh, const float* __restrict__ Zo, int64_t n,
                           latentam_image_cfg cfg, const double* __restrict__ acc, float* __restrict__ dZ) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    float g = 0.f;
    if (Zo[p] > 0.f && acc[3] > 0.0) {
        const float diff = Zh[p] - Zo[p];
        g = cfg.lambda_d * (diff > 0.f ? 1.f : (diff < 0.f ? -1.f : 0.f)) / (float)acc[3];
    }
    dZ[p] = g;
}

// parts[5] L1, [6] 1 - mean SSIM, [7] L_d, [8] pixels with depth, [9] the total of Eq. full_obj.
__global__ void finalize_full(const double* __restrict__ acc, int64_t n, latentam_image_cfg cfg,
                              double* __restrict__ parts) {
    const double N3 = 3.0 * (double)n;
    const double l1 = n > 0 ? acc[0] / N3 : 0.0;
    const double ls = n > 0 ? 1.0 - acc[1] / N3 : 0.0;
    const double ld = acc[3] > 0.0 ? acc[2] / acc[3] : 0.0;
    parts[5] = l1;
    parts[6] = ls;
    parts[7] = ld;
    parts[8] = acc[3];
    parts[9] = (double)cfg.lambda_rgb * ((double)cfg.lambda_I1 * l1 + (double)cfg.lambda_I2 * ls) +
               (double)cfg.lambda_d * ld + parts[3];
}

// ---- projection backward ------------------------------------------------------------------

// dgeo[i] = (d u, d v, d conic a, b, c, d opacity, d depth channel, -) -> d mean, d quat, d scale,
// d opacity, through the same forward arithmetic as project_kernel.
__global__ void __launch_bounds__(256) project_bwd_kernel(int N, const float* __restrict__ means,
                                                          const float* __restrict__ quats,
                                                          const float* __restrict__ scales,
                                                          const float* __restrict__ opac, CamParams cam,
                                                          const float* __restrict__ dgeo, float* __restrict__ dmean,
                                                          float* __restrict__ dquat, float* __restrict__ dscale,
                                                          float* __restrict__ dopac) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    float gm[3] = {0.f, 0.f, 0.f}, gq[4] = {0.f, 0.f, 0.f, 0.f}, gs[3] = {0.f, 0.f, 0.f};
    float go = 0.f;
    const float px = means[3 * i], py = means[3 * i + 1], pz = means[3 * i + 2];
    const float o = opac[i];
    const double zd = __dadd_rn(__dadd_rn(__dadd_rn(__dmul_rn((double)cam.R[6], (double)px),
                                                    __dmul_rn((double)cam.R[7], (double)py)),
                                          __dmul_rn((double)cam.R[8], (double)pz)),
                                (double)cam.t[2]);
    const bool vis = (zd > (double)cam.z_near) && !((double)o < 1.0 / 255.0);
    if (vis) {
        const float* G = dgeo + 8 * (size_t)i;
        const float gu = G[0], gv = G[1], ga = G[2], gb = G[3], gc = G[4];
        go = G[5];
        const float gzr = G[6];
        const float z = (float)zd;
        const float x = cam.R[0] * px + cam.R[1] * py + cam.R[2] * pz + cam.t[0];
        const float y = cam.R[3] * px + cam.R[4] * py + cam.R[5] * pz + cam.t[1];
        const float q0 = quats[4 * i], q1 = quats[4 * i + 1], q2 = quats[4 * i + 2], q3 = quats[4 * i + 3];
        const float qn = rsqrtf(q0 * q0 + q1 * q1 + q2 * q2 + q3 * q3);
        const float qw = q0 * qn, qx = q1 * qn, qy = q2 * qn, qz = q3 * qn;
        const float Rq[9] = {1.f - 2.f * (qy * qy + qz * qz), 2.f * (qx * qy - qw * qz), 2.f * (qx * qz + qw * qy),
                             2.f * (qx * qy + qw * qz), 1.f - 2.f * (qx * qx + qz * qz), 2.f * (qy * qz - qw * qx),
                             2.f * (qx * qz - qw * qy), 2.f * (qy * qz + qw * qx), 1.f - 2.f * (qx * qx + qy * qy)};
        const float s[3] = {scales[3 * i], scales[3 * i + 1], scales[3 * i + 2]};
        const float iz = 1.0f / z;
        const float j00 = cam.fx * iz, j02 = -cam.fx * x * iz * iz;
        const float j11 = cam.fy * iz, j12 = -cam.fy * y * iz * iz;
        float T[6];
        for (int b = 0; b < 3; ++b) {
            T[b] = j00 * cam.R[b] + j02 * cam.R[6 + b];
            T[3 + b] = j11 * cam.R[3 + b] + j12 * cam.R[6 + b];
        }
        float B[6];
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 3; ++b)
                B[3 * a + b] = (T[3 * a] * Rq[b] + T[3 * a + 1] * Rq[3 + b] + T[3 * a + 2] * Rq[6 + b]) * s[b];
        const float ca = B[0] * B[0] + B[1] * B[1] + B[2] * B[2] + kDilation;
        const float cb = B[0] * B[3] + B[1] * B[4] + B[2] * B[5];
        const float cc = B[3] * B[3] + B[4] * B[4] + B[5] * B[5] + kDilation;
        const float det = ca * cc - cb * cb;
        if (det > 0.0f) {
            const float idet = 1.0f / det;
            const float A = cc * idet, Bc = -cb * idet, Cc = ca * idet;
            // conic -> Sigma': dL/dSigma' = -P G P with P the conic and G = [[ga, gb/2], [gb/2, gc]]
            const float pg00 = A * ga + Bc * 0.5f * gb, pg01 = A * 0.5f * gb + Bc * gc;
            const float pg10 = Bc * ga + Cc * 0.5f * gb, pg11 = Bc * 0.5f * gb + Cc * gc;
            const float d00 = -(pg00 * A + pg01 * Bc), d01 = -(pg00 * Bc + pg01 * Cc);
            const float d10 = -(pg10 * A + pg11 * Bc), d11 = -(pg10 * Bc + pg11 * Cc);
            const float gca = d00, gcb = d01 + d10, gcc = d11;
            // Sigma' = B B^T + eps I: dB = 2 Gs B with Gs = [[gca, gcb/2], [gcb/2, gcc]]
            float gB[6];
            for (int b = 0; b < 3; ++b) {
                gB[b] = 2.0f * (gca * B[b] + 0.5f * gcb * B[3 + b]);
                gB[3 + b] = 2.0f * (0.5f * gcb * B[b] + gcc * B[3 + b]);
            }
            // B = T M, M = Rq S
            float M[9];
            for (int k = 0; k < 3; ++k)
                for (int b = 0; b < 3; ++b) M[3 * k + b] = Rq[3 * k + b] * s[b];
            float gT[6], gM[9];
            for (int a = 0; a < 2; ++a)
                for (int k = 0; k < 3; ++k)
                    gT[3 * a + k] = gB[3 * a] * M[3 * k] + gB[3 * a + 1] * M[3 * k + 1] + gB[3 * a + 2] * M[3 * k + 2];
            for (int k = 0; k < 3; ++k)
                for (int b = 0; b < 3; ++b) gM[3 * k + b] = T[k] * gB[b] + T[3 + k] * gB[3 + b];
            float gR[9];
            for (int k = 0; k < 3; ++k)
                for (int b = 0; b < 3; ++b) gR[3 * k + b] = gM[3 * k + b] * s[b];
            for (int b = 0; b < 3; ++b) gs[b] = gM[b] * Rq[b] + gM[3 + b] * Rq[3 + b] + gM[6 + b] * Rq[6 + b];
            // rotation matrix -> normalised quaternion (w, x, y, z)
            const float gw = 2.f * (-qz * gR[1] + qy * gR[2] + qz * gR[3] - qx * gR[5] - qy * gR[6] + qx * gR[7]);
            const float gx = 2.f * (qy * gR[1] + qz * gR[2] + qy * gR[3] - 2.f * qx * gR[4] - qw * gR[5] + qz * gR[6] +
                                    qw * gR[7] - 2.f * qx * gR[8]);
            const float gy = 2.f * (-2.f * qy * gR[0] + qx * gR[1] + qw * gR[2] + qx * gR[3] + qz * gR[5] - qw * gR[6] +
                                    qz * gR[7] - 2.f * qy * gR[8]);
            const float gz = 2.f * (-2.f * qz * gR[0] - qw * gR[1] + qx * gR[2] + qw * gR[3] - 2.f * qz * gR[4] +
                                    qy * gR[5] + qx * gR[6] + qy * gR[7]);
            // through the normalisation q_hat = q / |q|
            const float dot = qw * gw + qx * gx + qy * gy + qz * gz;
            gq[0] = (gw - qw * dot) * qn;
            gq[1] = (gx - qx * dot) * qn;
            gq[2] = (gy - qy * dot) * qn;
            gq[3] = (gz - qz * dot) * qn;
            // T = J W -> J -> camera-space mean
            float gj00 = 0.f, gj02 = 0.f, gj11 = 0.f, gj12 = 0.f;
            for (int b = 0; b < 3; ++b) {
                gj00 += gT[b] * cam.R[b];
                gj02 += gT[b] * cam.R[6 + b];
                gj11 += gT[3 + b] * cam.R[3 + b];
                gj12 += gT[3 + b] * cam.R[6 + b];
            }
            const float iz2 = iz * iz, iz3 = iz2 * iz;
            float gcx = gj02 * (-cam.fx * iz2) + gu * cam.fx * iz;
            float gcy = gj12 * (-cam.fy * iz2) + gv * cam.fy * iz;
            float gcz = gj00 * (-cam.fx * iz2) + gj02 * (2.f * cam.fx * x * iz3) + gj11 * (-cam.fy * iz2) +
                        gj12 * (2.f * cam.fy * y * iz3) + gu * (-cam.fx * x * iz2) + gv * (-cam.fy * y * iz2) + gzr;
            for (int k = 0; k < 3; ++k) gm[k] = cam.R[k] * gcx + cam.R[3 + k] * gcy + cam.R[6 + k] * gcz;
        } else {
            go = 0.f;
        }
    }
    for (int k = 0; k < 3; ++k) dmean[3 * i + k] = gm[k];
    for (int k = 0; k < 4; ++k) dquat[4 * i + k] = gq[k];
    for (int k = 0; k < 3; ++k) dscale[3 * i + k] = gs[k];
    dopac[i] = go;
}

unsigned nblk(int64_t n) { return (unsigned)((n + 255) / 256); }

}  // namespace

latentam_status launch_image_loss(latentam_ctx* ctx, const float* C, const float* Z, const float* image,
                                  const float* depth_obs, int W, int H, const latentam_image_cfg& cfg,
                                  double* parts, float* dC, float* dZ, cudaStream_t st) {
    const int64_t n = (int64_t)W * H;
    static unsigned long long win_set = 0;  // the window lives in each device's constant memory
    int dev = 0;
    cudaGetDevice(&dev);
    if (!(win_set & (1ull << (dev & 63)))) {
        float w[kWin];
        double s = 0.0;
        for (int k = 0; k < kWin; ++k) s += exp(-(double)((k - kHalf) * (k - kHalf)) / (2.0 * 1.5 * 1.5));
        for (int k = 0; k < kWin; ++k) w[k] = (float)(exp(-(double)((k - kHalf) * (k - kHalf)) / (2.0 * 1.5 * 1.5)) / s);
        cudaError_t e = cudaMemcpyToSymbol(c_win, w, sizeof(w));
        if (e != cudaSuccess) return cuda_error(e, "SSIM window");
        win_set |= 1ull << (dev & 63);
    }
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t nn = (size_t)std::max<int64_t>(n, 1);
    char* base = static_cast<char*>(ws(ctx, WS_FULL_AUX, up(sizeof(float) * 15 * nn) + up(sizeof(float) * 9 * nn) +
                                                             up(sizeof(double) * 4)));
    if (!base) return LATENTAM_ERR_OUT_OF_MEMORY;
    float* hm = reinterpret_cast<float*>(base);          // 15 planes, then the 9 blurred partial planes
    float* dpart = reinterpret_cast<float*>(base + up(sizeof(float) * 15 * nn));
    double* acc = reinterpret_cast<double*>(base + up(sizeof(float) * 15 * nn) + up(sizeof(float) * 9 * nn));
    cudaError_t e = cudaMemsetAsync(acc, 0, sizeof(double) * 4, st);
    if (e != cudaSuccess) return cuda_error(e, "memset image loss");
    if (n > 0) {
        ssim_moments_h<<<nblk(3 * n), 256, 0, st>>>(C, image, W, H, hm);
        LAT_CHECK_LAUNCH("ssim_moments_h");
        ssim_map_v<<<nblk(3 * n), 256, 0, st>>>(hm, W, H, dpart, acc);
        LAT_CHECK_LAUNCH("ssim_map_v");
        ssim_partials_h<<<nblk(9 * n), 256, 0, st>>>(dpart, W, H, hm);
        LAT_CHECK_LAUNCH("ssim_partials_h");
        rgb_grad<<<nblk(3 * n), 256, 0, st>>>(C, image, hm, W, H, cfg, dC, acc);
        LAT_CHECK_LAUNCH("rgb_grad");
        depth_sums<<<nblk(n), 256, 0, st>>>(Z, depth_obs, n, acc);
        LAT_CHECK_LAUNCH("depth_sums");
        depth_grad<<<nblk(n), 256, 0, st>>>(Z, depth_obs, n, cfg, acc, dZ);
        LAT_CHECK_LAUNCH("depth_grad");
    }
    finalize_full<<<1, 1, 0, st>>>(acc, n, cfg, parts);
    LAT_CHECK_LAUNCH("finalize_full");
    return LATENTAM_OK;
}

latentam_status launch_project_bwd(const latentam_gaussians& g, const CamParams& cam, const float* dgeo,
                                   float* dmean, float* dquat, float* dscale, float* dopac, cudaStream_t st) {
    if (g.n == 0) return LATENTAM_OK;
    project_bwd_kernel<<<nblk(g.n), 256, 0, st>>>(g.n, g.means, g.quats, g.scales, g.opacities, cam, dgeo, dmean,
                                                 dquat, dscale, dopac);
    LAT_CHECK_LAUNCH("project_bwd_kernel");
    return LATENTAM_OK;
}

}  // namespace lat
