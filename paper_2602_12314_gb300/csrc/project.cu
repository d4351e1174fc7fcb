// EWA projection of the Gaussian primitives (Sec. III-A; the footprint of the 3DGS
// renderer the paper cites for Eq. alpha_blending).  One thread per Gaussian; SoA
// inputs, one float2 + float4 + float + int4 + int store per Gaussian.
#include "internal.cuh"

namespace lat {
namespace {

__device__ __forceinline__ void tile_span(float lo, float hi, int npix, int& t0, int& t1) {
    float plo = ceilf(lo), phi = floorf(hi);
    plo = fmaxf(plo, 0.0f);
    phi = fminf(phi, (float)(npix - 1));
    if (!(plo <= phi)) {
        t0 = t1 = 0;
        return;
    }
    t0 = (int)plo / kTile;
    t1 = (int)phi / kTile + 1;
}

__global__ void __launch_bounds__(256) project_kernel(int N, const float* __restrict__ means,
                                                      const float* __restrict__ quats,
                                                      const float* __restrict__ scales,
                                                      const float* __restrict__ opac, CamParams cam,
                                                      float2* __restrict__ xy_out,
                                                      float4* __restrict__ conic_out,
                                                      float* __restrict__ depth_out,
                                                      int4* __restrict__ rect_out,
                                                      int32_t* __restrict__ tiles_out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const float px = means[3 * i], py = means[3 * i + 1], pz = means[3 * i + 2];
    const float o = opac[i];
    // Depth sort key: evaluated in binary32 with every rounding explicit (no contraction into
    // fused multiply-adds), so the front-to-back order is an exact function of the inputs.
    const float z = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(cam.R[6], px), __fmul_rn(cam.R[7], py)),
                                        __fmul_rn(cam.R[8], pz)),
                              cam.t[2]);
    depth_out[i] = z;
    int4 rect = make_int4(0, 0, 0, 0);
    float2 xy = make_float2(0.f, 0.f);
    float4 co = make_float4(0.f, 0.f, 0.f, 0.f);
    // o < 1/255 for a binary32 o is o < bf(1/255), the nearest binary32 (above 1/255)
    bool vis = (z > cam.z_near) && !(o < kAlphaMin);
    if (vis) {
        const float x = cam.R[0] * px + cam.R[1] * py + cam.R[2] * pz + cam.t[0];
        const float y = cam.R[3] * px + cam.R[4] * py + cam.R[5] * pz + cam.t[1];
        // rotation from the (normalised) quaternion
        float qw = quats[4 * i], qx = quats[4 * i + 1], qy = quats[4 * i + 2], qz = quats[4 * i + 3];
        const float qn = rsqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
        qw *= qn;
        qx *= qn;
        qy *= qn;
        qz *= qn;
        const float Rq[9] = {1.f - 2.f * (qy * qy + qz * qz), 2.f * (qx * qy - qw * qz), 2.f * (qx * qz + qw * qy),
                             2.f * (qx * qy + qw * qz), 1.f - 2.f * (qx * qx + qz * qz), 2.f * (qy * qz - qw * qx),
                             2.f * (qx * qz - qw * qy), 2.f * (qy * qz + qw * qx), 1.f - 2.f * (qx * qx + qy * qy)};
        const float s0 = scales[3 * i], s1 = scales[3 * i + 1], s2 = scales[3 * i + 2];
        // T = J W (2x3), then Sigma' = (T Rq S)(T Rq S)^T + dilation
        const float iz = 1.0f / z;
        const float j00 = cam.fx * iz, j02 = -cam.fx * x * iz * iz;
        const float j11 = cam.fy * iz, j12 = -cam.fy * y * iz * iz;
        float T[6];
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            T[b] = j00 * cam.R[b] + j02 * cam.R[6 + b];
            T[3 + b] = j11 * cam.R[3 + b] + j12 * cam.R[6 + b];
        }
        float B[6];  // T Rq S
#pragma unroll
        for (int a = 0; a < 2; ++a) {
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                const float sb = b == 0 ? s0 : (b == 1 ? s1 : s2);
                B[3 * a + b] = (T[3 * a] * Rq[b] + T[3 * a + 1] * Rq[3 + b] + T[3 * a + 2] * Rq[6 + b]) * sb;
            }
        }
        const float ca = B[0] * B[0] + B[1] * B[1] + B[2] * B[2] + kDilation;
        const float cb = B[0] * B[3] + B[1] * B[4] + B[2] * B[5];
        const float cc = B[3] * B[3] + B[4] * B[4] + B[5] * B[5] + kDilation;
        const float det = ca * cc - cb * cb;
        if (det > 0.0f) {
            const float idet = 1.0f / det;
            co = make_float4(cc * idet, -cb * idet, ca * idet, o);
            xy = make_float2(cam.fx * x * iz + cam.cx, cam.fy * y * iz + cam.cy);
            // axis-aligned extent of the alpha >= 1/255 ellipse d^T conic d <= 2 ln(255 o)
            const float mmax = fmaxf(2.0f * logf(255.0f * o), 0.0f);
            const float ex = sqrtf(mmax * ca), ey = sqrtf(mmax * cc);
            int x0, x1, y0, y1;
            tile_span(xy.x - ex, xy.x + ex, cam.W, x0, x1);
            tile_span(xy.y - ey, xy.y + ey, cam.H, y0, y1);
            if (x0 != x1 && y0 != y1) rect = make_int4(x0, y0, x1, y1);
        } else {
            vis = false;
        }
    }
    xy_out[i] = xy;
    conic_out[i] = co;
    rect_out[i] = rect;
    tiles_out[i] = (rect.z - rect.x) * (rect.w - rect.y);
}

}  // namespace

latentam_status launch_project(const latentam_gaussians& g, const CamParams& cam,
                               const latentam_projected& out, cudaStream_t st) {
    if (g.n == 0) return LATENTAM_OK;
    const int threads = 256;
    const int blocks = (g.n + threads - 1) / threads;
    project_kernel<<<blocks, threads, 0, st>>>(g.n, g.means, g.quats, g.scales, g.opacities, cam,
                                               reinterpret_cast<float2*>(out.xy),
                                               reinterpret_cast<float4*>(out.conic_opacity), out.depth,
                                               reinterpret_cast<int4*>(out.rect), out.tiles_touched);
    LAT_CHECK_LAUNCH("project_kernel");
    return LATENTAM_OK;
}

}  // namespace lat
