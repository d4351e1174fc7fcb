// The paper's own parameterisation of the dictionary decode (Eq. dict_recon, Sec. III-B):
// u_p = q_p W (W: d_s x d_f), similarities cos(u_p, D_j) after l2 normalisation divided by
// the temperature tau, Fhat = softmax_rows(.) D (D: M x d_f atoms).
//
// It is computed exactly through the free-key decode: with n_j = |D_j|, the keys
// k_j = W D_j^T / n_j (M x d_s), G = W W^T (d_s x d_s), r_p = 1 / |q_p W| = (q_p^T G q_p)^-1/2,
// the scaled queries q'_p = r_p q_p and the logit scale c = 1/tau,
//     cos(u_p, D_j) / tau = c <q'_p, k_j>,   values V = D,
// so the n x d_f product Q W is never formed.  The gradients of the free-key decode (dQ', dK,
// dV) chain back through the two small maps:
//     s_p = <q_p, dQ'_p>,  dQ_p = r_p (dQ'_p - r_p^2 s_p G q_p),
//     dW = sum_j dK_j^T D_j / n_j - C W,   C = sum_p s_p r_p^3 q_p q_p^T,
//     dD_j = dV_j + (g_j - (D_j . g_j) D_j / n_j^2) / n_j,   g_j = W^T dK_j
// (dV already holds the trust-region subgradient on the atoms).
#include <math.h>

#include <algorithm>

#include "internal.cuh"

namespace lat {
namespace {

constexpr float kNormFloor = 1e-12f;  // floor of |u_p| and |D_j|

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// One block per atom j: n_j = max(|D_j|, floor) and K_j = W D_j^T / n_j; warp w computes the
// key entries a = w, w + 8, ...
__global__ void __launch_bounds__(256) paper_keys(const float* __restrict__ W, const float* __restrict__ D, int ds,
                                                  int df, float* __restrict__ K, float* __restrict__ nrm) {
    extern __shared__ float dj[];  // df
    __shared__ float red[8];
    const int j = blockIdx.x, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    float s = 0.f;
    for (int f = threadIdx.x; f < df; f += blockDim.x) {
        const float x = D[(size_t)j * df + f];
        dj[f] = x;
        s += x * x;
    }
    s = warp_sum(s);
    if (lane == 0) red[w] = s;
    __syncthreads();
    float t = 0.f;
#pragma unroll
    for (int q = 0; q < 8; ++q) t += red[q];
    const float n = fmaxf(sqrtf(t), kNormFloor);
    if (threadIdx.x == 0) nrm[j] = n;
    for (int a = w; a < ds; a += 8) {
        float acc = 0.f;
        for (int f = lane; f < df; f += 32) acc += W[(size_t)a * df + f] * dj[f];
        acc = warp_sum(acc);
        if (lane == 0) K[(size_t)j * ds + a] = acc / n;
    }
}

// G = W W^T: one warp per entry.
__global__ void __launch_bounds__(256) paper_gram(const float* __restrict__ W, int ds, int df, float* __restrict__ G) {
    const int e = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (e >= ds * ds) return;
    const int a = e / ds, b = e % ds;
    float acc = 0.f;
    for (int f = lane; f < df; f += 32) acc += W[(size_t)a * df + f] * W[(size_t)b * df + f];
    acc = warp_sum(acc);
    if (lane == 0) G[e] = acc;
}

// r_p = 1 / max(sqrt(q_p^T G q_p), floor), Q'_p = r_p q_p (one thread per pixel, G staged).
template <int DS>
__global__ void __launch_bounds__(256) paper_queries(const float* __restrict__ Q, int64_t n, const float* __restrict__ G,
                                                     float* __restrict__ Qp, float* __restrict__ r) {
    __shared__ float g[DS * DS];
    for (int e = threadIdx.x; e < DS * DS; e += blockDim.x) g[e] = G[e];
    __syncthreads();
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    float q[DS];
#pragma unroll
    for (int a = 0; a < DS; a += 4) {
        const float4 v = *reinterpret_cast<const float4*>(Q + p * DS + a);
        q[a] = v.x, q[a + 1] = v.y, q[a + 2] = v.z, q[a + 3] = v.w;
    }
    float t = 0.f;
#pragma unroll
    for (int a = 0; a < DS; ++a) {
        float ga = 0.f;
#pragma unroll
        for (int b = 0; b < DS; ++b) ga += g[a * DS + b] * q[b];
        t += q[a] * ga;
    }
    const float rp = 1.0f / fmaxf(sqrtf(fmaxf(t, 0.f)), kNormFloor);
    r[p] = rp;
#pragma unroll
    for (int a = 0; a < DS; a += 4)
        *reinterpret_cast<float4*>(Qp + p * DS + a) = make_float4(rp * q[a], rp * q[a + 1], rp * q[a + 2], rp * q[a + 3]);
}

// dQ_p = r_p (dQ'_p - r_p^2 s_p G q_p) with s_p = <q_p, dQ'_p>, and the block's share of
// C = sum_p s_p r_p^3 q_p q_p^T (added to Cm with one atomic per entry per block).  Pixels go
// through shared memory 64 at a time; thread t owns the entries t, t + 256, ... of C.
template <int DS>
__global__ void __launch_bounds__(256) paper_query_grads(const float* __restrict__ Q, const float* __restrict__ r,
                                                         const float* __restrict__ dQp, int64_t n,
                                                         const float* __restrict__ G, float* __restrict__ dQ,
                                                         float* __restrict__ Cm) {
    constexpr int CH = 64;
    constexpr int PER = (DS * DS + 255) / 256;
    __shared__ float g[DS * DS];
    __shared__ float sq[CH][DS];  // q_p
    __shared__ float sw[CH][DS];  // s_p r_p^3 q_p
    for (int e = threadIdx.x; e < DS * DS; e += blockDim.x) g[e] = G[e];
    float c[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) c[k] = 0.f;
    __syncthreads();
    for (int64_t base = (int64_t)blockIdx.x * CH; base < n; base += (int64_t)gridDim.x * CH) {
        // the first CH threads handle one pixel each
        if (threadIdx.x < CH) {
            const int64_t p = base + threadIdx.x;
            float q[DS], dq[DS];
            float s = 0.f, rp = 0.f;
            if (p < n) {
                rp = r[p];
#pragma unroll
                for (int a = 0; a < DS; ++a) {
                    q[a] = Q[p * DS + a];
                    dq[a] = dQp[p * DS + a];
                    s += q[a] * dq[a];
                }
                const float k2 = rp * rp * s;
#pragma unroll
                for (int a = 0; a < DS; ++a) {
                    float ga = 0.f;
#pragma unroll
                    for (int b = 0; b < DS; ++b) ga += g[a * DS + b] * q[b];
                    dQ[p * DS + a] = rp * (dq[a] - k2 * ga);
                }
            } else {
#pragma unroll
                for (int a = 0; a < DS; ++a) q[a] = 0.f;
            }
            const float wgt = s * rp * rp * rp;
#pragma unroll
            for (int a = 0; a < DS; ++a) {
                sq[threadIdx.x][a] = q[a];
                sw[threadIdx.x][a] = wgt * q[a];
            }
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int e = threadIdx.x + 256 * k;
            if (e < DS * DS) {
                const int a = e / DS, b = e % DS;
                float acc = 0.f;
#pragma unroll 8
                for (int i = 0; i < CH; ++i) acc += sw[i][a] * sq[i][b];
                c[k] += acc;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int e = threadIdx.x + 256 * k;
        if (e < DS * DS) atomicAdd(&Cm[e], c[k]);
    }
}

// dW[a][f] = sum_j dK[j][a] D[j][f] / n_j - sum_b C[a][b] W[b][f]  (one thread per entry).
__global__ void __launch_bounds__(256) paper_dW(const float* __restrict__ W, const float* __restrict__ D,
                                                const float* __restrict__ nrm, const float* __restrict__ dK,
                                                const float* __restrict__ Cm, int M, int ds, int df,
                                                float* __restrict__ dW) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)ds * df) return;
    const int a = (int)(e / df), f = (int)(e % df);
    float acc = 0.f;
    for (int j = 0; j < M; ++j) acc += dK[(size_t)j * ds + a] * D[(size_t)j * df + f] / nrm[j];
    for (int b = 0; b < ds; ++b) acc -= Cm[a * ds + b] * W[(size_t)b * df + f];
    dW[e] = acc;
}

// dD_j = dV_j + (g_j - (D_j . g_j) D_j / n_j^2) / n_j with g_j = W^T dK_j (one block per atom).
__global__ void __launch_bounds__(256) paper_dD(const float* __restrict__ W, const float* __restrict__ D,
                                                const float* __restrict__ nrm, const float* __restrict__ dK,
                                                const float* __restrict__ dV, int ds, int df,
                                                float* __restrict__ dD) {
    extern __shared__ float gj[];  // df
    __shared__ float red[8];
    const int j = blockIdx.x, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    float s = 0.f;
    for (int f = threadIdx.x; f < df; f += blockDim.x) {
        float g = 0.f;
        for (int a = 0; a < ds; ++a) g += W[(size_t)a * df + f] * dK[(size_t)j * ds + a];
        gj[f] = g;
        s += D[(size_t)j * df + f] * g;
    }
    s = warp_sum(s);
    if (lane == 0) red[w] = s;
    __syncthreads();
    float dot = 0.f;
#pragma unroll
    for (int q = 0; q < 8; ++q) dot += red[q];
    const float n = nrm[j];
    const float k = dot / (n * n);
    for (int f = threadIdx.x; f < df; f += blockDim.x)
        dD[(size_t)j * df + f] = dV[(size_t)j * df + f] + (gj[f] - k * D[(size_t)j * df + f]) / n;
}

int cdiv(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

}  // namespace

latentam_status paper_prepare(latentam_ctx* ctx, const PaperArgs& a, const PaperBuffers& b, cudaStream_t st) {
    paper_keys<<<a.M, 256, sizeof(float) * a.df, st>>>(a.W, a.D, a.ds, a.df, b.K, b.nrm);
    LAT_CHECK_LAUNCH("paper_keys");
    paper_gram<<<cdiv(a.ds * a.ds, 8), 256, 0, st>>>(a.W, a.ds, a.df, b.G);
    LAT_CHECK_LAUNCH("paper_gram");
    if (a.n > 0) {
        const int blocks = cdiv(a.n, 256);
        if (a.ds == 16) paper_queries<16><<<blocks, 256, 0, st>>>(a.Q, a.n, b.G, b.Qp, b.r);
        else if (a.ds == 32) paper_queries<32><<<blocks, 256, 0, st>>>(a.Q, a.n, b.G, b.Qp, b.r);
        else paper_queries<64><<<blocks, 256, 0, st>>>(a.Q, a.n, b.G, b.Qp, b.r);
        LAT_CHECK_LAUNCH("paper_queries");
    }
    (void)ctx;
    return LATENTAM_OK;
}

latentam_status paper_chain(latentam_ctx* ctx, const PaperArgs& a, const PaperBuffers& b, float* dQ, float* dW,
                            float* dD, cudaStream_t st) {
    if (dQ || dW) {
        cudaError_t e = cudaMemsetAsync(b.Cm, 0, sizeof(float) * a.ds * a.ds, st);
        if (e != cudaSuccess) return cuda_error(e, "memset C");
        if (a.n > 0) {
            const int blocks = std::max(1, std::min(cdiv(a.n, 64), 2 * ctx->num_sms));
            float* out = dQ ? dQ : b.dQp;  // dQ' is not needed after this kernel: reuse it when dQ is not asked for
            if (a.ds == 16) paper_query_grads<16><<<blocks, 256, 0, st>>>(a.Q, b.r, b.dQp, a.n, b.G, out, b.Cm);
            else if (a.ds == 32) paper_query_grads<32><<<blocks, 256, 0, st>>>(a.Q, b.r, b.dQp, a.n, b.G, out, b.Cm);
            else paper_query_grads<64><<<blocks, 256, 0, st>>>(a.Q, b.r, b.dQp, a.n, b.G, out, b.Cm);
            LAT_CHECK_LAUNCH("paper_query_grads");
        }
    }
    if (dW) {
        paper_dW<<<cdiv((int64_t)a.ds * a.df, 256), 256, 0, st>>>(a.W, a.D, b.nrm, b.dK, b.Cm, a.M, a.ds, a.df, dW);
        LAT_CHECK_LAUNCH("paper_dW");
    }
    if (dD) {
        paper_dD<<<a.M, 256, sizeof(float) * a.df, st>>>(a.W, a.D, b.nrm, b.dK, b.dV, a.ds, a.df, dD);
        LAT_CHECK_LAUNCH("paper_dD");
    }
    return LATENTAM_OK;
}

}  // namespace lat
