// Dictionary decode (Sec. III-B, Eq. dict_recon), feature objective (Eq. feat_loss,
// Eq. full_obj) and its backward, plain FP32 form on the CUDA cores.
//
//   rows kernel (32 pixels / CTA):  S = c Q K^T -> row softmax A -> Fhat = A V
//        -> per-pixel cos / L2 against F -> dFhat = a_p Fhat_p + b_p F_p  (loss written FP64)
//   rows-backward kernel:           dA = dFhat V^T -> dS = A (dA - <A, dA>) -> dQ = c dS K
//   dictionary kernels (split-K):   dV = A^T dFhat + trust-region term, dK = c dS^T Q
//
// dL/dFhat_p = a_p Fhat_p + b_p F_p with
//   a_p = lambda_f/|Omega| (lambda_cos cos_p / |Fhat_p|^2 + 2 lambda_2 / D)
//   b_p = lambda_f/|Omega| (-lambda_cos / (|Fhat_p| |F_p|) - 2 lambda_2 / D),
// and <A_p, dA_p> = <Fhat_p, dFhat_p> = a_p |Fhat_p|^2 + b_p <Fhat_p, F_p>.
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>

#include "internal.cuh"

namespace lat {
namespace {

constexpr int kRows = 32;      // pixels per CTA in the row kernels
constexpr int kThreads = 256;  // 8 warps x 4 rows
constexpr int kAtomChunk = 128;
constexpr int kColChunk = 512;  // 32 lanes x 4 floats x 4 groups

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ float4 load_target4(const void* F, latentam_dtype dt, size_t idx4) {
    if (dt == LATENTAM_DTYPE_F32) return reinterpret_cast<const float4*>(F)[idx4];
    const uint2 raw = reinterpret_cast<const uint2*>(F)[idx4];
    const __nv_bfloat162 lo = *reinterpret_cast<const __nv_bfloat162*>(&raw.x);
    const __nv_bfloat162 hi = *reinterpret_cast<const __nv_bfloat162*>(&raw.y);
    const float2 a = __bfloat1622float2(lo), b = __bfloat1622float2(hi);
    return make_float4(a.x, a.y, b.x, b.y);
}

// Accumulators: [0] sum over valid pixels of (1 - cos), [1] sum of squared errors,
// [2] trust-region sum, [3] |Omega|.
struct LossAcc {
    double* acc;
};

__global__ void count_mask_kernel(const uint8_t* __restrict__ mask, int64_t n, double* __restrict__ acc) {
    __shared__ int s[kThreads / 32];
    int c = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        c += mask ? (mask[i] != 0) : 1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < kThreads / 32; ++w) t += s[w];
        atomicAdd(&acc[3], (double)t);
    }
}

// Trust-region term of Eq. (feat_loss) on the value rows: one warp per atom.  coef[j] =
// lambda_f lambda_D / |V_j - V0_j| when the atom is outside the radius, else 0.
__global__ void trust_region_kernel(const float* __restrict__ V, const float* __restrict__ V0, int M, int D,
                                    float delta, float weight, float* __restrict__ coef, double* __restrict__ acc) {
    const int j = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (j >= M) return;
    float s = 0.f;
    for (int k = lane; k < D; k += 32) {
        const float t = V[(size_t)j * D + k] - V0[(size_t)j * D + k];
        s += t * t;
    }
    s = warp_sum(s);
    if (lane == 0) {
        const float nrm = sqrtf(s);
        const bool out = nrm > delta;
        coef[j] = out ? weight / nrm : 0.f;
        if (out) atomicAdd(&acc[2], (double)(nrm - delta));
    }
}

// ---- rows kernel: S, softmax, Fhat, loss coefficients, dFhat ---------------------------
// smem: sA[kRows][M] | sKt[d][kAtomChunk + 1] | sQ[kRows][d] | stats
// MODE 0: Fhat only (inference); 1: the whole row pass of the loss; 2: S and the softmax only
// (A and its row statistics), for the tiled path.
template <int DQ, int MODE>
__global__ void __launch_bounds__(kThreads) dec_rows_fwd(const float* __restrict__ Q, int64_t n, const float* __restrict__ K,
                                                          const float* __restrict__ V, int M, int D, float c,
                                                          const void* __restrict__ F, latentam_dtype F_dtype,
                                                          const uint8_t* __restrict__ mask, latentam_loss_cfg cfg,
                                                          double* __restrict__ acc, float* __restrict__ A_out,
                                                          float* __restrict__ Fh_out, float* __restrict__ row_out,
                                                          float* __restrict__ stats_out) {
    extern __shared__ float smem[];
    float* sA = smem;                                  // kRows * M
    float* sKt = sA + kRows * M;                       // DQ * (kAtomChunk + 1)
    float* sQ = sKt + DQ * (kAtomChunk + 1);           // kRows * DQ
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int64_t row0 = (int64_t)blockIdx.x * kRows;
    // stage the query tile
    for (int e = t; e < kRows * DQ; e += kThreads) {
        const int r = e / DQ;
        sQ[e] = (row0 + r < n) ? Q[(row0 + r) * DQ + (e % DQ)] : 0.f;
    }
    // S = c Q K^T, atoms in chunks of 128 (lane owns atoms lane + 32u)
    for (int j0 = 0; j0 < M; j0 += kAtomChunk) {
        const int jc = min(kAtomChunk, M - j0);
        __syncthreads();
        for (int e = t; e < jc * DQ; e += kThreads) {
            const int jj = e / DQ, k = e % DQ;
            sKt[k * (kAtomChunk + 1) + jj] = K[(size_t)(j0 + jj) * DQ + k];
        }
        __syncthreads();
        float s[4][4];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int u = 0; u < 4; ++u) s[r][u] = 0.f;
#pragma unroll 8
        for (int k = 0; k < DQ; ++k) {
            float kv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) kv[u] = sKt[k * (kAtomChunk + 1) + lane + 32 * u];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const float q = sQ[(warp * 4 + r) * DQ + k];
#pragma unroll
                for (int u = 0; u < 4; ++u) s[r][u] += q * kv[u];
            }
        }
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (lane + 32 * u < jc) sA[(warp * 4 + r) * M + j0 + lane + 32 * u] = c * s[r][u];
    }
    __syncthreads();
    // row softmax (warp per 4 rows)
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int rr = warp * 4 + r;
        float* a = sA + rr * M;
        float m = -INFINITY;
        for (int j = lane; j < M; j += 32) m = fmaxf(m, a[j]);
        m = warp_max(m);
        float l = 0.f;
        for (int j = lane; j < M; j += 32) {
            const float e = __expf(a[j] - m);
            a[j] = e;
            l += e;
        }
        l = warp_sum(l);
        const float il = 1.0f / l;
        const int64_t p = row0 + rr;
        for (int j = lane; j < M; j += 32) {
            const float v = a[j] * il;
            a[j] = v;
            if (MODE >= 1 && p < n) A_out[p * M + j] = v;
        }
        if (lane == 0 && stats_out && p < n) {
            stats_out[2 * p] = m;
            stats_out[2 * p + 1] = l;
        }
    }
    if (MODE == 2) return;
    constexpr bool TRAIN = MODE == 1;
    __syncthreads();
    // Fhat = A V in column chunks; thread owns rows 4 warp + r, columns c0 + 4 lane + 128 g
    float pdot[4] = {0.f, 0.f, 0.f, 0.f}, pnh[4] = {0.f, 0.f, 0.f, 0.f}, pnf[4] = {0.f, 0.f, 0.f, 0.f},
          perr[4] = {0.f, 0.f, 0.f, 0.f};
    const float4* V4 = reinterpret_cast<const float4*>(V);
    const int D4 = D / 4;
    for (int c0 = 0; c0 < D; c0 += kColChunk) {
        const int ng = min(4, (D - c0) / 128);
        float4 accv[4][4];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int g = 0; g < 4; ++g) accv[r][g] = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int j = 0; j < M; ++j) {
            float a[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) a[r] = sA[(warp * 4 + r) * M + j];
#pragma unroll
            for (int g = 0; g < 4; ++g) {
                if (g < ng) {
                    const float4 v = __ldg(&V4[(size_t)j * D4 + (c0 / 4) + lane + 32 * g]);
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        accv[r][g].x += a[r] * v.x;
                        accv[r][g].y += a[r] * v.y;
                        accv[r][g].z += a[r] * v.z;
                        accv[r][g].w += a[r] * v.w;
                    }
                }
            }
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int64_t p = row0 + warp * 4 + r;
            if (p >= n) continue;
#pragma unroll
            for (int g = 0; g < 4; ++g) {
                if (g >= ng) continue;
                const size_t idx4 = (size_t)p * D4 + (c0 / 4) + lane + 32 * g;
                const float4 h = accv[r][g];
                reinterpret_cast<float4*>(Fh_out)[idx4] = h;
                if (TRAIN) {
                    const float4 f = load_target4(F, F_dtype, idx4);
                    pdot[r] += h.x * f.x + h.y * f.y + h.z * f.z + h.w * f.w;
                    pnh[r] += h.x * h.x + h.y * h.y + h.z * h.z + h.w * h.w;
                    pnf[r] += f.x * f.x + f.y * f.y + f.z * f.z + f.w * f.w;
                    const float ex = h.x - f.x, ey = h.y - f.y, ez = h.z - f.z, ew = h.w - f.w;
                    perr[r] += ex * ex + ey * ey + ez * ez + ew * ew;
                }
            }
        }
    }
    if (!TRAIN) return;
    // per-pixel coefficients of dL/dFhat; loss sums in FP64
    const double nv = acc[3];
    const float scale = nv > 0.0 ? (float)((double)cfg.lambda_f / nv) : 0.f;
    double loc_cos = 0.0, loc_err = 0.0;
    float ra[4], rb[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const float dot = warp_sum(pdot[r]), nh2 = warp_sum(pnh[r]), nf2 = warp_sum(pnf[r]), e2 = warp_sum(perr[r]);
        const int64_t p = row0 + warp * 4 + r;
        const bool valid = p < n && (mask == nullptr || mask[p] != 0);
        const float den = sqrtf(nh2) * sqrtf(nf2);
        const float cs = dot / fmaxf(den, 1e-8f);
        float a = 0.f, b = 0.f;
        if (valid) {
            loc_cos += 1.0 - (double)cs;
            loc_err += (double)e2;
            const float l2c = 2.0f * cfg.lambda_2 / (float)D;
            if (den > 1e-8f) {
                a = scale * (cfg.lambda_cos * cs / nh2 + l2c);
                b = scale * (-cfg.lambda_cos / den - l2c);
            } else {
                a = scale * l2c;
                b = scale * (-cfg.lambda_cos / 1e-8f - l2c);
            }
        }
        ra[r] = a;
        rb[r] = b;
        if (lane == 0 && p < n) {
            row_out[4 * p] = a;
            row_out[4 * p + 1] = b;
            row_out[4 * p + 2] = a * nh2 + b * dot;  // <A_p, dA_p>
            row_out[4 * p + 3] = cs;
        }
    }
    if (lane == 0) {
        atomicAdd(&acc[0], loc_cos);
        atomicAdd(&acc[1], loc_err);
    }
    // dFhat = a Fhat + b F in place over the Fhat buffer (rows of this warp only)
    for (int c0 = 0; c0 < D; c0 += 128) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int64_t p = row0 + warp * 4 + r;
            if (p >= n) continue;
            const size_t idx4 = (size_t)p * D4 + (c0 / 4) + lane;
            const float4 h = reinterpret_cast<const float4*>(Fh_out)[idx4];
            const float4 f = load_target4(F, F_dtype, idx4);
            reinterpret_cast<float4*>(Fh_out)[idx4] =
                make_float4(ra[r] * h.x + rb[r] * f.x, ra[r] * h.y + rb[r] * f.y, ra[r] * h.z + rb[r] * f.z,
                            ra[r] * h.w + rb[r] * f.w);
        }
    }
}

// ---- rows-backward kernel: dA, dS, dQ ----------------------------------------------------
// smem: sdS[kRows][M] | sV[kAtomChunk][33] | sdF[kRows][33]
template <int DQ>
__global__ void __launch_bounds__(kThreads) dec_rows_bwd(const float* __restrict__ dFh, const float* __restrict__ A,
                                                          const float* __restrict__ row, const float* __restrict__ K,
                                                          const float* __restrict__ V, int64_t n, int M, int D, float c,
                                                          float* __restrict__ dS_out, float* __restrict__ dQ) {
    extern __shared__ float smem[];
    float* sdS = smem;                     // kRows * M
    float* sV = sdS + kRows * M;           // kAtomChunk * 33
    float* sdF = sV + kAtomChunk * 33;     // kRows * 33
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int64_t row0 = (int64_t)blockIdx.x * kRows;
    for (int j0 = 0; j0 < M; j0 += kAtomChunk) {
        const int jc = min(kAtomChunk, M - j0);
        float s[4][4];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int u = 0; u < 4; ++u) s[r][u] = 0.f;
        for (int k0 = 0; k0 < D; k0 += 32) {
            __syncthreads();
            for (int e = t; e < jc * 32; e += kThreads) {
                const int jj = e >> 5, k = e & 31;
                sV[jj * 33 + k] = V[(size_t)(j0 + jj) * D + k0 + k];
            }
            for (int e = t; e < kRows * 32; e += kThreads) {
                const int r = e >> 5, k = e & 31;
                sdF[r * 33 + k] = (row0 + r < n) ? dFh[(row0 + r) * D + k0 + k] : 0.f;
            }
            __syncthreads();
#pragma unroll 8
            for (int k = 0; k < 32; ++k) {
                float vv[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) vv[u] = (lane + 32 * u < jc) ? sV[(lane + 32 * u) * 33 + k] : 0.f;
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const float g = sdF[(warp * 4 + r) * 33 + k];
#pragma unroll
                    for (int u = 0; u < 4; ++u) s[r][u] += g * vv[u];
                }
            }
        }
        // dS = A (dA - <A, dA>)
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int64_t p = row0 + warp * 4 + r;
            const float rd = p < n ? row[4 * p + 2] : 0.f;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int j = j0 + lane + 32 * u;
                if (lane + 32 * u >= jc) continue;
                float ds = 0.f;
                if (p < n) {
                    ds = A[p * M + j] * (s[r][u] - rd);
                    dS_out[p * M + j] = ds;
                }
                sdS[(warp * 4 + r) * M + j] = ds;
            }
        }
    }
    __syncthreads();
    if (!dQ) return;
    // dQ = c dS K : thread -> row t / 8, columns (t % 8) * DQ/8 ...
    constexpr int CPT = DQ / 8;
    const int r = t >> 3, cb = (t & 7) * CPT;
    float q[CPT];
#pragma unroll
    for (int i = 0; i < CPT; ++i) q[i] = 0.f;
    for (int j = 0; j < M; ++j) {
        const float ds = sdS[r * M + j];
#pragma unroll
        for (int i = 0; i < CPT; ++i) q[i] += ds * __ldg(&K[(size_t)j * DQ + cb + i]);
    }
    const int64_t p = row0 + r;
    if (p < n)
#pragma unroll
        for (int i = 0; i < CPT; ++i) dQ[p * DQ + cb + i] = c * q[i];
}

// ---- split-K C = X^T Y over pixels: X (n x ldx, columns [x0, x0+64)), Y (n x ldy) ----------
// Block tile: 64 atoms x (32 * VEC) columns; thread: 8 atoms x VEC columns.
template <int VEC>
__global__ void __launch_bounds__(kThreads) atb_splitk(const float* __restrict__ X, int ldx, int nx,
                                                        const float* __restrict__ Y, int ldy, int ny, int64_t n,
                                                        int64_t rows_per_split, float* __restrict__ part) {
    constexpr int CT = 32 * VEC;
    __shared__ __align__(16) float sX[32][64];
    __shared__ __align__(16) float sY[32][CT];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int x0 = blockIdx.x * 64, y0 = blockIdx.y * CT;
    const int64_t p_begin = (int64_t)blockIdx.z * rows_per_split;
    const int64_t p_end = min(n, p_begin + rows_per_split);
    float acc[8][VEC];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int v = 0; v < VEC; ++v) acc[i][v] = 0.f;
    for (int64_t p0 = p_begin; p0 < p_end; p0 += 32) {
        __syncthreads();
        for (int e = t; e < 32 * 64; e += kThreads) {
            const int pr = e >> 6, j = e & 63;
            const int64_t p = p0 + pr;
            sX[pr][j] = (p < p_end && x0 + j < nx) ? X[p * ldx + x0 + j] : 0.f;
        }
        for (int e = t; e < 32 * CT; e += kThreads) {
            const int pr = e / CT, k = e % CT;
            const int64_t p = p0 + pr;
            sY[pr][k] = (p < p_end && y0 + k < ny) ? Y[p * ldy + y0 + k] : 0.f;
        }
        __syncthreads();
#pragma unroll 4
        for (int pr = 0; pr < 32; ++pr) {
            float xv[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) xv[i] = sX[pr][warp * 8 + i];
            float yv[VEC];
#pragma unroll
            for (int v = 0; v < VEC; ++v) yv[v] = sY[pr][lane * VEC + v];
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int v = 0; v < VEC; ++v) acc[i][v] += xv[i] * yv[v];
        }
    }
    const size_t base = (size_t)blockIdx.z * nx * ny;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int j = x0 + warp * 8 + i;
        if (j >= nx) continue;
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
            const int k = y0 + lane * VEC + v;
            if (k < ny) part[base + (size_t)j * ny + k] = acc[i][v];
        }
    }
}

// out[j][k] = scale * sum_s part[s][j][k] (+ coef[j] (V - V0)[j][k] when coef != NULL).  A CTA
// owns 32 consecutive outputs (lane = output); warp w adds the splits w, w + 8, ... in order and
// the eight warp sums are added in warp order, so the result does not depend on scheduling and
// no thread walks more than splits / 8 dependent loads.
__global__ void __launch_bounds__(256) reduce_splits(const float* __restrict__ part, int splits, int nx, int ny,
                                                     float scale, const float* __restrict__ coef,
                                                     const float* __restrict__ V, const float* __restrict__ V0,
                                                     float* __restrict__ out) {
    __shared__ float s_w[8][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t total = (int64_t)nx * ny;
    const int64_t e = (int64_t)blockIdx.x * 32 + lane;
    float s = 0.f;
    if (e < total)
        for (int k = warp; k < splits; k += 8) s += part[(size_t)k * total + e];
    s_w[warp][lane] = s;
    __syncthreads();
    if (warp != 0 || e >= total) return;
    float r = 0.f;
#pragma unroll
    for (int w = 0; w < 8; ++w) r += s_w[w][lane];
    r *= scale;
    if (coef) {
        const int j = (int)(e / ny);
        r += coef[j] * (V[e] - V0[e]);
    }
    out[e] = r;
}

__global__ void finalize_loss(const double* __restrict__ acc, int D, latentam_loss_cfg cfg, double* __restrict__ parts) {
    const double nv = acc[3];
    const double lcos = nv > 0 ? acc[0] / nv : 0.0;
    const double l2 = nv > 0 ? acc[1] / (nv * D) : 0.0;
    const double tr = acc[2];
    parts[0] = lcos;
    parts[1] = l2;
    parts[2] = tr;
    parts[3] = (double)cfg.lambda_f * ((double)cfg.lambda_cos * lcos + (double)cfg.lambda_2 * l2 +
                                       (double)cfg.lambda_D * tr);
    parts[4] = nv;
}

// ---- register-tiled FP32 GEMM (CUDA cores) --------------------------------------------------
//
// C (128 x 128 tile) = sum_k A(m, k) B(k, n) over one K split (blockIdx.z), 256 threads with an
// 8 x 8 register tile each (rows ty*4 + {0..3} and 64 + ty*4 + {0..3}, likewise the columns),
// operands staged through double-buffered shared memory 16 K-steps at a time.  A is read from a
// matrix stored with k contiguous (A_KM) or m contiguous; B with k contiguous (B_KM) or n
// contiguous.  The epilogue receives the 8 x 8 accumulator.

constexpr int kGM = 128, kGN = 128, kGK = 16, kGPad = 4;

// Row-major source matrix X (row stride ld); four consecutive elements of a row at a time.
// The GEMM loads a K slice into registers (load_raw) before computing on the previous one and
// turns it into operand values (finish) only when it stages them in shared memory, so the
// loads' latency hides behind the compute.
struct PlainSrc {
    const float* X;
    int64_t ld, rows, cols;
    using Raw = float4;
    __device__ __forceinline__ float4 load4(int64_t r, int64_t c) const {
        if (r >= rows || c >= cols) return make_float4(0.f, 0.f, 0.f, 0.f);
        return *reinterpret_cast<const float4*>(X + r * ld + c);
    }
    __device__ __forceinline__ Raw load_raw(int64_t r, int64_t c) const { return load4(r, c); }
    static __device__ __forceinline__ Raw zero_raw() { return make_float4(0.f, 0.f, 0.f, 0.f); }
    __device__ __forceinline__ float4 finish(const Raw& x) const { return x; }
};

// dL/dFhat (n x D) formed on load: a_p Fhat_p + b_p F_p with a_p = coef[4p], b_p = coef[4p+1].
struct DFhatSrc {
    const float* Fh;
    const void* F;
    latentam_dtype F_dtype;
    const float* coef;
    int64_t rows, cols;  // n, D
    struct Raw {
        float4 h;
        uint4 f;  // four FP32 targets, or four BF16 targets in f.x, f.y
        float a, b;
    };
    __device__ __forceinline__ Raw load_raw(int64_t r, int64_t c) const {
        Raw x;
        if (r >= rows || c >= cols) return zero_raw();
        x.a = coef[4 * r];
        x.b = coef[4 * r + 1];
        x.h = *reinterpret_cast<const float4*>(Fh + r * cols + c);
        const size_t i4 = (size_t)((r * cols + c) / 4);
        if (F_dtype == LATENTAM_DTYPE_F32) {
            x.f = reinterpret_cast<const uint4*>(F)[i4];
        } else {
            const uint2 u = reinterpret_cast<const uint2*>(F)[i4];
            x.f = make_uint4(u.x, u.y, 0u, 0u);
        }
        return x;
    }
    static __device__ __forceinline__ Raw zero_raw() {
        Raw x;
        x.h = make_float4(0.f, 0.f, 0.f, 0.f);
        x.f = make_uint4(0u, 0u, 0u, 0u);
        x.a = x.b = 0.f;
        return x;
    }
    __device__ __forceinline__ float4 finish(const Raw& x) const {
        float4 f;
        if (F_dtype == LATENTAM_DTYPE_F32) {
            f = make_float4(__uint_as_float(x.f.x), __uint_as_float(x.f.y), __uint_as_float(x.f.z),
                            __uint_as_float(x.f.w));
        } else {
            const float2 lo = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&x.f.x));
            const float2 hi = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&x.f.y));
            f = make_float4(lo.x, lo.y, hi.x, hi.y);
        }
        return make_float4(x.a * x.h.x + x.b * f.x, x.a * x.h.y + x.b * f.y, x.a * x.h.z + x.b * f.z,
                           x.a * x.h.w + x.b * f.w);
    }
};

template <bool A_KM, bool B_KM, class SrcA, class SrcB, class Epi>
__global__ void __launch_bounds__(256, 2) sgemm_tile(SrcA sa, SrcB sb, int64_t m_ext, int64_t n_ext, int64_t k_ext,
                                                     int64_t k_per_split, typename Epi::Params ep) {
    __shared__ __align__(16) float sA[2][kGK][kGM + kGPad];
    __shared__ __align__(16) float sB[2][kGK][kGN + kGPad];
    const int t = threadIdx.x, ty = t >> 4, tx = t & 15;
    // x: column tile, y: row tile (the column tiles of a row tile run together and share its
    // A rows in L2)
    const int64_t m0 = (int64_t)blockIdx.y * kGM, n0 = (int64_t)blockIdx.x * kGN;
    const int64_t kb = (int64_t)blockIdx.z * k_per_split;
    const int64_t ke = min(k_ext, kb + k_per_split);
    typename SrcA::Raw ra[2];
    typename SrcB::Raw rb[2];
    // global -> registers for the K slice starting at k0
    auto fetch = [&](int64_t k0) {
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int e = t + 256 * i;
            if (A_KM) {
                const int mm = e >> 2, kq = (e & 3) * 4;
                ra[i] = (k0 + kq < ke) ? sa.load_raw(m0 + mm, k0 + kq) : SrcA::zero_raw();
            } else {
                const int kk = e >> 5, mq = (e & 31) * 4;
                ra[i] = (k0 + kk < ke) ? sa.load_raw(k0 + kk, m0 + mq) : SrcA::zero_raw();
            }
            if (B_KM) {
                const int nn = e >> 2, kq = (e & 3) * 4;
                rb[i] = (k0 + kq < ke) ? sb.load_raw(n0 + nn, k0 + kq) : SrcB::zero_raw();
            } else {
                const int kk = e >> 5, nq = (e & 31) * 4;
                rb[i] = (k0 + kk < ke) ? sb.load_raw(k0 + kk, n0 + nq) : SrcB::zero_raw();
            }
        }
    };
    // registers -> operand values -> shared buffer `buf`
    auto stash = [&](int buf) {
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int e = t + 256 * i;
            const float4 va = sa.finish(ra[i]), vb = sb.finish(rb[i]);
            if (A_KM) {
                const int mm = e >> 2, kq = (e & 3) * 4;
                sA[buf][kq][mm] = va.x;
                sA[buf][kq + 1][mm] = va.y;
                sA[buf][kq + 2][mm] = va.z;
                sA[buf][kq + 3][mm] = va.w;
            } else {
                *reinterpret_cast<float4*>(&sA[buf][e >> 5][(e & 31) * 4]) = va;
            }
            if (B_KM) {
                const int nn = e >> 2, kq = (e & 3) * 4;
                sB[buf][kq][nn] = vb.x;
                sB[buf][kq + 1][nn] = vb.y;
                sB[buf][kq + 2][nn] = vb.z;
                sB[buf][kq + 3][nn] = vb.w;
            } else {
                *reinterpret_cast<float4*>(&sB[buf][e >> 5][(e & 31) * 4]) = vb;
            }
        }
    };
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
    int buf = 0;
    if (kb < ke) {
        fetch(kb);
        stash(0);
    }
    __syncthreads();
    for (int64_t k0 = kb; k0 < ke; k0 += kGK) {
        const bool more = k0 + kGK < ke;
        if (more) fetch(k0 + kGK);
        else Epi::prefetch(ep, m0, n0, m_ext, n_ext);
#pragma unroll
        for (int k = 0; k < kGK; ++k) {
            const float4 a0 = *reinterpret_cast<const float4*>(&sA[buf][k][ty * 4]);
            const float4 a1 = *reinterpret_cast<const float4*>(&sA[buf][k][64 + ty * 4]);
            const float4 b0 = *reinterpret_cast<const float4*>(&sB[buf][k][tx * 4]);
            const float4 b1 = *reinterpret_cast<const float4*>(&sB[buf][k][64 + tx * 4]);
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] += av[i] * bv[j];
        }
        if (more) stash(buf ^ 1);
        __syncthreads();
        buf ^= 1;
    }
    Epi::store(ep, m0, n0, ty, tx, acc, m_ext, n_ext, (int)blockIdx.z);
}

// Narrow form for products with few columns (dQ = c dS K and dK = c dS^T Q, n <= 64): 128 x 32
// tiles, 256 threads with 4 x 4 each; B is read n-contiguous.  C[m][n] = scale * acc is stored
// at C + z * split_stride (row stride ld).
template <bool A_KM>
__global__ void __launch_bounds__(256) sgemm_narrow(PlainSrc sa, PlainSrc sb, int64_t m_ext, int64_t n_ext,
                                                    int64_t k_ext, int64_t k_per_split, float* __restrict__ C,
                                                    int64_t ld, int64_t split_stride, float scale) {
    constexpr int TN = 32;
    __shared__ __align__(16) float sA[2][kGK][kGM + kGPad];
    __shared__ __align__(16) float sB[2][kGK][TN + kGPad];
    const int t = threadIdx.x, ty = t >> 3, tx = t & 7;
    const int64_t m0 = (int64_t)blockIdx.y * kGM, n0 = (int64_t)blockIdx.x * TN;
    const int64_t kb = (int64_t)blockIdx.z * k_per_split;
    const int64_t ke = min(k_ext, kb + k_per_split);
    float4 ra[2], rb = make_float4(0.f, 0.f, 0.f, 0.f);
    auto fetch = [&](int64_t k0) {
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int e = t + 256 * i;
            if (A_KM) {
                const int mm = e >> 2, kq = (e & 3) * 4;
                ra[i] = (k0 + kq < ke) ? sa.load4(m0 + mm, k0 + kq) : make_float4(0.f, 0.f, 0.f, 0.f);
            } else {
                const int kk = e >> 5, mq = (e & 31) * 4;
                ra[i] = (k0 + kk < ke) ? sa.load4(k0 + kk, m0 + mq) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
        if (t < kGK * TN / 4) {
            const int kk = t >> 3, nq = (t & 7) * 4;
            rb = (k0 + kk < ke) ? sb.load4(k0 + kk, n0 + nq) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
    };
    auto stash = [&](int buf) {
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int e = t + 256 * i;
            if (A_KM) {
                const int mm = e >> 2, kq = (e & 3) * 4;
                sA[buf][kq][mm] = ra[i].x;
                sA[buf][kq + 1][mm] = ra[i].y;
                sA[buf][kq + 2][mm] = ra[i].z;
                sA[buf][kq + 3][mm] = ra[i].w;
            } else {
                *reinterpret_cast<float4*>(&sA[buf][e >> 5][(e & 31) * 4]) = ra[i];
            }
        }
        if (t < kGK * TN / 4) *reinterpret_cast<float4*>(&sB[buf][t >> 3][(t & 7) * 4]) = rb;
    };
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    int buf = 0;
    if (kb < ke) {
        fetch(kb);
        stash(0);
    }
    __syncthreads();
    for (int64_t k0 = kb; k0 < ke; k0 += kGK) {
        const bool more = k0 + kGK < ke;
        if (more) fetch(k0 + kGK);
#pragma unroll
        for (int k = 0; k < kGK; ++k) {
            const float4 a = *reinterpret_cast<const float4*>(&sA[buf][k][ty * 4]);
            const float4 b = *reinterpret_cast<const float4*>(&sB[buf][k][tx * 4]);
            const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] += av[i] * bv[j];
        }
        if (more) stash(buf ^ 1);
        __syncthreads();
        buf ^= 1;
    }
    float* Cz = C + (int64_t)blockIdx.z * split_stride;
    const int64_t c = n0 + tx * 4;
    if (c >= n_ext) return;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t m = m0 + ty * 4 + i;
        if (m < m_ext)
            *reinterpret_cast<float4*>(Cz + m * ld + c) =
                make_float4(scale * acc[i][0], scale * acc[i][1], scale * acc[i][2], scale * acc[i][3]);
    }
}

__device__ __forceinline__ int64_t tile_row(int64_t m0, int ty, int i) { return m0 + (i < 4 ? ty * 4 + i : 60 + ty * 4 + i); }
__device__ __forceinline__ int64_t tile_col(int64_t n0, int tx) { return n0 + tx * 4; }  // and + 64

// L2 prefetch of the 128 x 128 block of a row-major matrix (row stride ld elements of `esz`
// bytes) at (m0, n0), clipped to rows x cols: one 128-byte line per thread and step.
__device__ __forceinline__ void prefetch_tile_l2(const void* base, int64_t ld, int esz, int64_t m0, int64_t n0,
                                                 int64_t rows, int64_t cols) {
    const int lines_per_row = (kGN * esz + 127) / 128;
    for (int l = threadIdx.x; l < kGM * lines_per_row; l += blockDim.x) {
        const int64_t r = m0 + l / lines_per_row, c = n0 + (int64_t)(l % lines_per_row) * (128 / esz);
        if (r < rows && c < cols) {
            const char* ptr = static_cast<const char*>(base) + (r * ld + c) * esz;
            asm volatile("prefetch.global.L2 [%0];" ::"l"(ptr));
        }
    }
}

// Fhat tile: stored; with `stats`, the per-row partial sums <Fhat,F>, |Fhat|^2, |F|^2,
// |Fhat - F|^2 over the tile's 128 columns go to stats[(p * tiles + column tile) * 4 ...]
// (summed in a fixed order later: the result does not depend on the order the tiles run in).
struct FhatTileEpi {
    struct Params {
        float* Fh;
        int64_t D;
        const void* F;
        latentam_dtype F_dtype;
        float* stats;
    };
    // the targets the statistics read, while the last K slice computes
    static __device__ __forceinline__ void prefetch(const Params& p, int64_t m0, int64_t n0, int64_t m_ext,
                                                    int64_t n_ext) {
        if (p.stats)
            prefetch_tile_l2(p.F, p.D, p.F_dtype == LATENTAM_DTYPE_F32 ? 4 : 2, m0, n0, m_ext, n_ext);
    }
    static __device__ __forceinline__ void store(const Params& p, int64_t m0, int64_t n0, int ty, int tx,
                                                 float (&acc)[8][8], int64_t m_ext, int64_t n_ext, int) {
        // four rows at a time: their target loads are issued together, ahead of the stores
        float4 fr[4][2];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int64_t m = tile_row(m0, ty, i);
            if ((i & 3) == 0 && p.stats) {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int64_t mj = tile_row(m0, ty, i + j);
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int64_t c = tile_col(n0, tx) + 64 * h;
                        fr[j][h] = (mj < m_ext && c < n_ext) ? load_target4(p.F, p.F_dtype, (size_t)((mj * p.D + c) / 4))
                                                             : make_float4(0.f, 0.f, 0.f, 0.f);
                    }
                }
            }
            float s[4] = {0.f, 0.f, 0.f, 0.f};
            if (m < m_ext) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int64_t c = tile_col(n0, tx) + 64 * h;
                    if (c >= n_ext) continue;
                    const float4 v = make_float4(acc[i][4 * h], acc[i][4 * h + 1], acc[i][4 * h + 2], acc[i][4 * h + 3]);
                    *reinterpret_cast<float4*>(p.Fh + m * p.D + c) = v;
                    if (p.stats) {
                        const float4 f = fr[i & 3][h];
                        const float hv[4] = {v.x, v.y, v.z, v.w}, fv[4] = {f.x, f.y, f.z, f.w};
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            s[0] += hv[q] * fv[q];
                            s[1] += hv[q] * hv[q];
                            s[2] += fv[q] * fv[q];
                            const float e = hv[q] - fv[q];
                            s[3] += e * e;
                        }
                    }
                }
            }
            if (p.stats) {
                // the 16 threads of one tile row are 16 consecutive lanes
#pragma unroll
                for (int q = 0; q < 4; ++q)
#pragma unroll
                    for (int o = 8; o > 0; o >>= 1) s[q] += __shfl_xor_sync(0xffffffffu, s[q], o);
                if (tx == 0 && m < m_ext) {
                    const int64_t tiles = (p.D + kGN - 1) / kGN;
                    *reinterpret_cast<float4*>(p.stats + (m * tiles + n0 / kGN) * 4) = make_float4(s[0], s[1], s[2], s[3]);
                }
            }
        }
    }
};

// dS tile: dS = A (dA - <A, dA>_p) with <A, dA>_p = coef[4p + 2]; A and dS are n x M.
struct DsTileEpi {
    struct Params {
        const float* A;
        const float* coef;
        float* dS;
        int64_t M;
    };
    static __device__ __forceinline__ void prefetch(const Params& p, int64_t m0, int64_t n0, int64_t m_ext,
                                                    int64_t n_ext) {
        prefetch_tile_l2(p.A, p.M, 4, m0, n0, m_ext, n_ext);
        if (threadIdx.x < kGM * 16 / 128) {
            const int64_t r = m0 + threadIdx.x * 8;
            if (r < m_ext) asm volatile("prefetch.global.L2 [%0];" ::"l"(p.coef + 4 * r));
        }
    }
    static __device__ __forceinline__ void store(const Params& p, int64_t m0, int64_t n0, int ty, int tx,
                                                 float (&acc)[8][8], int64_t m_ext, int64_t n_ext, int) {
        // four rows at a time: their attention and coefficient loads are issued together,
        // ahead of the stores
#pragma unroll
        for (int g = 0; g < 2; ++g) {
            float4 av[4][2];
            float rd[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int64_t m = tile_row(m0, ty, 4 * g + j);
                rd[j] = m < m_ext ? p.coef[4 * m + 2] : 0.f;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int64_t c = tile_col(n0, tx) + 64 * h;
                    av[j][h] = (m < m_ext && c < n_ext) ? *reinterpret_cast<const float4*>(p.A + m * p.M + c)
                                                        : make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int i = 4 * g + j;
                const int64_t m = tile_row(m0, ty, i);
                if (m >= m_ext) continue;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int64_t c = tile_col(n0, tx) + 64 * h;
                    if (c >= n_ext) continue;
                    const float4 a = av[j][h];
                    *reinterpret_cast<float4*>(p.dS + m * p.M + c) =
                        make_float4(a.x * (acc[i][4 * h] - rd[j]), a.y * (acc[i][4 * h + 1] - rd[j]),
                                    a.z * (acc[i][4 * h + 2] - rd[j]), a.w * (acc[i][4 * h + 3] - rd[j]));
                }
            }
        }
    }
};

// Plain scaled store C[m][n] = scale * acc into a row-major (ld) matrix, split z at offset
// z * split_stride (the partial sums of a split-K product, or dQ).
struct StoreTileEpi {
    struct Params {
        float* C;
        int64_t ld, split_stride;
        float scale;
    };
    static __device__ __forceinline__ void prefetch(const Params&, int64_t, int64_t, int64_t, int64_t) {}
    static __device__ __forceinline__ void store(const Params& p, int64_t m0, int64_t n0, int ty, int tx,
                                                 float (&acc)[8][8], int64_t m_ext, int64_t n_ext, int z) {
        float* C = p.C + (int64_t)z * p.split_stride;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int64_t m = tile_row(m0, ty, i);
            if (m >= m_ext) continue;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int64_t c = tile_col(n0, tx) + 64 * h;
                if (c >= n_ext) continue;
                *reinterpret_cast<float4*>(C + m * p.ld + c) =
                    make_float4(p.scale * acc[i][4 * h], p.scale * acc[i][4 * h + 1], p.scale * acc[i][4 * h + 2],
                                p.scale * acc[i][4 * h + 3]);
            }
        }
    }
};

// Per-pixel coefficients of dL/dFhat from the row sums (a_p, b_p, <A_p, dA_p>, cos_p into
// coef) and the frame's loss sums (FP64, one atomic pair per warp).
__global__ void __launch_bounds__(256) coef_rows(const float* __restrict__ stats, int64_t n, int D,
                                                 const uint8_t* __restrict__ mask, latentam_loss_cfg cfg,
                                                 double* __restrict__ acc, float* __restrict__ coef) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float lc = 0.f, le = 0.f;
    if (p < n) {
        const int tiles = (D + kGN - 1) / kGN;
        float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int k = 0; k < tiles; ++k) {  // column tiles in order
            const float4 u = *reinterpret_cast<const float4*>(stats + ((int64_t)p * tiles + k) * 4);
            s.x += u.x, s.y += u.y, s.z += u.z, s.w += u.w;
        }
        const float dot = s.x, nh2 = s.y, nf2 = s.z, e2 = s.w;
        const bool valid = mask == nullptr || mask[p] != 0;
        const float nv = (float)acc[3];
        const float scale = nv > 0.f ? cfg.lambda_f / nv : 0.f;
        const float den = sqrtf(nh2) * sqrtf(nf2);
        const float cs = dot / fmaxf(den, 1e-8f);
        float a = 0.f, b = 0.f;
        if (valid) {
            lc = 1.0f - cs;
            le = e2;
            const float l2c = 2.0f * cfg.lambda_2 / (float)D;
            if (den > 1e-8f) {
                a = scale * (cfg.lambda_cos * cs / nh2 + l2c);
                b = scale * (-cfg.lambda_cos / den - l2c);
            } else {
                a = scale * l2c;
                b = scale * (-cfg.lambda_cos / 1e-8f - l2c);
            }
        }
        *reinterpret_cast<float4*>(coef + 4 * p) = make_float4(a, b, a * nh2 + b * dot, cs);
    }
    lc = warp_sum(lc);
    le = warp_sum(le);
    if ((threadIdx.x & 31) == 0 && (lc != 0.f || le != 0.f)) {
        atomicAdd(&acc[0], (double)lc);
        atomicAdd(&acc[1], (double)le);
    }
}

// *z_out (nullable) receives the number of K splits launched.
template <bool A_KM, bool B_KM, class SrcA, class SrcB, class Epi>
latentam_status launch_sgemm(const SrcA& a, const SrcB& b, int64_t m_ext, int64_t n_ext, int64_t k_ext, int splits,
                             const typename Epi::Params& ep, cudaStream_t st, int* z_out = nullptr) {
    if (z_out) *z_out = 0;
    if (m_ext <= 0 || n_ext <= 0 || k_ext <= 0) return LATENTAM_OK;
    const int64_t kps = ((k_ext + splits - 1) / splits + kGK - 1) / kGK * kGK;
    const int z = (int)std::max<int64_t>(1, (k_ext + kps - 1) / std::max<int64_t>(kps, 1));
    if (z_out) *z_out = z;
    dim3 grid((unsigned)((n_ext + kGN - 1) / kGN), (unsigned)((m_ext + kGM - 1) / kGM), (unsigned)z);
    sgemm_tile<A_KM, B_KM, SrcA, SrcB, Epi><<<grid, 256, 0, st>>>(a, b, m_ext, n_ext, k_ext, kps, ep);
    LAT_CHECK_LAUNCH("sgemm_tile");
    return LATENTAM_OK;
}

template <bool A_KM>
latentam_status launch_narrow(const PlainSrc& a, const PlainSrc& b, int64_t m_ext, int64_t n_ext, int64_t k_ext,
                              int splits, float* C, int64_t ld, int64_t split_stride, float scale, cudaStream_t st,
                              int* z_out = nullptr) {
    if (z_out) *z_out = 0;
    if (m_ext <= 0 || n_ext <= 0 || k_ext <= 0) return LATENTAM_OK;
    const int64_t kps = ((k_ext + splits - 1) / splits + kGK - 1) / kGK * kGK;
    const int z = (int)std::max<int64_t>(1, (k_ext + kps - 1) / kps);
    if (z_out) *z_out = z;
    dim3 grid((unsigned)((n_ext + 31) / 32), (unsigned)((m_ext + kGM - 1) / kGM), (unsigned)z);
    sgemm_narrow<A_KM><<<grid, 256, 0, st>>>(a, b, m_ext, n_ext, k_ext, kps, C, ld, split_stride, scale);
    LAT_CHECK_LAUNCH("sgemm_narrow");
    return LATENTAM_OK;
}

// Number of K splits of a pixel reduction: about two CTAs per SM over the output tiles.
int tile_splits(int num_sms, int64_t m_ext, int64_t n_ext, int64_t k_ext) {
    const int64_t tiles = ((m_ext + kGM - 1) / kGM) * ((n_ext + kGN - 1) / kGN);
    int64_t z = std::max<int64_t>(1, (2 * num_sms + tiles - 1) / tiles);
    z = std::min<int64_t>(z, std::max<int64_t>(1, k_ext / 256));
    return (int)z;
}

// S = c Q K^T and its row softmax for d = 32 queries and M = 32 MU <= 256 atoms (the attention
// weights A and the row statistics (max, sum) only): a persistent CTA stages K^T once, then
// takes 64-row tiles; warp w owns rows 8 w .. 8 w + 7 and lane l the atoms l + 32 u, so each row's
// max and sum are warp reductions and every K value read from shared memory feeds 8 rows.
// The arithmetic of every row is dec_rows_fwd's, in the same order (S accumulated over k in
// order and scaled by c, the per-lane sums over u in order, then the same warp reduction), so
// A and the statistics are the same numbers.
constexpr int kAttnRows = 64;
template <int MU>
__global__ void __launch_bounds__(256, 2) attn_rows_d32(const float* __restrict__ Q, int64_t n,
                                                         const float* __restrict__ K, float c,
                                                         float* __restrict__ A_out, float* __restrict__ stats_out) {
    constexpr int DQ = 32, M = 32 * MU;
    __shared__ __align__(16) float sKt[DQ][M];              // K transposed: atom j at column j
    __shared__ __align__(16) float sQt[DQ][kAttnRows + 4];  // the tile's queries transposed
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    for (int e = t; e < M * DQ; e += 256) {  // consecutive threads: consecutive atoms (no bank conflict)
        const int k = e / M, j = e % M;
        sKt[k][j] = K[j * DQ + k];
    }
    const int64_t tiles = (n + kAttnRows - 1) / kAttnRows;
    for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int64_t row0 = tile * kAttnRows;
        __syncthreads();  // K staged / the previous tile's queries read
        for (int e = t; e < kAttnRows * DQ / 4; e += 256) {
            const int r = e / (DQ / 4), k4 = (e % (DQ / 4)) * 4;
            const float4 q = (row0 + r < n) ? *reinterpret_cast<const float4*>(Q + (row0 + r) * DQ + k4)
                                            : make_float4(0.f, 0.f, 0.f, 0.f);
            sQt[k4][r] = q.x;
            sQt[k4 + 1][r] = q.y;
            sQt[k4 + 2][r] = q.z;
            sQt[k4 + 3][r] = q.w;
        }
        __syncthreads();
        float s[8][MU];
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
            for (int u = 0; u < MU; ++u) s[r][u] = 0.f;
#pragma unroll 4
        for (int k = 0; k < DQ; ++k) {
            const float4 q0 = *reinterpret_cast<const float4*>(&sQt[k][warp * 8]);
            const float4 q1 = *reinterpret_cast<const float4*>(&sQt[k][warp * 8 + 4]);
            const float q[8] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
            float kv[MU];
#pragma unroll
            for (int u = 0; u < MU; ++u) kv[u] = sKt[k][lane + 32 * u];
#pragma unroll
            for (int r = 0; r < 8; ++r)
#pragma unroll
                for (int u = 0; u < MU; ++u) s[r][u] += q[r] * kv[u];
        }
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const int64_t p = row0 + warp * 8 + r;
            float a[MU];
            float m = -INFINITY;
#pragma unroll
            for (int u = 0; u < MU; ++u) {
                a[u] = c * s[r][u];
                m = fmaxf(m, a[u]);
            }
            m = warp_max(m);
            float l = 0.f;
#pragma unroll
            for (int u = 0; u < MU; ++u) {
                a[u] = __expf(a[u] - m);
                l += a[u];
            }
            l = warp_sum(l);
            const float il = 1.0f / l;
            if (p < n) {
#pragma unroll
                for (int u = 0; u < MU; ++u) A_out[p * M + lane + 32 * u] = a[u] * il;
                if (lane == 0 && stats_out) {
                    stats_out[2 * p] = m;
                    stats_out[2 * p + 1] = l;
                }
            }
        }
    }
}

size_t rows_fwd_smem(int d, int M) { return sizeof(float) * ((size_t)kRows * M + (size_t)d * (kAtomChunk + 1) + (size_t)kRows * d); }
size_t rows_bwd_smem(int M) { return sizeof(float) * ((size_t)kRows * M + (size_t)kAtomChunk * 33 + (size_t)kRows * 33); }

template <int DQ, int MODE>
latentam_status launch_rows_fwd(const float* Q, int64_t n, const float* K, const float* V, int M, int D, float c,
                                const void* F, latentam_dtype F_dtype, const uint8_t* mask,
                                const latentam_loss_cfg& cfg, double* acc, float* A_out, float* Fh, float* row,
                                float* stats, cudaStream_t st) {
    if constexpr (DQ == 32 && MODE == 2) {
        if (M == 64 || M == 128 || M == 256) {
            int dev = 0, sms = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            const unsigned blocks =
                (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + kAttnRows - 1) / kAttnRows, 2 * (int64_t)sms));
            if (M == 64) attn_rows_d32<2><<<blocks, 256, 0, st>>>(Q, n, K, c, A_out, stats);
            else if (M == 128) attn_rows_d32<4><<<blocks, 256, 0, st>>>(Q, n, K, c, A_out, stats);
            else attn_rows_d32<8><<<blocks, 256, 0, st>>>(Q, n, K, c, A_out, stats);
            LAT_CHECK_LAUNCH("attn_rows_d32");
            return LATENTAM_OK;
        }
    }
    const size_t smem = rows_fwd_smem(DQ, M);
    auto kern = dec_rows_fwd<DQ, MODE>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_error(e, "dec_rows_fwd smem attribute");
    const unsigned blocks = (unsigned)((n + kRows - 1) / kRows);
    kern<<<blocks, kThreads, smem, st>>>(Q, n, K, V, M, D, c, F, F_dtype, mask, cfg, acc, A_out, Fh, row, stats);
    LAT_CHECK_LAUNCH("dec_rows_fwd");
    return LATENTAM_OK;
}

template <int DQ>
latentam_status launch_rows_bwd(const float* dFh, const float* A, const float* row, const float* K, const float* V,
                                int64_t n, int M, int D, float c, float* dS, float* dQ, cudaStream_t st) {
    const size_t smem = rows_bwd_smem(M);
    auto kern = dec_rows_bwd<DQ>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_error(e, "dec_rows_bwd smem attribute");
    const unsigned blocks = (unsigned)((n + kRows - 1) / kRows);
    kern<<<blocks, kThreads, smem, st>>>(dFh, A, row, K, V, n, M, D, c, dS, dQ);
    LAT_CHECK_LAUNCH("dec_rows_bwd");
    return LATENTAM_OK;
}

// The FP32 form: S and the softmax in the row kernel, then register-tiled GEMMs:
//   Fhat = A V (+ per-row loss sums)  ->  per-pixel coefficients a_p, b_p  ->
//   dA = dFhat V^T (dFhat = a_p Fhat + b_p F formed on load) -> dS = A (dA - <A, dA>),
//   dQ = c dS K,  dV = A^T dFhat (split over pixels),  dK = c dS^T Q (split over pixels).
template <int DQ>
latentam_status loss_bwd_t(latentam_ctx* ctx, const DecodeArgs& a, cudaStream_t st) {
    const int64_t n = a.n, nn = std::max<int64_t>(n, 1);
    const int M = a.M, D = a.D;
    double* acc = static_cast<double*>(ws(ctx, WS_LOSS, sizeof(double) * 8));
    float* A = static_cast<float*>(ws(ctx, WS_DEC_A, sizeof(float) * (size_t)nn * M));
    float* Fh = static_cast<float*>(ws(ctx, WS_DEC_DF, sizeof(float) * (size_t)nn * D));
    float* dS = static_cast<float*>(ws(ctx, WS_DEC_DS, sizeof(float) * (size_t)nn * M));
    float* coef = static_cast<float*>(ws(ctx, WS_DEC_ROW, sizeof(float) * 4 * (size_t)nn));
    const int ctiles = (D + kGN - 1) / kGN;
    float* stats = static_cast<float*>(ws(ctx, WS_DEC_AUX, sizeof(float) * 4 * (size_t)nn * ctiles));
    float* trc = static_cast<float*>(ws(ctx, WS_DEC_AUX3, sizeof(float) * (size_t)M));
    if (!acc || !A || !Fh || !dS || !coef || !stats || !trc) return LATENTAM_ERR_OUT_OF_MEMORY;
    cudaError_t e = cudaMemsetAsync(acc, 0, sizeof(double) * 8, st);
    if (e != cudaSuccess) return cuda_error(e, "memset loss");
    if (n > 0) {
        const unsigned cb = (unsigned)std::min<int64_t>((n + kThreads - 1) / kThreads, 4 * ctx->num_sms);
        count_mask_kernel<<<cb, kThreads, 0, st>>>(a.mask, n, acc);
        LAT_CHECK_LAUNCH("count_mask_kernel");
    }
    trust_region_kernel<<<(unsigned)((M + 7) / 8), 256, 0, st>>>(a.V, a.V0, M, D, a.cfg.delta,
                                                                 a.cfg.lambda_f * a.cfg.lambda_D, trc, acc);
    LAT_CHECK_LAUNCH("trust_region_kernel");
    const PlainSrc Asrc{A, M, n, M}, Vsrc{a.V, D, M, D}, dSsrc{dS, M, n, M};
    const DFhatSrc dFsrc{Fh, a.F, a.F_dtype, coef, n, D};
    if (n > 0) {
        LAT_TRY((launch_rows_fwd<DQ, 2>(a.Q, n, a.K, a.V, M, D, a.c, nullptr, LATENTAM_DTYPE_F32, nullptr, a.cfg,
                                        nullptr, A, nullptr, nullptr, nullptr, st)));
        LAT_TRY((launch_sgemm<true, false, PlainSrc, PlainSrc, FhatTileEpi>(
            Asrc, Vsrc, n, D, M, 1, FhatTileEpi::Params{Fh, D, a.F, a.F_dtype, stats}, st)));
        coef_rows<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(stats, n, D, a.mask, a.cfg, acc, coef);
        LAT_CHECK_LAUNCH("coef_rows");
        if (a.dQ || a.dK)
            LAT_TRY((launch_sgemm<true, true, DFhatSrc, PlainSrc, DsTileEpi>(dFsrc, Vsrc, n, M, D, 1,
                                                                             DsTileEpi::Params{A, coef, dS, M}, st)));
        if (a.dQ) {
            const PlainSrc Ksrc{a.K, DQ, M, DQ};
            LAT_TRY(launch_narrow<true>(dSsrc, Ksrc, n, DQ, M, 1, a.dQ, DQ, 0, a.c, st));
        }
    }
    if (a.dV) {
        const int z0 = n > 0 ? tile_splits(ctx->num_sms, M, D, n) : 1;
        float* part = static_cast<float*>(ws(ctx, WS_DEC_PART, sizeof(float) * (size_t)z0 * M * D));
        if (!part) return LATENTAM_ERR_OUT_OF_MEMORY;
        int z = 0;
        LAT_TRY((launch_sgemm<false, false, PlainSrc, DFhatSrc, StoreTileEpi>(
            Asrc, dFsrc, M, D, n, z0, StoreTileEpi::Params{part, D, (int64_t)M * D, 1.0f}, st, &z)));
        reduce_splits<<<(unsigned)(((int64_t)M * D + 31) / 32), 256, 0, st>>>(part, z, M, D, 1.0f, trc, a.V, a.V0,
                                                                               a.dV);
        LAT_CHECK_LAUNCH("reduce_splits");
    }
    if (a.dK) {
        // narrow tiles: (M / 128) x (d / 32) of them, so more pixel splits
        const int64_t ntiles = ((M + kGM - 1) / kGM) * ((DQ + 31) / 32);
        const int z0 = n > 0 ? (int)std::max<int64_t>(1, std::min<int64_t>((4 * ctx->num_sms + ntiles - 1) / ntiles,
                                                                            std::max<int64_t>(1, n / 256)))
                             : 1;
        float* part = static_cast<float*>(ws(ctx, WS_DEC_PART, sizeof(float) * (size_t)z0 * M * DQ));
        if (!part) return LATENTAM_ERR_OUT_OF_MEMORY;
        const PlainSrc Qsrc{a.Q, DQ, n, DQ};
        int z = 0;
        LAT_TRY(launch_narrow<false>(dSsrc, Qsrc, M, DQ, n, z0, part, DQ, (int64_t)M * DQ, 1.0f, st, &z));
        reduce_splits<<<(unsigned)(((int64_t)M * DQ + 31) / 32), 256, 0, st>>>(part, z, M, DQ, a.c, nullptr,
                                                                                nullptr, nullptr, a.dK);
        LAT_CHECK_LAUNCH("reduce_splits");
    }
    finalize_loss<<<1, 1, 0, st>>>(acc, D, a.cfg, a.loss_parts);
    LAT_CHECK_LAUNCH("finalize_loss");
    return LATENTAM_OK;
}

template <int DQ>
latentam_status decode_fwd_t(latentam_ctx* ctx, const float* Q, int64_t n, const float* K, const float* V, int M,
                             int D, float c, float* F_hat, float* row_stats, cudaStream_t st) {
    if (n == 0) return LATENTAM_OK;
    float* A = static_cast<float*>(ws(ctx, WS_DEC_A, sizeof(float) * (size_t)n * M));
    if (!A) return LATENTAM_ERR_OUT_OF_MEMORY;
    latentam_loss_cfg cfg{};
    LAT_TRY((launch_rows_fwd<DQ, 2>(Q, n, K, V, M, D, c, nullptr, LATENTAM_DTYPE_F32, nullptr, cfg, nullptr, A,
                                    nullptr, nullptr, row_stats, st)));
    if (!F_hat) return LATENTAM_OK;
    const PlainSrc Asrc{A, M, n, M}, Vsrc{V, D, M, D};
    return launch_sgemm<true, false, PlainSrc, PlainSrc, FhatTileEpi>(
        Asrc, Vsrc, n, D, M, 1, FhatTileEpi::Params{F_hat, D, nullptr, LATENTAM_DTYPE_F32, nullptr}, st);
}

// ---- allocation-free variant -------------------------------------------------------------
// Scratch of decode_loss_bwd_f32_noalloc: one file-scope device array.  Host code only ever
// sees a host-side stand-in for the symbol; the device address comes from cudaGetSymbolAddress,
// called by decode_noalloc_setup when a context is created (that device current), which also
// loads this module and so commits the array on the device before the first call.
constexpr size_t kStaticScratchBytes = (size_t)16 << 20;
__device__ __align__(256) unsigned char g_noalloc_scratch[kStaticScratchBytes];

struct NoallocPlan {
    size_t acc, A, dF, dS, row, coef, partV, partK, total;
    int64_t splitsV, rpsV, splitsK, rpsK;
};

// Split of a pixel reduction over atb_splitk: about two CTAs per SM, at least 256 pixels per split.
void plan_split(int num_sms, int nx, int ny, int64_t n, int64_t* splits_out, int64_t* rps_out) {
    const int vec = ny >= 128 ? 4 : 1;
    const int ct = 32 * vec;
    const int bx = (nx + 63) / 64, by = (ny + ct - 1) / ct;
    int64_t splits = std::max<int64_t>(1, (2 * num_sms + bx * by - 1) / (bx * by));
    splits = std::min<int64_t>(splits, std::max<int64_t>(1, (n + 255) / 256));
    const int64_t rps = std::max<int64_t>(32, ((n + splits - 1) / splits + 31) / 32 * 32);
    *rps_out = rps;
    *splits_out = std::max<int64_t>(1, (n + rps - 1) / rps);
}

NoallocPlan plan_noalloc(int num_sms, int64_t n, int M, int D, int d) {
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    NoallocPlan p{};
    plan_split(num_sms, M, D, n, &p.splitsV, &p.rpsV);
    plan_split(num_sms, M, d, n, &p.splitsK, &p.rpsK);
    size_t o = 0;
    p.acc = o;
    o += up(sizeof(double) * 8);
    p.A = o;
    o += up(sizeof(float) * (size_t)n * M);
    p.dF = o;
    o += up(sizeof(float) * (size_t)n * D);
    p.dS = o;
    o += up(sizeof(float) * (size_t)n * M);
    p.row = o;
    o += up(sizeof(float) * 4 * (size_t)n);
    p.coef = o;
    o += up(sizeof(float) * (size_t)M);
    p.partV = o;
    o += up(sizeof(float) * (size_t)p.splitsV * M * D);
    p.partK = o;
    o += up(sizeof(float) * (size_t)p.splitsK * M * d);
    p.total = o;
    return p;
}

latentam_status atb_noalloc(const float* X, int ldx, int nx, const float* Y, int ldy, int ny, int64_t n, float scale,
                            const float* coef, const float* V, const float* V0, float* out, float* part,
                            int64_t splits, int64_t rps, cudaStream_t st) {
    const int vec = ny >= 128 ? 4 : 1;
    const int ct = 32 * vec;
    dim3 grid((unsigned)((nx + 63) / 64), (unsigned)((ny + ct - 1) / ct), (unsigned)splits);
    if (vec == 4)
        atb_splitk<4><<<grid, kThreads, 0, st>>>(X, ldx, nx, Y, ldy, ny, n, rps, part);
    else
        atb_splitk<1><<<grid, kThreads, 0, st>>>(X, ldx, nx, Y, ldy, ny, n, rps, part);
    LAT_CHECK_LAUNCH("atb_splitk");
    const int64_t total = (int64_t)nx * ny;
    reduce_splits<<<(unsigned)((total + 31) / 32), 256, 0, st>>>(part, (int)splits, nx, ny, scale, coef, V, V0, out);
    LAT_CHECK_LAUNCH("reduce_splits");
    return LATENTAM_OK;
}

template <int DQ>
latentam_status loss_bwd_noalloc_t(latentam_ctx* ctx, const DecodeArgs& a, cudaStream_t st) {
    const int64_t n = a.n;
    const int M = a.M, D = a.D;
    const NoallocPlan p = plan_noalloc(ctx->num_sms, n, M, D, DQ);
    if (p.total > kStaticScratchBytes) {
        set_error("allocation-free decode needs %zu bytes of scratch for n=%lld, M=%d, D=%d, d=%d; the static "
                  "scratch holds %zu bytes (use fewer pixels per call)",
                  p.total, (long long)n, M, D, DQ, kStaticScratchBytes);
        return LATENTAM_ERR_UNSUPPORTED_SHAPE;
    }
    unsigned char* base = static_cast<unsigned char*>(ctx->noalloc_scratch);
    if (!base) {
        set_error("the context holds no address of the static decode scratch");
        return LATENTAM_ERR_INVALID_ARG;
    }
    double* acc = reinterpret_cast<double*>(base + p.acc);
    float* A = reinterpret_cast<float*>(base + p.A);
    float* dF = reinterpret_cast<float*>(base + p.dF);
    float* dS = reinterpret_cast<float*>(base + p.dS);
    float* row = reinterpret_cast<float*>(base + p.row);
    float* coef = reinterpret_cast<float*>(base + p.coef);
    // the accumulators keep the previous call's sums: clear them first
    cudaError_t e = cudaMemsetAsync(acc, 0, sizeof(double) * 8, st);
    if (e != cudaSuccess) return cuda_error(e, "memset static loss accumulators");
    if (n > 0) {
        const unsigned cb = (unsigned)std::min<int64_t>((n + kThreads - 1) / kThreads, 4 * ctx->num_sms);
        count_mask_kernel<<<cb, kThreads, 0, st>>>(a.mask, n, acc);
        LAT_CHECK_LAUNCH("count_mask_kernel");
    }
    trust_region_kernel<<<(unsigned)((M + 7) / 8), 256, 0, st>>>(a.V, a.V0, M, D, a.cfg.delta,
                                                                 a.cfg.lambda_f * a.cfg.lambda_D, coef, acc);
    LAT_CHECK_LAUNCH("trust_region_kernel");
    if (n > 0) {
        LAT_TRY((launch_rows_fwd<DQ, 1>(a.Q, n, a.K, a.V, M, D, a.c, a.F, a.F_dtype, a.mask, a.cfg, acc, A, dF, row,
                                           nullptr, st)));
        if (a.dQ || a.dK)
            LAT_TRY(launch_rows_bwd<DQ>(dF, A, row, a.K, a.V, n, M, D, a.c, dS, a.dQ, st));
    }
    if (a.dV)
        LAT_TRY(atb_noalloc(A, M, M, dF, D, D, n, 1.0f, coef, a.V, a.V0, a.dV, reinterpret_cast<float*>(base + p.partV),
                            p.splitsV, p.rpsV, st));
    if (a.dK)
        LAT_TRY(atb_noalloc(dS, M, M, a.Q, DQ, DQ, n, a.c, nullptr, nullptr, nullptr, a.dK,
                            reinterpret_cast<float*>(base + p.partK), p.splitsK, p.rpsK, st));
    finalize_loss<<<1, 1, 0, st>>>(acc, D, a.cfg, a.loss_parts);
    LAT_CHECK_LAUNCH("finalize_loss");
    return LATENTAM_OK;
}

}  // namespace

latentam_status decode_loss_bwd_f32_noalloc(latentam_ctx* ctx, const DecodeArgs& a, cudaStream_t st) {
    switch (a.d) {
        case 16: return loss_bwd_noalloc_t<16>(ctx, a, st);
        case 32: return loss_bwd_noalloc_t<32>(ctx, a, st);
        case 64: return loss_bwd_noalloc_t<64>(ctx, a, st);
        default: set_error("query dimension d=%d not in {16, 32, 64}", a.d); return LATENTAM_ERR_UNSUPPORTED_SHAPE;
    }
}

latentam_status decode_noalloc_setup(latentam_ctx* ctx) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(static decode scratch)");
    ctx->noalloc_scratch = ptr;
    return LATENTAM_OK;
}

latentam_status sgemm_abt(const float* A, int64_t m, const float* B, int64_t n, int64_t k, float* C, int64_t ldc,
                          float scale, cudaStream_t st) {
    const PlainSrc a{A, k, m, k}, b{B, k, n, k};
    const StoreTileEpi::Params ep{C, ldc, 0, scale};
    return launch_sgemm<true, true, PlainSrc, PlainSrc, StoreTileEpi>(a, b, m, n, k, 1, ep, st);
}

latentam_status decode_loss_bwd_f32(latentam_ctx* ctx, const DecodeArgs& a, cudaStream_t st) {
    switch (a.d) {
        case 16: return loss_bwd_t<16>(ctx, a, st);
        case 32: return loss_bwd_t<32>(ctx, a, st);
        case 64: return loss_bwd_t<64>(ctx, a, st);
        default: set_error("query dimension d=%d not in {16, 32, 64}", a.d); return LATENTAM_ERR_UNSUPPORTED_SHAPE;
    }
}

latentam_status decode_fwd_f32(latentam_ctx* ctx, const float* Q, int64_t n, int d, const float* K, const float* V,
                               int M, int D, float c, float* F_hat, float* row_stats, cudaStream_t st) {
    switch (d) {
        case 16: return decode_fwd_t<16>(ctx, Q, n, K, V, M, D, c, F_hat, row_stats, st);
        case 32: return decode_fwd_t<32>(ctx, Q, n, K, V, M, D, c, F_hat, row_stats, st);
        case 64: return decode_fwd_t<64>(ctx, Q, n, K, V, M, D, c, F_hat, row_stats, st);
        default: set_error("query dimension d=%d not in {16, 32, 64}", d); return LATENTAM_ERR_UNSUPPORTED_SHAPE;
    }
}

}  // namespace lat
