// Dictionary decode (Eq. dict_recon), feature objective (Eq. feat_loss, Eq. full_obj) and
// its backward on the tcgen05 tensor cores: BF16 operands, FP32 accumulation in TMEM, FP32
// softmax and loss arithmetic, FP64 frame sums.  Six contractions share tc_gemm_kernel:
//
//   G1  S = Q K^T            epilogue: row softmax (logit scale c) -> A (BF16), row stats
//   G2  Fhat = A V           epilogue: cos / L2 against F, a_p, b_p -> dFhat (BF16)
//   G3  dA = dFhat V^T       epilogue: dS = A (dA - <A, dA>) -> dS (BF16)
//   G4  dQ = c dS K          epilogue: FP32 dQ
//   G5  dV = A^T dFhat       split over pixels -> FP32 partials -> sum + trust-region term
//   G6  dK = c dS^T Q        split over pixels -> FP32 partials -> sum
//
// Every intermediate is stored once, row-major (pixel x atom / pixel x feature); the
// contractions that reduce over pixels (G5, G6) and those whose B operand runs along its
// contiguous dimension (G2, G4) read it as an MN-major operand, so nothing is transposed.
#include <cuda_fp8.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

#include "tc_gemm.cuh"

namespace lat {
namespace {

using tc::kTileM;
using bf16 = __nv_bfloat16;

constexpr int kPad = 64;  // query / key rows padded to one 64-wide K chunk

// ---- operand preparation ----------------------------------------------------------------

// Qb[p][0..63] = bf16(Q[p][0..d)) zero-padded; thread t writes 8 columns (16 bytes) of row t / 8,
// so a warp reads and writes contiguous memory.  SPLIT: Qb holds two planes [2][n][64], the hi
// terms bf16(q) and the lo terms bf16(q - hi).
template <bool SPLIT>
__global__ void prep_queries(const float* __restrict__ Q, int64_t n, int d, bf16* __restrict__ Qb) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * (kPad / 8)) return;
    const int64_t p = t / (kPad / 8);
    const int c = (int)(t % (kPad / 8)) * 8;
    uint4 hi = make_uint4(0u, 0u, 0u, 0u), lo = hi;
    if (c < d) {  // d is a multiple of 8 and Q rows are 16-byte aligned
        const float4 a = *reinterpret_cast<const float4*>(Q + p * d + c);
        const float4 b = *reinterpret_cast<const float4*>(Q + p * d + c + 4);
        tc::pack_split_bf16x2(a.x, a.y, hi.x, lo.x);
        tc::pack_split_bf16x2(a.z, a.w, hi.y, lo.y);
        tc::pack_split_bf16x2(b.x, b.y, hi.z, lo.z);
        tc::pack_split_bf16x2(b.z, b.w, hi.w, lo.w);
    }
    reinterpret_cast<uint4*>(Qb + p * kPad)[t % (kPad / 8)] = hi;
    if (SPLIT) reinterpret_cast<uint4*>(Qb + n * kPad + p * kPad)[t % (kPad / 8)] = lo;
}

// Kb[j][0..63] (zero-padded) and Vb[j][c]: BF16 copies of the dictionary (SPLIT: hi planes
// followed by lo planes, Kb [2][M][64], Vb [2][M][D]).
template <bool SPLIT>
__global__ void prep_dict(const float* __restrict__ K, const float* __restrict__ V, int M, int d, int D,
                          bf16* __restrict__ Kb, bf16* __restrict__ Vb) {
    const int64_t nv = (int64_t)M * D, nk = (int64_t)M * kPad;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nv + nk; e += (int64_t)gridDim.x * blockDim.x) {
        float v;
        bf16* dst;
        int64_t plane;
        if (e < nv) {
            v = V[e];
            dst = Vb + e;
            plane = nv;
        } else {
            const int64_t f = e - nv;
            const int j = (int)(f / kPad), k = (int)(f % kPad);
            v = k < d ? K[(int64_t)j * d + k] : 0.f;
            dst = Kb + f;
            plane = nk;
        }
        *dst = __float2bfloat16_rn(v);
        if (SPLIT) dst[plane] = __float2bfloat16_rn(tc::split_lo(v));
    }
}

// ---- E4M3 operands of the value contraction ----------------------------------------------

// Aq[p][j] = e4m3(A[p][j] * 448 l_p): the largest weight of a softmax row is 1 / l_p (the
// largest logit contributes exp(0)), so every scaled row peaks at the E4M3 maximum 448.
// Thread t converts 8 weights (16 bytes in, 8 out).
__global__ void fp8_rows(const bf16* __restrict__ A, const float* __restrict__ stats, int64_t n, int M,
                         uint8_t* __restrict__ Aq) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int per_row = M / 8;
    if (t >= n * per_row) return;
    const int64_t p = t / per_row;
    const float s = 448.0f * stats[2 * p + 1];
    const uint4 u = reinterpret_cast<const uint4*>(A)[t];
    const uint32_t w[4] = {u.x, u.y, u.z, u.w};
    uint16_t o[4];
#pragma unroll
    for (int h = 0; h < 4; ++h) {
        const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w[h]));
        o[h] = __nv_cvt_float2_to_fp8x2(make_float2(f.x * s, f.y * s), __NV_SATFINITE, __NV_E4M3);
    }
    reinterpret_cast<uint2*>(Aq)[t] = make_uint2((uint32_t)o[0] | ((uint32_t)o[1] << 16),
                                                 (uint32_t)o[2] | ((uint32_t)o[3] << 16));
}

// Vtq[c][j] = e4m3(V[j][c] / inv_t[c]) with inv_t[c] = max_j |V_jc| / 448 (the transpose makes
// the atoms the contiguous K dimension of the operand).  One thread per feature column.
__global__ void fp8_values(const float* __restrict__ V, int M, int D, uint8_t* __restrict__ Vtq,
                           float* __restrict__ inv_t) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= D) return;
    float mx = 0.f;
    for (int j = 0; j < M; ++j) mx = fmaxf(mx, fabsf(V[(size_t)j * D + c]));
    const float it = mx > 0.f ? mx / 448.0f : 1.0f;
    inv_t[c] = it;
    const float s = 1.0f / it;
    for (int j = 0; j < M; j += 2) {
        const uint16_t o = __nv_cvt_float2_to_fp8x2(make_float2(V[(size_t)j * D + c] * s, V[(size_t)(j + 1) * D + c] * s),
                                                   __NV_SATFINITE, __NV_E4M3);
        *reinterpret_cast<uint16_t*>(Vtq + (size_t)c * M + j) = o;
    }
}

// Accumulators: [0] sum (1 - cos) over valid pixels, [1] sum of squared errors, [2] trust
// region, [3] |Omega|.  The tensor-core kernels raise the context's sticky device flag when a
// bounded wait gives up; the loss of that call is then NaN and the next synchronising call
// (binning, or a step that reads its loss back) returns LATENTAM_ERR_TIMEOUT.
__global__ void tc_count_mask(const uint8_t* __restrict__ mask, int64_t n, double* __restrict__ acc) {
    __shared__ int s[8];
    int c = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        c += mask ? (mask[i] != 0) : 1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s[w];
        atomicAdd(&acc[3], (double)t);
    }
}

// Trust region on the value rows (FP32 values): coef[j] = lambda_f lambda_D / |V_j - V0_j|
// outside the radius, else 0; the ReLU sum goes to acc[2].
__global__ void tc_trust_region(const float* __restrict__ V, const float* __restrict__ V0, int M, int D, float delta,
                                float weight, float* __restrict__ coef, double* __restrict__ acc) {
    const int j = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (j >= M) return;
    float s = 0.f;
    for (int k = lane; k < D; k += 32) {
        const float t = V[(size_t)j * D + k] - V0[(size_t)j * D + k];
        s += t * t;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
        const float nrm = sqrtf(s);
        const bool out = nrm > delta;
        coef[j] = out ? weight / nrm : 0.f;
        if (out) atomicAdd(&acc[2], (double)(nrm - delta));
    }
}

// out[j][k] = scale * sum_z part[z][j][k] (+ coef[j] (V - V0)[j][k]) for k < ncols (of ld columns).
// A block owns 32 consecutive outputs (one per lane); its W warps take every W-th split, so the
// reads of each split are contiguous and many splits are summed in parallel (W = 32 for the
// thousands of per-tile partials of the fused dK).
// Eight loads of a warp's splits are in flight before their (in-order) additions.  T: the sum
// goes to out[k][j] instead (partials stored transposed).
template <int W, bool T = false>
__global__ void __launch_bounds__(32 * W, W >= 32 ? 2 : 8)
    tc_reduce_parts(const float* __restrict__ part, int splits, int rows, int ld, int ncols, float scale,
                    const float* __restrict__ coef, const float* __restrict__ V, const float* __restrict__ V0,
                    float* __restrict__ out) {
    __shared__ float acc[W][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t e = (int64_t)blockIdx.x * 32 + lane;
    const bool live = e < (int64_t)rows * ncols;
    const int j = live ? (int)(e / ncols) : 0, k = live ? (int)(e % ncols) : 0;
    float s = 0.f;
    if (live) {
        const int64_t step = (int64_t)W * rows * ld;  // W splits
        const float* p = part + (int64_t)j * ld + k + (int64_t)w * rows * ld;
        int z = w;
        for (; W >= 32 && z + 7 * W < splits; z += 8 * W) {  // (fewer registers for W = 8: more blocks)
            float v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u, p += step) v[u] = __ldg(p);
#pragma unroll
            for (int u = 0; u < 8; ++u) s += v[u];
        }
#pragma unroll 4
        for (; z < splits; z += W, p += step) s += __ldg(p);
    }
    acc[w][lane] = s;
    __syncthreads();
    if (w == 0 && live) {
        float t = 0.f;
#pragma unroll
        for (int q = 0; q < W; ++q) t += acc[q][lane];
        t *= scale;
        if (coef) t += coef[j] * (V[e] - V0[e]);
        out[T ? (int64_t)k * rows + j : e] = t;
    }
}

// The same sums (the same order per output) with each lane owning four consecutive outputs of
// one row: 16-byte loads, for the wide dV partials (ncols and ld multiples of 4, part 16-byte
// aligned).
template <int W>
__global__ void __launch_bounds__(32 * W, 8)
    tc_reduce_parts4(const float* __restrict__ part, int splits, int rows, int ld, int ncols, float scale,
                     const float* __restrict__ coef, const float* __restrict__ V, const float* __restrict__ V0,
                     float* __restrict__ out) {
    __shared__ float4 acc[W][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t e = 4 * ((int64_t)blockIdx.x * 32 + lane);  // first of the lane's four outputs
    const bool live = e < (int64_t)rows * ncols;
    const int j = live ? (int)(e / ncols) : 0, k = live ? (int)(e % ncols) : 0;
    float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
    if (live) {
        const int64_t step = (int64_t)W * rows * ld;  // W splits
        const float* p = part + (int64_t)j * ld + k + (int64_t)w * rows * ld;
#pragma unroll 4
        for (int z = w; z < splits; z += W, p += step) {
            const float4 u = __ldg(reinterpret_cast<const float4*>(p));
            s.x += u.x;
            s.y += u.y;
            s.z += u.z;
            s.w += u.w;
        }
    }
    acc[w][lane] = s;
    __syncthreads();
    if (w == 0 && live) {
        float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int q = 0; q < W; ++q) {
            const float4 u = acc[q][lane];
            t.x += u.x;
            t.y += u.y;
            t.z += u.z;
            t.w += u.w;
        }
        t = make_float4(t.x * scale, t.y * scale, t.z * scale, t.w * scale);
        if (coef) {
            const float c = coef[j];
            const float4 v = *reinterpret_cast<const float4*>(V + e), v0 = *reinterpret_cast<const float4*>(V0 + e);
            t = make_float4(t.x + c * (v.x - v0.x), t.y + c * (v.y - v0.y), t.z + c * (v.z - v0.z), t.w + c * (v.w - v0.w));
        }
        *reinterpret_cast<float4*>(out + e) = t;
    }
}

__global__ void tc_finalize(const double* __restrict__ acc, const int* __restrict__ err, int D, latentam_loss_cfg cfg,
                            double* __restrict__ parts) {
    const double nv = acc[3];
    const double lcos = nv > 0 ? acc[0] / nv : 0.0;
    const double l2 = nv > 0 ? acc[1] / (nv * D) : 0.0;
    parts[0] = lcos;
    parts[1] = l2;
    parts[2] = acc[2];
    parts[3] = (double)cfg.lambda_f *
               ((double)cfg.lambda_cos * lcos + (double)cfg.lambda_2 * l2 + (double)cfg.lambda_D * acc[2]);
    parts[4] = nv;
    if (*err) parts[3] = __longlong_as_double(0x7ff8000000000000ll);  // a device wait gave up: NaN loss
}

// ---- epilogues ---------------------------------------------------------------------------

__device__ __forceinline__ void load_row_bf16x32(const bf16* src, float (&v)[32]) {
    const uint4* s4 = reinterpret_cast<const uint4*>(src);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const uint4 u = s4[q];
        const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w[h]));
            v[8 * q + 2 * h] = f.x;
            v[8 * q + 2 * h + 1] = f.y;
        }
    }
}

__device__ __forceinline__ void load_target32(const void* F, latentam_dtype dt, int64_t off, float (&v)[32]) {
    if (dt == LATENTAM_DTYPE_BF16) {
        load_row_bf16x32(reinterpret_cast<const bf16*>(F) + off, v);
    } else {
        const float4* s4 = reinterpret_cast<const float4*>(reinterpret_cast<const float*>(F) + off);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const float4 f = s4[q];
            v[4 * q] = f.x;
            v[4 * q + 1] = f.y;
            v[4 * q + 2] = f.z;
            v[4 * q + 3] = f.w;
        }
    }
}

// Column chunks of 32 are dealt to the epilogue warpgroups round-robin: group g owns the
// chunks c0 = 32 (g + G k).

// G1: row softmax of c S over the M atoms.
struct SoftmaxParams {
    int64_t n;
    int M;
    float c;
    bf16* A;       // n x M
    float* stats;  // n x 2 (row max of c S, softmax denominator), nullable
};

// One CTA holds the logits of 256 atoms; when M > 256 the CTAs of a row block form a cluster
// and combine their (row max, partial denominator) pairs before normalising.
// SPLIT_: the FP32 form (queries, keys and A as hi / lo BF16 planes, three MMAs per product):
// 16-wide K chunks over the d query columns, three ring stages.
template <bool SPLIT_ = false>
struct SoftmaxEpi {
    // plain: one K chunk (the padded queries) per tile
    static constexpr bool SPLIT = SPLIT_, INPLACE = false;
    static constexpr int BN = 256, BK = SPLIT_ ? 16 : 64, ELEM = 2, STAGES = SPLIT_ ? 3 : 1, BOX_B = 256;
    static constexpr int EPI_WG = 4, E_BOXES = 0, O_BOXES = 4;
    static constexpr int XROUNDS = 1;
    static constexpr bool A_MN = false, B_MN = false;
    using Params = SoftmaxParams;
    static __device__ int run(const Params& p, const tc::EpiCtx& ec) {
        const uint32_t taddr = ec.taddr;
        const int row = ec.row, m0 = ec.m0, g = ec.g;
        const int ncols = min(BN, p.M - ec.n0);  // atoms of this CTA's slice
        float* scr = ec.scratch;
        const int64_t pix = (int64_t)m0 + row;
        const bool valid = pix < p.n;
        float mx = -INFINITY;
        for (int c0 = 32 * g; c0 < ncols; c0 += 32 * EPI_WG) {
            float v[32];
            tc::tmem_ld32(taddr + c0, v);
#pragma unroll
            for (int i = 0; i < 32; ++i) mx = fmaxf(mx, v[i]);
        }
        mx = tc::group_max<EPI_WG>(mx, scr, 0, g, row);
        float cm = p.c * mx;  // c > 0
        // the exponentials are taken once and written back over S in TMEM (this thread's lane
        // and chunks only), then scaled by the row's normaliser on the way out
        float sum = 0.f;
        for (int c0 = 32 * g; c0 < ncols; c0 += 32 * EPI_WG) {
            float v[32];
            tc::tmem_ld32(taddr + c0, v);
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                v[i] = __expf(p.c * v[i] - cm);
                sum += v[i];
            }
            tc::tmem_st32(taddr + c0, v);
        }
        sum = tc::group_sum<EPI_WG>(sum, scr, 1, g, row);
        const float mine[tc::kXchgVals] = {cm, sum, 0.f, 0.f};
        ec.exchange(mine);
        float rescale = 1.f;  // exp(cm - global max) when the row spans a cluster
        if (ec.csize > 1) {
            float gm = cm;
            for (int q = 0; q < ec.csize; ++q)
                if (q != ec.crank) gm = fmaxf(gm, ec.xval(q, 0));
            float l = 0.f;
            for (int q = 0; q < ec.csize; ++q)
                l += q == ec.crank ? sum * __expf(cm - gm) : ec.xval(q, 1) * __expf(ec.xval(q, 0) - gm);
            rescale = __expf(cm - gm);
            cm = gm;
            sum = l;
        }
        const float il = rescale / sum;
        ec.wait_out();
        for (int c0 = 32 * g; c0 < ncols; c0 += 32 * EPI_WG) {
            float v[32];
            tc::tmem_ld32(taddr + c0, v);
#pragma unroll
            for (int i = 0; i < 32; ++i) v[i] *= il;
            ec.put32(c0, v);
        }
        if (valid && p.stats && g == 0 && ec.crank == 0) {
            p.stats[2 * pix] = cm;
            p.stats[2 * pix + 1] = sum;
        }
        return (ncols + 63) / 64;
    }
};

// G2: Fhat = A V, the per-pixel loss terms and dL/dFhat = a_p Fhat + b_p F.  One CTA holds
// 256 features of its rows; when D > 256 the CTAs of a row block form a cluster and add up
// their per-row partial sums (<Fhat, F>, |Fhat|^2, |F|^2, |Fhat - F|^2) before dFhat is formed.
struct FhatParams {
    int64_t n;
    int D;
    const void* F;
    latentam_dtype F_dtype;
    const uint8_t* mask;
    latentam_loss_cfg cfg;
    double* acc;
    bf16* dF;     // n x D
    float* row;   // n x 4: a_p, b_p, <A_p, dA_p>, cos_p
    float* Fout;  // n x D FP32 Fhat (inference form: no loss) or NULL
    // E4M3 form: row statistics of the softmax (the per-pixel scale 448 l_p) and the
    // per-feature scale inverses max_j |V_jc| / 448
    const float* stats;
    const float* inv_t;
};

// ETILE: the BF16 target rows come through shared memory (TMA, after the MMAs); otherwise
// (FP32 targets) each thread reads its own row from global memory, one chunk ahead.
// Q8: the contraction runs on E4M3 operands (attention rows scaled per pixel, values per
// feature, both K-major) and the accumulator is rescaled before any use.
// SPLIT_ (the FP32 form): A and V as hi / lo BF16 planes, three MMAs per product, dFhat out as
// hi / lo planes, 32-byte K chunks so that three ring stages fit beside the staged tile.  With
// ETILE (FP32 targets) the tile's target rows come by TMA as eight 32-column FP32 chunks filling
// both box buffers and dFhat is written over them (INPLACE); without, the targets (FP32 or BF16)
// are read per thread and dFhat is staged as two planes across the buffers.
template <bool ETILE, bool Q8 = false, bool SPLIT_ = false>
struct FhatEpi {
    static_assert(!SPLIT_ || !Q8, "the split form has no E4M3 operands");
    static constexpr bool SPLIT = SPLIT_, INPLACE = SPLIT_ && ETILE;
    // persistent, 64-byte K chunks (three ring stages fit beside two epilogue buffers)
    static constexpr int ELEM = Q8 ? 1 : 2, BK = SPLIT_ ? 16 : 64 / ELEM;
    static constexpr int BN = 256, STAGES = 3, BOX_B = 256, EPI_WG = ETILE ? 4 : 2, XROUNDS = 1;
    // dFhat staged over the target
    static constexpr int E_BOXES = INPLACE ? 8 : ETILE ? BN / 64 : 0, O_BOXES = BN / 64;
    // B = V (atoms x features, features contiguous: MN-major) or, for E4M3, V^T (K-major)
    static constexpr bool A_MN = false, B_MN = !Q8;
    using Params = FhatParams;
    // Fhat chunk c0 of this thread's row from TMEM (E4M3: times 1 / (scale_p scale_c))
    static __device__ __forceinline__ void fhat32(const Params& p, const tc::EpiCtx& ec, int c0, float isp,
                                                  float (&h)[32]) {
        tc::tmem_ld32(ec.taddr + c0, h);
        if constexpr (Q8) {
            const float4* it = reinterpret_cast<const float4*>(p.inv_t + ec.n0 + c0);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const float4 v = it[q];
                h[4 * q] *= isp * v.x;
                h[4 * q + 1] *= isp * v.y;
                h[4 * q + 2] *= isp * v.z;
                h[4 * q + 3] *= isp * v.w;
            }
        }
    }
    static __device__ __forceinline__ float row_scale_inv(const Params& p, int64_t pix, bool valid) {
        if constexpr (Q8) return valid ? 1.0f / (448.0f * p.stats[2 * pix + 1]) : 0.f;
        return 1.f;
    }
    // body(c0, h, f) for each 32-column chunk of this thread's share of the slice: h = Fhat
    // (TMEM), f = target
    template <class Body>
    static __device__ __forceinline__ void sweep(const Params& p, const tc::EpiCtx& ec, int64_t frow, int ncols,
                                                 float isp, Body&& body) {
        constexpr int step = 32 * EPI_WG;
        float h[32], f[32];
        if constexpr (ETILE) {
            for (int c0 = 32 * ec.g; c0 < ncols; c0 += step) {
                if (INPLACE)
                    ec.row32f(c0, f);
                else
                    ec.row32(c0, f);
                fhat32(p, ec, c0, isp, h);
                body(c0, h, f);
            }
        } else {
            float fn[32];
            load_target32(p.F, p.F_dtype, frow + 32 * ec.g, f);
            for (int c0 = 32 * ec.g; c0 < ncols; c0 += step) {
                if (c0 + step < ncols) load_target32(p.F, p.F_dtype, frow + c0 + step, fn);
                fhat32(p, ec, c0, isp, h);
                body(c0, h, f);
#pragma unroll
                for (int i = 0; i < 32; ++i) f[i] = fn[i];
            }
        }
    }
    static __device__ int run(const Params& p, const tc::EpiCtx& ec) {
        const int row = ec.row, m0 = ec.m0, g = ec.g;
        const int ncols = min(BN, p.D - ec.n0);  // features of this CTA's slice
        float* scr = ec.scratch;
        const int64_t pix = (int64_t)m0 + row;
        const bool valid = pix < p.n;
        const float isp = row_scale_inv(p, pix, valid);
        if (p.Fout) {  // inference form, launched without a cluster
            ec.wait_out();
            float h[32];
            for (int c0 = 32 * g; c0 < ncols; c0 += 32 * EPI_WG) {
                fhat32(p, ec, c0, isp, h);
                if (valid) {
                    float4* d4 = reinterpret_cast<float4*>(p.Fout + pix * p.D + ec.n0 + c0);
#pragma unroll
                    for (int q = 0; q < 8; ++q) d4[q] = make_float4(h[4 * q], h[4 * q + 1], h[4 * q + 2], h[4 * q + 3]);
                }
            }
            const float none[tc::kXchgVals] = {0.f, 0.f, 0.f, 0.f};
            ec.exchange(none);
            return 0;
        }
        // invalid rows read row 0 (discarded)
        const int64_t frow = (valid ? pix * p.D : 0) + ec.n0;
        // per-row and per-frame inputs first: their latency hides behind the first pass
        const bool in_loss = valid && (p.mask == nullptr || p.mask[pix] != 0);
        const float nv = (float)p.acc[3];
        if (ETILE)
            for (int b = 0; b < E_BOXES; ++b) (void)ec.wait_box(b);  // a timeout raises the error flag
        float t[4] = {0.f, 0.f, 0.f, 0.f};  // <Fhat, F>, |Fhat|^2, |F|^2, |Fhat - F|^2
        sweep(p, ec, frow, ncols, isp, [&](int, const float(&h)[32], const float(&f)[32]) {
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                t[0] += h[i] * f[i];
                t[1] += h[i] * h[i];
                t[2] += f[i] * f[i];
                const float e = h[i] - f[i];
                t[3] += e * e;
            }
        });
        tc::group_sum4<EPI_WG>(t, scr, g, row);
        ec.exchange(t);
        for (int q = 0; q < ec.csize; ++q) {
            if (q == ec.crank) continue;
#pragma unroll
            for (int k = 0; k < 4; ++k) t[k] += ec.xval(q, k);
        }
        const float dot = t[0], nh2 = t[1], nf2 = t[2], e2 = t[3];
        // FP32 arithmetic per row (FP64 only in the frame sums below)
        const float scale = nv > 0.f ? p.cfg.lambda_f / nv : 0.f;
        const float den = sqrtf(nh2) * sqrtf(nf2);
        const float cs = dot / fmaxf(den, 1e-8f);
        float a = 0.f, b = 0.f;
        if (in_loss) {
            const float l2c = 2.0f * p.cfg.lambda_2 / (float)p.D;
            if (den > 1e-8f) {
                a = scale * (p.cfg.lambda_cos * cs / nh2 + l2c);
                b = scale * (-p.cfg.lambda_cos / den - l2c);
            } else {
                a = scale * l2c;
                b = scale * (-p.cfg.lambda_cos / 1e-8f - l2c);
            }
        }
        const bool lead = g == 0 && ec.crank == 0;  // one thread per row writes the row's results
        if (valid && lead)
            *reinterpret_cast<float4*>(p.row + 4 * pix) = make_float4(a, b, a * nh2 + b * dot, cs);
        if (lead) {
            // warp partial sums in FP32 (32 rows), added to the frame sums in FP64
            float lc = in_loss ? 1.0f - cs : 0.f, le = in_loss ? e2 : 0.f;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                lc += __shfl_xor_sync(0xffffffffu, lc, o);
                le += __shfl_xor_sync(0xffffffffu, le, o);
            }
            if ((threadIdx.x & 31) == 0) {
                atomicAdd(&p.acc[0], (double)lc);
                atomicAdd(&p.acc[1], (double)le);
            }
        }
        // dFhat overwrites the target chunk it was formed from (plain: same thread, same bytes;
        // in place: the chunk's two planes replace its FP32 rows once its warpgroup read them)
        ec.wait_out();
        sweep(p, ec, frow, ncols, isp, [&](int c0, const float(&h)[32], const float(&f)[32]) {
            float v[32];
#pragma unroll
            for (int i = 0; i < 32; ++i) v[i] = a * h[i] + b * f[i];
            if (INPLACE) {
                ec.group_sync();
                ec.put32s(c0, v);
            } else {
                ec.put32(c0, v);
            }
        });
        return (ncols + 63) / 64;
    }
};

// G3: dS = A (dA - <A, dA>).
struct DsParams {
    int64_t n;
    int M;
    const bf16* A;
    const float* row;
    bf16* dS;  // n x M
    // G4 fused as the trailing product dQ = c dS K (K padded to 64 columns), or dQ == NULL;
    // dq_add: the CTAs along y (two at most) add their partial rows into a zeroed dQ
    float* dQ;
    int d;
    float c;
    int dq_add;
    // G6 fused as a second trailing product (needs dQ fused): dKpart[tile][j][atom], j < d, = the
    // tile's share of dS^T Q (unscaled, transposed so that a warp's stores are contiguous), and
    // dS is not stored; or dKpart == NULL
    float* dKpart;
};

// One CTA holds 256 atoms of its rows (M > 256: several CTAs along y, nothing to trade: the
// row term <A, dA> comes from G2).  SPLIT_: the FP32 form (hi / lo planes in and out).
template <bool SPLIT_ = false>
struct DsEpi {
    static constexpr bool SPLIT = SPLIT_;
    // split form: 32-wide K stages and the epilogue in two passes over the column halves, so
    // that the tile fits in half the shared memory and two CTAs share an SM (one CTA's epilogue
    // runs during the other's main loop), as in the plain form
    static constexpr int MSUB = 1, BKC = SPLIT_ ? 32 : 64, EPASS = SPLIT_ ? 2 : 1;
    // the attention rows of the tile come through shared memory
    static constexpr int BN = 256, STAGES = 2, BOX_B = 256, EPI_WG = 2, XROUNDS = 0, MIN_SMEM = 0;
    static constexpr int MIN_BLOCKS = 2;
    static constexpr int E_BOXES = BN / 64, O_BOXES = BN / 64;  // dS staged over the attention rows
    static constexpr bool A_MN = false, B_MN = false;
    static constexpr int XPROD = 64;  // dQ = c dS K on the staged dS tile
    static constexpr int XPROD2 = 1;  // dK partial = dS^T Q on the same staged tile
    // its Q tile preloaded into 16 KB of its own (the BF16 form: two CTAs per SM still fit; the
    // split form's 32 KB do not, and it waits for the dQ product's operand space)
    static constexpr int X2PRE = SPLIT_ ? 0 : 1;
    using Params = DsParams;
    static __device__ bool x_active(const Params& p) { return p.dQ != nullptr; }
    static __device__ bool x2_active(const Params& p) { return p.dKpart != nullptr; }
    // this tile's dK partial: atoms n0 + 128 G + row from TMEM columns 64 + 64 G .. + d - 1, one
    // 128-byte row of atoms per warp and column
    static __device__ void run_k(const Params& p, const tc::EpiCtx& ec, int tile) {
        float v[32];
        for (int G = ec.g; G < BN / 128; G += EPI_WG) {
            const int atom = ec.n0 + 128 * G + ec.row;
            for (int c0 = 0; c0 < p.d; c0 += 32) {
                tc::tmem_ld32(ec.taddr + 64u + 64u * (uint32_t)G + (uint32_t)c0, v);
                if (atom >= p.M) continue;
                float* dst = p.dKpart + ((int64_t)tile * p.d + c0) * p.M + atom;
                const int nc = min(32, p.d - c0);
#pragma unroll
                for (int c = 0; c < 32; ++c) {
                    if (c >= nc) break;
                    dst[(int64_t)c * p.M] = v[c];
                }
            }
        }
    }
    // dQ rows of this tile from TMEM columns 0 .. d - 1 (the padded columns hold zeros); with free
    // shared memory, each warp's 32 rows x 32 columns go through it (4 KB, 16-byte chunks
    // swizzled by row) so that every store covers four whole 128-byte rows
    static __device__ void run_x(const Params& p, const tc::EpiCtx& ec) {
        const int64_t pix = (int64_t)ec.m0 + ec.row;
        float v[32];
        if (ec.xstage) {
            const int lane = ec.row & 31, quarter = ec.row >> 5;
            const int64_t pix0 = (int64_t)ec.m0 + 32 * quarter;  // the warp's first row
            for (int c0 = 32 * ec.g; c0 < p.d; c0 += 32 * EPI_WG) {
                tc::tmem_ld32(ec.taddr + c0, v);
                uint8_t* stage = ec.xstage + (ec.g * 4 + quarter) * 4096;
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    *reinterpret_cast<float4*>(stage + lane * 128 + ((q ^ (lane & 7)) << 4)) =
                        make_float4(p.c * v[4 * q], p.c * v[4 * q + 1], p.c * v[4 * q + 2], p.c * v[4 * q + 3]);
                __syncwarp();
                const int nq = min(32, p.d - c0) / 4, cq = lane & 7;
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int r = 4 * i + (lane >> 3);
                    const float4 u = *reinterpret_cast<const float4*>(stage + r * 128 + ((cq ^ (r & 7)) << 4));
                    if (pix0 + r < p.n && cq < nq) {
                        float4* d4 = reinterpret_cast<float4*>(p.dQ + (pix0 + r) * p.d + c0) + cq;
                        if (p.dq_add)
                            atomicAdd(d4, u);  // two addends onto zero: the same sum in either order
                        else
                            *d4 = u;
                    }
                }
                __syncwarp();  // (the next column block reuses the warp's staging rows)
            }
            return;
        }
        for (int c0 = 32 * ec.g; c0 < p.d; c0 += 32 * EPI_WG) {
            tc::tmem_ld32(ec.taddr + c0, v);
            if (pix >= p.n) continue;
            float4* d4 = reinterpret_cast<float4*>(p.dQ + pix * p.d + c0);
            const int nq = min(32, p.d - c0) / 4;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                if (q >= nq) break;
                const float4 u = make_float4(p.c * v[4 * q], p.c * v[4 * q + 1], p.c * v[4 * q + 2], p.c * v[4 * q + 3]);
                if (p.dq_add)
                    atomicAdd(d4 + q, u);  // two addends onto zero: the same sum in either order
                else
                    d4[q] = u;
            }
        }
    }
    // the columns [col0, col0 + BN / EPASS) of the tile (one epilogue pass)
    static __device__ int run(const Params& p, const tc::EpiCtx& ec) {
        const int64_t pix = (int64_t)ec.m0 + ec.row;
        const bool valid = pix < p.n;
        const float rd = valid ? p.row[4 * pix + 2] : 0.f;
        for (int b = 0; b < E_BOXES / EPASS; ++b) (void)ec.wait_box(b);
        const int cend = min(min(BN, p.M - ec.n0), ec.col0 + BN / EPASS);
        float dA[32], a[32];
        for (int c0 = ec.col0 + 32 * ec.g; c0 < cend; c0 += 32 * EPI_WG) {
            ec.row32(c0, a);
            tc::tmem_ld32(ec.taddr + c0, dA);
#pragma unroll
            for (int i = 0; i < 32; ++i) dA[i] = valid ? a[i] * (dA[i] - rd) : 0.f;  // (the dK product sums rows)
            ec.put32(c0, dA);
        }
        return cend > ec.col0 ? (cend - ec.col0 + 63) / 64 : 0;
    }
};

// G4: dQ = c dS K (the first d of the 64 padded query columns).
struct DqParams {
    int64_t n;
    int d;
    float c;
    float* dQ;
};

template <int BN_, bool SPLIT_ = false>
struct DqEpi {
    static constexpr bool SPLIT = SPLIT_;
    static constexpr int MSUB = 1, BKC = 64;
    static constexpr int BN = BN_, STAGES = 2, BOX_B = BN_, EPI_WG = 1, E_BOXES = 0, O_BOXES = 0, XROUNDS = 0;
    static constexpr int MIN_SMEM = 0, MIN_BLOCKS = 1;
    static constexpr bool A_MN = false, B_MN = true;  // B = K padded (atoms x 64), queries contiguous
    static constexpr int XPROD = 0, XPROD2 = 0, X2PRE = 0, EPASS = 1;
    using Params = DqParams;
    static __device__ int run(const Params& p, const tc::EpiCtx& ec) {
        const uint32_t taddr = ec.taddr;
        const int row = ec.row, m0 = ec.m0;
        const int64_t pix = (int64_t)m0 + row;
        float v[32];
#pragma unroll
        for (int c0 = 0; c0 < BN; c0 += 32) {
            if (c0 >= p.d) break;  // d is CTA-uniform
            tc::tmem_ld32(taddr + c0, v);
            if (pix < p.n) {
                float4* d4 = reinterpret_cast<float4*>(p.dQ + pix * p.d + c0);
                if (c0 + 32 <= p.d) {
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        d4[q] = make_float4(p.c * v[4 * q], p.c * v[4 * q + 1], p.c * v[4 * q + 2], p.c * v[4 * q + 3]);
                } else {
#pragma unroll
                    for (int q = 0; q < 4; ++q)  // d = 16
                        d4[q] = make_float4(p.c * v[4 * q], p.c * v[4 * q + 1], p.c * v[4 * q + 2], p.c * v[4 * q + 3]);
                }
            }
        }
        return 0;
    }
};

// G5 / G6: FP32 partial sums of one pixel split, part[z][row][col].
struct PartParams {
    int rows, ld, ncols;
    float* part;
};

// MSUB_ = 2: one CTA covers 256 rows (two accumulators) so that each B stage (the pixel block
// of the wide operand) is read once for both; with 32-wide pixel stages in the split form.
template <int BN_, bool SPLIT_ = false, int MSUB_ = 1>
struct PartEpi {
    static constexpr bool SPLIT = SPLIT_;
    static constexpr int MSUB = MSUB_, BKC = MSUB_ == 2 && SPLIT_ ? 32 : 64;
    static constexpr int BN = BN_, BOX_B = BN_, EPI_WG = 1;
    static constexpr int STAGES = MSUB_ == 2 ? 3 : (BN_ <= 64 ? 6 : 4) / (SPLIT_ ? 2 : 1);
    static constexpr int E_BOXES = 0, O_BOXES = 0;
    static constexpr int XROUNDS = 0;
    static constexpr int MIN_SMEM = 0, MIN_BLOCKS = 1;
    static constexpr bool A_MN = true, B_MN = true;  // both pixel-major: K = pixels runs along rows
    static constexpr int XPROD = 0, XPROD2 = 0, X2PRE = 0, EPASS = 1;
    using Params = PartParams;
    static __device__ int run(const Params& p, const tc::EpiCtx& ec) {
#pragma unroll
        for (int ms = 0; ms < MSUB; ++ms) sub(p, ec, ms);
        return 0;
    }
    static __device__ void sub(const Params& p, const tc::EpiCtx& ec, int ms) {
        const uint32_t taddr = ec.taddr + (uint32_t)(ms * BN);
        const int row = ec.row, m0 = ec.m0 + ms * tc::kTileM, n0 = ec.n0, z = ec.z;
        const int j = m0 + row;
        float v[32];
#pragma unroll
        for (int c0 = 0; c0 < BN; c0 += 32) {
            tc::tmem_ld32(taddr + c0, v);
            if (j < p.rows) {
                float* dst = p.part + ((int64_t)z * p.rows + j) * p.ld + n0 + c0;
                if (n0 + c0 + 32 <= p.ncols) {
                    float4* d4 = reinterpret_cast<float4*>(dst);
#pragma unroll
                    for (int q = 0; q < 8; ++q) d4[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                } else {
#pragma unroll
                    for (int i = 0; i < 32; ++i)
                        if (n0 + c0 + i < p.ncols) dst[i] = v[i];
                }
            }
        }
    }
};

// ---- host side ---------------------------------------------------------------------------

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

std::once_flag g_encode_once;
EncodeTiledFn g_encode = nullptr;

latentam_status encoder(EncodeTiledFn* out) {
    std::call_once(g_encode_once, [] {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = reinterpret_cast<EncodeTiledFn>(fn);
        (void)cudaGetLastError();
    });
    if (!g_encode) {
        set_error("cuTensorMapEncodeTiled is not available from the driver");
        return LATENTAM_ERR_CUDA;
    }
    *out = g_encode;
    return LATENTAM_OK;
}

// Tensor map of a row-major BF16 matrix (rows x inner, row stride ld elements), boxes of
// box_inner (64: 128-byte swizzle, 32: 64-byte swizzle) x box_rows; out-of-range elements read
// as zero.
latentam_status bf16_map(CUtensorMap* m, const void* base, int64_t inner, int64_t rows, int64_t ld, int box_rows,
                         int box_inner = tc::kChunkK) {
    EncodeTiledFn enc;
    LAT_TRY(encoder(&enc));
    if ((reinterpret_cast<uintptr_t>(base) & 15u) || (ld * 2) % 16) {
        set_error("tensor-core operand not 16-byte aligned");
        return LATENTAM_ERR_INVALID_ARG;
    }
    const cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
    const cuuint32_t box[2] = {(cuuint32_t)box_inner, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    const CUtensorMapSwizzle sw = box_inner == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B;
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed (%d) for a %lld x %lld operand", (int)r, (long long)rows,
                  (long long)inner);
        return LATENTAM_ERR_CUDA;
    }
    return LATENTAM_OK;
}

// Tensor map of a row-major FP32 matrix read in boxes of 32 columns (128 bytes, 128-byte
// swizzle) x box_rows.
latentam_status f32_map(CUtensorMap* m, const void* base, int64_t inner, int64_t rows, int box_rows) {
    EncodeTiledFn enc;
    LAT_TRY(encoder(&enc));
    if ((reinterpret_cast<uintptr_t>(base) & 15u) || (inner * 4) % 16) {
        set_error("FP32 tensor-core epilogue operand not 16-byte aligned");
        return LATENTAM_ERR_INVALID_ARG;
    }
    const cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)(inner * 4)};
    const cuuint32_t box[2] = {32, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed (%d) for a %lld x %lld FP32 operand", (int)r, (long long)rows,
                  (long long)inner);
        return LATENTAM_ERR_CUDA;
    }
    return LATENTAM_OK;
}

// Tensor map of a split operand: two row-major BF16 planes [2][rows][ld] (hi, then lo) as a 3D
// tensor with the plane as z, boxes of box_inner (64 / 32 / 16: 128 / 64 / 32-byte swizzle) x
// box_rows x box_planes (2: one load brings both planes, [plane][row][inner]; 1: one plane, for
// the epilogue operands and outputs and the MN-major A operands); out-of-range elements read as
// zero.
latentam_status split_map(CUtensorMap* m, const void* base, int64_t inner, int64_t rows, int64_t ld, int box_rows,
                          int box_inner, int box_planes) {
    EncodeTiledFn enc;
    LAT_TRY(encoder(&enc));
    if ((reinterpret_cast<uintptr_t>(base) & 15u) || (ld * 2) % 16 || (rows * ld * 2) % 16) {
        set_error("split tensor-core operand not 16-byte aligned");
        return LATENTAM_ERR_INVALID_ARG;
    }
    const cuuint64_t dims[3] = {(cuuint64_t)inner, (cuuint64_t)rows, 2};
    const cuuint64_t strides[2] = {(cuuint64_t)(ld * 2), (cuuint64_t)(rows * ld * 2)};
    const cuuint32_t box[3] = {(cuuint32_t)box_inner, (cuuint32_t)box_rows, (cuuint32_t)box_planes};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUtensorMapSwizzle sw = box_inner == 16   ? CU_TENSOR_MAP_SWIZZLE_32B
                                  : box_inner == 32 ? CU_TENSOR_MAP_SWIZZLE_64B
                                                    : CU_TENSOR_MAP_SWIZZLE_128B;
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed (%d) for a split %lld x %lld operand", (int)r, (long long)rows,
                  (long long)inner);
        return LATENTAM_ERR_CUDA;
    }
    return LATENTAM_OK;
}

// Tensor map of a split operand read MN-major (K rows of `inner` contiguous MN elements, inner a
// multiple of 64): a 4D view (64 elements, K row, 64-element block, plane) whose box of 64 x
// box_rows x nblk x 2 lands in shared memory as [plane][block][K row][128 B], the MN-major
// layout of both planes of a BN = 64 nblk tile, in one load.
latentam_status split_map_mn(CUtensorMap* m, const void* base, int64_t inner, int64_t rows, int64_t ld, int box_rows,
                             int nblk) {
    EncodeTiledFn enc;
    LAT_TRY(encoder(&enc));
    if ((reinterpret_cast<uintptr_t>(base) & 15u) || (ld * 2) % 16 || (rows * ld * 2) % 16 || inner % 64) {
        set_error("split MN-major operand not 16-byte aligned or not made of 64-wide blocks");
        return LATENTAM_ERR_INVALID_ARG;
    }
    const cuuint64_t dims[4] = {64, (cuuint64_t)rows, (cuuint64_t)(inner / 64), 2};
    const cuuint64_t strides[3] = {(cuuint64_t)(ld * 2), 128, (cuuint64_t)(rows * ld * 2)};
    const cuuint32_t box[4] = {64, (cuuint32_t)box_rows, (cuuint32_t)nblk, 2};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(base), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed (%d) for a split MN-major %lld x %lld operand", (int)r,
                  (long long)rows, (long long)inner);
        return LATENTAM_ERR_CUDA;
    }
    return LATENTAM_OK;
}

// Maps of the plain (BF16, 2D) or split (FP32, hi / lo planes) form: op_map for a K-major MMA
// operand (split: both planes per box), mn_map for an MN-major B operand (split: both planes
// and nblk 64-wide blocks per box), io_map for epilogue operands, staged outputs and MN-major A
// operands (split: one plane per box).
latentam_status op_map(bool split, CUtensorMap* m, const void* base, int64_t inner, int64_t rows, int64_t ld,
                       int box_rows, int box_inner = tc::kChunkK) {
    return split ? split_map(m, base, inner, rows, ld, box_rows, box_inner, 2)
                 : bf16_map(m, base, inner, rows, ld, box_rows, box_inner);
}
latentam_status mn_map(bool split, CUtensorMap* m, const void* base, int64_t inner, int64_t rows, int64_t ld,
                       int box_rows, int nblk) {
    return split ? split_map_mn(m, base, inner, rows, ld, box_rows, nblk)
                 : bf16_map(m, base, inner, rows, ld, box_rows);
}
latentam_status io_map(bool split, CUtensorMap* m, const void* base, int64_t inner, int64_t rows, int64_t ld,
                       int box_rows, int box_inner = tc::kChunkK) {
    return split ? split_map(m, base, inner, rows, ld, box_rows, box_inner, 1)
                 : bf16_map(m, base, inner, rows, ld, box_rows, box_inner);
}

// Launch one tile grid of Epi (emap: epilogue operand, omap: staged output); cluster_y > 1
// groups that many consecutive y tiles of each row block into a thread-block cluster (the
// epilogue's row exchange).
// Tensor map of a row-major 8-bit matrix (rows x inner bytes, row stride ld bytes), boxes of
// 64 x box_rows bytes with 64-byte swizzle.
latentam_status u8_map(CUtensorMap* m, const void* base, int64_t inner, int64_t rows, int64_t ld, int box_rows) {
    EncodeTiledFn enc;
    LAT_TRY(encoder(&enc));
    if ((reinterpret_cast<uintptr_t>(base) & 15u) || ld % 16) {
        set_error("tensor-core operand not 16-byte aligned");
        return LATENTAM_ERR_INVALID_ARG;
    }
    const cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld};
    const cuuint32_t box[2] = {64, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void*>(base), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed (%d) for a %lld x %lld 8-bit operand", (int)r, (long long)rows,
                  (long long)inner);
        return LATENTAM_ERR_CUDA;
    }
    return LATENTAM_OK;
}

template <class Epi>
latentam_status launch_gemm(const CUtensorMap& a, const CUtensorMap& b, dim3 grid, tc::GemmGrid g,
                            const typename Epi::Params& p, int* err, cudaStream_t st, const CUtensorMap* emap = nullptr,
                            const CUtensorMap* omap = nullptr, int cluster_y = 1, const CUtensorMap* xmap = nullptr,
                            const CUtensorMap* xmap2 = nullptr) {
    constexpr size_t smem = tc::gemm_smem_bytes<Epi>();
    static_assert(smem <= 227 * 1024, "tile does not fit in shared memory");
    if (cluster_y > tc::kMaxCluster || (int)grid.y % cluster_y != 0 || (cluster_y > 1 && Epi::XROUNDS == 0)) {
        set_error("bad cluster shape %d for a grid of %u row tiles", cluster_y, grid.y);
        return LATENTAM_ERR_INVALID_ARG;
    }
    auto kern = tc::tc_gemm_kernel<Epi>;
    static unsigned long long attr_set = 0;  // per instantiation and device; setting it twice is harmless
    int dev = 0;
    cudaGetDevice(&dev);
    if (!(attr_set & (1ull << (dev & 63)))) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return cuda_error(e, "tc_gemm smem attribute");
        attr_set |= 1ull << (dev & 63);
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(tc::gemm_threads(Epi::EPI_WG), 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    if (cluster_y > 1) {
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = 1;
        attr[0].val.clusterDim.y = (unsigned)cluster_y;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
    }
    cudaError_t e =
        cudaLaunchKernelEx(&cfg, kern, a, b, emap ? *emap : a, omap ? *omap : a, xmap ? *xmap : a, xmap2 ? *xmap2 : a, g,
                           p, err);
    if (e != cudaSuccess) return cuda_error(e, "tc_gemm_kernel launch");
    LAT_CHECK_LAUNCH("tc_gemm_kernel");
    return LATENTAM_OK;
}

// Launch the persistent form of Epi over row_tiles 128-row tiles and gy column tiles (a
// cluster of gy CTAs when the epilogue trades row partials): as many CTAs (clusters) as can be
// resident at once, each walking its share of the row tiles.
template <class Epi>
latentam_status launch_persist(latentam_ctx* ctx, const CUtensorMap& a, const CUtensorMap& b, int row_tiles,
                               int k_chunks, int gy, bool cluster, const typename Epi::Params& p, int* err,
                               cudaStream_t st, const CUtensorMap* emap = nullptr,
                               const CUtensorMap* omap = nullptr) {
    constexpr size_t smem = tc::persist_smem_bytes<Epi>();
    static_assert(smem <= 227 * 1024, "persistent tile does not fit in shared memory");
    if (row_tiles <= 0) return LATENTAM_OK;
    if (gy < 1 || (cluster && (gy > tc::kMaxCluster || Epi::XROUNDS == 0))) {
        set_error("bad cluster shape %d", gy);
        return LATENTAM_ERR_INVALID_ARG;
    }
    auto kern = tc::tc_persist_kernel<Epi>;
    static unsigned long long attr_set = 0;  // per instantiation and device
    int dev = 0;
    cudaGetDevice(&dev);
    if (!(attr_set & (1ull << (dev & 63)))) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return cuda_error(e, "tc_persist smem attribute");
        attr_set |= 1ull << (dev & 63);
    }
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(tc::persist_threads(Epi::EPI_WG), 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    int slots = ctx->num_sms / gy;  // one CTA per SM
    if (cluster && gy > 1) {
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = 1;
        attr[0].val.clusterDim.y = (unsigned)gy;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        static int cached[tc::kMaxCluster + 1] = {0};
        if (cached[gy] == 0) {
            cfg.gridDim = dim3((unsigned)std::max(1, ctx->num_sms / gy), (unsigned)gy, 1);
            int nc = 0;
            if (cudaOccupancyMaxActiveClusters(&nc, kern, &cfg) != cudaSuccess || nc <= 0) {
                (void)cudaGetLastError();
                nc = std::max(1, ctx->num_sms / gy);
            }
            cached[gy] = nc;
        }
        slots = cached[gy];
    }
    cfg.gridDim = dim3((unsigned)std::max(1, std::min(row_tiles, slots)), (unsigned)gy, 1);
    const tc::PersistGrid pg{k_chunks, row_tiles};
    cudaError_t e = cudaLaunchKernelEx(&cfg, kern, a, b, emap ? *emap : a, omap ? *omap : a, pg, p, err);
    if (e != cudaSuccess) return cuda_error(e, "tc_persist_kernel launch");
    LAT_CHECK_LAUNCH("tc_persist_kernel");
    return LATENTAM_OK;
}

struct TcBuffers {
    bf16 *Qb, *Kb, *Vb, *A, *dF, *dS;
    float *row, *coef, *part;
    double* acc;
    int* err;
    // E4M3 form
    uint8_t *Aq, *Vtq;
    float *stats, *inv_t;
};

// split: Qb, Kb, Vb, A, dF and dS each hold a hi and a lo plane.
latentam_status tc_buffers(latentam_ctx* ctx, int64_t n, int M, int D, bool train, bool fp8, TcBuffers* b,
                           bool split = false) {
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const int64_t nn = std::max<int64_t>(n, 1);
    const size_t e2 = sizeof(bf16) * (split ? 2 : 1);  // bytes per element over all planes
    size_t o = 0, off[9];
    off[0] = o, o += up(e2 * nn * kPad);                      // Qb
    off[1] = o, o += up(e2 * (size_t)M * kPad);               // Kb
    off[2] = o, o += up(e2 * (size_t)M * D);                  // Vb
    off[3] = o, o += up(sizeof(float) * 4 * nn);              // row
    off[4] = o, o += up(sizeof(float) * (size_t)M);           // coef
    off[5] = o, o += fp8 ? up((size_t)nn * M) : 0;            // Aq
    off[6] = o, o += fp8 ? up((size_t)D * M) : 0;             // Vtq
    off[7] = o, o += fp8 ? up(sizeof(float) * 2 * nn) : 0;    // stats
    off[8] = o, o += fp8 ? up(sizeof(float) * (size_t)D) : 0; // inv_t
    char* ops = static_cast<char*>(ws(ctx, WS_DEC_AUX3, o));
    // dS, or (dK fused into G3) the per-tile dK partials: 128-pixel tiles x M x (d <= 64) FP32
    const size_t ds_bytes = std::max(up(e2 * nn * M), up(sizeof(float) * (size_t)((nn + 127) / 128) * M * kPad));
    const size_t rows_bytes = up(e2 * nn * M) + (train ? up(e2 * nn * D) + ds_bytes : 0);
    char* rows = static_cast<char*>(ws(ctx, WS_DEC_A, rows_bytes));
    double* acc = static_cast<double*>(ws(ctx, WS_LOSS, 256));
    if (!ops || !rows || !acc) return LATENTAM_ERR_OUT_OF_MEMORY;
    b->Qb = reinterpret_cast<bf16*>(ops + off[0]);
    b->Kb = reinterpret_cast<bf16*>(ops + off[1]);
    b->Vb = reinterpret_cast<bf16*>(ops + off[2]);
    b->row = reinterpret_cast<float*>(ops + off[3]);
    b->coef = reinterpret_cast<float*>(ops + off[4]);
    b->A = reinterpret_cast<bf16*>(rows);
    b->dF = train ? reinterpret_cast<bf16*>(rows + up(e2 * nn * M)) : nullptr;
    b->dS = train ? reinterpret_cast<bf16*>(rows + up(e2 * nn * M) + up(e2 * nn * D)) : nullptr;
    b->acc = acc;
    b->err = ctx->dev_flags;  // sticky: reported by the next synchronising call
    b->part = nullptr;
    b->Aq = fp8 ? reinterpret_cast<uint8_t*>(ops + off[5]) : nullptr;
    b->Vtq = fp8 ? reinterpret_cast<uint8_t*>(ops + off[6]) : nullptr;
    b->stats = fp8 ? reinterpret_cast<float*>(ops + off[7]) : nullptr;
    b->inv_t = fp8 ? reinterpret_cast<float*>(ops + off[8]) : nullptr;
    return LATENTAM_OK;
}

// Split of the pixel reduction (K) of G5/G6 into about z parts of at least four chunks of
// `chunk` pixels; *z_out receives the number of parts.
tc::GemmGrid pixel_split(int64_t n, int z, int* z_out, int chunk = tc::kChunkK) {
    const int chunks = (int)((n + chunk - 1) / chunk);
    z = std::max(1, std::min(z, std::max(1, chunks / 4)));
    const int cpz = (chunks + z - 1) / z;
    *z_out = (chunks + cpz - 1) / cpz;
    return tc::GemmGrid{chunks, cpz};
}

// The split the tile grid starts from: about one wave of CTAs.
int wave_split(int tiles_xy, int num_sms) { return std::max(1, (num_sms + tiles_xy - 1) / tiles_xy); }

// Autotuned launch shape of a pixel reduction: the first time a shape (n, M, D, which) is seen
// outside stream capture, `launch(shape, z)` runs for every tile shape 0 .. nshapes - 1 with its
// wave split z0[shape], half of it and twice it (one untimed warm-up run first), timed with CUDA
// events on the stream, and the fastest (tile shape, split) is kept in the context.
template <class Launch>
latentam_status tuned_shape(latentam_ctx* ctx, int64_t n, int M, int D, int which, int nshapes, const int* z0,
                            cudaStream_t st, Launch&& launch, int* shape_out, int* z_out) {
    *shape_out = 0;
    *z_out = z0[0];
    for (int i = 0; i < ctx->tune_used; ++i) {
        const auto& t = ctx->tune[i];
        if (t.n == n && t.M == M && t.D == D && t.which == which) {
            *shape_out = t.shape;
            *z_out = t.z;
            return LATENTAM_OK;
        }
    }
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (!ctx->autotune || cudaStreamIsCapturing(st, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone)
        return LATENTAM_OK;
    cudaEvent_t ev[2];
    for (auto& e : ev)
        if (cudaEventCreate(&e) != cudaSuccess) return cuda_error(cudaGetLastError(), "tuning events");
    latentam_status s = launch(0, z0[0]);  // warm-up
    float best = 1e30f;
    for (int sh = 0; sh < nshapes && s == LATENTAM_OK; ++sh) {
        const int cand[3] = {z0[sh], std::max(1, z0[sh] / 2), 2 * z0[sh]};
        for (int i = 0; i < 3 && s == LATENTAM_OK; ++i) {
            cudaEventRecord(ev[0], st);
            s = launch(sh, cand[i]);
            cudaEventRecord(ev[1], st);
            cudaEventSynchronize(ev[1]);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ev[0], ev[1]);
            if (s == LATENTAM_OK && ms < best) best = ms, *shape_out = sh, *z_out = cand[i];
        }
    }
    for (auto& e : ev) cudaEventDestroy(e);
    LAT_TRY(s);
    auto& t = ctx->tune[ctx->tune_next];
    t = latentam_ctx::TuneEntry{n, M, D, which, *shape_out, *z_out, best};
    ctx->tune_next = (ctx->tune_next + 1) % 32;
    if (ctx->tune_used < 32) ++ctx->tune_used;
    return LATENTAM_OK;
}

}  // namespace

namespace {

int cdiv(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// Rows of S and of Fhat are spread over clusters of up to kMaxCluster CTAs of 256 columns.
constexpr int kMaxCols = 256 * tc::kMaxCluster;

latentam_status check_tc_shape(int M, int D) {
    if (M > kMaxCols || D > kMaxCols) {
        set_error("the BF16 tensor-core decode spreads a row of S (M=%d) and of Fhat (D=%d) over at most %d CTAs "
                  "of 256 columns: both must be <= %d",
                  M, D, tc::kMaxCluster, kMaxCols);
        return LATENTAM_ERR_UNSUPPORTED_SHAPE;
    }
    return LATENTAM_OK;
}

// Operand preparation + G1 (softmax).  SPLIT: the FP32 form (hi / lo planes, 16-wide K chunks
// over the d query columns).
template <bool SPLIT>
latentam_status tc_forward(latentam_ctx* ctx, const float* Q, int64_t n, int d, const float* K, const float* V, int M,
                           int D, float c, const TcBuffers& b, float* stats, cudaStream_t st) {
    prep_dict<SPLIT><<<std::min(4 * ctx->num_sms, cdiv((int64_t)M * (D + kPad), 256)), 256, 0, st>>>(K, V, M, d, D,
                                                                                                      b.Kb, b.Vb);
    LAT_CHECK_LAUNCH("prep_dict");
    prep_queries<SPLIT><<<cdiv(n * (kPad / 8), 256), 256, 0, st>>>(Q, n, d, b.Qb);
    LAT_CHECK_LAUNCH("prep_queries");
    if (b.Vtq) {
        fp8_values<<<cdiv(D, 128), 128, 0, st>>>(V, M, D, b.Vtq, b.inv_t);
        LAT_CHECK_LAUNCH("fp8_values");
    }
    using Epi = SoftmaxEpi<SPLIT>;
    CUtensorMap mQ, mK;
    LAT_TRY(op_map(SPLIT, &mQ, b.Qb, kPad, n, kPad, kTileM, Epi::BK));
    LAT_TRY(op_map(SPLIT, &mK, b.Kb, kPad, M, kPad, 256, Epi::BK));
    CUtensorMap mA;  // the attention rows leave through the TMA
    LAT_TRY(io_map(SPLIT, &mA, b.A, M, n, M, kTileM));
    SoftmaxParams sp{n, M, c, b.A, stats};
    const int cy = cdiv(M, 256);
    const int kc = SPLIT ? d / Epi::BK : 1;  // plain: the padded queries are one 64-wide chunk
    return launch_persist<Epi>(ctx, mQ, mK, cdiv(n, kTileM), kc, cy, true, sp, b.err, st, nullptr, &mA);
}

// G2: Fhat = A V (A in 32-wide K chunks, 64-byte swizzle), B = V read MN-major in 64 x 32
// boxes (features x atoms).
latentam_status tc_fhat8(latentam_ctx* ctx, const TcBuffers& b, int64_t n, int M, int D, const FhatParams& fp,
                         cudaStream_t st);

template <bool SPLIT>
latentam_status tc_fhat(latentam_ctx* ctx, const TcBuffers& b, int64_t n, int M, int D, const FhatParams& fp,
                        cudaStream_t st) {
    if (!SPLIT && b.Aq) return tc_fhat8(ctx, b, n, M, D, fp, st);
    using EpiF = FhatEpi<false, false, SPLIT>;  // targets read per thread (FP32 or BF16)
    constexpr int BK = EpiF::BK;
    CUtensorMap mA, mV;
    LAT_TRY(op_map(SPLIT, &mA, b.A, M, n, M, kTileM, BK));
    LAT_TRY(mn_map(SPLIT, &mV, b.Vb, D, M, D, BK, EpiF::BN / 64));
    const int cy = cdiv(D, 256), tiles = cdiv(n, kTileM), kc = cdiv(M, BK);
    if (fp.Fout)  // no row terms: independent column tiles
        return launch_persist<EpiF>(ctx, mA, mV, tiles, kc, cy, false, fp, b.err, st);
    CUtensorMap mdF;  // dFhat leaves through the TMA
    if (SPLIT && fp.F_dtype == LATENTAM_DTYPE_F32) {
        // FP32 targets by TMA, 32 columns at a time; dFhat written over them as 32-column planes
        CUtensorMap mF;
        LAT_TRY(f32_map(&mF, fp.F, D, n, kTileM));
        LAT_TRY(io_map(true, &mdF, fp.dF, D, n, D, kTileM, 32));
        return launch_persist<FhatEpi<true, false, true>>(ctx, mA, mV, tiles, kc, cy, true, fp, b.err, st, &mF, &mdF);
    }
    LAT_TRY(io_map(SPLIT, &mdF, fp.dF, D, n, D, kTileM));
    if (!SPLIT && fp.F_dtype == LATENTAM_DTYPE_BF16) {
        // BF16 targets: the tile's target rows are TMA-loaded into shared memory for the epilogue
        CUtensorMap mF;
        LAT_TRY(bf16_map(&mF, fp.F, D, n, D, kTileM));
        return launch_persist<FhatEpi<true>>(ctx, mA, mV, tiles, kc, cy, true, fp, b.err, st, &mF, &mdF);
    }
    return launch_persist<EpiF>(ctx, mA, mV, tiles, kc, cy, true, fp, b.err, st, nullptr, &mdF);
}

// G2 on E4M3 operands: the attention rows scaled per pixel (from the softmax row statistics)
// and V^T scaled per feature, both in 64-byte K chunks; the epilogue undoes both scales.
latentam_status tc_fhat8(latentam_ctx* ctx, const TcBuffers& b, int64_t n, int M, int D, const FhatParams& fp0,
                         cudaStream_t st) {
    fp8_rows<<<cdiv(n * (M / 8), 256), 256, 0, st>>>(b.A, b.stats, n, M, b.Aq);
    LAT_CHECK_LAUNCH("fp8_rows");
    FhatParams fp = fp0;
    fp.stats = b.stats;
    fp.inv_t = b.inv_t;
    CUtensorMap mA, mV;
    LAT_TRY(u8_map(&mA, b.Aq, M, n, M, kTileM));
    LAT_TRY(u8_map(&mV, b.Vtq, M, D, M, 256));
    const int cy = cdiv(D, 256), tiles = cdiv(n, kTileM), kc = cdiv(M, 64);
    if (fp.Fout) return launch_persist<FhatEpi<false, true>>(ctx, mA, mV, tiles, kc, cy, false, fp, b.err, st);
    CUtensorMap mdF;
    LAT_TRY(bf16_map(&mdF, fp.dF, D, n, D, kTileM));
    if (fp.F_dtype == LATENTAM_DTYPE_BF16) {
        CUtensorMap mF;
        LAT_TRY(bf16_map(&mF, fp.F, D, n, D, kTileM));
        return launch_persist<FhatEpi<true, true>>(ctx, mA, mV, tiles, kc, cy, true, fp, b.err, st, &mF, &mdF);
    }
    return launch_persist<FhatEpi<false, true>>(ctx, mA, mV, tiles, kc, cy, true, fp, b.err, st, nullptr, &mdF);
}

// The six contractions of the decode, its loss and its backward.  SPLIT: the FP32 form, every
// operand a hi / lo pair of BF16 planes and every product three MMAs (see tc::mma_step).
template <bool SPLIT>
latentam_status tc_loss_bwd(latentam_ctx* ctx, const DecodeArgs& a, cudaStream_t st, bool fp8) {
    const int64_t n = a.n;
    const int M = a.M, D = a.D, d = a.d;
    LAT_TRY(check_tc_shape(M, D));
    TcBuffers b;
    LAT_TRY(tc_buffers(ctx, n, M, D, true, fp8, &b, SPLIT));
    cudaError_t e = cudaMemsetAsync(b.acc, 0, 256, st);
    if (e != cudaSuccess) return cuda_error(e, "memset accumulators");
    if (n > 0) {
        tc_count_mask<<<std::min(4 * ctx->num_sms, cdiv(n, 256)), 256, 0, st>>>(a.mask, n, b.acc);
        LAT_CHECK_LAUNCH("tc_count_mask");
    }
    tc_trust_region<<<cdiv(M, 8), 256, 0, st>>>(a.V, a.V0, M, D, a.cfg.delta, a.cfg.lambda_f * a.cfg.lambda_D, b.coef,
                                              b.acc);
    LAT_CHECK_LAUNCH("tc_trust_region");
    constexpr int BNq = kPad;  // queries padded to 64 columns
    // dV tile shapes: 0 = 256 atoms per CTA (two accumulators: each dFhat block read once for
    // both halves), 1 = 128 atoms per CTA (twice the CTAs, each dFhat block read twice)
    using EpiV = PartEpi<256, SPLIT, 2>;
    using EpiV1 = PartEpi<256, SPLIT, 1>;
    const int tilesV[2] = {cdiv(M, 2 * kTileM) * cdiv(D, 256), cdiv(M, kTileM) * cdiv(D, 256)};
    const int tilesK = cdiv(M, kTileM);
    const int zV0[2] = {wave_split(tilesV[0], ctx->num_sms), wave_split(tilesV[1], ctx->num_sms)};
    const int zK0 = wave_split(tilesK, ctx->num_sms);
    // partial sums for the largest split a tuner may try
    const size_t part_floats = std::max({(size_t)2 * zV0[0] * M * D, (size_t)2 * zV0[1] * M * D,
                                         (size_t)2 * zK0 * M * BNq});
    b.part = static_cast<float*>(ws(ctx, WS_DEC_PART, sizeof(float) * part_floats));
    if (!b.part) return LATENTAM_ERR_OUT_OF_MEMORY;
    const int which = SPLIT ? 16 : 0;  // autotuner key offset of the split form
    bool dk_fused = false;
    if (n > 0) {
        // G1: S = Q K^T -> softmax
        LAT_TRY(tc_forward<SPLIT>(ctx, a.Q, n, d, a.K, a.V, M, D, a.c, b, b.stats, st));
        // G2: Fhat = A V -> loss terms -> dFhat
        FhatParams fp{n, D, a.F, a.F_dtype, a.mask, a.cfg, b.acc, b.dF, b.row, nullptr, nullptr, nullptr};
        LAT_TRY(tc_fhat<SPLIT>(ctx, b, n, M, D, fp, st));
        // G3: dA = dFhat V^T -> dS
        CUtensorMap mdF, mV, mdS, mK;
        constexpr int BK3 = DsEpi<SPLIT>::BKC;  // K (feature) elements per ring stage
        LAT_TRY(op_map(SPLIT, &mdF, b.dF, D, n, D, kTileM, BK3));
        LAT_TRY(op_map(SPLIT, &mV, b.Vb, D, M, D, 256, BK3));
        // G4 (dQ = c dS K, B = K padded, read MN-major) runs as G3's trailing product on the
        // staged dS tile when a row's atoms span at most two CTAs, else as its own GEMM
        const int ty = cdiv(M, 256);
        const bool dq_fused = a.dQ != nullptr && ty <= 2;
        // G6 (dK partials = dS^T Q per tile, Q read MN-major as the tile's 128 x 64 block) runs as
        // its second trailing product when G4 is fused: dS then never leaves the chip
        dk_fused = dq_fused && a.dK != nullptr;
        if (a.dQ) LAT_TRY(mn_map(SPLIT, &mK, b.Kb, kPad, M, kPad, 64, kPad / 64));
        CUtensorMap mQt;
        if (dk_fused) LAT_TRY(op_map(SPLIT, &mQt, b.Qb, kPad, n, kPad, kTileM));
        if (dq_fused && ty > 1) {
            e = cudaMemsetAsync(a.dQ, 0, sizeof(float) * (size_t)n * d, st);
            if (e != cudaSuccess) return cuda_error(e, "memset dQ");
        }
        DsParams dp{n,   M, b.A, b.row, b.dS, dq_fused ? a.dQ : nullptr, d, a.c, ty > 1 ? 1 : 0,
                    dk_fused ? reinterpret_cast<float*>(b.dS) : nullptr};
        const dim3 grow(cdiv(n, kTileM), 1, 1);
        const tc::GemmGrid g3{cdiv(D, BK3), cdiv(D, BK3)};
        CUtensorMap mAe, mdSo;  // attention rows for the epilogue, dS out through the TMA
        LAT_TRY(io_map(SPLIT, &mAe, b.A, M, n, M, kTileM));
        LAT_TRY(io_map(SPLIT, &mdSo, b.dS, M, n, M, kTileM));
        LAT_TRY((launch_gemm<DsEpi<SPLIT>>(mdF, mV, dim3(cdiv(n, kTileM), ty, 1), g3, dp, b.err, st, &mAe, &mdSo, 1,
                                           dq_fused ? &mK : nullptr, dk_fused ? &mQt : nullptr)));
        if (a.dQ && !dq_fused) {
            LAT_TRY(op_map(SPLIT, &mdS, b.dS, M, n, M, kTileM));
            DqParams qp{n, d, a.c, a.dQ};
            const tc::GemmGrid g4{cdiv(M, tc::kChunkK), cdiv(M, tc::kChunkK)};
            LAT_TRY((launch_gemm<DqEpi<BNq, SPLIT>>(mdS, mK, grow, g4, qp, b.err, st)));
        }
    }
    // dQ is final: work of the caller's that needs only dQ may branch off here
    if (ctx->after_dq && a.dQ) {
        LAT_TRY((*ctx->after_dq)(st));
        ctx->after_dq_called = 1;
    }
    // G5: dV = A^T dFhat (+ trust region), both operands pixel-major (MN-major); each candidate
    // the tuner times includes the reduction of its partials (more splits, more partials to sum)
    auto reduce_dV = [&](int z) -> latentam_status {
        const bool v4 = D % 4 == 0 && !(reinterpret_cast<uintptr_t>(a.dV) & 15u) &&
                        !(reinterpret_cast<uintptr_t>(a.V) & 15u) && !(reinterpret_cast<uintptr_t>(a.V0) & 15u);
        if (v4)
            tc_reduce_parts4<8><<<cdiv((int64_t)M * D, 128), 256, 0, st>>>(b.part, z, M, D, D, 1.0f, b.coef, a.V,
                                                                          a.V0, a.dV);
        else
            tc_reduce_parts<8><<<cdiv((int64_t)M * D, 32), 256, 0, st>>>(b.part, z, M, D, D, 1.0f, b.coef, a.V, a.V0,
                                                                         a.dV);
        LAT_CHECK_LAUNCH("tc_reduce_parts");
        return LATENTAM_OK;
    };
    auto reduce_dK = [&](int z) -> latentam_status {
        tc_reduce_parts<8><<<cdiv((int64_t)M * d, 32), 256, 0, st>>>(b.part, z, M, BNq, d, a.c, nullptr, nullptr,
                                                                     nullptr, a.dK);
        LAT_CHECK_LAUNCH("tc_reduce_parts");
        return LATENTAM_OK;
    };
    if (a.dV) {
        if (n == 0) LAT_TRY(reduce_dV(0));  // the trust-region term alone
        if (n > 0) {
            CUtensorMap mA[2], mdF[2];  // per tile shape (pixel block of a ring stage: BKC)
            LAT_TRY(io_map(SPLIT, &mA[0], b.A, M, n, M, EpiV::BKC));
            LAT_TRY(mn_map(SPLIT, &mdF[0], b.dF, D, n, D, EpiV::BKC, 256 / 64));
            LAT_TRY(io_map(SPLIT, &mA[1], b.A, M, n, M, EpiV1::BKC));
            LAT_TRY(mn_map(SPLIT, &mdF[1], b.dF, D, n, D, EpiV1::BKC, 256 / 64));
            PartParams pp{M, D, D, b.part};
            auto g5 = [&](int shape, int z) -> latentam_status {
                int zz;
                if (shape == 0) {
                    const tc::GemmGrid g = pixel_split(n, z, &zz, EpiV::BKC);
                    LAT_TRY(launch_gemm<EpiV>(mA[0], mdF[0], dim3(cdiv(M, 2 * kTileM), cdiv(D, 256), zz), g, pp,
                                              b.err, st));
                } else {
                    const tc::GemmGrid g = pixel_split(n, z, &zz, EpiV1::BKC);
                    LAT_TRY(launch_gemm<EpiV1>(mA[1], mdF[1], dim3(cdiv(M, kTileM), cdiv(D, 256), zz), g, pp, b.err,
                                               st));
                }
                return reduce_dV(zz);
            };
            int shape, z;
            LAT_TRY(tuned_shape(ctx, n, M, D, 5 + which, 2, zV0, st, g5, &shape, &z));
            LAT_TRY(g5(shape, z));
        }
    }
    // G6: dK = c dS^T Q
    if (a.dK && dk_fused) {
        // the per-tile partials G3 left in the dS buffer, summed in tile order
        tc_reduce_parts<32, true><<<cdiv((int64_t)M * d, 32), 1024, 0, st>>>(
            reinterpret_cast<const float*>(b.dS), (int)cdiv(n, kTileM), d, M, M, a.c, nullptr, nullptr, nullptr, a.dK);
        LAT_CHECK_LAUNCH("tc_reduce_parts");
    } else if (a.dK) {
        if (n == 0) LAT_TRY(reduce_dK(0));  // zero
        if (n > 0) {
            CUtensorMap mdS, mQ;
            LAT_TRY(io_map(SPLIT, &mdS, b.dS, M, n, M, 64));
            LAT_TRY(mn_map(SPLIT, &mQ, b.Qb, kPad, n, kPad, 64, kPad / 64));
            PartParams pp{M, BNq, BNq, b.part};
            auto g6 = [&](int, int z) -> latentam_status {
                int zz;
                const tc::GemmGrid g = pixel_split(n, z, &zz);
                LAT_TRY((launch_gemm<PartEpi<BNq, SPLIT>>(mdS, mQ, dim3(cdiv(M, kTileM), 1, zz), g, pp, b.err, st)));
                return reduce_dK(zz);
            };
            int shape, z;
            LAT_TRY(tuned_shape(ctx, n, M, D, 6 + which, 1, &zK0, st, g6, &shape, &z));
            LAT_TRY(g6(0, z));
        }
    }
    tc_finalize<<<1, 1, 0, st>>>(b.acc, b.err, D, a.cfg, a.loss_parts);
    LAT_CHECK_LAUNCH("tc_finalize");
    return LATENTAM_OK;
}

template <bool SPLIT>
latentam_status tc_fwd(latentam_ctx* ctx, const float* Q, int64_t n, int d, const float* K, const float* V, int M,
                       int D, float c, float* F_hat, float* row_stats, cudaStream_t st, bool fp8) {
    LAT_TRY(check_tc_shape(M, D));
    if (n == 0) return LATENTAM_OK;
    TcBuffers b;
    LAT_TRY(tc_buffers(ctx, n, M, D, false, fp8, &b, SPLIT));
    cudaError_t e = cudaMemsetAsync(b.acc, 0, 256, st);
    if (e != cudaSuccess) return cuda_error(e, "memset accumulators");
    float* stats = fp8 ? b.stats : row_stats;
    LAT_TRY(tc_forward<SPLIT>(ctx, Q, n, d, K, V, M, D, c, b, stats, st));
    if (fp8 && row_stats) {
        e = cudaMemcpyAsync(row_stats, b.stats, sizeof(float) * 2 * n, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return cuda_error(e, "copy row statistics");
    }
    if (F_hat) {
        FhatParams fp{n, D, nullptr, LATENTAM_DTYPE_F32, nullptr, latentam_loss_cfg{}, b.acc, nullptr, b.row, F_hat,
                      nullptr, nullptr};
        LAT_TRY(tc_fhat<SPLIT>(ctx, b, n, M, D, fp, st));
    }
    return LATENTAM_OK;
}

}  // namespace

latentam_status decode_loss_bwd_bf16(latentam_ctx* ctx, const DecodeArgs& a, cudaStream_t st, bool fp8) {
    return tc_loss_bwd<false>(ctx, a, st, fp8);
}

latentam_status decode_fwd_bf16(latentam_ctx* ctx, const float* Q, int64_t n, int d, const float* K, const float* V,
                                int M, int D, float c, float* F_hat, float* row_stats, cudaStream_t st, bool fp8) {
    return tc_fwd<false>(ctx, Q, n, d, K, V, M, D, c, F_hat, row_stats, st, fp8);
}

bool decode_split_supported(int d, int M, int D) {
    return (d == 16 || d == 32 || d == 64) && M <= kMaxCols && D <= kMaxCols;
}

latentam_status decode_loss_bwd_split(latentam_ctx* ctx, const DecodeArgs& a, cudaStream_t st) {
    return tc_loss_bwd<true>(ctx, a, st, false);
}

latentam_status decode_fwd_split(latentam_ctx* ctx, const float* Q, int64_t n, int d, const float* K, const float* V,
                                 int M, int D, float c, float* F_hat, float* row_stats, cudaStream_t st) {
    return tc_fwd<true>(ctx, Q, n, d, K, V, M, D, c, F_hat, row_stats, st, false);
}

}  // namespace lat
