// Query rendering Q = R_f(G, T) (Sec. III-B, Eq. render_query): the depth-ordered alpha
// blending of Eq. (alpha_blending) applied to the d-dimensional query vectors f_i, and its
// backward with respect to f.
//
// One CTA per 16x16 tile, one thread per pixel.  The tile's Gaussians are staged through
// shared memory in batches of 256 (mean, exponent coefficients/opacity, query as
// float4 rows), so every query row is read from L2/HBM once per tile and broadcast to the
// 256 pixels.
#include <cuda_bf16.h>

#include <algorithm>

#include "internal.cuh"

namespace lat {
namespace {

constexpr int kBatch = kTilePixels;  // 256 Gaussians staged per round

// Staged form of one splat: exponent coefficients q = (-a/2, -b, -c/2, opacity) of the conic
// (a, b, c).
__device__ __forceinline__ float4 stage_splat(float4 co) {
    return make_float4(__fmul_rn(-0.5f, co.x), -co.y, __fmul_rn(-0.5f, co.z), co.w);
}

// The hi and lo BF16 terms of (x0, x1), packed: hi = bf16(x), lo = bf16(x - hi).
__device__ __forceinline__ void tc_split(float x0, float x1, uint32_t& hi, uint32_t& lo) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
    const float2 hf = __bfloat1622float2(h);
    const __nv_bfloat162 l = __floats2bfloat162_rn(x0 - hf.x, x1 - hf.y);
    hi = *reinterpret_cast<const uint32_t*>(&h);
    lo = *reinterpret_cast<const uint32_t*>(&l);
}

// alpha of a splat at a pixel centre, or -1 when the exponent is positive.  Every rounding
// is explicit (fused multiply-adds written out), so the forward and backward kernels take
// bit-identical decisions for the same inputs.
__device__ __forceinline__ float splat_alpha(float2 m, float4 q, float px, float py) {
    const float dx = __fsub_rn(m.x, px), dy = __fsub_rn(m.y, py);
    const float power = __fmaf_rn(dx, __fmaf_rn(q.x, dx, __fmul_rn(q.y, dy)), __fmul_rn(__fmul_rn(q.z, dy), dy));
    if (power > 0.0f) return -1.0f;
    return fminf(kAlphaMax, __fmul_rn(q.w, __expf(power)));
}

template <int DQ>
struct FwdSmem {
    float2 xy[kBatch];
    float4 co[kBatch];
    float4 f[kBatch][DQ / 4];
};

// Front-to-back blend of one tile (256 threads, one pixel each).
template <int DQ>
__device__ __forceinline__ void render_fwd_tile(const TileJob& job, FwdSmem<DQ>& sm) {
    constexpr int DV = DQ / 4;
    const int tile = job.tile;
    const int tx = tile % job.tiles_x, ty = tile / job.tiles_x;
    const int t = threadIdx.x;
    const int px = tx * kTile + (t % kTile), py = ty * kTile + (t / kTile);
    const bool inside = px < job.W && py < job.H;
    const float fpx = (float)px, fpy = (float)py;
    const int2 range = job.ranges[tile];
    float4 acc[DV];
#pragma unroll
    for (int k = 0; k < DV; ++k) acc[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    float T = 1.0f;
    int count = 0;
    bool done = !inside;
    for (int start = range.x; start < range.y; start += kBatch) {
        if (__syncthreads_count(done) == kTilePixels) break;
        const int k = start + t;
        if (k < range.y) {
            const int g = job.pair_ids[k];
            sm.xy[t] = job.xy[g];
            sm.co[t] = stage_splat(job.conic_opac[g]);
#pragma unroll
            for (int c = 0; c < DV; ++c) sm.f[t][c] = job.f[(size_t)g * DV + c];
        }
        __syncthreads();
        const int cnt = min(kBatch, range.y - start);
        for (int j = 0; j < cnt && !done; ++j) {
            const float alpha = splat_alpha(sm.xy[j], sm.co[j], fpx, fpy);
            if (alpha < kAlphaMin) continue;
            const float test_T = __fmul_rn(T, __fsub_rn(1.0f, alpha));
            if (test_T < kTMin) {
                done = true;
                break;
            }
            const float w = __fmul_rn(alpha, T);
#pragma unroll
            for (int c = 0; c < DV; ++c) {
                const float4 v = sm.f[j][c];
                acc[c].x += w * v.x;
                acc[c].y += w * v.y;
                acc[c].z += w * v.z;
                acc[c].w += w * v.w;
            }
            T = test_T;
            ++count;
        }
    }
    if (inside) {
        const size_t p = (size_t)py * job.W + px;
#pragma unroll
        for (int c = 0; c < DV; ++c) job.Q[p * DV + c] = acc[c];
        job.T_final[p] = T;
        job.n_contrib[p] = count;
    }
}

template <int DQ>
__global__ void __launch_bounds__(kTilePixels) render_fwd_kernel(CamParams cam, const int2* __restrict__ ranges,
                                                                 const int32_t* __restrict__ pair_ids,
                                                                 const float2* __restrict__ xy,
                                                                 const float4* __restrict__ conic_opac,
                                                                 const float4* __restrict__ f, float4* __restrict__ Q,
                                                                 float* __restrict__ T_final,
                                                                 int32_t* __restrict__ n_contrib) {
    __shared__ FwdSmem<DQ> sm;
    const int tile = cam.tile_order ? cam.tile_order[blockIdx.x] : (int)blockIdx.x;
    const TileJob job{tile, cam.tiles_x, cam.W, cam.H, ranges, pair_ids, xy, conic_opac, f, Q, T_final, n_contrib,
                      nullptr, nullptr};
    render_fwd_tile<DQ>(job, sm);
}

// Next (frame, tile) of a batch from the global work list (frame in the top 12 bits), taken in
// list order by an atomic ticket; -1 when the list is exhausted.  Every thread returns the same
// item; the two barriers also keep the previous item's shared memory until every thread is done.
__device__ __forceinline__ int next_item(int* counter, const int32_t* order, int total) {
    __shared__ int s_item;
    if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
    __syncthreads();
    const int it = s_item;
    __syncthreads();
    return it < total ? order[it] : -1;
}

// Persistent render forward over every tile of every frame of a batch, longest lists first.
template <int DQ>
__global__ void __launch_bounds__(kTilePixels) render_fwd_batch_kernel(const __grid_constant__ BatchJobs jobs,
                                                                       const int32_t* __restrict__ order, int total,
                                                                       int* __restrict__ counter) {
    __shared__ FwdSmem<DQ> sm;
    for (int item = next_item(counter, order, total); item >= 0; item = next_item(counter, order, total)) {
        TileJob job = jobs.fr[item >> 20];
        job.tile = item & 0xFFFFF;
        render_fwd_tile<DQ>(job, sm);
    }
}

// Reduce-scatter of 32 per-lane channels over the warp: lane l ends with the warp-wide
// sum of channel l (31 shuffles instead of 32 x 5).
__device__ __forceinline__ float warp_reduce_scatter32(float (&v)[32], int lane) {
#pragma unroll
    for (int half = 16; half >= 1; half >>= 1) {
        const bool upper = (lane & half) != 0;
#pragma unroll
        for (int i = 0; i < half; ++i) {
            const float send = upper ? v[i] : v[i + half];
            const float keep = upper ? v[i + half] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, half);
        }
    }
    return v[0];
}

// Backward of the query blend, df_i = sum_p w_ip dQ_p, as one small GEMM per tile and batch on
// the tensor cores: the weights w_ip of a batch of kBwdBatch Gaussians are first recomputed front
// to back by the pixel threads (the forward's arithmetic, so the same contributions are taken: a
// pixel stops after its n_contrib-th one) into a shared-memory matrix W^T (Gaussians x pixels),
// each weight as two BF16 terms w = hi + lo (hi = bf16(w), lo = bf16(w - hi)); the tile's dQ
// rows are held the same way.  Then warp (m, h) takes Gaussians 16m..16m+15 and channel half h
// and sums over the tile's 256 pixels with mma.sync m16n8k16 (BF16 in, FP32 accumulate) as
// W_hi dQ_hi + W_hi dQ_lo + W_lo dQ_hi (each product within 2^-16 of the FP32 one), and each
// non-zero (Gaussian, channel) sum goes to df with one atomic per tile.  A per-tile contraction
// of 64 x 256 x d does not amortise TMEM allocation and completion waits; the warp-level MMA
// runs in the registers of the warps that computed the weights.
constexpr int kBwdBatch = 64;
constexpr int kWtStride = kTilePixels + 8;  // bf16 per W^T row (528 B: ldmatrix rows on distinct banks)

template <int DQ>
constexpr int dq_stride() {
    return DQ + 8;  // bf16 per dQ row (16 B of padding: ldmatrix rows on distinct banks)
}

template <int DQ>
constexpr size_t render_bwd_smem() {
    // W^T hi / lo, dQ hi / lo, staged splats
    return 2 * sizeof(__nv_bfloat16) * (size_t)kBwdBatch * kWtStride +
           2 * sizeof(__nv_bfloat16) * (size_t)kTilePixels * dq_stride<DQ>() +
           (sizeof(float4) + sizeof(float2) + sizeof(int)) * kBwdBatch;
}

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t (&r)[4]) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(addr));
}
__device__ __forceinline__ void ldsm_x2_trans(uint32_t addr, uint32_t (&r)[2]) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0, %1}, [%2];" : "=r"(r[0]), "=r"(r[1]) : "r"(addr));
}
// c += a b, m16n8k16, BF16 operands, FP32 accumulators
__device__ __forceinline__ void mma_bf16_16816(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Backward of one tile (256 threads); smem is the dynamic shared memory of render_bwd_smem.
template <int DQ>
__device__ __forceinline__ void render_bwd_tile(const TileJob& job, float4* smem) {
    constexpr int DV = DQ / 4;
    constexpr int DQS = dq_stride<DQ>();
    constexpr int NT = DQ / 16;  // n-tiles of 8 channels per warp (a warp covers DQ / 2 channels)
    using bf16 = __nv_bfloat16;
    bf16* wt_hi = reinterpret_cast<bf16*>(smem);      // [Gaussian][pixel]
    bf16* wt_lo = wt_hi + (size_t)kBwdBatch * kWtStride;
    bf16* dq_hi = wt_lo + (size_t)kBwdBatch * kWtStride;  // [pixel][channel]
    bf16* dq_lo = dq_hi + (size_t)kTilePixels * DQS;
    float4* s_co = reinterpret_cast<float4*>(dq_lo + (size_t)kTilePixels * DQS);
    float2* s_xy = reinterpret_cast<float2*>(s_co + kBwdBatch);
    int* s_id = reinterpret_cast<int*>(s_xy + kBwdBatch);
    static_assert(((size_t)kBwdBatch * kWtStride * 2 * 2 + (size_t)kTilePixels * DQS * 2 * 2) % 16 == 0,
                  "staged splats stay 16-byte aligned");

    const int tile = job.tile;
    const int tx = tile % job.tiles_x, ty = tile / job.tiles_x;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int px = tx * kTile + (t % kTile), py = ty * kTile + (t / kTile);
    const bool inside = px < job.W && py < job.H;
    const float fpx = (float)px, fpy = (float)py;
    const int2 range = job.ranges[tile];
    int remaining = 0;
    {
        // this pixel's dQ row as hi / lo terms
        float4 g[DV];
        if (inside) {
            const size_t p = (size_t)py * job.W + px;
#pragma unroll
            for (int c = 0; c < DV; ++c) g[c] = job.dQ[p * DV + c];
            remaining = job.n_contrib[p];
        } else {
#pragma unroll
            for (int c = 0; c < DV; ++c) g[c] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int c = 0; c < DV; c += 2) {
            uint32_t h[4], l[4];
            const float4 a = g[c], b = c + 1 < DV ? g[c + 1] : make_float4(0.f, 0.f, 0.f, 0.f);
            tc_split(a.x, a.y, h[0], l[0]);
            tc_split(a.z, a.w, h[1], l[1]);
            tc_split(b.x, b.y, h[2], l[2]);
            tc_split(b.z, b.w, h[3], l[3]);
            if (c + 1 < DV) {
                *reinterpret_cast<uint4*>(dq_hi + (size_t)t * DQS + 4 * c) = make_uint4(h[0], h[1], h[2], h[3]);
                *reinterpret_cast<uint4*>(dq_lo + (size_t)t * DQS + 4 * c) = make_uint4(l[0], l[1], l[2], l[3]);
            } else {
                *reinterpret_cast<uint2*>(dq_hi + (size_t)t * DQS + 4 * c) = make_uint2(h[0], h[1]);
                *reinterpret_cast<uint2*>(dq_lo + (size_t)t * DQS + 4 * c) = make_uint2(l[0], l[1]);
            }
        }
    }
    const int mt = warp & 3, nh = warp >> 2;  // GEMM role: Gaussian rows 16 mt.., channel half nh
    float T = 1.0f;
    bool done = remaining == 0;
    for (int start = range.x; start < range.y; start += kBwdBatch) {
        if (__syncthreads_count(done) == kTilePixels) break;
        const int cnt = min(kBwdBatch, range.y - start);
        if (t < cnt) {
            const int gid = job.pair_ids[start + t];
            s_xy[t] = job.xy[gid];
            s_co[t] = stage_splat(job.conic_opac[gid]);
            s_id[t] = gid;
        }
        __syncthreads();
        // 1. this pixel's weights for the batch (identical arithmetic to the forward pass); the
        //    columns of the Gaussians past the batch are zero
        for (int j = 0; j < kBwdBatch; ++j) {
            float w = 0.0f;
            if (j < cnt && !done) {
                const float alpha = splat_alpha(s_xy[j], s_co[j], fpx, fpy);
                if (alpha >= kAlphaMin) {
                    w = __fmul_rn(alpha, T);
                    T = __fmul_rn(T, __fsub_rn(1.0f, alpha));
                    if (--remaining == 0) done = true;
                }
            }
            const __nv_bfloat16 wh = __float2bfloat16_rn(w);
            wt_hi[(size_t)j * kWtStride + t] = wh;
            wt_lo[(size_t)j * kWtStride + t] = __float2bfloat16_rn(w - __bfloat162float(wh));
        }
        __syncthreads();
        // 2. warp (mt, nh): df rows 16 mt.. (Gaussians) x channels nh DQ/2.. over the 256 pixels
        if (16 * mt < cnt) {
            float acc[NT][4];
#pragma unroll
            for (int n = 0; n < NT; ++n) acc[n][0] = acc[n][1] = acc[n][2] = acc[n][3] = 0.f;
            const int ar = 16 * mt + (lane & 15), ac = (lane >> 4) * 8;  // A fragment row / column
            const int br = lane & 15;                                     // B fragment row (pixel)
#pragma unroll 4
            for (int kt = 0; kt < kTilePixels / 16; ++kt) {
                uint32_t ah[4], al[4];
                ldsm_x4(smem_addr(wt_hi + (size_t)ar * kWtStride + 16 * kt + ac), ah);
                ldsm_x4(smem_addr(wt_lo + (size_t)ar * kWtStride + 16 * kt + ac), al);
#pragma unroll
                for (int n = 0; n < NT; ++n) {
                    const int col = nh * (DQ / 2) + 8 * n;
                    uint32_t bh[2], bl[2];
                    ldsm_x2_trans(smem_addr(dq_hi + (size_t)(16 * kt + br) * DQS + col), bh);
                    ldsm_x2_trans(smem_addr(dq_lo + (size_t)(16 * kt + br) * DQS + col), bl);
                    mma_bf16_16816(acc[n], ah, bh);
                    mma_bf16_16816(acc[n], ah, bl);
                    mma_bf16_16816(acc[n], al, bh);
                }
            }
            // 3. one atomic per non-zero (Gaussian, channel) of the tile
            const int g0 = 16 * mt + (lane >> 2);
#pragma unroll
            for (int n = 0; n < NT; ++n) {
                const int c = nh * (DQ / 2) + 8 * n + 2 * (lane & 3);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int g = g0 + 8 * h;
                    if (g >= cnt) continue;
                    float* dst = job.df + (size_t)s_id[g] * DQ + c;
                    if (acc[n][2 * h] != 0.0f) atomicAdd(dst, acc[n][2 * h]);
                    if (acc[n][2 * h + 1] != 0.0f) atomicAdd(dst + 1, acc[n][2 * h + 1]);
                }
            }
        }
        // the next batch's staging and W writes come after the barrier at the loop head
    }
}

template <int DQ>
__global__ void __launch_bounds__(kTilePixels) render_bwd_kernel(CamParams cam, const int2* __restrict__ ranges,
                                                                 const int32_t* __restrict__ pair_ids,
                                                                 const float2* __restrict__ xy,
                                                                 const float4* __restrict__ conic_opac,
                                                                 const int32_t* __restrict__ n_contrib,
                                                                 const float4* __restrict__ dQ, float* __restrict__ df) {
    extern __shared__ float4 smem_f4[];
    const int tile = cam.tile_order ? cam.tile_order[blockIdx.x] : (int)blockIdx.x;
    const TileJob job{tile, cam.tiles_x, cam.W, cam.H, ranges, pair_ids, xy, conic_opac, nullptr, nullptr, nullptr,
                      const_cast<int32_t*>(n_contrib), dQ, df};
    render_bwd_tile<DQ>(job, smem_f4);
}

// Persistent render backward over every tile of every frame of a batch, longest lists first
// (frames that share their queries add into the same df).
template <int DQ>
__global__ void __launch_bounds__(kTilePixels) render_bwd_batch_kernel(const __grid_constant__ BatchJobs jobs,
                                                                       const int32_t* __restrict__ order, int total,
                                                                       int* __restrict__ counter) {
    extern __shared__ float4 smem_f4[];
    for (int item = next_item(counter, order, total); item >= 0; item = next_item(counter, order, total)) {
        TileJob job = jobs.fr[item >> 20];
        job.tile = item & 0xFFFFF;
        render_bwd_tile<DQ>(job, smem_f4);
    }
}

// ---- the full Stage I render: queries, colours and depth blended together ---------------
//
// The colour c_i (view-independent) and the camera depth z_i of every Gaussian are blended with
// the same weights as its query (Eq. alpha_blending; the depth image uses the same blend).  The
// backward adds the gradients of the blend weights: with G = dL/dX the pixel's gradient over all
// blended channels X, and x_i the channels of contribution i,
//   dL/dalpha_i = T_i <G, x_i> - (<G, X> - P_i) / (1 - alpha_i),  P_i = sum_{k <= i} w_k <G, x_k>,
// so one running scalar per pixel replaces the back-to-front pass.  alpha = min(0.99, o e^power)
// passes dL/dalpha to o (e^power) and to power (alpha) unless it is clamped, and power to the
// screen mean and the conic.

constexpr int kBatchFull = 128;  // Gaussians staged per round (f rows, colour + depth, geometry)

template <int DQ>
__global__ void __launch_bounds__(kTilePixels) render_fwd_full_kernel(
    CamParams cam, const int2* __restrict__ ranges, const int32_t* __restrict__ pair_ids,
    const float2* __restrict__ xy, const float4* __restrict__ conic_opac, const float4* __restrict__ f,
    const float* __restrict__ colours, const float* __restrict__ depth, float4* __restrict__ Q,
    float* __restrict__ C, float* __restrict__ Z, float* __restrict__ T_final, int32_t* __restrict__ n_contrib) {
    constexpr int DV = DQ / 4;
    __shared__ float2 s_xy[kBatchFull];
    __shared__ float4 s_co[kBatchFull];
    __shared__ float4 s_cz[kBatchFull];
    __shared__ float4 s_f[kBatchFull][DV];
    const int tile = cam.tile_order ? cam.tile_order[blockIdx.x] : (int)blockIdx.x;
    const int tx = tile % cam.tiles_x, ty = tile / cam.tiles_x;
    const int t = threadIdx.x;
    const int px = tx * kTile + (t % kTile), py = ty * kTile + (t / kTile);
    const bool inside = px < cam.W && py < cam.H;
    const float fpx = (float)px, fpy = (float)py;
    const int2 range = ranges[tile];
    float4 acc[DV];
#pragma unroll
    for (int k = 0; k < DV; ++k) acc[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    float4 acz = make_float4(0.f, 0.f, 0.f, 0.f);
    float T = 1.0f;
    int count = 0;
    bool done = !inside;
    for (int start = range.x; start < range.y; start += kBatchFull) {
        if (__syncthreads_count(done) == kTilePixels) break;
        const int k = start + t;
        if (t < kBatchFull && k < range.y) {
            const int g = pair_ids[k];
            s_xy[t] = xy[g];
            s_co[t] = stage_splat(conic_opac[g]);
            s_cz[t] = make_float4(colours[3 * g], colours[3 * g + 1], colours[3 * g + 2], depth[g]);
#pragma unroll
            for (int c = 0; c < DV; ++c) s_f[t][c] = f[(size_t)g * DV + c];
        }
        __syncthreads();
        const int cnt = min(kBatchFull, range.y - start);
        for (int j = 0; j < cnt && !done; ++j) {
            const float alpha = splat_alpha(s_xy[j], s_co[j], fpx, fpy);
            if (alpha < kAlphaMin) continue;
            const float test_T = __fmul_rn(T, __fsub_rn(1.0f, alpha));
            if (test_T < kTMin) {
                done = true;
                break;
            }
            const float w = __fmul_rn(alpha, T);
#pragma unroll
            for (int c = 0; c < DV; ++c) {
                const float4 v = s_f[j][c];
                acc[c].x += w * v.x;
                acc[c].y += w * v.y;
                acc[c].z += w * v.z;
                acc[c].w += w * v.w;
            }
            const float4 v = s_cz[j];
            acz.x += w * v.x;
            acz.y += w * v.y;
            acz.z += w * v.z;
            acz.w += w * v.w;
            T = test_T;
            ++count;
        }
    }
    if (inside) {
        const size_t p = (size_t)py * cam.W + px;
#pragma unroll
        for (int c = 0; c < DV; ++c) Q[p * DV + c] = acc[c];
        C[3 * p] = acz.x;
        C[3 * p + 1] = acz.y;
        C[3 * p + 2] = acz.z;
        Z[p] = acz.w;
        T_final[p] = T;
        n_contrib[p] = count;
    }
}

// Per-Gaussian gradients: df (N x DQ), dcol (N x 3) and dgeo (N x 8: d mean2d x, y, d conic
// a, b, c, d opacity, d depth channel, unused), accumulated with one atomic per warp and channel.
template <int DQ>
__global__ void __launch_bounds__(kTilePixels) render_bwd_full_kernel(
    CamParams cam, const int2* __restrict__ ranges, const int32_t* __restrict__ pair_ids,
    const float2* __restrict__ xy, const float4* __restrict__ conic_opac, const float4* __restrict__ f,
    const float* __restrict__ colours, const float* __restrict__ depth, const int32_t* __restrict__ n_contrib,
    const float4* __restrict__ Qf, const float* __restrict__ Cf, const float* __restrict__ Zf,
    const float4* __restrict__ dQ, const float* __restrict__ dC, const float* __restrict__ dZ,
    float* __restrict__ df, float* __restrict__ dcol, float* __restrict__ dgeo) {
    constexpr int DV = DQ / 4;
    constexpr int NG = DQ / 32 > 0 ? DQ / 32 : 1;
    __shared__ float2 s_xy[kBatchFull];
    __shared__ float4 s_co[kBatchFull];
    __shared__ float4 s_cz[kBatchFull];
    __shared__ float4 s_f[kBatchFull][DV];
    __shared__ int s_id[kBatchFull];
    const int tile = cam.tile_order ? cam.tile_order[blockIdx.x] : (int)blockIdx.x;
    const int tx = tile % cam.tiles_x, ty = tile / cam.tiles_x;
    const int t = threadIdx.x, lane = t & 31;
    const int px = tx * kTile + (t % kTile), py = ty * kTile + (t / kTile);
    const bool inside = px < cam.W && py < cam.H;
    const float fpx = (float)px, fpy = (float)py;
    const int2 range = ranges[tile];
    float g[DQ];
    float4 gcz = make_float4(0.f, 0.f, 0.f, 0.f);  // dL/dC (3), dL/dZ
    float GX = 0.f;
    int remaining = 0;
    if (inside) {
        const size_t p = (size_t)py * cam.W + px;
#pragma unroll
        for (int c = 0; c < DV; ++c) {
            const float4 v = dQ[p * DV + c], q = Qf[p * DV + c];
            g[4 * c] = v.x;
            g[4 * c + 1] = v.y;
            g[4 * c + 2] = v.z;
            g[4 * c + 3] = v.w;
            GX += v.x * q.x + v.y * q.y + v.z * q.z + v.w * q.w;
        }
        gcz = make_float4(dC[3 * p], dC[3 * p + 1], dC[3 * p + 2], dZ[p]);
        GX += gcz.x * Cf[3 * p] + gcz.y * Cf[3 * p + 1] + gcz.z * Cf[3 * p + 2] + gcz.w * Zf[p];
        remaining = n_contrib[p];
    } else {
#pragma unroll
        for (int c = 0; c < DQ; ++c) g[c] = 0.f;
    }
    float T = 1.0f, P = 0.0f;
    bool done = remaining == 0;
    for (int start = range.x; start < range.y; start += kBatchFull) {
        if (__syncthreads_count(done) == kTilePixels) break;
        const int k = start + t;
        if (t < kBatchFull && k < range.y) {
            const int gid = pair_ids[k];
            s_xy[t] = xy[gid];
            s_co[t] = stage_splat(conic_opac[gid]);
            s_cz[t] = make_float4(colours[3 * gid], colours[3 * gid + 1], colours[3 * gid + 2], depth[gid]);
#pragma unroll
            for (int c = 0; c < DV; ++c) s_f[t][c] = f[(size_t)gid * DV + c];
            s_id[t] = gid;
        }
        __syncthreads();
        const int cnt = min(kBatchFull, range.y - start);
        for (int j = 0; j < cnt; ++j) {
            float w = 0.0f;
            float geo[10] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            if (!done) {
                const float2 m = s_xy[j];
                const float4 q = s_co[j];
                const float dx = __fsub_rn(m.x, fpx), dy = __fsub_rn(m.y, fpy);
                const float power =
                    __fmaf_rn(dx, __fmaf_rn(q.x, dx, __fmul_rn(q.y, dy)), __fmul_rn(__fmul_rn(q.z, dy), dy));
                if (power <= 0.0f) {
                    const float raw = __fmul_rn(q.w, __expf(power));
                    const float alpha = fminf(kAlphaMax, raw);
                    if (alpha >= kAlphaMin) {
                        const float Tb = T;
                        w = __fmul_rn(alpha, T);
                        T = __fmul_rn(T, __fsub_rn(1.0f, alpha));
                        if (--remaining == 0) done = true;
                        // <G, x_j>
                        float gx = gcz.x * s_cz[j].x + gcz.y * s_cz[j].y + gcz.z * s_cz[j].z + gcz.w * s_cz[j].w;
#pragma unroll
                        for (int c = 0; c < DV; ++c) {
                            const float4 v = s_f[j][c];
                            gx += g[4 * c] * v.x + g[4 * c + 1] * v.y + g[4 * c + 2] * v.z + g[4 * c + 3] * v.w;
                        }
                        P += w * gx;
                        const float dalpha = Tb * gx - (GX - P) / (1.0f - alpha);
                        geo[0] = w * gcz.x;
                        geo[1] = w * gcz.y;
                        geo[2] = w * gcz.z;
                        geo[3] = w * gcz.w;
                        if (raw <= kAlphaMax) {
                            const float dpow = dalpha * raw;
                            const float a = -2.0f * q.x, b = -q.y, cc = -2.0f * q.z;
                            geo[4] = dpow * (-a * dx - b * dy);  // d mean2d x
                            geo[5] = dpow * (-b * dx - cc * dy);
                            geo[6] = dpow * (-0.5f * dx * dx);    // d conic a, b, c
                            geo[7] = dpow * (-dx * dy);
                            geo[8] = dpow * (-0.5f * dy * dy);
                            geo[9] = dalpha * (raw / q.w);         // d opacity
                        }
                    }
                }
            }
            if (__any_sync(0xffffffffu, w != 0.0f)) {
                const int gid = s_id[j];
#pragma unroll
                for (int grp = 0; grp < NG; ++grp) {
                    float v[32];
                    if (DQ >= 32) {
#pragma unroll
                        for (int c = 0; c < 32; ++c) v[c] = w * g[grp * 32 + c];
                    } else {
#pragma unroll
                        for (int c = 0; c < 32; ++c) v[c] = c < DQ ? w * g[c] : 0.0f;
                    }
                    const float s = warp_reduce_scatter32(v, lane);
                    if (lane < (DQ < 32 ? DQ : 32)) atomicAdd(&df[(size_t)gid * DQ + grp * 32 + lane], s);
                }
                float v[32];
#pragma unroll
                for (int c = 0; c < 32; ++c) v[c] = c < 10 ? geo[c] : 0.0f;
                const float s = warp_reduce_scatter32(v, lane);
                if (lane < 3) atomicAdd(&dcol[(size_t)gid * 3 + lane], s);
                else if (lane < 10) {
                    // lanes 3..9: depth channel, mean2d x, y, conic a, b, c, opacity
                    const int slot = lane == 3 ? 6 : lane - 4;
                    atomicAdd(&dgeo[(size_t)gid * 8 + slot], s);
                }
            }
        }
    }
}

template <int DQ>
latentam_status render_fwd_t(const CamParams& cam, const latentam_projected& proj, const latentam_bins& bins,
                             const float* f, float* Q, float* T_final, int32_t* n_contrib, cudaStream_t st) {
    const int tiles = cam.tiles_x * cam.tiles_y;
    render_fwd_kernel<DQ><<<tiles, kTilePixels, 0, st>>>(
        cam, reinterpret_cast<const int2*>(bins.tile_ranges), bins.pair_ids, reinterpret_cast<const float2*>(proj.xy),
        reinterpret_cast<const float4*>(proj.conic_opacity), reinterpret_cast<const float4*>(f),
        reinterpret_cast<float4*>(Q), T_final, n_contrib);
    LAT_CHECK_LAUNCH("render_fwd_kernel");
    return LATENTAM_OK;
}

template <int DQ>
latentam_status render_bwd_t(const CamParams& cam, const latentam_projected& proj, const latentam_bins& bins,
                             const int32_t* n_contrib, const float* dQ, float* df, int32_t n, cudaStream_t st,
                             bool accumulate) {
    if (!accumulate) {
        cudaError_t e = cudaMemsetAsync(df, 0, sizeof(float) * (size_t)n * DQ, st);
        if (e != cudaSuccess) return cuda_error(e, "memset df");
    }
    const int tiles = cam.tiles_x * cam.tiles_y;
    constexpr size_t smem = render_bwd_smem<DQ>();
    static_assert(smem <= 227 * 1024, "render backward tile does not fit in shared memory");
    auto kern = render_bwd_kernel<DQ>;
    static unsigned long long attr_set = 0;  // per instantiation and device
    int dev = 0;
    cudaGetDevice(&dev);
    if (!(attr_set & (1ull << (dev & 63)))) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return cuda_error(e, "render backward smem attribute");
        attr_set |= 1ull << (dev & 63);
    }
    kern<<<tiles, kTilePixels, smem, st>>>(
        cam, reinterpret_cast<const int2*>(bins.tile_ranges), bins.pair_ids, reinterpret_cast<const float2*>(proj.xy),
        reinterpret_cast<const float4*>(proj.conic_opacity), n_contrib, reinterpret_cast<const float4*>(dQ), df);
    LAT_CHECK_LAUNCH("render_bwd_kernel");
    return LATENTAM_OK;
}

// Longest tiles first: class b holds the tiles whose list length has its highest set bit at b
// (empty tiles last); within a class the order is that of the atomics (it only schedules).
__global__ void __launch_bounds__(1024) tile_order_kernel(const int2* __restrict__ ranges, int tiles,
                                                          int32_t* __restrict__ order) {
    __shared__ int s_cnt[33], s_pos[33];
    const int t = threadIdx.x;
    if (t < 33) s_cnt[t] = 0;
    __syncthreads();
    auto cls = [&](int i) {
        const int2 r = ranges[i];
        const int len = r.y - r.x;
        return len > 0 ? 32 - __clz(len) : 0;  // 1..31, 0 for an empty tile
    };
    for (int i = t; i < tiles; i += blockDim.x) atomicAdd(&s_cnt[cls(i)], 1);
    __syncthreads();
    if (t == 0) {
        int run = 0;
        for (int c = 32; c >= 0; --c) {
            s_pos[c] = run;
            run += s_cnt[c];
        }
    }
    __syncthreads();
    for (int i = t; i < tiles; i += blockDim.x) order[atomicAdd(&s_pos[cls(i)], 1)] = i;
}

// Longest tiles first over every frame of a batch (the same length classes as
// tile_order_kernel); entries are (frame << 20) | tile.
__global__ void __launch_bounds__(1024) batch_order_kernel(const __grid_constant__ BatchJobs jobs,
                                                           int32_t* __restrict__ order) {
    __shared__ int s_cnt[33], s_pos[33];
    const int t = threadIdx.x;
    if (t < 33) s_cnt[t] = 0;
    __syncthreads();
    auto cls = [&](const TileJob& fr, int i) {
        const int2 r = fr.ranges[i];
        const int len = r.y - r.x;
        return len > 0 ? 32 - __clz(len) : 0;
    };
    for (int k = 0; k < jobs.n; ++k) {
        const TileJob& fr = jobs.fr[k];
        const int tiles = fr.tiles_x * ((fr.H + kTile - 1) / kTile);
        for (int i = t; i < tiles; i += blockDim.x) atomicAdd(&s_cnt[cls(fr, i)], 1);
    }
    __syncthreads();
    if (t == 0) {
        int run = 0;
        for (int c = 32; c >= 0; --c) {
            s_pos[c] = run;
            run += s_cnt[c];
        }
    }
    __syncthreads();
    for (int k = 0; k < jobs.n; ++k) {
        const TileJob& fr = jobs.fr[k];
        const int tiles = fr.tiles_x * ((fr.H + kTile - 1) / kTile);
        for (int i = t; i < tiles; i += blockDim.x) order[atomicAdd(&s_pos[cls(fr, i)], 1)] = (k << 20) | i;
    }
}

// CTAs of a persistent batch kernel: as many as can be resident at once, at most `total`.
template <class Kernel>
int persistent_grid(Kernel kern, size_t smem, int total) {
    static int per_sm[64] = {0};
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) sms = 1;
    int& b = per_sm[dev & 63];
    if (b == 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, kTilePixels, smem) != cudaSuccess || b < 1) b = 1;
        (void)cudaGetLastError();
    }
    return std::max(1, std::min(total, b * sms));
}

template <int DQ>
latentam_status render_fwd_batch_t(const BatchJobs& jobs, const int32_t* order, int total, int* counter,
                                   cudaStream_t st) {
    auto kern = render_fwd_batch_kernel<DQ>;
    kern<<<persistent_grid(kern, 0, total), kTilePixels, 0, st>>>(jobs, order, total, counter);
    LAT_CHECK_LAUNCH("render_fwd_batch_kernel");
    return LATENTAM_OK;
}

template <int DQ>
latentam_status render_bwd_batch_t(const BatchJobs& jobs, const int32_t* order, int total, int* counter,
                                   cudaStream_t st) {
    constexpr size_t smem = render_bwd_smem<DQ>();
    auto kern = render_bwd_batch_kernel<DQ>;
    static unsigned long long attr_set = 0;  // per instantiation and device
    int dev = 0;
    cudaGetDevice(&dev);
    if (!(attr_set & (1ull << (dev & 63)))) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return cuda_error(e, "batched render backward smem attribute");
        attr_set |= 1ull << (dev & 63);
    }
    kern<<<persistent_grid(kern, smem, total), kTilePixels, smem, st>>>(jobs, order, total, counter);
    LAT_CHECK_LAUNCH("render_bwd_batch_kernel");
    return LATENTAM_OK;
}

}  // namespace

latentam_status launch_batch_order(const BatchJobs& jobs, int32_t* order, cudaStream_t st) {
    batch_order_kernel<<<1, 1024, 0, st>>>(jobs, order);
    LAT_CHECK_LAUNCH("batch_order_kernel");
    return LATENTAM_OK;
}

latentam_status launch_render_fwd_batch(const BatchJobs& jobs, int d, const int32_t* order, int total, int* counter,
                                        cudaStream_t st) {
    if (total <= 0) return LATENTAM_OK;
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int), st);
    if (e != cudaSuccess) return cuda_error(e, "reset the render work ticket");
    switch (d) {
        case 16: return render_fwd_batch_t<16>(jobs, order, total, counter, st);
        case 32: return render_fwd_batch_t<32>(jobs, order, total, counter, st);
        case 64: return render_fwd_batch_t<64>(jobs, order, total, counter, st);
        default: set_error("query dimension d=%d not in {16, 32, 64}", d); return LATENTAM_ERR_UNSUPPORTED_SHAPE;
    }
}

latentam_status launch_render_bwd_batch(const BatchJobs& jobs, int d, const int32_t* order, int total, int* counter,
                                        cudaStream_t st) {
    if (total <= 0) return LATENTAM_OK;
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int), st);
    if (e != cudaSuccess) return cuda_error(e, "reset the render work ticket");
    switch (d) {
        case 16: return render_bwd_batch_t<16>(jobs, order, total, counter, st);
        case 32: return render_bwd_batch_t<32>(jobs, order, total, counter, st);
        case 64: return render_bwd_batch_t<64>(jobs, order, total, counter, st);
        default: set_error("query dimension d=%d not in {16, 32, 64}", d); return LATENTAM_ERR_UNSUPPORTED_SHAPE;
    }
}

latentam_status launch_tile_order(const CamParams& cam, const latentam_bins& bins, int32_t* order, cudaStream_t st) {
    const int tiles = cam.tiles_x * cam.tiles_y;
    tile_order_kernel<<<1, 1024, 0, st>>>(reinterpret_cast<const int2*>(bins.tile_ranges), tiles, order);
    LAT_CHECK_LAUNCH("tile_order_kernel");
    return LATENTAM_OK;
}

latentam_status launch_render_fwd(const CamParams& cam, const latentam_projected& proj, const latentam_bins& bins,
                                  const float* f, int d, float* Q, float* T_final, int32_t* n_contrib,
                                  cudaStream_t st) {
    switch (d) {
        case 16: return render_fwd_t<16>(cam, proj, bins, f, Q, T_final, n_contrib, st);
        case 32: return render_fwd_t<32>(cam, proj, bins, f, Q, T_final, n_contrib, st);
        case 64: return render_fwd_t<64>(cam, proj, bins, f, Q, T_final, n_contrib, st);
        default: set_error("query dimension d=%d not in {16, 32, 64}", d); return LATENTAM_ERR_UNSUPPORTED_SHAPE;
    }
}

latentam_status launch_render_full(const CamParams& cam, const latentam_projected& proj, const latentam_bins& bins,
                                   const float* f, int d, const float* colours, float* Q, float* C, float* Z,
                                   float* T_final, int32_t* n_contrib, cudaStream_t st) {
    const int tiles = cam.tiles_x * cam.tiles_y;
    auto args = [&](auto kernel) {
        kernel<<<tiles, kTilePixels, 0, st>>>(cam, reinterpret_cast<const int2*>(bins.tile_ranges), bins.pair_ids,
                                              reinterpret_cast<const float2*>(proj.xy),
                                              reinterpret_cast<const float4*>(proj.conic_opacity),
                                              reinterpret_cast<const float4*>(f), colours, proj.depth,
                                              reinterpret_cast<float4*>(Q), C, Z, T_final, n_contrib);
    };
    switch (d) {
        case 16: args(render_fwd_full_kernel<16>); break;
        case 32: args(render_fwd_full_kernel<32>); break;
        case 64: args(render_fwd_full_kernel<64>); break;
        default: set_error("query dimension d=%d not in {16, 32, 64}", d); return LATENTAM_ERR_UNSUPPORTED_SHAPE;
    }
    LAT_CHECK_LAUNCH("render_fwd_full_kernel");
    return LATENTAM_OK;
}

latentam_status launch_render_bwd_full(const CamParams& cam, const latentam_projected& proj,
                                       const latentam_bins& bins, const float* f, int d, const float* colours,
                                       const int32_t* n_contrib, const float* Q, const float* C, const float* Z,
                                       const float* dQ, const float* dC, const float* dZ, float* df, float* dcol,
                                       float* dgeo, int32_t n, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(df, 0, sizeof(float) * (size_t)n * d, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(dcol, 0, sizeof(float) * (size_t)n * 3, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(dgeo, 0, sizeof(float) * (size_t)n * 8, st);
    if (e != cudaSuccess) return cuda_error(e, "memset full gradients");
    const int tiles = cam.tiles_x * cam.tiles_y;
    auto args = [&](auto kernel) {
        kernel<<<tiles, kTilePixels, 0, st>>>(
            cam, reinterpret_cast<const int2*>(bins.tile_ranges), bins.pair_ids, reinterpret_cast<const float2*>(proj.xy),
            reinterpret_cast<const float4*>(proj.conic_opacity), reinterpret_cast<const float4*>(f), colours, proj.depth,
            n_contrib, reinterpret_cast<const float4*>(Q), C, Z, reinterpret_cast<const float4*>(dQ), dC, dZ, df, dcol,
            dgeo);
    };
    switch (d) {
        case 16: args(render_bwd_full_kernel<16>); break;
        case 32: args(render_bwd_full_kernel<32>); break;
        case 64: args(render_bwd_full_kernel<64>); break;
        default: set_error("query dimension d=%d not in {16, 32, 64}", d); return LATENTAM_ERR_UNSUPPORTED_SHAPE;
    }
    LAT_CHECK_LAUNCH("render_bwd_full_kernel");
    return LATENTAM_OK;
}

latentam_status launch_render_bwd(const CamParams& cam, const latentam_projected& proj, const latentam_bins& bins,
                                  const int32_t* n_contrib, const float* dQ, int d, float* df, int32_t n,
                                  cudaStream_t st, bool accumulate) {
    switch (d) {
        case 16: return render_bwd_t<16>(cam, proj, bins, n_contrib, dQ, df, n, st, accumulate);
        case 32: return render_bwd_t<32>(cam, proj, bins, n_contrib, dQ, df, n, st, accumulate);
        case 64: return render_bwd_t<64>(cam, proj, bins, n_contrib, dQ, df, n, st, accumulate);
        default: set_error("query dimension d=%d not in {16, 32, 64}", d); return LATENTAM_ERR_UNSUPPORTED_SHAPE;
    }
}

}  // namespace lat
