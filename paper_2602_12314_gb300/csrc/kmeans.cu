// Streaming K-means update of the dictionary atoms (Algorithm 1, Eq. stream_kmeans_init,
// Sec. III-C): the new keyframe's embeddings are summarised into k micro-clusters by a local
// K-means, which are merged with the weighted global centres and re-clustered to the fixed
// dictionary size K.  Global centres keep their slots (row j stays row j); weight 0 marks an
// empty slot, and the empty slots take the heaviest micro-centres first.
//
// Local phase (n rows, k <= 32 centres): one warp per row finds the nearest centre against the
// centres staged in shared memory (squared distance as |c|^2 - 2 <x, c>, ties to the lower
// index); each block then sums its row range per cluster with every thread owning fixed
// columns of a per-row-group accumulator (no atomics), and the cluster means are formed by
// summing the blocks' partials in block order, so the result does not depend on scheduling.
// Global phase (at most K + k weighted points against K centres): the dot products of all
// points with all centres come from the FP32 tiled GEMM, one warp per point takes the argmin
// over the occupied slots, and one block per centre gathers its points' weighted sum in point
// order.
#include <algorithm>

#include "internal.cuh"

namespace lat {
namespace {

constexpr int kMaxMicro = 32;
constexpr int kAccumThreads = 256;

__device__ __forceinline__ float warp_allsum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ---- local phase ------------------------------------------------------------------------

// C[c] = F[init_idx[c]]; an index outside [0, n) starts its centre at the origin.
__global__ void local_init(const float* __restrict__ F, int64_t n, int D, const int32_t* __restrict__ init_idx,
                           float* __restrict__ C) {
    const int c = blockIdx.x;
    const int32_t r = init_idx[c];
    const bool ok = r >= 0 && (int64_t)r < n;
    for (int j = threadIdx.x; j < D; j += blockDim.x) C[(int64_t)c * D + j] = ok ? F[(int64_t)r * D + j] : 0.f;
}

// assign[r] = nearest of the k centres (-1 for an invalid row); warp per row.  Shared memory:
// the centres (k x D) and their squared norms.  D % 4 == 0, D <= 1024.
__global__ void __launch_bounds__(256) local_assign(const float* __restrict__ F, int64_t n, int D,
                                                    const uint8_t* __restrict__ valid, const float* __restrict__ C,
                                                    int k, int32_t* __restrict__ assign) {
    extern __shared__ __align__(16) float sm[];
    float* sC = sm;
    float* sN = sm + (size_t)k * D;
    const int D4 = D / 4;
    const float4* C4 = reinterpret_cast<const float4*>(C);
    float4* sC4 = reinterpret_cast<float4*>(sC);
    for (int i = threadIdx.x; i < k * D4; i += blockDim.x) sC4[i] = C4[i];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int c = warp; c < k; c += 8) {
        float s = 0.f;
        for (int j = lane; j < D; j += 32) s += sC[(size_t)c * D + j] * sC[(size_t)c * D + j];
        s = warp_allsum(s);
        if (lane == 0) sN[c] = s;
    }
    __syncthreads();
    const float4* F4 = reinterpret_cast<const float4*>(F);
    for (int64_t r = (int64_t)blockIdx.x * 8 + warp; r < n; r += (int64_t)gridDim.x * 8) {
        if (valid && !valid[r]) {
            if (lane == 0) assign[r] = -1;
            continue;
        }
        float4 x[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int q = lane + 32 * i;
            x[i] = q < D4 ? F4[r * D4 + q] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        float best = INFINITY;
        int bi = 0;
        for (int c = 0; c < k; ++c) {
            float s = 0.f;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int q = lane + 32 * i;
                if (q < D4) {
                    const float4 cc = sC4[(size_t)c * D4 + q];
                    s += x[i].x * cc.x + x[i].y * cc.y + x[i].z * cc.z + x[i].w * cc.w;
                }
            }
            s = warp_allsum(s);
            const float v = sN[c] - 2.0f * s;
            if (v < best) {
                best = v;
                bi = c;
            }
        }
        if (lane == 0) assign[r] = bi;
    }
}

// Per-block cluster sums of rows [b R, (b+1) R): G = 256 / (D/4) row groups, each with its
// own accumulator copy (k x D) in shared memory; thread t of group g owns columns
// 4 (t mod D/4) .. +3 and adds rows g, g+G, ... of the range in order.  The copies are added in
// group order into part[b] (k x D); pcnt[b] (k) counts the rows.
__global__ void __launch_bounds__(kAccumThreads) local_accum(const float* __restrict__ F, int64_t n, int D,
                                                             const int32_t* __restrict__ assign, int k, int64_t R,
                                                             float* __restrict__ part, float* __restrict__ pcnt) {
    extern __shared__ __align__(16) float acc[];  // G x k x D
    __shared__ float cnt[kMaxMicro];
    const int D4 = D / 4;
    const int G = kAccumThreads / D4;  // row groups; threads past G * D4 (D4 not dividing 256) idle
    const int t = threadIdx.x, g = t / D4, q = t % D4;
    for (int i = t; i < G * k * D; i += kAccumThreads) acc[i] = 0.f;
    if (t < k) cnt[t] = 0.f;
    __syncthreads();
    const int64_t r0 = (int64_t)blockIdx.x * R, r1 = min(n, r0 + R);
    const float4* F4 = reinterpret_cast<const float4*>(F);
    float4* a4 = reinterpret_cast<float4*>(acc) + (size_t)min(g, G - 1) * k * D4;
    constexpr int U = 4;
    for (int64_t rb = r0 + g; g < G && rb < r1; rb += (int64_t)G * U) {
        int cs[U];
        float4 v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t r = rb + (int64_t)u * G;
            cs[u] = r < r1 ? assign[r] : -1;
            v[u] = cs[u] >= 0 ? F4[r * D4 + q] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (cs[u] < 0) continue;
            float4& s = a4[(size_t)cs[u] * D4 + q];
            s.x += v[u].x, s.y += v[u].y, s.z += v[u].z, s.w += v[u].w;
        }
    }
    __syncthreads();
    if (t == 0) {  // row counts, in row order
        for (int64_t r = r0; r < r1; ++r) {
            const int c = assign[r];
            if (c >= 0) cnt[c] += 1.f;
        }
    }
    __syncthreads();
    for (int i = t; i < k * D; i += kAccumThreads) {
        float s = 0.f;
        for (int h = 0; h < G; ++h) s += acc[(size_t)h * k * D + i];
        part[(int64_t)blockIdx.x * k * D + i] = s;
    }
    if (t < k) pcnt[(int64_t)blockIdx.x * k + t] = cnt[t];
}

// C[c][j] = (sum over blocks, in order, of part[b][c][j]) / count_c, kept when the cluster is
// empty; W[c] = count_c.
__global__ void local_finish(const float* __restrict__ part, const float* __restrict__ pcnt, int nb, int k, int D,
                             float* __restrict__ C, float* __restrict__ W) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)k * D) return;
    const int c = (int)(i / D), j = (int)(i % D);
    float s = 0.f, m = 0.f;
    for (int b = 0; b < nb; ++b) {
        s += part[(int64_t)b * k * D + i];
        m += pcnt[(int64_t)b * k + c];
    }
    if (m > 0.f) C[i] = s / m;
    if (j == 0) W[c] = m;
}

// ---- global phase -----------------------------------------------------------------------

struct MergeBufs {
    int32_t* n_points;   // [0] = |P|
    int32_t* pt_src;     // K + k: slot j >= 0, or micro c as -1 - c
    float* pt_w;         // K + k
    int32_t* slot_fill;  // K: micro index copied into an empty slot, or -1
    int32_t* active;     // K: 1 = the slot competes in the re-clustering
};

// One block of 1024 threads: the point list, the fill of the empty slots and the active set.
__global__ void __launch_bounds__(1024) global_merge(const float* __restrict__ w, int K, const float* __restrict__ mW,
                                                     int k, MergeBufs b) {
    __shared__ int by_rank[kMaxMicro];
    __shared__ int live_before[kMaxMicro + 1];
    __shared__ int warp_tot[2][32];
    __shared__ int carry[2];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    if (t == 0) {
        int lv = 0;
        for (int c = 0; c < k; ++c) {
            live_before[c] = lv;
            lv += mW[c] > 0.f ? 1 : 0;
        }
        live_before[k] = lv;
        carry[0] = carry[1] = 0;
    }
    if (t < k && mW[t] > 0.f) {  // rank among the live micro-centres: heavier first, then lower index
        int r = 0;
        for (int c = 0; c < k; ++c)
            if (mW[c] > 0.f && (mW[c] > mW[t] || (mW[c] == mW[t] && c < t))) ++r;
        by_rank[r] = t;
    }
    __syncthreads();
    const int n_live = live_before[k];
    for (int base = 0; base < K; base += 1024) {
        const int j = base + t;
        const int used = (j < K && w[j] > 0.f) ? 1 : 0;
        const int empty = (j < K && !used) ? 1 : 0;
        int xu = used, xe = empty;
        for (int o = 1; o < 32; o <<= 1) {
            const int yu = __shfl_up_sync(0xffffffffu, xu, o), ye = __shfl_up_sync(0xffffffffu, xe, o);
            if (lane >= o) xu += yu, xe += ye;
        }
        if (lane == 31) warp_tot[0][warp] = xu, warp_tot[1][warp] = xe;
        __syncthreads();
        if (warp == 0) {
            int wu = warp_tot[0][lane], we = warp_tot[1][lane];
            for (int o = 1; o < 32; o <<= 1) {
                const int yu = __shfl_up_sync(0xffffffffu, wu, o), ye = __shfl_up_sync(0xffffffffu, we, o);
                if (lane >= o) wu += yu, we += ye;
            }
            warp_tot[0][lane] = wu, warp_tot[1][lane] = we;
        }
        __syncthreads();
        const int ub = carry[0] + (warp ? warp_tot[0][warp - 1] : 0) + xu - used;
        const int eb = carry[1] + (warp ? warp_tot[1][warp - 1] : 0) + xe - empty;
        if (j < K) {
            b.slot_fill[j] = -1;
            if (used) {
                b.pt_src[ub] = j;
                b.pt_w[ub] = w[j];
                b.active[j] = 1;
            } else if (eb < n_live) {
                b.slot_fill[j] = by_rank[eb];
                b.active[j] = 1;
            } else {
                b.active[j] = 0;
            }
        }
        __syncthreads();
        if (t == 1023) carry[0] = ub + used, carry[1] = eb + empty;
        __syncthreads();
    }
    const int U = carry[0];
    if (t < k && mW[t] > 0.f) {
        b.pt_src[U + live_before[t]] = -1 - t;
        b.pt_w[U + live_before[t]] = mW[t];
    }
    if (t == 0) b.n_points[0] = U + n_live;
}

// Pm[p] = the point's row (an occupied slot of C, or a micro-centre), p < |P|.
__global__ void global_points(const float* __restrict__ C, const float* __restrict__ mC, int D, MergeBufs b,
                              float* __restrict__ Pm) {
    const int p = blockIdx.x;
    if (p >= b.n_points[0]) return;
    const int s = b.pt_src[p];
    const float* src = s >= 0 ? C + (int64_t)s * D : mC + (int64_t)(-1 - s) * D;
    for (int j = threadIdx.x; j < D; j += blockDim.x) Pm[(int64_t)p * D + j] = src[j];
}

// The empty slots that take a micro-centre start there.
__global__ void global_fill(const float* __restrict__ mC, int D, MergeBufs b, float* __restrict__ C) {
    const int j = blockIdx.x;
    const int c = b.slot_fill[j];
    if (c < 0) return;
    for (int i = threadIdx.x; i < D; i += blockDim.x) C[(int64_t)j * D + i] = mC[(int64_t)c * D + i];
}

// nrm[c] = |C_c|^2; warp per centre.
__global__ void centre_norms(const float* __restrict__ C, int K, int D, float* __restrict__ nrm) {
    const int lane = threadIdx.x & 31;
    const int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (c >= K) return;
    float s = 0.f;
    for (int j = lane; j < D; j += 32) s += C[(int64_t)c * D + j] * C[(int64_t)c * D + j];
    s = warp_allsum(s);
    if (lane == 0) nrm[c] = s;
}

// pa[p] = argmin over active c of nrm[c] - 2 G[p][c] (ties to the lower index); warp per point.
__global__ void global_assign(const float* __restrict__ G, int64_t ldg, const float* __restrict__ nrm, int K,
                              MergeBufs b, int32_t* __restrict__ pa) {
    const int lane = threadIdx.x & 31;
    const int p = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (p >= b.n_points[0]) return;
    float best = INFINITY;
    int bi = 0x7fffffff;
    for (int c = lane; c < K; c += 32) {
        if (!b.active[c]) continue;
        const float v = nrm[c] - 2.0f * G[(int64_t)p * ldg + c];
        if (v < best) best = v, bi = c;  // c increases along the lane's list
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob < best || (ob == best && oi < bi)) best = ob, bi = oi;
    }
    if (lane == 0) pa[p] = bi;
}

// Block per centre: the weighted mean of its points (in point order) and their total weight;
// an active centre without points keeps its position with weight 0; inactive slots are left.
__global__ void __launch_bounds__(256) global_update(const float* __restrict__ Pm, int D, MergeBufs b,
                                                     const int32_t* __restrict__ pa, float* __restrict__ C,
                                                     float* __restrict__ W) {
    const int c = blockIdx.x;
    if (!b.active[c]) return;
    const int P = b.n_points[0];
    constexpr int kCols = 4;  // D <= 1024 = 4 x 256
    float acc[kCols] = {0.f, 0.f, 0.f, 0.f};
    float wsum = 0.f;
    for (int p = 0; p < P; ++p) {
        if (pa[p] != c) continue;
        const float wp = b.pt_w[p];
        wsum += wp;
#pragma unroll
        for (int u = 0; u < kCols; ++u) {
            const int j = threadIdx.x + 256 * u;
            if (j < D) acc[u] += wp * Pm[(int64_t)p * D + j];
        }
    }
    if (wsum > 0.f) {
#pragma unroll
        for (int u = 0; u < kCols; ++u) {
            const int j = threadIdx.x + 256 * u;
            if (j < D) C[(int64_t)c * D + j] = acc[u] / wsum;
        }
    }
    if (threadIdx.x == 0) W[c] = wsum;
}

}  // namespace

size_t kmeans_scratch_bytes(int64_t n, int D, int k, int K, int nb, bool need_mc, bool need_mw, bool need_assign) {
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t KP = (size_t)K + k, ldg = ((size_t)K + 3) & ~(size_t)3;
    size_t b = 0;
    if (need_mc) b += up(4 * (size_t)k * D);
    if (need_mw) b += up(4 * (size_t)k);
    if (need_assign) b += up(4 * (size_t)std::max<int64_t>(n, 1));
    b += up(4 * (size_t)nb * k * D) + up(4 * (size_t)nb * k);
    b += up(4) + up(4 * KP) * 3 + up(4 * (size_t)K) * 3;
    b += up(4 * KP * D) + up(4 * KP * ldg);
    return b;
}

latentam_status stream_kmeans(latentam_ctx* ctx, const KMeansArgs& a, cudaStream_t st) {
    const int k = a.k, K = a.K, D = a.D;
    const int64_t n = a.n;
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const int nb = (int)std::max<int64_t>(1, std::min<int64_t>((n + 63) / 64, 2 * (int64_t)ctx->num_sms));
    const int64_t R = (n + nb - 1) / nb;
    const size_t KP = (size_t)K + k, ldg = ((size_t)K + 3) & ~(size_t)3;
    char* base = static_cast<char*>(
        ws(ctx, WS_KMEANS, kmeans_scratch_bytes(n, D, k, K, nb, !a.micro_C, !a.micro_W, !a.micro_assign)));
    if (!base) return LATENTAM_ERR_OUT_OF_MEMORY;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        char* p = base + o;
        o += up(bytes);
        return p;
    };
    // the buffers whose sizes do not depend on n first: their addresses (and the global
    // phase's captured graph) then stay the same from one keyframe to the next
    float* mC = a.micro_C ? a.micro_C : reinterpret_cast<float*>(take(4 * (size_t)k * D));
    float* mW = a.micro_W ? a.micro_W : reinterpret_cast<float*>(take(4 * (size_t)k));
    MergeBufs mb;
    mb.n_points = reinterpret_cast<int32_t*>(take(4));
    mb.pt_src = reinterpret_cast<int32_t*>(take(4 * KP));
    mb.pt_w = reinterpret_cast<float*>(take(4 * KP));
    int32_t* pa = a.point_assign ? a.point_assign : reinterpret_cast<int32_t*>(take(4 * KP));
    mb.slot_fill = reinterpret_cast<int32_t*>(take(4 * (size_t)K));
    mb.active = reinterpret_cast<int32_t*>(take(4 * (size_t)K));
    float* nrm = reinterpret_cast<float*>(take(4 * (size_t)K));
    float* Pm = reinterpret_cast<float*>(take(4 * KP * D));
    float* G = reinterpret_cast<float*>(take(4 * KP * ldg));
    int32_t* asg = a.micro_assign ? a.micro_assign : reinterpret_cast<int32_t*>(take(4 * (size_t)std::max<int64_t>(n, 1)));
    float* part = reinterpret_cast<float*>(take(4 * (size_t)nb * k * D));
    float* pcnt = reinterpret_cast<float*>(take(4 * (size_t)nb * k));

    // Both phases are chains of small dependent launches with no host round trip: each replays
    // a captured CUDA graph once the same shapes and buffers recur (the global phase's shapes
    // are the dictionary's, the same for every keyframe; the local phase's depend on the
    // number of targets).
    const size_t sm_assign = 4 * ((size_t)k * D + k);
    const int G_rows = kAccumThreads / (D / 4);
    const size_t sm_accum = 4 * (size_t)G_rows * k * D;
    const int ga = (int)std::max<int64_t>(1, std::min<int64_t>((n + 7) / 8, 4 * (int64_t)ctx->num_sms));
    auto local = [&](cudaStream_t s) -> latentam_status {
        cudaFuncSetAttribute(local_assign, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_assign);
        cudaFuncSetAttribute(local_accum, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_accum);
        local_init<<<k, 256, 0, s>>>(a.F, n, D, a.init_idx, mC);
        LAT_CHECK_LAUNCH("kmeans local_init");
        for (int it = 0; it < a.iters_local; ++it) {
            if (n > 0) {
                local_assign<<<ga, 256, sm_assign, s>>>(a.F, n, D, a.valid, mC, k, asg);
                LAT_CHECK_LAUNCH("kmeans local_assign");
                local_accum<<<nb, kAccumThreads, sm_accum, s>>>(a.F, n, D, asg, k, R, part, pcnt);
                LAT_CHECK_LAUNCH("kmeans local_accum");
            } else {
                cudaError_t e = cudaMemsetAsync(pcnt, 0, 4 * (size_t)nb * k, s);
                if (e != cudaSuccess) return cuda_error(e, "clear kmeans counts");
                e = cudaMemsetAsync(part, 0, 4 * (size_t)nb * k * D, s);
                if (e != cudaSuccess) return cuda_error(e, "clear kmeans sums");
            }
            local_finish<<<(unsigned)(((int64_t)k * D + 255) / 256), 256, 0, s>>>(part, pcnt, nb, k, D, mC, mW);
            LAT_CHECK_LAUNCH("kmeans local_finish");
        }
        return LATENTAM_OK;
    };
    auto global = [&](cudaStream_t s) -> latentam_status {
        cudaError_t e = cudaMemsetAsync(Pm, 0, 4 * KP * D, s);
        if (e != cudaSuccess) return cuda_error(e, "clear kmeans points");
        e = cudaMemsetAsync(pa, 0xff, 4 * KP, s);  // -1 past the last point
        if (e != cudaSuccess) return cuda_error(e, "clear kmeans point assignment");
        global_merge<<<1, 1024, 0, s>>>(a.weights, K, mW, k, mb);
        LAT_CHECK_LAUNCH("kmeans global_merge");
        global_points<<<(unsigned)KP, 256, 0, s>>>(a.centres, mC, D, mb, Pm);
        LAT_CHECK_LAUNCH("kmeans global_points");
        global_fill<<<K, 256, 0, s>>>(mC, D, mb, a.centres);
        LAT_CHECK_LAUNCH("kmeans global_fill");
        for (int it = 0; it < a.iters_global; ++it) {
            centre_norms<<<(K + 7) / 8, 256, 0, s>>>(a.centres, K, D, nrm);
            LAT_CHECK_LAUNCH("kmeans centre_norms");
            LAT_TRY(sgemm_abt(Pm, (int64_t)KP, a.centres, K, D, G, (int64_t)ldg, 1.0f, s));
            global_assign<<<(unsigned)((KP + 7) / 8), 256, 0, s>>>(G, (int64_t)ldg, nrm, K, mb, pa);
            LAT_CHECK_LAUNCH("kmeans global_assign");
            global_update<<<K, 256, 0, s>>>(Pm, D, mb, pa, a.centres, a.weights);
            LAT_CHECK_LAUNCH("kmeans global_update");
        }
        return LATENTAM_OK;
    };
    const uint64_t lkey[] = {0x6b6d2d6c6f63616cull /* tag: local phase */, (uint64_t)n, (uint64_t)D, (uint64_t)k,
                             (uint64_t)a.iters_local, reinterpret_cast<uint64_t>(a.F),
                             reinterpret_cast<uint64_t>(a.valid), reinterpret_cast<uint64_t>(a.init_idx),
                             reinterpret_cast<uint64_t>(mC), reinterpret_cast<uint64_t>(mW),
                             reinterpret_cast<uint64_t>(asg), reinterpret_cast<uint64_t>(base),
                             reinterpret_cast<uint64_t>(st), ctx->ws_generation};
    LAT_TRY(cached_launch(ctx, lkey, (int)(sizeof(lkey) / sizeof(lkey[0])), st, local));
    const uint64_t gkey[] = {0x6b6d2d676c6f6262ull /* tag: global phase */, (uint64_t)D, (uint64_t)k, (uint64_t)K,
                             (uint64_t)a.iters_global, reinterpret_cast<uint64_t>(a.centres),
                             reinterpret_cast<uint64_t>(a.weights), reinterpret_cast<uint64_t>(mC),
                             reinterpret_cast<uint64_t>(mW), reinterpret_cast<uint64_t>(pa),
                             reinterpret_cast<uint64_t>(Pm), reinterpret_cast<uint64_t>(G),
                             reinterpret_cast<uint64_t>(base), reinterpret_cast<uint64_t>(st), ctx->ws_generation};
    LAT_TRY(cached_launch(ctx, gkey, (int)(sizeof(gkey) / sizeof(gkey[0])), st, global));
    return LATENTAM_OK;
}

}  // namespace lat
