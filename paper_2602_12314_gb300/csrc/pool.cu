// Mask pooling of the rendered queries: with SAM-based targets the rows of the decode are the
// n valid masks, not the pixels (Sec. III-B, Eq. render_query), and the query of mask m is the
// mean of the rendered per-pixel queries over its pixels.  Its backward hands dQm_m / |m| to
// every pixel of the mask (summed where masks overlap).
//
// Masks arrive as CSR lists (offsets[S+1], pixel indices).  Each mask's entry range is cut into
// chunks of kChunk entries; a per-keyframe plan holds the first chunk of every mask (an
// exclusive scan of the chunk counts) and the number of valid entries per mask.  The forward
// pools each chunk in one warp (rows of d floats read as float4, several rows per warp step,
// reduced by a fixed shuffle tree) and then sums each mask's chunk partials in chunk order, so
// the result does not depend on scheduling.  The backward scatters the scaled mask gradient
// into the zeroed per-pixel gradient with float4 atomic adds (one add per pixel and channel
// group when the masks do not overlap, which is then exact).
#include "internal.cuh"

namespace lat {
namespace {

constexpr int kChunk = 256;        // entries per chunk
constexpr int kWarpsPerBlock = 8;  // chunks (or masks) per 256-thread block

struct PlanDev {
    const int32_t* off;
    const int32_t* pix;
    int64_t E;
    int S;
    int64_t npix;
    const int32_t* chunk_start;
    const int32_t* count;
};

// Entry range of mask m: offsets clamped into [0, E] and made non-decreasing.
__device__ __forceinline__ void mask_span(const int32_t* off, int64_t E, int m, int64_t& s0, int64_t& s1) {
    s0 = min(max((int64_t)off[m], (int64_t)0), E);
    s1 = min(max((int64_t)off[m + 1], s0), E);
}

// The mask owning chunk c: the largest m with chunk_start[m] <= c (c < chunk_start[S]).
__device__ __forceinline__ int chunk_mask(const int32_t* cs, int S, int64_t c) {
    int lo = 0, hi = S - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (cs[mid] <= c) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ void chunk_range(const PlanDev& p, int m, int64_t c, int64_t& e0, int64_t& e1) {
    int64_t s0, s1;
    mask_span(p.off, p.E, m, s0, s1);
    e0 = s0 + (c - p.chunk_start[m]) * kChunk;
    e1 = min(e0 + kChunk, s1);
}

__device__ __forceinline__ bool valid_pixel(int32_t q, int64_t npix) { return q >= 0 && (int64_t)q < npix; }

__device__ __forceinline__ float4 add4(float4 a, float4 b) {
    return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}

__device__ __forceinline__ float4 shfl_xor4(float4 v, int o) {
    return make_float4(__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o),
                       __shfl_xor_sync(0xffffffffu, v.z, o), __shfl_xor_sync(0xffffffffu, v.w, o));
}

// chunk_start[m] = sum_{k < m} ceil(|span k| / kChunk), chunk_start[S] = total; one block.
__global__ void __launch_bounds__(1024) plan_scan(const int32_t* off, int64_t E, int S, int32_t* chunk_start) {
    __shared__ int warp_tot[32];
    __shared__ int carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < S; base += 1024) {
        const int m = base + (int)threadIdx.x;
        int v = 0;
        if (m < S) {
            int64_t s0, s1;
            mask_span(off, E, m, s0, s1);
            v = (int)((s1 - s0 + kChunk - 1) / kChunk);
        }
        int x = v;  // inclusive scan within the warp
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_tot[warp] = x;
        __syncthreads();
        if (warp == 0) {
            int w = warp_tot[lane];
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            warp_tot[lane] = w;
        }
        __syncthreads();
        const int before = carry + (warp ? warp_tot[warp - 1] : 0) + x - v;
        if (m < S) chunk_start[m] = before;
        __syncthreads();
        if (threadIdx.x == 1023) carry = before + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) chunk_start[S] = carry;
}

// count[m] += valid entries of each of its chunks (count zeroed before); warp per chunk.
__global__ void __launch_bounds__(256) plan_count(PlanDev p, int32_t* count) {
    const int lane = threadIdx.x & 31;
    const int64_t c = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    if (p.S <= 0 || c >= p.chunk_start[p.S]) return;
    const int m = chunk_mask(p.chunk_start, p.S, c);
    int64_t e0, e1;
    chunk_range(p, m, c, e0, e1);
    int k = 0;
    for (int64_t e = e0 + lane; e < e1; e += 32) k += valid_pixel(p.pix[e], p.npix) ? 1 : 0;
    k = __reduce_add_sync(0xffffffffu, (unsigned)k);
    if (lane == 0 && k) atomicAdd(count + m, k);
}

// part[c] = sum of the valid rows of chunk c; warp per chunk, D4 = d / 4 lanes per row.
template <int D4>
__global__ void __launch_bounds__(256) pool_partial(PlanDev p, const float4* __restrict__ Q, float4* __restrict__ part) {
    constexpr int R = 32 / D4;  // rows per warp step
    const int lane = threadIdx.x & 31, r = lane / D4, q = lane % D4;
    const int64_t c = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    if (p.S <= 0 || c >= p.chunk_start[p.S]) return;
    const int m = chunk_mask(p.chunk_start, p.S, c);
    int64_t e0, e1;
    chunk_range(p, m, c, e0, e1);
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 8
    for (int64_t e = e0 + r; e < e1; e += R) {
        const int32_t px = p.pix[e];
        if (valid_pixel(px, p.npix)) acc = add4(acc, Q[(int64_t)px * D4 + q]);
    }
#pragma unroll
    for (int o = D4; o < 32; o <<= 1) acc = add4(acc, shfl_xor4(acc, o));
    if (r == 0) part[c * D4 + q] = acc;
}

// Qm[m] = (sum of its chunk partials, in chunk order) / count[m]; zero for an empty mask.
template <int D4>
__global__ void __launch_bounds__(256) pool_finish(PlanDev p, const float4* __restrict__ part, float4* __restrict__ Qm) {
    constexpr int R = 32 / D4;
    const int lane = threadIdx.x & 31, r = lane / D4, q = lane % D4;
    const int m = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    if (m >= p.S) return;
    const int c0 = p.chunk_start[m], c1 = p.chunk_start[m + 1];
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int c = c0 + r; c < c1; c += R) acc = add4(acc, part[(int64_t)c * D4 + q]);
#pragma unroll
    for (int o = D4; o < 32; o <<= 1) acc = add4(acc, shfl_xor4(acc, o));
    if (r == 0) {
        const int n = p.count[m];
        float4 out = make_float4(0.f, 0.f, 0.f, 0.f);
        if (n > 0) {
            const float fn = (float)n;
            out = make_float4(acc.x / fn, acc.y / fn, acc.z / fn, acc.w / fn);
        }
        Qm[(int64_t)m * D4 + q] = out;
    }
}

// dQ[p] += dQm[m] / count[m] for every valid entry p of chunk c (dQ zeroed before).
template <int D4>
__global__ void __launch_bounds__(256) pool_scatter(PlanDev p, const float4* __restrict__ dQm, float4* __restrict__ dQ) {
    constexpr int R = 32 / D4;
    const int lane = threadIdx.x & 31, r = lane / D4, q = lane % D4;
    const int64_t c = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    if (p.S <= 0 || c >= p.chunk_start[p.S]) return;
    const int m = chunk_mask(p.chunk_start, p.S, c);
    const int n = p.count[m];
    if (n <= 0) return;
    int64_t e0, e1;
    chunk_range(p, m, c, e0, e1);
    const float fn = (float)n;
    const float4 g0 = dQm[(int64_t)m * D4 + q];
    const float4 g = make_float4(g0.x / fn, g0.y / fn, g0.z / fn, g0.w / fn);
#pragma unroll 8
    for (int64_t e = e0 + r; e < e1; e += R) {
        const int32_t px = p.pix[e];
        if (valid_pixel(px, p.npix)) atomicAdd(dQ + (int64_t)px * D4 + q, g);
    }
}

PlanDev dev_view(const MaskPlan& p) {
    return PlanDev{p.offsets, p.pixels, p.n_entries, p.S, p.npix, p.chunk_start, p.count};
}

int chunk_blocks(const MaskPlan& p) { return (int)((p.max_chunks + kWarpsPerBlock - 1) / kWarpsPerBlock); }

}  // namespace

int64_t mask_max_chunks(int32_t S, int64_t E) { return E / kChunk + S + 1; }

size_t mask_plan_bytes(int32_t S, int64_t E, int d) {
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    return up(sizeof(int32_t) * ((size_t)S + 1)) + up(sizeof(int32_t) * ((size_t)S + 1)) +
           up(sizeof(float) * (size_t)d * (size_t)mask_max_chunks(S, E));
}

void mask_plan_carve(void* base, const int32_t* offsets, const int32_t* pixels, int64_t E, int32_t S, int64_t npix,
                     int d, MaskPlan* p) {
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    char* b = static_cast<char*>(base);
    p->offsets = offsets;
    p->pixels = pixels;
    p->n_entries = E;
    p->S = S;
    p->npix = npix;
    p->max_chunks = mask_max_chunks(S, E);
    p->chunk_start = reinterpret_cast<int32_t*>(b);
    b += up(sizeof(int32_t) * ((size_t)S + 1));
    p->count = reinterpret_cast<int32_t*>(b);
    b += up(sizeof(int32_t) * ((size_t)S + 1));
    p->part = reinterpret_cast<float*>(b);
    (void)d;
}

latentam_status launch_mask_plan(const MaskPlan& p, cudaStream_t st) {
    if (p.S <= 0) return LATENTAM_OK;
    cudaError_t e = cudaMemsetAsync(p.count, 0, sizeof(int32_t) * (size_t)p.S, st);
    if (e != cudaSuccess) return cuda_error(e, "clear mask counts");
    plan_scan<<<1, 1024, 0, st>>>(p.offsets, p.n_entries, p.S, p.chunk_start);
    LAT_CHECK_LAUNCH("mask plan_scan");
    plan_count<<<chunk_blocks(p), 256, 0, st>>>(dev_view(p), p.count);
    LAT_CHECK_LAUNCH("mask plan_count");
    return LATENTAM_OK;
}

latentam_status launch_pool_fwd(const MaskPlan& p, const float* Q, int d, float* Qm, cudaStream_t st) {
    if (p.S <= 0) return LATENTAM_OK;
    const PlanDev v = dev_view(p);
    const float4* Q4 = reinterpret_cast<const float4*>(Q);
    float4* part = reinterpret_cast<float4*>(p.part);
    float4* out = reinterpret_cast<float4*>(Qm);
    const int gm = (p.S + kWarpsPerBlock - 1) / kWarpsPerBlock;
    switch (d) {
        case 16:
            pool_partial<4><<<chunk_blocks(p), 256, 0, st>>>(v, Q4, part);
            LAT_CHECK_LAUNCH("pool_partial");
            pool_finish<4><<<gm, 256, 0, st>>>(v, part, out);
            break;
        case 32:
            pool_partial<8><<<chunk_blocks(p), 256, 0, st>>>(v, Q4, part);
            LAT_CHECK_LAUNCH("pool_partial");
            pool_finish<8><<<gm, 256, 0, st>>>(v, part, out);
            break;
        case 64:
            pool_partial<16><<<chunk_blocks(p), 256, 0, st>>>(v, Q4, part);
            LAT_CHECK_LAUNCH("pool_partial");
            pool_finish<16><<<gm, 256, 0, st>>>(v, part, out);
            break;
        default:
            set_error("mask pooling: d=%d not in {16, 32, 64}", d);
            return LATENTAM_ERR_UNSUPPORTED_SHAPE;
    }
    LAT_CHECK_LAUNCH("pool_finish");
    return LATENTAM_OK;
}

latentam_status launch_pool_bwd(const MaskPlan& p, const float* dQm, int d, float* dQ, cudaStream_t st) {
    if (p.npix > 0) {
        cudaError_t e = cudaMemsetAsync(dQ, 0, sizeof(float) * (size_t)p.npix * d, st);
        if (e != cudaSuccess) return cuda_error(e, "clear dQ");
    }
    if (p.S <= 0) return LATENTAM_OK;
    const PlanDev v = dev_view(p);
    const float4* g = reinterpret_cast<const float4*>(dQm);
    float4* out = reinterpret_cast<float4*>(dQ);
    switch (d) {
        case 16: pool_scatter<4><<<chunk_blocks(p), 256, 0, st>>>(v, g, out); break;
        case 32: pool_scatter<8><<<chunk_blocks(p), 256, 0, st>>>(v, g, out); break;
        case 64: pool_scatter<16><<<chunk_blocks(p), 256, 0, st>>>(v, g, out); break;
        default:
            set_error("mask pooling: d=%d not in {16, 32, 64}", d);
            return LATENTAM_ERR_UNSUPPORTED_SHAPE;
    }
    LAT_CHECK_LAUNCH("pool_scatter");
    return LATENTAM_OK;
}

}  // namespace lat
