// Tile binning and sorting of the splats (the depth-ordered lists that Eq. alpha_blending
// walks, Sec. III-A):
//   0. exclusive scan of tiles-touched -> pair offsets and the pair count P (the one host
//      round trip)
//   1. emission of one (tile, Gaussian) pair per covered tile, Gaussians in index order
//   2. stable radix sort of the pairs on the ceil(log2(tiles)) tile bits only
//   3. per-tile [start, end) ranges
//   4. each tile's list sorted by (binary32 depth key, index) in shared memory
// Sorting each short list on its own replaces a global depth sort of the visible Gaussians;
// each radix pass is one launch (decoupled look-back across blocks) after one launch that
// counts the digits of every pass.
#include <algorithm>

#include "internal.cuh"

namespace lat {
namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;  // 4096

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

// Exclusive scan of one 4096-item tile per block; block totals to sums[blockIdx].
__global__ void __launch_bounds__(kScanThreads) scan_tiles(const uint32_t* __restrict__ in, uint32_t* __restrict__ out,
                                                           uint32_t* __restrict__ sums, int64_t n) {
    __shared__ uint32_t warp_tot[32];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)t * kScanItems;
    uint32_t v[kScanItems];
    uint32_t tsum = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = (base + k < n) ? in[base + k] : 0u;
        tsum += v[k];
    }
    const uint32_t incl = warp_incl_scan(tsum, lane);
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = warp_tot[lane];
        uint32_t wi = warp_incl_scan(w, lane);
        warp_tot[lane] = wi - w;
        if (lane == 31 && sums) sums[blockIdx.x] = wi;
    }
    __syncthreads();
    uint32_t run = warp_tot[warp] + incl - tsum;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < n) out[base + k] = run;
        run += v[k];
    }
}

// In-place exclusive scan of up to 4096 block sums by a single block; total to *total.
__global__ void __launch_bounds__(kScanThreads) scan_sums(uint32_t* __restrict__ sums, int n, uint32_t* __restrict__ total) {
    __shared__ uint32_t warp_tot[32];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    uint32_t v[kScanItems];
    uint32_t tsum = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const int i = t * kScanItems + k;
        v[k] = i < n ? sums[i] : 0u;
        tsum += v[k];
    }
    const uint32_t incl = warp_incl_scan(tsum, lane);
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = warp_tot[lane];
        uint32_t wi = warp_incl_scan(w, lane);
        warp_tot[lane] = wi - w;
        if (lane == 31 && total) *total = wi;
    }
    __syncthreads();
    uint32_t run = warp_tot[warp] + incl - tsum;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const int i = t * kScanItems + k;
        if (i < n) sums[i] = run;
        run += v[k];
    }
}

__global__ void __launch_bounds__(kScanThreads) scan_add(uint32_t* __restrict__ out, const uint32_t* __restrict__ sums, int64_t n) {
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    const uint32_t add = sums[blockIdx.x];
    for (int k = threadIdx.x; k < kScanTile; k += kScanThreads)
        if (base + k < n) out[base + k] += add;
}

// ---- radix sort ---------------------------------------------------------------------

constexpr int kRsThreads = 256;
constexpr int kRsItems = 4;
constexpr int kRsTile = kRsThreads * kRsItems;  // 1024; warp w owns items [128 w, 128 w + 128)
constexpr int kRadix = 256;

// Look-back words of the one-sweep passes: per (block, digit) the block's own count of the
// digit, flagged as an aggregate, later replaced by the inclusive count of every block up to
// and including it.  Counts stay below 2^30.
constexpr uint32_t kLbAggregate = 1u << 30;
constexpr uint32_t kLbInclusive = 2u << 30;
constexpr uint32_t kLbValue = kLbAggregate - 1u;
constexpr int kLbSpinLimit = 1 << 20;
constexpr int kTestSpinLimit = 1 << 12;  // the short limit of an armed test stall

__device__ __forceinline__ uint32_t ld_relaxed_gpu(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_gpu(uint32_t* p, uint32_t v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Digit mask of LSD pass p over key bits [0, bits): 8-bit digits, the last one narrower.
__host__ __device__ __forceinline__ uint32_t pass_mask(int bits, int p) {
    const int pb = min(8, max(bits - 8 * p, 1));
    return (1u << pb) - 1u;
}

// Digit counts over all n keys for every pass at once (counts[p * 256 + digit]).  One read of
// the keys; the counts do not depend on the order the earlier passes leave behind.
__global__ void __launch_bounds__(kRsThreads) radix_digit_counts(const uint32_t* __restrict__ keys, int64_t n,
                                                                 int passes, int bits,
                                                                 uint32_t* __restrict__ counts) {
    __shared__ uint32_t h[4][kRadix];
    const int t = threadIdx.x, lane = t & 31;
#pragma unroll
    for (int p = 0; p < 4; ++p) h[p][t] = 0;
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * kRsThreads;
    for (int64_t base = (int64_t)blockIdx.x * kRsThreads + (t & ~31); base < n; base += stride) {
        const int64_t i = base + lane;
        const bool valid = i < n;
        const uint32_t k = valid ? keys[i] : 0u;
        for (int p = 0; p < passes; ++p) {
            const uint32_t dig = valid ? ((k >> (8 * p)) & pass_mask(bits, p)) : 0xffffffffu;
            const uint32_t peers = __match_any_sync(0xffffffffu, dig);
            if (valid && lane == __ffs(peers) - 1) atomicAdd(&h[p][dig], (uint32_t)__popc(peers));
        }
    }
    __syncthreads();
    for (int p = 0; p < passes; ++p)
        if (h[p][t]) atomicAdd(&counts[p * kRadix + t], h[p][t]);
}

// One stable LSD pass in a single launch.  Each block takes the next 1024-key tile in input
// order (a ticket, so that every tile before it belongs to a block already running), ranks
// its keys by digit in input order (warp w owns keys [128 w, 128 w + 128) of the tile), posts
// its per-digit counts, and adds the counts of the earlier tiles by walking back over their
// posted words until it meets an inclusive one (decoupled look-back).  The waits are bounded
// (spin_limit polls): a walk that gives up raises *err and uses what it summed (every position
// stays below n).  stall_tile >= 0 (a test of that path) makes that tile's first look-back poll
// stall_word, a zero word that nothing writes, so that its wait runs out.
__global__ void __launch_bounds__(kRsThreads) radix_onesweep(const uint32_t* __restrict__ keys_in,
                                                             const uint32_t* __restrict__ vals_in,
                                                             uint32_t* __restrict__ keys_out,
                                                             uint32_t* __restrict__ vals_out, int64_t n, int shift,
                                                             uint32_t mask, const uint32_t* __restrict__ counts,
                                                             uint32_t* status, uint32_t* ticket, uint32_t* err,
                                                             int spin_limit, int64_t stall_tile,
                                                             const uint32_t* stall_word) {
    __shared__ uint32_t s_off[kRadix];
    __shared__ uint32_t s_cnt[kRsThreads / 32][kRadix];
    __shared__ uint32_t s_wsum[kRsThreads / 32];
    __shared__ uint32_t s_tile;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    if (t == 0) s_tile = atomicAdd(ticket, 1u);
#pragma unroll
    for (int w = 0; w < kRsThreads / 32; ++w) s_cnt[w][t] = 0;
    // first output position of digit t: exclusive scan of the digit counts
    const uint32_t c_all = counts[t];
    const uint32_t c_incl = warp_incl_scan(c_all, lane);
    if (lane == 31) s_wsum[warp] = c_incl;
    __syncthreads();
    uint32_t digit_start = c_incl - c_all;
    for (int w = 0; w < warp; ++w) digit_start += s_wsum[w];
    const int64_t tile = s_tile;

    const uint32_t lt_mask = (1u << lane) - 1u;
    uint32_t kk[kRsItems], vv[kRsItems], dd[kRsItems], rr[kRsItems];
    const int64_t base = tile * kRsTile + warp * (32 * kRsItems);
#pragma unroll
    for (int it = 0; it < kRsItems; ++it) {
        const int64_t i = base + it * 32 + lane;
        const bool valid = i < n;
        const uint32_t key = valid ? keys_in[i] : 0u;
        const uint32_t val = valid ? (vals_in ? vals_in[i] : (uint32_t)i) : 0u;
        const uint32_t dig = valid ? ((key >> shift) & mask) : 0xffffffffu;
        const uint32_t peers = __match_any_sync(0xffffffffu, dig);
        const uint32_t rank = __popc(peers & lt_mask);
        const uint32_t before = valid ? s_cnt[warp][dig] : 0u;
        __syncwarp();
        if (valid && rank == 0) s_cnt[warp][dig] = before + __popc(peers);
        __syncwarp();
        kk[it] = key;
        vv[it] = val;
        dd[it] = dig;
        rr[it] = before + rank;
    }
    __syncthreads();
    uint32_t own = 0;  // keys of digit t in this tile; s_cnt becomes the per-warp exclusive prefix
#pragma unroll
    for (int w = 0; w < kRsThreads / 32; ++w) {
        const uint32_t c = s_cnt[w][t];
        s_cnt[w][t] = own;
        own += c;
    }
    uint32_t* word = status + tile * kRadix + t;
    st_relaxed_gpu(word, (tile == 0 ? kLbInclusive : kLbAggregate) | own);
    uint32_t earlier = 0;  // keys of digit t in the tiles before this one
    if (tile > 0) {
        bool ok = true;
        for (int64_t j = tile - 1; j >= 0 && ok; --j) {
            const uint32_t* w = (tile == stall_tile && j == tile - 1) ? stall_word : status + j * kRadix + t;
            uint32_t v = ld_relaxed_gpu(w);
            for (int spins = 0; (v & ~kLbValue) == 0; ++spins) {
                if (spins >= spin_limit) {
                    ok = false;
                    break;
                }
                if (spins >= 32) __nanosleep(64);
                v = ld_relaxed_gpu(w);
            }
            if (!ok) break;
            earlier += v & kLbValue;
            if (v & kLbInclusive) break;
        }
        if (!ok) atomicExch(err, 1u);
        st_relaxed_gpu(word, kLbInclusive | (earlier + own));
    }
    s_off[t] = digit_start + earlier;
    __syncthreads();
#pragma unroll
    for (int it = 0; it < kRsItems; ++it) {
        const int64_t i = base + it * 32 + lane;
        if (i < n) {
            const uint32_t pos = s_off[dd[it]] + s_cnt[warp][dd[it]] + rr[it];
            keys_out[pos] = kk[it];
            vals_out[pos] = vv[it];
        }
    }
}

// ---- binning ---------------------------------------------------------------------------

// One (tile, Gaussian) pair per covered tile, Gaussians in index order, at the exclusive scan
// of tiles_touched; writes beyond the P pairs counted are dropped.
__global__ void emit_pairs(int N, const int32_t* __restrict__ tiles, const uint32_t* __restrict__ offsets,
                           const int4* __restrict__ rect, int tiles_x, int64_t P, uint32_t* __restrict__ pair_tile,
                           uint32_t* __restrict__ pair_gauss) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= N) return;
    const int4 r = rect[g];
    const int n = max(0, min(tiles[g], (r.z - r.x) * (r.w - r.y)));
    int64_t o = offsets[g];
    int k = 0;
    for (int ty = r.y; ty < r.w && k < n; ++ty)
        for (int tx = r.x; tx < r.z && k < n; ++tx, ++k, ++o) {
            if (o >= P) return;
            pair_tile[o] = (uint32_t)(ty * tiles_x + tx);
            pair_gauss[o] = (uint32_t)g;
        }
}

// Per-tile depth order.  The tile lists arrive in Gaussian index order (the stable tile sort of
// the index-ordered pairs); each is sorted on the 64-bit key (binary32 depth bits, index), i.e.
// by depth with ties in index order (visible depths are > z_near > 0, so their bits order like
// the values).  Lists of up to kTsCap keys are sorted in shared memory by a bitonic network;
// longer ones are cut into kTsCap runs sorted the same way and merged pairwise through the
// scratch buffers (two arrays of P keys, each tile using its own segment).
constexpr int kTsThreads = 256;
constexpr int kTsCap = 4096;

__device__ __forceinline__ uint64_t depth_index_key(const float* __restrict__ depth, uint32_t g) {
    return ((uint64_t)__float_as_uint(depth[g]) << 32) | g;
}

// Bitonic sort of s[0, n2) (n2 a power of two) by the whole block, ascending.
__device__ void block_bitonic(uint64_t* s, int n2) {
    for (int k = 2; k <= n2; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < n2; i += blockDim.x) {
                const int l = i ^ j;
                if (l > i) {
                    const uint64_t a = s[i], b = s[l];
                    if ((a > b) == ((i & k) == 0)) {
                        s[i] = b;
                        s[l] = a;
                    }
                }
            }
            __syncthreads();
        }
}

// Number of elements taken from a (length na) among the first `diag` outputs of the merge of
// a and b (length nb): the merge-path split, ties taken from a first.
__device__ __forceinline__ int merge_split(const uint64_t* a, int na, const uint64_t* b, int nb, int diag) {
    int lo = max(0, diag - nb), hi = min(diag, na);
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (a[mid] <= b[diag - 1 - mid]) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__global__ void __launch_bounds__(kTsThreads) tile_depth_sort(const int2* __restrict__ ranges,
                                                              const float* __restrict__ depth,
                                                              int32_t* __restrict__ ids, uint64_t* __restrict__ buf0,
                                                              uint64_t* __restrict__ buf1, const uint32_t* err) {
    __shared__ uint64_t s[kTsCap];
    if (*err) return;
    const int2 r = ranges[blockIdx.x];
    const int L = r.y - r.x;
    if (L <= 1) return;
    int32_t* list = ids + r.x;
    if (L <= kTsCap) {
        int n2 = 1;
        while (n2 < L) n2 <<= 1;
        for (int i = threadIdx.x; i < n2; i += blockDim.x)
            s[i] = i < L ? depth_index_key(depth, (uint32_t)list[i]) : ~0ull;
        __syncthreads();
        block_bitonic(s, n2);
        for (int i = threadIdx.x; i < L; i += blockDim.x) list[i] = (int32_t)(uint32_t)s[i];
        return;
    }
    // long list: sorted runs of kTsCap keys, then pairwise merges
    uint64_t* src = buf0 + r.x;
    uint64_t* dst = buf1 + r.x;
    for (int c0 = 0; c0 < L; c0 += kTsCap) {
        const int n = min(kTsCap, L - c0);
        for (int i = threadIdx.x; i < kTsCap; i += blockDim.x)
            s[i] = i < n ? depth_index_key(depth, (uint32_t)list[c0 + i]) : ~0ull;
        __syncthreads();
        block_bitonic(s, kTsCap);
        for (int i = threadIdx.x; i < n; i += blockDim.x) src[c0 + i] = s[i];
        __syncthreads();
    }
    for (int width = kTsCap; width < L; width <<= 1) {
        for (int m0 = 0; m0 < L; m0 += 2 * width) {
            const int na = min(width, L - m0), nb = max(0, min(width, L - m0 - width));
            const uint64_t* a = src + m0;
            const uint64_t* b = a + na;
            const int total = na + nb;
            const int per = (total + blockDim.x - 1) / blockDim.x;
            const int d0 = min(total, (int)threadIdx.x * per), d1 = min(total, d0 + per);
            int ia = merge_split(a, na, b, nb, d0), ib = d0 - ia;
            for (int o = d0; o < d1; ++o) {
                const bool take_a = ib >= nb || (ia < na && a[ia] <= b[ib]);
                dst[m0 + o] = take_a ? a[ia++] : b[ib++];
            }
        }
        __syncthreads();
        uint64_t* t = src;
        src = dst;
        dst = t;
    }
    for (int i = threadIdx.x; i < L; i += blockDim.x) list[i] = (int32_t)(uint32_t)src[i];
}

// A sort whose look-back gave up (*err) leaves every tile empty (the ranges were cleared).
__global__ void tile_ranges(const uint32_t* __restrict__ keys, int64_t P, const uint32_t* __restrict__ err,
                            int2* __restrict__ ranges) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P || *err) return;
    const uint32_t t = keys[i];
    if (i == 0 || keys[i - 1] != t) ranges[t].x = (int)i;
    if (i == P - 1 || keys[i + 1] != t) ranges[t].y = (int)(i + 1);
}

int ceil_log2(int64_t v) {
    int b = 0;
    while (((int64_t)1 << b) < v) ++b;
    return b;
}

}  // namespace

size_t scan_scratch_words(int64_t n) { return (size_t)((n + kScanTile - 1) / kScanTile + 1); }

latentam_status scan_exclusive_u32(latentam_ctx* ctx, const uint32_t* in, uint32_t* out, int64_t n,
                                   uint32_t* total_dev, cudaStream_t st, uint32_t* sums) {
    if (n <= 0) {
        if (total_dev) {
            cudaError_t e = cudaMemsetAsync(total_dev, 0, sizeof(uint32_t), st);
            if (e != cudaSuccess) return cuda_error(e, "scan memset");
        }
        return LATENTAM_OK;
    }
    const int64_t nb = (n + kScanTile - 1) / kScanTile;
    if (nb > kScanTile) {
        set_error("scan of %lld items exceeds the supported %lld", (long long)n, (long long)kScanTile * kScanTile);
        return LATENTAM_ERR_UNSUPPORTED_SHAPE;
    }
    if (!sums) sums = static_cast<uint32_t*>(ws(ctx, WS_SCAN_SUMS, sizeof(uint32_t) * (size_t)(nb + 1)));
    if (!sums) return LATENTAM_ERR_OUT_OF_MEMORY;
    scan_tiles<<<(unsigned)nb, kScanThreads, 0, st>>>(in, out, sums, n);
    LAT_CHECK_LAUNCH("scan_tiles");
    scan_sums<<<1, kScanThreads, 0, st>>>(sums, (int)nb, total_dev);
    LAT_CHECK_LAUNCH("scan_sums");
    if (nb > 1) {
        scan_add<<<(unsigned)nb, kScanThreads, 0, st>>>(out, sums, n);
        LAT_CHECK_LAUNCH("scan_add");
    }
    return LATENTAM_OK;
}

size_t radix_scratch_words(int64_t n, int bits) {
    const int passes = bits <= 0 ? 1 : (bits + 7) / 8;
    const int64_t nb = (n + kRsTile - 1) / kRsTile;
    return (size_t)(passes + 1) * kRadix + (size_t)passes * (size_t)nb * kRadix;
}

latentam_status radix_sort_pairs(latentam_ctx* ctx, uint32_t* const keys[2], uint32_t* const vals[2], bool vals_iota,
                                 int64_t n, int bits, int* result, uint32_t* err, cudaStream_t st,
                                 uint32_t* counters) {
    const int passes = bits <= 0 ? 1 : (bits + 7) / 8;
    *result = passes % 2;
    if (n <= 0) return LATENTAM_OK;
    if (passes > 4 || n > (int64_t)kLbValue) {
        set_error("radix sort of %lld keys on %d bits is not supported", (long long)n, bits);
        return LATENTAM_ERR_UNSUPPORTED_SHAPE;
    }
    const int64_t nb = (n + kRsTile - 1) / kRsTile;
    // [digit counts: passes x 256 | tickets: 256 | look-back words: passes x nb x 256], zeroed;
    // tickets[255] is never written (the word an armed test stall polls)
    const size_t words = radix_scratch_words(n, bits);
    uint32_t* buf = counters ? counters : static_cast<uint32_t*>(ws(ctx, WS_SORT_HIST, sizeof(uint32_t) * words));
    if (!buf) return LATENTAM_ERR_OUT_OF_MEMORY;
    cudaError_t e = cudaMemsetAsync(buf, 0, sizeof(uint32_t) * words, st);
    if (e != cudaSuccess) return cuda_error(e, "clear radix sort counters");
    uint32_t* counts = buf;
    uint32_t* tickets = buf + (size_t)passes * kRadix;
    uint32_t* status = tickets + kRadix;
    const unsigned cblocks = (unsigned)std::min<int64_t>(nb, 2 * (int64_t)ctx->num_sms);
    radix_digit_counts<<<cblocks, kRsThreads, 0, st>>>(keys[0], n, passes, bits, counts);
    LAT_CHECK_LAUNCH("radix_digit_counts");
    // an armed test stall applies to the last tile of the first pass (once)
    const bool stall = ctx->test_stall_sort && nb > 1;
    if (stall) ctx->test_stall_sort = 0;
    for (int p = 0; p < passes; ++p) {
        const int src = p % 2, dst = 1 - src;
        const uint32_t* vin = (p == 0 && vals_iota) ? nullptr : vals[src];
        radix_onesweep<<<(unsigned)nb, kRsThreads, 0, st>>>(
            keys[src], vin, keys[dst], vals[dst], n, 8 * p, pass_mask(bits, p), counts + p * kRadix,
            status + (size_t)p * (size_t)nb * kRadix, tickets + p, err, stall ? kTestSpinLimit : kLbSpinLimit,
            (stall && p == 0) ? nb - 1 : -1, tickets + (kRadix - 1));
        LAT_CHECK_LAUNCH("radix_onesweep");
    }
    return LATENTAM_OK;
}

// Counters of binning slot k (a keyframe of a batch; a single binning uses slot 0): on the
// device 4 words at cnt + 16 k ([1] the pair count P, [2] the sort error word), read back into
// 4 pinned host words at host_counts + 8 + 4 k with the tensor-core wait flag.
namespace {
// Scratch buffer j of binning slot k (j: 0 scan sums, 1-2 sort keys, 3 sort values, 4 long-list
// merge buffers, 5 radix counters): slot 0 uses the context's workspace slots, the others their
// own buffers, so that the keyframes of a batch can be binned at the same time.
void* bin_scratch(latentam_ctx* ctx, int slot, int j, size_t bytes) {
    static const Slot shared[6] = {WS_SCAN_SUMS, WS_SORT_K0, WS_SORT_K1, WS_SORT_V0, WS_SORT_V1, WS_SORT_HIST};
    if (slot == 0) return ws(ctx, shared[j], bytes);
    return frame_ws(ctx, 2 * LATENTAM_MAX_BATCH + 6 * slot + j, bytes);
}

latentam_status bin_slot(latentam_ctx* ctx, int slot, uint32_t** cnt, uint32_t** host) {
    if (slot < 0 || slot >= LATENTAM_MAX_BATCH) {
        set_error("binning slot %d outside 0..%d", slot, LATENTAM_MAX_BATCH - 1);
        return LATENTAM_ERR_INVALID_ARG;
    }
    uint32_t* c = static_cast<uint32_t*>(ws(ctx, WS_COUNTERS, 64 * LATENTAM_MAX_BATCH));
    if (!c) return LATENTAM_ERR_OUT_OF_MEMORY;
    *cnt = c + 16 * slot;
    *host = ctx->host_counts + 8 + 4 * slot;
    return LATENTAM_OK;
}
}  // namespace

latentam_status bin_count(latentam_ctx* ctx, int32_t N, const latentam_projected& proj, const CamParams& cam,
                          latentam_bins* bins, uint32_t* off, int slot, cudaStream_t st) {
    const int64_t num_tiles = (int64_t)cam.tiles_x * cam.tiles_y;
    if (N == 0) {
        cudaError_t e = cudaMemsetAsync(bins->tile_ranges, 0, sizeof(int2) * (size_t)num_tiles, st);
        if (e != cudaSuccess) return cuda_error(e, "memset tile_ranges");
        return LATENTAM_OK;
    }
    uint32_t *cnt, *host;
    LAT_TRY(bin_slot(ctx, slot, &cnt, &host));
    // cleared ranges, pair offsets (exclusive scan of tiles_touched) and the pair count P into
    // cnt[1], read back with cnt[2]: raised by a sort pass whose look-back gave up; it outlives
    // the call and is reported (and cleared) by the slot's next binning.  The same frame size
    // and buffers replay one captured graph.
    uint32_t* sums = static_cast<uint32_t*>(bin_scratch(ctx, slot, 0, sizeof(uint32_t) * scan_scratch_words(N)));
    if (!sums) return LATENTAM_ERR_OUT_OF_MEMORY;
    auto pre = [&](cudaStream_t s) -> latentam_status {
        cudaError_t e2 = cudaMemsetAsync(bins->tile_ranges, 0, sizeof(int2) * (size_t)num_tiles, s);
        if (e2 == cudaSuccess) e2 = cudaMemsetAsync(cnt, 0, 2 * sizeof(uint32_t), s);
        if (e2 != cudaSuccess) return cuda_error(e2, "clear ranges and counters");
        LAT_TRY(scan_exclusive_u32(ctx, reinterpret_cast<const uint32_t*>(proj.tiles_touched), off, N, cnt + 1, s,
                                   sums));
        e2 = cudaMemcpyAsync(host, cnt, 3 * sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
        if (e2 == cudaSuccess)  // and the tensor-core kernels' sticky wait flag
            e2 = cudaMemcpyAsync(host + 3, ctx->dev_flags, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
        if (e2 != cudaSuccess) return cuda_error(e2, "read the pair count");
        return LATENTAM_OK;
    };
    const uint64_t pre_key[] = {0x62696e302d707265ull /* tag: counting phase */, (uint64_t)N, (uint64_t)num_tiles,
                                reinterpret_cast<uint64_t>(proj.tiles_touched),
                                reinterpret_cast<uint64_t>(bins->tile_ranges), reinterpret_cast<uint64_t>(host),
                                reinterpret_cast<uint64_t>(off), reinterpret_cast<uint64_t>(sums),
                                reinterpret_cast<uint64_t>(st), ctx->ws_generation};
    return cached_launch(ctx, pre_key, (int)(sizeof(pre_key) / sizeof(pre_key[0])), st, pre);
}

latentam_status bin_finish(latentam_ctx* ctx, int32_t N, const latentam_projected& proj, const CamParams& cam,
                           latentam_bins* bins, const uint32_t* off, int slot, cudaStream_t st) {
    const int64_t num_tiles = (int64_t)cam.tiles_x * cam.tiles_y;
    cudaError_t e;
    if (N == 0) {
        bins->num_pairs = 0;
        return LATENTAM_OK;
    }
    uint32_t *cnt, *host;
    LAT_TRY(bin_slot(ctx, slot, &cnt, &host));
    const uint32_t pairs = host[1], sort_error = host[2], tc_error = host[3];
    if (sort_error) {
        e = cudaMemsetAsync(cnt + 2, 0, sizeof(uint32_t), st);
        if (e != cudaSuccess) return cuda_error(e, "clear the sort error word");
        set_error("a radix sort look-back wait gave up in an earlier binning (its tiles were left empty)");
        return LATENTAM_ERR_TIMEOUT;
    }
    if (tc_error) {
        host[3] = 0;  // reported once, by this slot
        e = cudaMemsetAsync(ctx->dev_flags, 0, sizeof(int), st);
        if (e != cudaSuccess) return cuda_error(e, "clear the tensor-core wait flag");
        set_error("a bounded wait of a tensor-core decode kernel gave up in an earlier call (its loss was NaN)");
        return LATENTAM_ERR_TIMEOUT;
    }
    const int64_t P = (int64_t)pairs;
    bins->num_pairs = P;
    if (P > bins->capacity) {
        set_error("pair buffer holds %lld pairs, %lld needed", (long long)bins->capacity, (long long)P);
        return LATENTAM_ERR_CAPACITY;
    }
    if (P == 0) return LATENTAM_OK;
    // Steps 1-4 depend on the host only through P: the same frame binned again (the iterations
    // of one keyframe, each call of Stage I and II) replays one captured graph.
    const size_t pbytes = sizeof(uint32_t) * (size_t)P;
    const int tile_bits = std::max(1, ceil_log2(num_tiles));
    const int passes = (tile_bits + 7) / 8;
    uint32_t* pk[2] = {static_cast<uint32_t*>(bin_scratch(ctx, slot, 1, pbytes)),
                       static_cast<uint32_t*>(bin_scratch(ctx, slot, 2, pbytes))};
    uint32_t* scratch = static_cast<uint32_t*>(bin_scratch(ctx, slot, 3, pbytes));
    uint64_t* lng = static_cast<uint64_t*>(bin_scratch(ctx, slot, 4, 2 * sizeof(uint64_t) * (size_t)P));
    uint32_t* rcnt =
        static_cast<uint32_t*>(bin_scratch(ctx, slot, 5, sizeof(uint32_t) * radix_scratch_words(P, tile_bits)));
    if (!pk[0] || !pk[1] || !scratch || !lng || !rcnt) return LATENTAM_ERR_OUT_OF_MEMORY;
    // the tile sort's result lands in buffer passes % 2: make that the caller's pair list
    uint32_t* ids = reinterpret_cast<uint32_t*>(bins->pair_ids);
    uint32_t* pv[2] = {passes % 2 == 0 ? ids : scratch, passes % 2 == 0 ? scratch : ids};
    const int threads = 256;
    const unsigned blocks = (unsigned)((N + threads - 1) / threads);
    auto rest = [&, P](cudaStream_t s) -> latentam_status {
        // 1. pairs in Gaussian index order
        emit_pairs<<<blocks, threads, 0, s>>>(N, proj.tiles_touched, off, reinterpret_cast<const int4*>(proj.rect),
                                              cam.tiles_x, P, pk[0], pv[0]);
        LAT_CHECK_LAUNCH("emit_pairs");
        // 2. stable sort on the tile bits (index order kept within a tile)
        int r = 0;
        LAT_TRY(radix_sort_pairs(ctx, pk, pv, false, P, tile_bits, &r, cnt + 2, s, rcnt));
        // 3. ranges
        tile_ranges<<<(unsigned)((P + 255) / 256), 256, 0, s>>>(pk[r], P, cnt + 2,
                                                                 reinterpret_cast<int2*>(bins->tile_ranges));
        LAT_CHECK_LAUNCH("tile_ranges");
        // 4. depth order within each tile
        tile_depth_sort<<<(unsigned)num_tiles, kTsThreads, 0, s>>>(reinterpret_cast<const int2*>(bins->tile_ranges),
                                                                   proj.depth, bins->pair_ids, lng, lng + P, cnt + 2);
        LAT_CHECK_LAUNCH("tile_depth_sort");
        return LATENTAM_OK;
    };
    const uint64_t key[] = {0x62696e312d706169ull /* tag: pair phase */, (uint64_t)N, (uint64_t)P,
                            (uint64_t)num_tiles, (uint64_t)cam.tiles_x,
                            reinterpret_cast<uint64_t>(proj.depth), reinterpret_cast<uint64_t>(proj.tiles_touched),
                            reinterpret_cast<uint64_t>(proj.rect), reinterpret_cast<uint64_t>(bins->pair_ids),
                            reinterpret_cast<uint64_t>(bins->tile_ranges), reinterpret_cast<uint64_t>(off),
                            reinterpret_cast<uint64_t>(cnt), reinterpret_cast<uint64_t>(rcnt),
                            reinterpret_cast<uint64_t>(lng), reinterpret_cast<uint64_t>(st), ctx->ws_generation,
                            (uint64_t)ctx->test_stall_sort};
    return cached_launch(ctx, key, (int)(sizeof(key) / sizeof(key[0])), st, rest);
}

latentam_status bin_and_sort(latentam_ctx* ctx, int32_t N, const latentam_projected& proj,
                             const CamParams& cam, latentam_bins* bins, cudaStream_t st) {
    uint32_t* off = nullptr;
    if (N > 0) {
        off = static_cast<uint32_t*>(ws(ctx, WS_OFFSETS, sizeof(uint32_t) * ((size_t)N + 1)));
        if (!off) return LATENTAM_ERR_OUT_OF_MEMORY;
    }
    LAT_TRY(bin_count(ctx, N, proj, cam, bins, off, 0, st));
    if (N > 0) {
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_error(e, "sync for the pair count");
    }
    return bin_finish(ctx, N, proj, cam, bins, off, 0, st);
}

}  // namespace lat
