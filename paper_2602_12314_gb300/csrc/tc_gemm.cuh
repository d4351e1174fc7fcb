// One tcgen05 GEMM tile kernel shared by every tensor-core contraction of the decode:
//   C[128 x BN] = A[128 x K] * B[BN x K]^T, A and B BF16 K-major in global memory,
// TMA-loaded in 64-wide K chunks (128-byte swizzle) through a STAGES-deep mbarrier pipeline,
// accumulated in FP32 in tensor memory, then handed row by row to an epilogue.
//
// Warp roles (192 threads): warp 0 issues the TMA loads, warp 1 owns the TMEM allocation and
// issues the MMAs (one thread), warps 2..5 run the epilogue; epilogue thread r owns tile row r
// (TMEM lane r; warp w reads the lane quarter w % 4).
// blockIdx.x: 128-row tile of A, blockIdx.y: BN-row tile of B, blockIdx.z: split of the K range.
// When a row reduction spans several BN tiles, the tiles of one row block run as a thread-block
// cluster along y and trade their per-row partial results through distributed shared memory.
#pragma once

#include "internal.cuh"
#include "tc_common.cuh"

namespace lat {
namespace tc {

constexpr int kTileM = 128;
// epilogue row-reduction scratch: 4 slots x G warpgroups
__host__ __device__ constexpr int scratch_bytes(int groups) { return 4 * groups * kTileM * 4; }
constexpr int kScratchBytes = scratch_bytes(2);
constexpr int kMaxCluster = 4;                         // CTAs of a cluster that trade row partials
constexpr int kXchgVals = 4;                           // values per row per CTA in one exchange
constexpr int kXchgMsg = kXchgVals * kTileM * 4;       // one CTA's partials of a tile (bytes)
constexpr int kXchgBytes = kMaxCluster * kXchgMsg;     // one outgoing + (kMaxCluster - 1) incoming
constexpr int kChunkK = 64;                       // BF16 elements per 128-byte row
constexpr uint32_t kTileABytes = kTileM * 128;    // 16 KB

__host__ __device__ constexpr uint32_t tmem_cols_for(int n) {
    return n <= 32 ? 32u : n <= 64 ? 64u : n <= 128 ? 128u : n <= 256 ? 256u : 512u;
}

// Planes per operand: 2 for the split form (every FP32 operand held as a BF16 hi and lo term,
// stored [2][rows][inner]), 1 otherwise.
template <class Epi>
__host__ __device__ constexpr int planes() {
    return Epi::SPLIT ? 2 : 1;
}

// One-tile kernel with a trailing product (Epi::XPROD > 0): the B operand of that product,
// BN (K) x XPROD (N) BF16 per plane, stored MN-major as BN / 64 boxes of 64 x 64.
// (One epilogue pass's share of it when the epilogue runs in Epi::EPASS passes.)
template <class Epi>
__host__ __device__ constexpr uint32_t xprod_bytes() {
    return Epi::XPROD > 0 ? (uint32_t)(Epi::BN / 64 / Epi::EPASS) * planes<Epi>() * 64u * 64u * 2u : 0u;
}

// Shared memory at the start of the tile: the operand pipeline, reused once the MMAs are done
// for the epilogue operand (E_BOXES boxes of 64 x 128 BF16 per plane) and the staged output
// (O_BOXES per plane), then the trailing product's B operand; with Epi::EPASS passes over
// column slices of the tile, one pass's share of each at a time.
template <class Epi>
__host__ __device__ constexpr uint32_t tile_region_bytes() {
    const uint32_t pipe = (uint32_t)Epi::STAGES * planes<Epi>() *
                          ((uint32_t)Epi::MSUB * kTileM + (uint32_t)Epi::BN) * Epi::BKC * 2;
    const uint32_t boxes = (uint32_t)(Epi::E_BOXES > Epi::O_BOXES ? Epi::E_BOXES : Epi::O_BOXES) / Epi::EPASS *
                               planes<Epi>() * kTileABytes +
                           xprod_bytes<Epi>();
    return pipe > boxes ? pipe : boxes;
}

// A second trailing product whose B tile (128 pixels x 64, per plane) has a region of its own,
// loaded when the CTA starts (Epi::X2PRE), instead of taking the first product's operand space
// once that product has completed.
template <class Epi>
__host__ __device__ constexpr uint32_t x2_pre_bytes() {
    return Epi::XPROD2 > 0 && Epi::X2PRE ? (uint32_t)planes<Epi>() * kTileM * 128 : 0u;
}

// Compact layout (with a preloaded second product): no row-reduction scratch, and the 256 bytes
// of barriers in the alignment slack in front of the tile when it has room for them, else right
// behind the regions; either way within the regions + 1024 bytes.
template <class Epi>
__host__ __device__ constexpr size_t gemm_smem_bytes() {
    if (x2_pre_bytes<Epi>() > 0) return (size_t)tile_region_bytes<Epi>() + x2_pre_bytes<Epi>() + 1024;
    const size_t need = (size_t)tile_region_bytes<Epi>() + 1024 /* alignment */ + 256 /* barriers */ +
                        kScratchBytes;
    // MIN_SMEM caps the CTAs resident on one SM (so that their TMEM allocations never wait)
    return need > (size_t)Epi::MIN_SMEM ? need : (size_t)Epi::MIN_SMEM;
}

__host__ __device__ constexpr int gemm_threads(int epi_warpgroups) { return 64 + 128 * epi_warpgroups; }

// Barrier among the epilogue threads only (named barrier 1).
__device__ __forceinline__ void epi_sync(int nthreads) {
    asm volatile("bar.sync 1, %0;" ::"r"(nthreads) : "memory");
}

// Sum (or max) of one value per row over the G epilogue warpgroups, through shared memory.
// `slot` (0..3) must differ between reductions of the same tile.
template <int G>
__device__ __forceinline__ float group_sum(float v, float* scratch, int slot, int g, int row) {
    if (G == 1) return v;
    scratch[(slot * G + g) * kTileM + row] = v;
    epi_sync(128 * G);
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < G; ++k) s += scratch[(slot * G + k) * kTileM + row];
    return s;
}
// The four per-row values v[0..3] summed over the G epilogue warpgroups with one barrier
// (slots 0..3).
template <int G>
__device__ __forceinline__ void group_sum4(float (&v)[4], float* scratch, int g, int row) {
    if (G == 1) return;
#pragma unroll
    for (int k = 0; k < 4; ++k) scratch[(k * G + g) * kTileM + row] = v[k];
    epi_sync(128 * G);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        float s = 0.f;
#pragma unroll
        for (int j = 0; j < G; ++j) s += scratch[(k * G + j) * kTileM + row];
        v[k] = s;
    }
}
template <int G>
__device__ __forceinline__ float group_max(float v, float* scratch, int slot, int g, int row) {
    if (G == 1) return v;
    scratch[(slot * G + g) * kTileM + row] = v;
    epi_sync(128 * G);
    float s = -INFINITY;
#pragma unroll
    for (int k = 0; k < G; ++k) s = fmaxf(s, scratch[(slot * G + k) * kTileM + row]);
    return s;
}

struct GemmGrid {
    int k_chunks;      // total 64-wide K chunks
    int chunks_per_z;  // chunks handled by one blockIdx.z
};

// Epi must provide: static constexpr int BN, STAGES, BOX_B (rows per TMA box of a K-major B,
// divides BN, <= 256); static constexpr int MSUB (one-tile kernel: 128-row sub-tiles of A per CTA
// sharing each B stage, 1 or 2 (MN-major A), each its own TMEM accumulator of BN columns) and
// BKC (one-tile kernel: K elements per ring stage, 64, or 32 when both operands are MN-major);
// static constexpr bool SPLIT (every operand, epilogue operand and staged
// output held as a BF16 hi and lo plane, 3D tensor maps with the plane as z, and each product
// taken as three MMAs); static constexpr bool A_MN, B_MN (operand stored MN-major: the tile is
// loaded as 64 (MN) x 64 (K) boxes of a row-major K x MN matrix, x = MN, y = K); struct
// Params; static constexpr int EPI_WG (1 or 2 epilogue warpgroups: warpgroup g owns the
// 32-column chunks c with c % EPI_WG == g of every row); static constexpr int E_BOXES (number
// of 64-column boxes of a row-major BF16 "epilogue operand" (tmE) loaded for the tile's 128
// rows into the pipeline shared memory once the MMAs are done, 0 for none); static __device__
// void run(const Params&, const EpiCtx&) executed by the 128 * EPI_WG epilogue threads
// (warp-convergent), returning the number of 64-column boxes of output it staged with
// EpiCtx::put32 (CTA-uniform; stored to tmO at (n0 + 64 b, m0) by TMA); static constexpr int
// O_BOXES (boxes the epilogue may stage, 0 for none); static constexpr int XROUNDS (0 or 1: run() calls EpiCtx::exchange exactly
// that many times, whatever the CTA's rows hold), MIN_SMEM (bytes of shared memory to request
// at least) and MIN_BLOCKS (CTAs per SM the register allocation must allow).  One-tile kernel
// only: static constexpr int XPROD (0, or the N = 64 of a trailing product: once the output
// tile is staged, its 128 x BN BF16 values, K-major as staged, are multiplied on the tensor
// cores by a BN x 64 operand tmX (MN-major, rows n0 .. n0 + BN) into TMEM columns 0 .. 63,
// after which static __device__ void run_x(const Params&, const EpiCtx&) reads them; static
// __device__ bool x_active(const Params&) says, CTA-uniformly, whether this launch takes it);
// static constexpr int EPASS (1, or 2: the epilogue runs in two passes over the two column
// halves of the tile, each with its half of the epilogue-operand boxes, of the staged output
// and of the trailing product's K, in half the shared memory; run() then covers the columns
// [EpiCtx::col0, col0 + BN / EPASS) and is called once per pass); static constexpr int XPROD2
// (0, or 1 with XPROD: a second trailing product of the staged output, transposed: its 128-column
// groups (MN-major, M = the output's columns) times tmX2's 128 x 64 tile at (0, m0) (MN-major,
// K = the tile's rows), group G into TMEM columns 64 + 64 G; static __device__ bool
// x2_active(const Params&) says whether this launch takes it, and then the staged output is not
// stored; static __device__ void run_k(const Params&, const EpiCtx&, int tile) reads it at the
// end.  With static constexpr int X2PRE = 1 the tile has 16 KB (per plane) of shared memory of
// its own and is loaded when the CTA starts; otherwise it takes the first product's operand
// space once pass 0's first product has read it, and later passes run the second product first,
// on that tile, before the first product's operand returns.  Either way run_x then finds the
// first product's 32 KB operand space free in EpiCtx::xstage).
struct EpiCtx {
    uint32_t taddr;        // TMEM address of this thread's row, column 0
    int row, m0, n0, z;    // tile row owned by this thread, tile origin, K split
    int g;                 // epilogue warpgroup
    float* scratch;        // row-reduction scratch
    const uint8_t* etile;  // epilogue operand tile (128-byte swizzled 64 x 128 boxes), or null
    uint8_t* otile;        // staging tile of the output, same layout (may alias etile)
    uint64_t* ebar;        // one barrier per box
    volatile int* abort;
    int crank, csize;      // rank of this CTA in its cluster, cluster size
    uint64_t* xbar;        // completes when every other CTA's partials of this tile arrived
    float* xbuf;           // [value][row] outgoing partials, then [peer slot][value][row] incoming
    uint32_t ephase = 0;   // phase parity of the epilogue-operand barriers for this tile
    uint32_t xphase = 0;   // phase parity of xbar for this tile
    int ngroups = 1;       // epilogue warpgroups
    int leader = 64;       // first epilogue thread
    int col0 = 0;          // one-tile kernel, epilogue pass: first tile column of the pass's boxes
    uint32_t eplane = 0;   // split form: bytes from the hi to the lo plane of the epilogue operand
    uint32_t oplane = 0;   // split form: bytes from the hi to the lo plane of the staged output
    uint64_t* ofree = nullptr;  // split persistent form: completes when the staging buffers are free
    uint32_t ofree_phase = 0;
    uint8_t* xstage = nullptr;  // one-tile kernel, run_x: 32 KB of free shared memory, or null

    // In-place split form (Epi::INPLACE): the tile's FP32 epilogue operand sits in the box
    // buffers as 32-column chunks (128 rows x 128 B, 128-byte swizzle, chunk c at c x 16 KB), and
    // the output of chunk c replaces it as two 32-column BF16 boxes (hi at the chunk's first
    // 8 KB, lo at its second, 64-byte swizzle).
    // 32 FP32 values of this thread's row from chunk c0 / 32 of the epilogue operand.
    __device__ __forceinline__ void row32f(int c0, float (&v)[32]) const {
        const uint8_t* base = etile + (c0 >> 5) * 16384 + row * 128;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const float4 u = *reinterpret_cast<const float4*>(base + ((q ^ (row & 7)) << 4));
            v[4 * q] = u.x;
            v[4 * q + 1] = u.y;
            v[4 * q + 2] = u.z;
            v[4 * q + 3] = u.w;
        }
    }
    // The hi and lo terms of 32 values of this thread's row into chunk c0 / 32 (every thread that
    // reads the chunk must have read it first: the caller synchronises its warpgroup).
    __device__ __forceinline__ void put32s(int c0, const float (&v)[32]) const {
        uint8_t* base = otile + (c0 >> 5) * 16384 + row * 64;
        const int sw = (row >> 1) & 3;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            uint32_t h[4], l[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) pack_split_bf16x2(v[8 * q + 2 * k], v[8 * q + 2 * k + 1], h[k], l[k]);
            const int off = (q ^ sw) << 4;
            *reinterpret_cast<uint4*>(base + off) = make_uint4(h[0], h[1], h[2], h[3]);
            *reinterpret_cast<uint4*>(base + 8192 + off) = make_uint4(l[0], l[1], l[2], l[3]);
        }
    }
    // Barrier of this thread's epilogue warpgroup only (named barriers 2 + g).
    __device__ __forceinline__ void group_sync() const {
        asm volatile("bar.sync %0, 128;" ::"r"(2 + g) : "memory");
    }

    // Split persistent form: wait until the previous tile's staged output has been read by its
    // TMA stores (call before the first put32; a no-op elsewhere).  Bounded.
    __device__ __forceinline__ bool wait_out() const {
        if (!ofree) return true;
        const bool ok = mbar_wait(ofree, ofree_phase, abort);
        if (!ok) *abort = 1;
        return ok;
    }

    // Give this row's kXchgVals partials to every other CTA of the cluster and wait for theirs
    // (read back with xval).  Warpgroup 0 stages the CTA's partials in shared memory; one thread
    // arms this CTA's barrier for the incoming bytes and sends the block to each peer with one
    // bulk copy that completes on the peer's barrier.  Called by every epilogue thread.
    // Bounded: false (and the error flag raised) if the partials did not all arrive.
    __device__ __forceinline__ bool exchange(const float (&v)[kXchgVals]) const {
        if (csize <= 1) return true;
        if (g == 0) {
#pragma unroll
            for (int k = 0; k < kXchgVals; ++k) xbuf[k * kTileM + row] = v[k];
            fence_proxy_async();
        }
        epi_sync(128 * ngroups);
        if ((int)threadIdx.x == leader) {
            mbar_expect_tx(xbar, (uint32_t)((csize - 1) * kXchgMsg));
            for (int q = 0; q < csize; ++q) {
                if (q == crank) continue;
                const int slot = 1 + (crank < q ? crank : crank - 1);  // this CTA's slot at q
                bulk_copy_to_peer(peer_addr(xbuf + slot * (kXchgMsg / 4), (uint32_t)q), xbuf, kXchgMsg,
                                  peer_addr(xbar, (uint32_t)q));
            }
        }
        const bool ok = mbar_wait_long(xbar, xphase);
        if (!ok) *abort = 1;
        return ok;
    }
    // Partial k of this thread's row from CTA q (q != crank) of the cluster.
    __device__ __forceinline__ float xval(int q, int k) const {
        const int slot = 1 + (q < crank ? q : q - 1);
        return xbuf[slot * (kXchgMsg / 4) + k * kTileM + row];
    }

    // Wait for box b of the epilogue operand (bounded; false if it gave up).
    __device__ __forceinline__ bool wait_box(int b) const { return mbar_wait(&ebar[b], ephase, abort); }
    // Stage 32 values of this thread's row as BF16 at column c0 (a multiple of 32) of the output
    // (split form: the hi terms in the hi plane, the lo terms in the lo plane).
    __device__ __forceinline__ void put32(int c0, const float (&v)[32]) const {
        uint8_t* base = otile + ((c0 - col0) >> 6) * (kTileM * 128) + row * 128;
        const int j0 = (c0 & 63) >> 3;
        if (oplane) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                uint32_t h[4], l[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) pack_split_bf16x2(v[8 * q + 2 * k], v[8 * q + 2 * k + 1], h[k], l[k]);
                const int off = ((j0 + q) ^ (row & 7)) << 4;
                *reinterpret_cast<uint4*>(base + off) = make_uint4(h[0], h[1], h[2], h[3]);
                *reinterpret_cast<uint4*>(base + oplane + off) = make_uint4(l[0], l[1], l[2], l[3]);
            }
            return;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q)
            *reinterpret_cast<uint4*>(base + (((j0 + q) ^ (row & 7)) << 4)) =
                make_uint4(pack_bf16x2(v[8 * q], v[8 * q + 1]), pack_bf16x2(v[8 * q + 2], v[8 * q + 3]),
                           pack_bf16x2(v[8 * q + 4], v[8 * q + 5]), pack_bf16x2(v[8 * q + 6], v[8 * q + 7]));
    }
    // 32 values of this thread's row from column c0 (a multiple of 32) of the operand (split
    // form: hi + lo).
    __device__ __forceinline__ void row32(int c0, float (&v)[32]) const {
        const uint8_t* base = etile + ((c0 - col0) >> 6) * (kTileM * 128) + row * 128;
        const int j0 = (c0 & 63) >> 3;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int off = ((j0 + q) ^ (row & 7)) << 4;
            const uint4 u = *reinterpret_cast<const uint4*>(base + off);
            const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w[h]));
                v[8 * q + 2 * h] = f.x;
                v[8 * q + 2 * h + 1] = f.y;
            }
            if (eplane) {
                const uint4 ul = *reinterpret_cast<const uint4*>(base + eplane + off);
                const uint32_t wl[4] = {ul.x, ul.y, ul.z, ul.w};
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&wl[h]));
                    v[8 * q + 2 * h] += f.x;
                    v[8 * q + 2 * h + 1] += f.y;
                }
            }
        }
    }
};

// One MMA step of the product: A x B (plain) or, split, A_hi B_hi + A_hi B_lo + A_lo B_hi.
template <bool SPLIT>
__device__ __forceinline__ void mma_step(uint32_t d, uint64_t a_hi, uint64_t a_lo, uint64_t b_hi, uint64_t b_lo,
                                         uint32_t idesc, uint32_t acc) {
    mma_bf16(d, a_hi, b_hi, idesc, acc);
    if (SPLIT) {
        mma_bf16(d, a_hi, b_lo, idesc, 1u);
        mma_bf16(d, a_lo, b_hi, idesc, 1u);
    }
}

// 2D (plain, z < 0) or 3D (split plane z) tile store.
__device__ __forceinline__ void tma_store(const CUtensorMap* map, const void* src, int x, int y, int z) {
    if (z < 0)
        tma_store_2d(map, src, x, y);
    else
        tma_store_3d(map, src, x, y, z);
}

template <class Epi>
__global__ void __launch_bounds__(gemm_threads(Epi::EPI_WG), Epi::MIN_BLOCKS)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const __grid_constant__ CUtensorMap tmE, const __grid_constant__ CUtensorMap tmO,
                   const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmX2, GemmGrid g,
                   typename Epi::Params ep, int* __restrict__ err) {
    constexpr int BN = Epi::BN;
    constexpr int STAGES = Epi::STAGES;
    constexpr int BOX_B = Epi::BOX_B;
    constexpr int NSUB = BN <= 256 ? 1 : 2;      // MMA instructions per K step (N <= 256 each)
    constexpr int SUBN = BN / NSUB;
    constexpr bool SPLIT = Epi::SPLIT;
    constexpr int PL = planes<Epi>();
    constexpr int MSUB = Epi::MSUB;  // 128-row sub-tiles of A sharing every B stage
    constexpr int BKC = Epi::BKC;    // K elements per ring stage
    constexpr uint32_t A_BYTES = (uint32_t)MSUB * kTileM * BKC * 2;  // per plane
    constexpr uint32_t B_BYTES = (uint32_t)BN * BKC * 2;             // per plane
    constexpr uint32_t MNBOX = 64u * BKC * 2;  // one 64 (MN) x BKC (K) box of an MN-major operand
    constexpr uint32_t STAGE_BYTES = PL * (A_BYTES + B_BYTES);  // [A planes][B planes]
    constexpr uint32_t TMEM_COLS = tmem_cols_for(MSUB * BN);
    constexpr bool A_MN = Epi::A_MN, B_MN = Epi::B_MN;
    constexpr uint32_t IDESC = idesc_bf16(kTileM, SUBN, A_MN, B_MN);
    static_assert(BKC == kChunkK || BKC == 32, "64- or 32-wide K stages");
    static_assert(BKC == kChunkK || (A_MN && B_MN) || (!A_MN && !B_MN && MSUB == 1 && BN <= 256),
                  "32-wide K stages: both operands MN-major, or both K-major (64-byte rows)");
    constexpr uint32_t KROW = (uint32_t)BKC * 2;  // bytes per row of a K-major operand stage
    static_assert(MSUB == 1 || (A_MN && MSUB == 2 && MSUB * BN <= 512), "two A sub-tiles: MN-major, <= 512 columns");
    static_assert(BN % 16 == 0 && SUBN % 16 == 0 && SUBN <= 256, "MMA N must be a multiple of 16, <= 256");
    static_assert(BN % BOX_B == 0 && BOX_B <= 256 && (BOX_B * 128) % 1024 == 0, "bad B box");
    static_assert(!B_MN || SUBN % 64 == 0, "an MN-major B tile is made of 64-wide boxes");
    constexpr int E_BOXES = Epi::E_BOXES;
    constexpr uint32_t TILE_REGION = tile_region_bytes<Epi>();
    static_assert(E_BOXES * PL <= 8 && Epi::O_BOXES * PL <= 8, "at most 8 boxes of epilogue operand / output");
    static_assert(!SPLIT || B_MN || BOX_B == BN, "a split K-major B tile is one box");
    static_assert(Epi::XROUNDS == 0, "row exchanges run in the persistent form");
    // epilogue passes over column slices of the tile: EB operand boxes, OB output boxes and XC
    // trailing-product K chunks (64 atoms each) per pass
    constexpr int EPASS = Epi::EPASS;
    constexpr int EB = E_BOXES / EPASS, OB = Epi::O_BOXES / EPASS;
    static_assert(EPASS == 1 || (EPASS == 2 && E_BOXES % 2 == 0 && Epi::O_BOXES % 2 == 0 && MSUB == 1),
                  "one or two epilogue passes");
    // trailing product: staged output (K-major, 64 columns per box) x tmX (MN-major 64 x 64 boxes)
    constexpr int XN = Epi::XPROD;
    constexpr int XC = BN / 64 / EPASS;
    constexpr uint32_t X_BOX = 64u * 64u * 2u;  // one 64 (N) x 64 (K) box per plane
    constexpr uint32_t X_OFF = (uint32_t)(EB > OB ? EB : OB) * PL * kTileABytes;
    static_assert(XN == 0 || (XN == 64 && MSUB == 1 && !A_MN && Epi::O_BOXES * 64 == BN && BN <= 256 &&
                              X_OFF + xprod_bytes<Epi>() <= TILE_REGION),
                  "a trailing product multiplies the whole staged tile by a 64-column operand");
    constexpr uint32_t XDESC = idesc_bf16(kTileM, XN > 0 ? XN : 64, false, true);
    // second trailing product: (staged output)^T x tmX2's tile, 128 output columns per group
    constexpr int X2 = Epi::XPROD2;
    constexpr int X2G = BN / EPASS / 128;                        // groups per pass
    constexpr uint32_t X2_BYTES = (uint32_t)PL * kTileM * 128;  // 128 rows x 64 BF16 per plane
    constexpr uint32_t X2DESC = idesc_bf16(kTileM, 64, true, true);
    static_assert(X2 == 0 || (XN == 64 && BN % (128 * EPASS) == 0 && X2_BYTES <= xprod_bytes<Epi>() &&
                              64 + 64 * EPASS * X2G <= (int)tmem_cols_for(MSUB * BN)),
                  "the second trailing product reuses the first one's operand space and free TMEM columns");
    constexpr bool X2PRE = x2_pre_bytes<Epi>() > 0;  // its B tile preloaded into a region of its own
    constexpr uint32_t Q_OFF = X2PRE ? TILE_REGION : X_OFF;
    static_assert(X2 == 0 || xprod_bytes<Epi>() >= 32768, "run_x's staging space is the first product's operand");

    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t* bar_base = smem + TILE_REGION;
    if constexpr (X2PRE)  // compact layout (see gemm_smem_bytes)
        bar_base = smem - smem_raw >= 256 ? smem - 256 : smem + TILE_REGION + x2_pre_bytes<Epi>();
    uint64_t* full = reinterpret_cast<uint64_t*>(bar_base);
    uint64_t* empty = full + STAGES;
    uint64_t* accum = empty + STAGES;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accum + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    volatile int* decision = abort_flag + 1;
    uint64_t* ebar = reinterpret_cast<uint64_t*>(tmem_slot + 4);  // 8-byte aligned, 8 barriers
    uint64_t* x_loaded = ebar + 8;  // trailing product: its B operand arrived
    uint64_t* x_staged = ebar + 9;  //   the staged output is complete
    uint64_t* x_done = ebar + 10;   //   its MMAs have completed
    uint64_t* p_free = ebar + 11;   // epilogue pass: its staged output has been read by its stores
    uint64_t* q_loaded = ebar + 12;  // second trailing product: its B operand arrived
    uint64_t* k_done = ebar + 13;    //   its MMAs have completed
    float* scratch = X2PRE ? nullptr : reinterpret_cast<float*>(smem + TILE_REGION + 256);
    static_assert(STAGES * 16 + 8 + 16 + 14 * 8 <= 256, "barriers fit their 256 bytes");
    bool x_on = false, x2_on = false;
    if constexpr (XN > 0) x_on = Epi::x_active(ep);
    if constexpr (X2 > 0) x2_on = x_on && Epi::x2_active(ep);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * MSUB * kTileM;
    const int n0 = blockIdx.y * BN;
    const int k_begin = blockIdx.z * g.chunks_per_z;
    const int k_end = min(g.k_chunks, k_begin + g.chunks_per_z);
    const int nk = k_end - k_begin;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(accum, 1);
        for (int b = 0; b < E_BOXES; ++b) mbar_init(&ebar[b], 1);
        if (XN > 0) {
            mbar_init(x_loaded, 1);
            mbar_init(x_staged, 1);
            mbar_init(x_done, 1);
        }
        if (X2 > 0) {
            mbar_init(q_loaded, 1);
            mbar_init(k_done, 1);
        }
        if (EPASS > 1) mbar_init(p_free, 1);
        *abort_flag = 0;
        fence_mbar_init();
        prefetch_tmap(&tmA);
        prefetch_tmap(&tmB);
    }
    if (warp == 1) tmem_alloc(tmem_slot, TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            // ---- TMA producer ----
            if (X2 > 0 && x2_on) {  // the second trailing product's tile: loaded now, or to L2 now
                if (X2PRE) {
                    mbar_expect_tx(q_loaded, X2_BYTES);
                    tma_load(smem + Q_OFF, &tmX2, q_loaded, 0, m0, SPLIT ? 0 : -1);
                } else if (SPLIT) {
                    tma_prefetch_3d(&tmX2, 0, m0, 0);
                } else {
                    tma_prefetch_2d(&tmX2, 0, m0);
                }
            }
            int issued = 0;
            for (int i = 0; i < nk; ++i) {
                const int s = i % STAGES;
                const uint32_t ph = (uint32_t)(i / STAGES) & 1u;
                if (i >= STAGES && !mbar_wait(&empty[s], ph ^ 1u, abort_flag)) {
                    *abort_flag = 1;
                    break;
                }
                const int kx = (k_begin + i) * BKC;
                mbar_expect_tx(&full[s], STAGE_BYTES);
                uint8_t* sa = smem + s * STAGE_BYTES;
                uint8_t* sb = sa + PL * A_BYTES;
                if (SPLIT) {
                    // one box holds both planes: K-major [plane][row][128 B] (3D), MN-major B
                    // [plane][block][K row][128 B] (4D); an MN-major A loads each plane's blocks
                    if (A_MN) {
#pragma unroll
                        for (int z = 0; z < 2; ++z)
#pragma unroll
                            for (int b = 0; b < MSUB * kTileM / 64; ++b)
                                tma_load_3d(sa + z * A_BYTES + b * MNBOX, &tmA, &full[s], m0 + 64 * b, kx, z);
                    } else {
                        tma_load_3d(sa, &tmA, &full[s], kx, m0, 0);
                    }
                    if (B_MN)
                        tma_load_4d(sb, &tmB, &full[s], 0, kx, n0 / 64, 0);
                    else
                        tma_load_3d(sb, &tmB, &full[s], kx, n0, 0);
                } else {
                    if (A_MN) {
#pragma unroll
                        for (int b = 0; b < MSUB * kTileM / 64; ++b)
                            tma_load_2d(sa + b * MNBOX, &tmA, &full[s], m0 + 64 * b, kx);
                    } else {
                        tma_load_2d(sa, &tmA, &full[s], kx, m0);
                    }
                    if (B_MN) {
#pragma unroll
                        for (int b = 0; b < BN / 64; ++b)
                            tma_load_2d(sb + b * MNBOX, &tmB, &full[s], n0 + 64 * b, kx);
                    } else {
#pragma unroll
                        for (int b = 0; b < BN / BOX_B; ++b)
                            tma_load_2d(sb + b * BOX_B * 128, &tmB, &full[s], kx, n0 + b * BOX_B);
                    }
                }
                ++issued;
            }
            // never leave the CTA with copies in flight: drain the stages still being filled
            if (*abort_flag) {
                for (int i = max(0, issued - STAGES); i < issued; ++i)
                    (void)mbar_wait(&full[i % STAGES], (uint32_t)(i / STAGES) & 1u, nullptr);
            } else if (E_BOXES > 0) {
                // the pipeline buffers are free once every MMA has completed: bring in the
                // epilogue operand rows of this tile
                if (mbar_wait(accum, 0, abort_flag) && !*abort_flag) {
                    prefetch_tmap(&tmE);
                    for (int h = 0; h < EPASS; ++h) {
                        // a second product whose tile shares the first one's operand space runs
                        // first in the later passes, on the tile pass 0 left there
                        const bool swap = X2 > 0 && !X2PRE && x2_on && h > 0;
                        // pass h reuses pass h - 1's buffers once its stores and products read them
                        if (h > 0 && (!mbar_wait(p_free, (uint32_t)(h - 1) & 1u, abort_flag) ||
                                      (XN > 0 && x_on && !mbar_wait(x_done, (uint32_t)(h - 1) & 1u, abort_flag)) ||
                                      (X2 > 0 && x2_on && !mbar_wait(k_done, (uint32_t)(h - 1) & 1u, abort_flag)))) {
                            *abort_flag = 1;
                            break;
                        }
                        for (int b = 0; b < EB; ++b) {
                            mbar_expect_tx(&ebar[b], PL * kTileM * 128);
                            for (int z = 0; z < PL; ++z)
                                tma_load(smem + (z * EB + b) * (kTileM * 128), &tmE, &ebar[b], n0 + 64 * (h * EB + b),
                                         m0, SPLIT ? z : -1);
                        }
                        auto load_x = [&]() {
                            // the trailing product's B rows of the pass (both planes per box when split)
                            mbar_expect_tx(x_loaded, xprod_bytes<Epi>());
                            for (int c = 0; c < XC; ++c) {
                                uint8_t* dst = smem + X_OFF + c * PL * X_BOX;
                                if (SPLIT)
                                    tma_load_4d(dst, &tmX, x_loaded, 0, n0 + 64 * (h * XC + c), 0, 0);
                                else
                                    tma_load_2d(dst, &tmX, x_loaded, 0, n0 + 64 * (h * XC + c));
                            }
                        };
                        if (XN > 0 && x_on && !swap) load_x();
                        for (int b = 0; b < EB; ++b) (void)mbar_wait(&ebar[b], (uint32_t)h & 1u, nullptr);
                        if (XN > 0 && x_on && !swap) (void)mbar_wait(x_loaded, (uint32_t)h & 1u, nullptr);
                        if (X2 > 0 && !X2PRE && x2_on) {
                            // pass 0: the first product has read its operand, the second's tile
                            // takes its place (both planes in one box when split); later passes:
                            // the second product has read the tile, the first one's operand returns
                            if (!mbar_wait(swap ? k_done : x_done, (uint32_t)h & 1u, abort_flag)) {
                                *abort_flag = 1;
                                break;
                            }
                            if (swap) {
                                load_x();
                                (void)mbar_wait(x_loaded, (uint32_t)h & 1u, nullptr);
                            } else {
                                mbar_expect_tx(q_loaded, X2_BYTES);
                                tma_load(smem + X_OFF, &tmX2, q_loaded, 0, m0, SPLIT ? 0 : -1);
                                (void)mbar_wait(q_loaded, 0, nullptr);
                            }
                        }
                    }
                } else {
                    *abort_flag = 1;
                }
            }
            if (X2 > 0 && X2PRE && x2_on) (void)mbar_wait(q_loaded, 0, nullptr);  // no copy left in flight
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---- MMA issuer ----
            bool ok = true;
            for (int i = 0; i < nk && ok; ++i) {
                const int s = i % STAGES;
                const uint32_t ph = (uint32_t)(i / STAGES) & 1u;
                if (!mbar_wait(&full[s], ph, abort_flag)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t sa = smem_u32(smem + s * STAGE_BYTES);  // A hi (then A lo)
                const uint32_t sb = sa + PL * A_BYTES;                 // B hi (then B lo)
                auto kdesc = [&](uint32_t a) { return KROW == 128 ? sw128_desc(a) : sw64_desc(a); };
                auto adesc = [&](uint32_t base, int ms, int kk) {
                    return A_MN ? mn128_desc(base + (uint32_t)(ms * 2) * MNBOX + kk * 16 * 128, MNBOX)
                                : kdesc(base + kk * 32);
                };
                auto bdesc = [&](uint32_t base, int j, int kk) {
                    return B_MN ? mn128_desc(base + (uint32_t)(j * (SUBN / 64)) * MNBOX + kk * 16 * 128, MNBOX)
                                : kdesc(base + (uint32_t)j * SUBN * KROW + kk * 32);
                };
#pragma unroll
                for (int kk = 0; kk < BKC / 16; ++kk) {
#pragma unroll
                    for (int ms = 0; ms < MSUB; ++ms) {
                        const uint64_t da = adesc(sa, ms, kk), dal = adesc(sa + A_BYTES, ms, kk);
#pragma unroll
                        for (int j = 0; j < NSUB; ++j)
                            mma_step<SPLIT>(tmem_base + (uint32_t)(ms * BN + j * SUBN), da, dal, bdesc(sb, j, kk),
                                            bdesc(sb + B_BYTES, j, kk), IDESC, (i > 0 || kk > 0) ? 1u : 0u);
                    }
                }
                mma_commit(&empty[s]);  // frees the stage once these MMAs have read it
            }
            if (!ok) *abort_flag = 1;
            mma_commit(accum);  // accumulator complete (or the pipeline was abandoned)
            if (XN > 0 && x_on) {
                // trailing product into columns 0 .. XN - 1, once the epilogue has read them
                // (x_staged) and the pass's staged slice and B operand are in shared memory;
                // each pass adds its K (atoms) slice into the same accumulator
                auto first = [&](int h, bool go) {
                    if (go) {
                        tc_fence_after();
                        const uint32_t so = smem_u32(smem);         // staged output, hi plane (then lo)
                        const uint32_t sx = smem_u32(smem + X_OFF);  // B boxes [c][plane]
                        constexpr uint32_t OPL = (uint32_t)OB * kTileABytes;
#pragma unroll
                        for (int c = 0; c < XC; ++c)
#pragma unroll
                            for (int kk = 0; kk < 4; ++kk) {
                                const uint32_t oa = so + (uint32_t)c * kTileABytes + kk * 32;
                                const uint32_t ob = sx + (uint32_t)c * PL * X_BOX + kk * 16 * 128;
                                mma_step<SPLIT>(tmem_base, sw128_desc(oa), sw128_desc(oa + OPL), mn128_desc(ob, X_BOX),
                                                mn128_desc(ob + X_BOX, X_BOX), XDESC,
                                                (h > 0 || c > 0 || kk > 0) ? 1u : 0u);
                            }
                    }
                    mma_commit(x_done);  // at once when nothing was issued
                };
                // (staged output)^T x tile: group G of 128 output columns (two 64-column boxes,
                // MN-major) over the tile's 128 rows into TMEM columns 64 + 64 G
                auto second = [&](int h, bool go) {
                    if (go) {
                        tc_fence_after();
                        const uint32_t so = smem_u32(smem);
                        const uint32_t sq = smem_u32(smem + Q_OFF);
                        constexpr uint32_t OPL = (uint32_t)OB * kTileABytes;
#pragma unroll
                        for (int gi = 0; gi < X2G; ++gi)
#pragma unroll
                            for (int kk = 0; kk < kTileM / 16; ++kk) {
                                const uint32_t oa = so + (uint32_t)(2 * gi) * kTileABytes + kk * 16 * 128;
                                const uint32_t qb = sq + kk * 16 * 128;
                                mma_step<SPLIT>(tmem_base + 64u + 64u * (uint32_t)(h * X2G + gi),
                                                mn128_desc(oa, kTileABytes), mn128_desc(oa + OPL, kTileABytes),
                                                mn128_desc(qb), mn128_desc(qb + kTileM * 128), X2DESC,
                                                kk > 0 ? 1u : 0u);
                            }
                    }
                    mma_commit(k_done);  // at once when nothing was issued
                };
                for (int h = 0; h < EPASS; ++h) {
                    const uint32_t ph = (uint32_t)h & 1u;
                    if (X2 > 0 && !X2PRE && x2_on && h > 0) {
                        // later passes: the second product first, on the tile pass 0 left in the
                        // operand space, then the first one once its operand has replaced it
                        const bool go2 = ok && mbar_wait(x_staged, ph, abort_flag) && !*abort_flag;
                        second(h, go2);
                        first(h, go2 && mbar_wait(x_loaded, ph, abort_flag) && !*abort_flag);
                        continue;
                    }
                    const bool go = ok && mbar_wait(x_loaded, ph, abort_flag) && mbar_wait(x_staged, ph, abort_flag) &&
                                    !*abort_flag;
                    first(h, go);
                    if (X2 > 0 && x2_on) second(h, go && mbar_wait(q_loaded, 0, abort_flag) && !*abort_flag);
                }
            }
        }
    } else {
        // ---- epilogue warps ----
        const bool ready = mbar_wait(accum, 0, abort_flag);
        tc_fence_after();
        const int quarter = warp & 3;
        const int group = (warp - 2) >> 2;
        const int row = quarter * 32 + lane;
        if (!ready) *abort_flag = 1;
        // one CTA-uniform decision, taken by one thread: the epilogue's TMEM loads are
        // warp-collective and its row reductions synchronise all epilogue warps
        epi_sync(128 * Epi::EPI_WG);
        if (threadIdx.x == 64) *decision = (nk > 0 && !*abort_flag) ? 1 : 0;
        epi_sync(128 * Epi::EPI_WG);
        EpiCtx ec{tmem_base + ((uint32_t)(quarter * 32) << 16), row, m0, n0, (int)blockIdx.z, group, scratch,
                  E_BOXES > 0 ? smem : nullptr, smem, ebar, abort_flag, 0, 1, nullptr, nullptr};
        if (SPLIT) {
            ec.eplane = (uint32_t)EB * kTileM * 128;
            ec.oplane = (uint32_t)OB * kTileABytes;
        }
        int any_boxes = 0;
        for (int h = 0; h < EPASS; ++h) {
            ec.col0 = h * (BN / EPASS);
            ec.ephase = (uint32_t)h & 1u;
            int out_boxes = 0;
            if (*decision) out_boxes = Epi::run(ep, ec);
            any_boxes |= out_boxes;
            if (Epi::O_BOXES > 0) {
                // the staged output slice goes out through the TMA once every epilogue thread
                // wrote its part (coalesced and asynchronous, instead of one row per thread)
                fence_proxy_async();
                if (XN > 0) tc_fence_before();  // this thread's TMEM reads precede the trailing product
                epi_sync(128 * Epi::EPI_WG);
                if (threadIdx.x == 64) {
                    if (XN > 0 && x_on) mbar_arrive(x_staged);  // the slice is staged (or abandoned)
                    if (out_boxes > 0 && !*abort_flag && !x2_on) {  // (consumed on chip otherwise)
                        for (int b = 0; b < out_boxes && b < OB; ++b)
                            for (int z = 0; z < PL; ++z)
                                tma_store(&tmO, smem + (z * OB + b) * kTileABytes, n0 + ec.col0 + 64 * b, m0,
                                          SPLIT ? z : -1);
                        bulk_commit();
                        bulk_wait_read();  // shared memory stays valid until the copies have read it
                    }
                    if (EPASS > 1) mbar_arrive(p_free);  // the next pass may refill the buffers
                }
            }
        }
        if constexpr (XN > 0) {
            if (x_on) {
                if (!mbar_wait(x_done, (uint32_t)(EPASS - 1) & 1u, abort_flag)) *abort_flag = 1;
                // one CTA-uniform decision again: run_x's TMEM loads are warp-collective
                epi_sync(128 * Epi::EPI_WG);
                if (threadIdx.x == 64) *decision = (*decision && any_boxes > 0 && !*abort_flag) ? 1 : 0;
                epi_sync(128 * Epi::EPI_WG);
                tc_fence_after();
                // the first product's operand space is free once its last pass completed (with a
                // second product, that one completed before: preloaded, or run first in that pass)
                if (X2 > 0 && x2_on && (X2PRE || EPASS > 1)) ec.xstage = smem + X_OFF;
                if (*decision) Epi::run_x(ep, ec);
                if constexpr (X2 > 0) {
                    if (x2_on) {
                        if (!mbar_wait(k_done, (uint32_t)(EPASS - 1) & 1u, abort_flag)) *abort_flag = 1;
                        epi_sync(128 * Epi::EPI_WG);
                        if (threadIdx.x == 64) *decision = (*decision && !*abort_flag) ? 1 : 0;
                        epi_sync(128 * Epi::EPI_WG);
                        tc_fence_after();
                        if (*decision) Epi::run_k(ep, ec, (int)blockIdx.x);
                    }
                }
            }
        }
        tc_fence_before();
    }
    __syncthreads();
    if (*abort_flag && threadIdx.x == 0) atomicExch(err, 1);
    // an abandoned pipeline may still have MMAs in flight: let them finish before freeing TMEM
    if (*abort_flag && warp == 1 && lane == 0) {
        (void)mbar_wait(accum, 0, nullptr);
        if (XN > 0 && x_on) {
            // the trailing products' MMAs too: one more commit tracks everything this thread issued
            mma_commit(accum);
            (void)mbar_wait(accum, 1, nullptr);
        }
    }
    __syncwarp();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem_base, TMEM_COLS);
    }
}


// ---- persistent form ----------------------------------------------------------------------
//
// One CTA per SM (or one cluster of CTAs along y per group of SMs) walks the 128-row tiles
// blockIdx.x, blockIdx.x + gridDim.x, ...  Two TMEM accumulators of BN columns alternate
// between tiles, so the MMAs of tile t+1 run while the epilogue of tile t drains the other
// accumulator; the operand ring runs on across tiles.  The epilogue operand and the staged
// output of a tile share one of two box buffers: for tile t a second producer thread sends the
// staged output of tile t-2 out of buffer t % 2 with TMA stores, waits until they have read it,
// and loads the epilogue operand of tile t there, while the epilogue works on tile t-1 from the
// other buffer.
//
// Warp roles (96 + 128 G threads): warp 0 queues the operand ring, warp 1 owns TMEM and issues
// the MMAs, warp 2 moves the box buffers (stores out, epilogue operands in), warps 3.. run the
// epilogue (thread 96 leads it).
//
// Barriers (phase parity in brackets; lt = this CTA's tile counter, it = k-chunk counter,
// e = lt & 1, u = lt >> 1):
//   full[s] / empty[s]   operand ring                                  [(it / STAGES) & 1]
//   acc_full[e]          MMAs of tile lt done -> epilogue              [u & 1]
//   acc_empty[e]         epilogue done reading TMEM -> MMA (tile lt+2) [(u - 1) & 1]
//   e_full[e][k]         epilogue operand box k of tile lt loaded      [u & 1]
//   e_free[e]            buffer e free for tile lt's output (no operand) [u & 1]
//   staged[e]            output of tile lt staged in buffer e          [u & 1]
//   xbar[e]              cluster row exchange of tile lt               [u & 1]
struct PersistGrid {
    int k_chunks;   // Epi::BK-wide K chunks per tile
    int row_tiles;  // 128-row tiles of A
};

template <class Epi>
__host__ __device__ constexpr uint32_t persist_box_bytes() {  // one box buffer
    // in place (split): the eight 16 KB operand chunks of one tile fill both buffers
    return Epi::INPLACE ? 4 * kTileABytes
                        : (uint32_t)(Epi::E_BOXES > Epi::O_BOXES ? Epi::E_BOXES : Epi::O_BOXES) * kTileABytes;
}

// One ring stage: A (128 x BK) and B (BN x BK) elements of Epi::ELEM bytes (2: BF16, 1: E4M3),
// each in both planes in the split form ([A hi][A lo][B hi][B lo]).
template <class Epi>
__host__ __device__ constexpr uint32_t persist_stage_bytes() {
    return (uint32_t)planes<Epi>() * (kTileM + Epi::BN) * Epi::BK * Epi::ELEM;
}

__host__ __device__ constexpr int persist_threads(int epi_warpgroups) { return 96 + 128 * epi_warpgroups; }

template <class Epi>
__host__ __device__ constexpr size_t persist_smem_bytes() {
    return (size_t)Epi::STAGES * persist_stage_bytes<Epi>() + 2 * persist_box_bytes<Epi>() +
           1024 /* alignment */ + 512 /* barriers */ + scratch_bytes(Epi::EPI_WG) +
           (Epi::XROUNDS > 0 ? 2 * kXchgBytes : 0);  // one exchange buffer per accumulator
}

template <class Epi>
__global__ void __launch_bounds__(persist_threads(Epi::EPI_WG), 1)
    tc_persist_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                      const __grid_constant__ CUtensorMap tmE, const __grid_constant__ CUtensorMap tmO,
                      PersistGrid pg, typename Epi::Params ep, int* __restrict__ err) {
    constexpr int BN = Epi::BN;
    constexpr int STAGES = Epi::STAGES;
    constexpr int BOX_B = Epi::BOX_B;
    constexpr int G = Epi::EPI_WG;
    constexpr int BK = Epi::BK;      // K elements per chunk
    constexpr int ELEM = Epi::ELEM;  // 2: BF16 operands (kind::f16), 1: E4M3 (kind::f8f6f4)
    constexpr int ROWB = BK * ELEM;  // bytes per K-major row: 128, 64 or 32 (that swizzle)
    constexpr bool SPLIT = Epi::SPLIT;
    constexpr int PL = planes<Epi>();
    constexpr uint32_t A_BYTES = (uint32_t)kTileM * ROWB;          // per plane
    constexpr uint32_t B_BYTES = (uint32_t)Epi::BN * BK * ELEM;    // per plane
    constexpr uint32_t STAGE_BYTES = persist_stage_bytes<Epi>();
    constexpr uint32_t PIPE_BYTES = STAGES * STAGE_BYTES;
    constexpr uint32_t MN_BOX = 64u * BK * 2;  // one 64 (MN) x BK (K) box of an MN-major operand
    constexpr uint32_t BOX_BYTES = persist_box_bytes<Epi>();
    constexpr bool A_MN = Epi::A_MN, B_MN = Epi::B_MN;
    constexpr uint32_t IDESC = ELEM == 1 ? idesc_e4m3(kTileM, BN) : idesc_bf16(kTileM, BN, A_MN, B_MN);
    constexpr int E_BOXES = Epi::E_BOXES, O_BOXES = Epi::O_BOXES;
    static_assert(BN % 16 == 0 && BN <= 256, "two accumulators of BN <= 256 columns fill TMEM");
    static_assert(ELEM == 2 || (ELEM == 1 && !B_MN), "E4M3 operands are read K-major");
    static_assert(BN % BOX_B == 0 && BOX_B <= 256 && (BOX_B * 128) % 1024 == 0, "bad B box");
    static_assert(!B_MN || BN % 64 == 0, "an MN-major B tile is made of 64-wide boxes");
    constexpr bool INPLACE = Epi::INPLACE;  // split: FP32 operand chunks in, output over them
    static_assert((E_BOXES <= 4 || INPLACE) && O_BOXES <= 4 && Epi::XROUNDS <= 1 && G <= 4, "epilogue shape");
    static_assert(ROWB == 128 || ROWB == 64 || ROWB == 32, "K chunk rows of 128, 64 or 32 bytes");
    static_assert(!A_MN, "the persistent tile reads A K-major");
    static_assert(!SPLIT || (ELEM == 2 && (E_BOXES == 0 || INPLACE)), "split form: BF16 planes");
    static_assert(!INPLACE || (SPLIT && E_BOXES == 8 && 2 * BOX_BYTES == 8 * 16384), "in-place chunks fill both buffers");
    static_assert(!SPLIT || B_MN || BOX_B == BN, "a split K-major B tile is one box");
    static_assert(STAGE_BYTES % 1024 == 0 && A_BYTES % 1024 == 0, "stages stay 1024-byte aligned");

    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t* boxes = smem + PIPE_BYTES;  // [2][BOX_BYTES]
    uint64_t* bars = reinterpret_cast<uint64_t*>(boxes + 2 * BOX_BYTES);
    uint64_t* full = bars;                // [STAGES]
    uint64_t* empty = full + STAGES;      // [STAGES]
    uint64_t* acc_full = empty + STAGES;  // [2]
    uint64_t* acc_empty = acc_full + 2;   // [2]
    uint64_t* e_full = acc_empty + 2;     // [2][4]
    uint64_t* e_free = e_full + 8;        // [2]
    uint64_t* staged = e_free + 2;        // [2]
    uint64_t* xbars = staged + 2;         // [2]
    uint64_t* drain = xbars + 2;          // [1]
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(drain + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    volatile int* decision = abort_flag + 1;
    volatile int* nbox = decision + 1;  // [2]: output boxes staged in each buffer
    float* scratch = reinterpret_cast<float*>(reinterpret_cast<uint8_t*>(bars) + 512);
    float* xbufs = scratch + scratch_bytes(G) / 4;

    uint32_t csize = 1;
    if (Epi::XROUNDS > 0) asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(csize));
    const uint32_t crank = csize > 1 ? cluster_rank() : 0u;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n0 = blockIdx.y * BN;
    const int nk = pg.k_chunks;
    const int first = blockIdx.x, stride = gridDim.x;
    const int my_tiles = first < pg.row_tiles ? (pg.row_tiles - first + stride - 1) / stride : 0;

    if (threadIdx.x == 0) {
        for (int i = 0; i < STAGES; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        for (int e = 0; e < 2; ++e) {
            mbar_init(&acc_full[e], 1);
            mbar_init(&acc_empty[e], 1);
            for (int b = 0; b < (INPLACE ? 4 : E_BOXES); ++b) mbar_init(&e_full[4 * e + b], 1);
            mbar_init(&e_free[e], 1);
            mbar_init(&staged[e], 1);
            if (csize > 1) mbar_init(&xbars[e], 1);  // this CTA's expect-tx arrival
        }
        mbar_init(drain, 1);
        *abort_flag = 0;
        fence_mbar_init();
        prefetch_tmap(&tmA);
        prefetch_tmap(&tmB);
        if (E_BOXES > 0) prefetch_tmap(&tmE);
        if (O_BOXES > 0) prefetch_tmap(&tmO);
    }
    if (warp == 1) tmem_alloc(tmem_slot, 512);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (csize > 1) cluster_sync_all();
    const uint32_t tmem_base = *tmem_slot;

    if (warp == 0) {
        if (lane == 0 && nk > 0) {
            // ---- TMA producer: operand ring ----
            int it = 0;
            bool ok = true;
            for (int lt = 0; lt < my_tiles && ok; ++lt) {
                const int m0 = (first + lt * stride) * kTileM;
                // the next tile's A rows go to L2 now, so that its ring refills at L2 latency
                if (lt + 1 < my_tiles)
                    for (int i = 0; i < nk; ++i) {
                        if (SPLIT)
                            tma_prefetch_3d(&tmA, i * BK, m0 + stride * kTileM, 0);  // both planes
                        else
                            tma_prefetch_2d(&tmA, i * BK, m0 + stride * kTileM);
                    }
                for (int i = 0; i < nk; ++i, ++it) {
                    const int s = it % STAGES;
                    if (it >= STAGES && !mbar_wait(&empty[s], ((uint32_t)(it / STAGES) & 1u) ^ 1u, abort_flag)) {
                        ok = false;
                        break;
                    }
                    const int kx = i * BK;
                    mbar_expect_tx(&full[s], STAGE_BYTES);
                    uint8_t* sa = smem + s * STAGE_BYTES;
                    uint8_t* sb = sa + PL * A_BYTES;
                    if (SPLIT) {  // one box holds both planes (see tc_gemm_kernel)
                        tma_load_3d(sa, &tmA, &full[s], kx, m0, 0);
                        if (B_MN)
                            tma_load_4d(sb, &tmB, &full[s], 0, kx, n0 / 64, 0);
                        else
                            tma_load_3d(sb, &tmB, &full[s], kx, n0, 0);
                    } else {
                        tma_load_2d(sa, &tmA, &full[s], kx, m0);
                        if (B_MN) {
#pragma unroll
                            for (int b = 0; b < BN / 64; ++b)
                                tma_load_2d(sb + b * MN_BOX, &tmB, &full[s], n0 + 64 * b, kx);
                        } else {
#pragma unroll
                            for (int b = 0; b < BN / BOX_B; ++b)
                                tma_load_2d(sb + b * BOX_B * ROWB, &tmB, &full[s], kx, n0 + b * BOX_B);
                        }
                    }
                }
            }
            if (!ok) {
                *abort_flag = 1;
                // never leave the CTA with copies in flight
                for (int j = max(0, it - STAGES); j < it; ++j)
                    (void)mbar_wait(&full[j % STAGES], (uint32_t)(j / STAGES) & 1u, nullptr);
            }
        }
    } else if (warp == 2 && INPLACE) {
        if (lane == 0 && nk > 0) {
            // ---- in-place split form: the FP32 operand chunks of tile t are loaded once the
            // stores of tile t - 1 (written over its chunks) have read them ----
            bool ok = true;
            int loaded = -1;
            auto store_tile = [&](int t) -> bool {
                if (!mbar_wait(&staged[0], (uint32_t)t & 1u, abort_flag)) return false;
                const int nb = nbox[0];
                const int m0t = (first + t * stride) * kTileM;
                for (int c = 0; c < 2 * nb && c < 8; ++c) {
                    tma_store_3d(&tmO, boxes + c * 16384, n0 + 32 * c, m0t, 0);
                    tma_store_3d(&tmO, boxes + c * 16384 + 8192, n0 + 32 * c, m0t, 1);
                }
                bulk_commit();
                bulk_wait_read();
                return true;
            };
            for (int t = 0; t < my_tiles && ok; ++t) {
                if (t >= 1 && !store_tile(t - 1)) {
                    ok = false;
                    break;
                }
                const int m0t = (first + t * stride) * kTileM;
                for (int c = 0; c < 8; ++c) {
                    mbar_expect_tx(&e_full[c], 16384);
                    tma_load_2d(boxes + c * 16384, &tmE, &e_full[c], n0 + 32 * c, m0t);
                }
                loaded = t;
            }
            if (ok && my_tiles > 0) ok = store_tile(my_tiles - 1);
            if (!ok) {
                *abort_flag = 1;
                if (loaded >= 0)  // never leave the CTA with copies in flight
                    for (int c = 0; c < 8; ++c) (void)mbar_wait(&e_full[c], (uint32_t)loaded & 1u, nullptr);
                bulk_wait_read();
            }
        }
    } else if (warp == 2 && SPLIT) {
        if (lane == 0 && nk > 0) {
            // ---- split form: one staged output per tile, its hi plane in buffer 0 and its lo
            // plane in buffer 1; tile t + 1 stages once the stores of tile t have read them ----
            bool ok = true;
            mbar_arrive(&e_free[0]);  // tile 0 may stage
            for (int t = 0; t < my_tiles && ok; ++t) {
                if (!mbar_wait(&staged[0], (uint32_t)t & 1u, abort_flag)) {
                    ok = false;
                    break;
                }
                const int nb = nbox[0];
                const int m0t = (first + t * stride) * kTileM;
                for (int b = 0; b < nb && b < O_BOXES; ++b) {
                    tma_store_3d(&tmO, boxes + b * kTileABytes, n0 + 64 * b, m0t, 0);
                    tma_store_3d(&tmO, boxes + BOX_BYTES + b * kTileABytes, n0 + 64 * b, m0t, 1);
                }
                bulk_commit();
                bulk_wait_read();
                mbar_arrive(&e_free[0]);  // tile t + 1 may stage
            }
            if (!ok) {
                *abort_flag = 1;
                bulk_wait_read();
            }
        }
    } else if (warp == 2) {
        if (lane == 0 && nk > 0) {
            // ---- box buffers: staged outputs out, epilogue operands in ----
            int stored = 0, e_issued = -1;
            bool ok = true;
            // send the staged output of tile t (its buffer is t & 1) and wait until it was read
            auto store_tile = [&](int t) -> bool {
                if (!mbar_wait(&staged[t & 1], (uint32_t)(t >> 1) & 1u, abort_flag)) return false;
                const int nb = nbox[t & 1];
                const int m0t = (first + t * stride) * kTileM;
                for (int b = 0; b < nb && b < O_BOXES; ++b)
                    tma_store_2d(&tmO, boxes + (t & 1) * BOX_BYTES + b * kTileABytes, n0 + 64 * b, m0t);
                bulk_commit();
                bulk_wait_read();
                return true;
            };
            for (int lt = 0; lt < my_tiles && ok; ++lt) {
                // buffer lt & 1 last held tile lt - 2
                if (lt >= 2) {
                    if (!store_tile(lt - 2)) {
                        ok = false;
                        break;
                    }
                    stored = lt - 1;
                }
                const int e = lt & 1;
                if (E_BOXES > 0) {
                    const int m0 = (first + lt * stride) * kTileM;
                    for (int b = 0; b < E_BOXES; ++b) {
                        mbar_expect_tx(&e_full[4 * e + b], kTileABytes);
                        tma_load_2d(boxes + e * BOX_BYTES + b * kTileABytes, &tmE, &e_full[4 * e + b], n0 + 64 * b,
                                    m0);
                    }
                    e_issued = lt;
                } else {
                    mbar_arrive(&e_free[e]);
                }
            }
            if (ok) {
                for (int t = stored; t < my_tiles && ok; ++t) ok = store_tile(t);
            }
            if (!ok) {
                *abort_flag = 1;
                for (int t = max(0, e_issued - 1); t <= e_issued; ++t)
                    for (int b = 0; b < E_BOXES; ++b)
                        (void)mbar_wait(&e_full[4 * (t & 1) + b], (uint32_t)(t >> 1) & 1u, nullptr);
                bulk_wait_read();
            }
        }
    } else if (warp == 1) {
        if (lane == 0 && nk > 0) {
            // ---- MMA issuer ----
            int it = 0;
            bool ok = true;
            for (int lt = 0; lt < my_tiles && ok; ++lt) {
                const int buf = lt & 1, use = lt >> 1;
                if (use > 0 && !mbar_wait(&acc_empty[buf], (uint32_t)(use - 1) & 1u, abort_flag)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t dst = tmem_base + (uint32_t)(buf * BN);
                for (int i = 0; i < nk; ++i, ++it) {
                    const int s = it % STAGES;
                    if (!mbar_wait(&full[s], (uint32_t)(it / STAGES) & 1u, abort_flag)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t sa = smem_u32(smem + s * STAGE_BYTES);  // A hi (then A lo)
                    const uint32_t sb = sa + PL * A_BYTES;                 // B hi (then B lo)
                    auto kdesc = [&](uint32_t a) {
                        return ROWB == 128 ? sw128_desc(a) : ROWB == 64 ? sw64_desc(a) : sw32_desc(a);
                    };
#pragma unroll
                    for (int kk = 0; kk < ROWB / 32; ++kk) {  // one MMA consumes 32 bytes of K
                        const uint64_t da = kdesc(sa + kk * 32);
                        const uint64_t db = B_MN ? mn128_desc(sb + kk * 16 * 128, MN_BOX) : kdesc(sb + kk * 32);
                        if (ELEM == 1) {
                            mma_e4m3(dst, da, db, IDESC, (i > 0 || kk > 0) ? 1u : 0u);
                        } else {
                            const uint64_t dal = kdesc(sa + A_BYTES + kk * 32);
                            const uint64_t dbl =
                                B_MN ? mn128_desc(sb + B_BYTES + kk * 16 * 128, MN_BOX) : kdesc(sb + B_BYTES + kk * 32);
                            mma_step<SPLIT>(dst, da, dal, db, dbl, IDESC, (i > 0 || kk > 0) ? 1u : 0u);
                        }
                    }
                    mma_commit(&empty[s]);
                }
                if (!ok) break;
                mma_commit(&acc_full[buf]);
            }
            if (!ok) *abort_flag = 1;
            // every MMA issued by this thread has completed before TMEM is released
            mma_commit(drain);
            (void)mbar_wait(drain, 0, nullptr);
        }
    } else {
        // ---- epilogue warps (3 ..) ----
        const int quarter = warp & 3;
        const int group = (warp - 3) >> 2;
        const int row = quarter * 32 + lane;
        for (int lt = 0; lt < my_tiles; ++lt) {
            const int e = lt & 1, use = lt >> 1;
            const int tile = first + lt * stride;
            bool ready = nk > 0 && mbar_wait(&acc_full[e], (uint32_t)use & 1u, abort_flag);
            if (!SPLIT && ready && E_BOXES == 0 && O_BOXES > 0)
                ready = mbar_wait(&e_free[e], (uint32_t)use & 1u, abort_flag);
            tc_fence_after();
            if (!ready) *abort_flag = 1;
            epi_sync(128 * G);
            if (threadIdx.x == 96) *decision = *abort_flag ? 0 : 1;
            epi_sync(128 * G);
            uint8_t* box = boxes + e * BOX_BYTES;
            EpiCtx ec{tmem_base + (uint32_t)(e * BN) + ((uint32_t)(quarter * 32) << 16),
                      row, tile * kTileM, n0, 0, group, scratch, E_BOXES > 0 ? box : nullptr, box,
                      &e_full[4 * e], abort_flag, (int)crank, (int)csize, &xbars[e],
                      xbufs + e * (kXchgBytes / 4), (uint32_t)use & 1u, (uint32_t)use & 1u, G, 96};
            if (INPLACE) {  // the operand chunks of this tile, the output written over them
                ec.etile = boxes;
                ec.otile = boxes;
                ec.ebar = e_full;
                ec.ephase = (uint32_t)lt & 1u;
            } else if (SPLIT) {  // both buffers hold this tile's output; run() waits for them (wait_out)
                ec.otile = boxes;
                ec.oplane = BOX_BYTES;
                ec.ofree = &e_free[0];
                ec.ofree_phase = (uint32_t)lt & 1u;
            }
            int out_boxes = 0;
            if (*decision) {
                out_boxes = Epi::run(ep, ec);  // split form: run() calls ec.wait_out() once, on every path
            } else {
                if (Epi::XROUNDS > 0) {
                    const float zero[kXchgVals] = {0.f, 0.f, 0.f, 0.f};
                    (void)ec.exchange(zero);
                }
                if (SPLIT && !INPLACE) (void)ec.wait_out();
            }
            // TMEM and the staged output are handed over once every epilogue thread is done
            tc_fence_before();
            fence_proxy_async();
            epi_sync(128 * G);
            if (threadIdx.x == 96) {
                mbar_arrive(&acc_empty[e]);
                const int sb = SPLIT ? 0 : e;
                nbox[sb] = *abort_flag ? 0 : out_boxes;
                mbar_arrive(&staged[sb]);
            }
        }
    }
    __syncthreads();
    // no CTA leaves while a peer may still read or write its shared memory (the row exchange)
    if (csize > 1) cluster_sync_all();
    if (*abort_flag && threadIdx.x == 0) atomicExch(err, 1);
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem_base, 512);
    }
}

}  // namespace tc
}  // namespace lat
