// Voxel-hashed global map and the active local map around the camera (Sec. III-E, "Local-
// Global Map Management via Voxel Hashing").
//
// The global store (Gaussian attributes in index order) and its slot table live in HBM: at
// 172 bytes per Gaussian (d = 32) the 280 GB of a GB300 hold on the order of 10^9 of them, so
// the radius gather, the de-duplication and the write-back run as kernels instead of host loops.
// Each Gaussian owns the slot of the voxel floor(p / s_v) it was inserted from; slots hold no key
// (two voxels with the same hash collide and the later one counts as occupied), at most one
// Gaussian per slot.  Insert-if-free is deterministic: every candidate whose slot is empty claims
// it with an atomic minimum of its input index, the lowest index wins, and the winners are
// appended in input order (an exclusive scan), exactly as a sequential insertion would.
//
// Synchronisation: Local -> Global (local Gaussians that came from the store overwrite their
// entries, new ones are inserted if their slot is free), then Global -> Local (local Gaussians
// outside the radius are dropped, kept ones are marked in a per-row epoch array, and the store's
// unmarked Gaussians inside the radius are appended in index order) into the second of two local
// buffers.  The local map also carries the Adam moments of the queries (zero for appended rows).
#include <algorithm>
#include <climits>
#include <cstring>

#include "internal.cuh"

using namespace lat;

namespace {

constexpr int kMapThreads = 256;
constexpr int64_t kScanChunk = 1ll << 24;  // the largest exclusive scan one call supports

struct Rows {  // SoA rows of Gaussians (any may be null where not used)
    float *means, *quats, *scales, *opac, *f, *m_f, *v_f;
    int32_t* gidx;
    bool host;  // pinned host memory (read and written by the kernels through unified addressing)
};

}  // namespace

struct latentam_map {
    int device;
    int d;
    int table_log2;
    float voxel_size;
    int64_t capacity, count;  // global store (count mirrored on the host)
    bool host_store;          // the store's rows in pinned host memory
    int32_t* table;           // 2^table_log2 slots, -1 = empty
    int32_t* claim;           // per-slot claims of one insertion, INT_MAX when idle
    int32_t* epoch_mark;      // per global row: the last synchronisation that found it local
    int32_t epoch;
    Rows g;
    Rows loc[2];
    int64_t loc_capacity[2];
    int cur;                  // the current local buffer
    int64_t local_count;
    // scratch of one operation
    int32_t* slot;
    uint32_t *flag, *pos;
    int64_t scratch_n;
    uint32_t* total;          // device counters
};

namespace {

void free_rows(Rows& r) {
    for (void* p : {(void*)r.means, (void*)r.quats, (void*)r.scales, (void*)r.opac, (void*)r.f, (void*)r.m_f,
                    (void*)r.v_f, (void*)r.gidx})
        if (p) {
            if (r.host) cudaFreeHost(p);
            else cudaFree(p);
        }
    r = Rows{};
}

// Rows of `cap` Gaussians (moments and gidx only when `local`); the first `keep` rows of `old`
// are copied over and `old` is freed.
latentam_status alloc_rows(Rows& r, int64_t cap, int d, bool local, Rows* old, int64_t keep, bool host = false) {
    Rows n{};
    n.host = host;
    auto alloc = [&](void** p, size_t bytes) {
        return host ? cudaHostAlloc(p, bytes, cudaHostAllocMapped) : cudaMalloc(p, bytes);
    };
    const size_t c = (size_t)std::max<int64_t>(cap, 1);
    struct Field {
        float** dst;
        float* src;
        int w;
    } fields[] = {{&n.means, old ? old->means : nullptr, 3},  {&n.quats, old ? old->quats : nullptr, 4},
                  {&n.scales, old ? old->scales : nullptr, 3}, {&n.opac, old ? old->opac : nullptr, 1},
                  {&n.f, old ? old->f : nullptr, d},           {&n.m_f, old ? old->m_f : nullptr, local ? d : 0},
                  {&n.v_f, old ? old->v_f : nullptr, local ? d : 0}};
    for (auto& fl : fields) {
        if (fl.w == 0) continue;
        if (alloc(reinterpret_cast<void**>(fl.dst), sizeof(float) * c * fl.w) != cudaSuccess) {
            cudaGetLastError();
            free_rows(n);
            set_error("voxel map: out of device memory for %lld rows", (long long)cap);
            return LATENTAM_ERR_OUT_OF_MEMORY;
        }
        if (fl.src && keep > 0) cudaMemcpy(*fl.dst, fl.src, sizeof(float) * (size_t)keep * fl.w, cudaMemcpyDefault);
    }
    if (local) {
        if (cudaMalloc(&n.gidx, sizeof(int32_t) * c) != cudaSuccess) {
            cudaGetLastError();
            free_rows(n);
            set_error("voxel map: out of device memory for %lld rows", (long long)cap);
            return LATENTAM_ERR_OUT_OF_MEMORY;
        }
        if (old && old->gidx && keep > 0)
            cudaMemcpy(n.gidx, old->gidx, sizeof(int32_t) * (size_t)keep, cudaMemcpyDeviceToDevice);
    }
    if (old) free_rows(*old);
    r = n;
    return LATENTAM_OK;
}

latentam_status grow_global(latentam_map* m, int64_t need) {
    if (need <= m->capacity) return LATENTAM_OK;
    if (need > INT32_MAX) {
        set_error("voxel map: %lld Gaussians exceed the int32 indices", (long long)need);
        return LATENTAM_ERR_UNSUPPORTED_SHAPE;
    }
    const int64_t cap = std::min<int64_t>(INT32_MAX, std::max<int64_t>(need, 2 * m->capacity));
    cudaDeviceSynchronize();
    Rows old = m->g;
    LAT_TRY(alloc_rows(m->g, cap, m->d, false, &old, m->count, m->host_store));
    int32_t* mark = nullptr;
    if (cudaMalloc(&mark, sizeof(int32_t) * (size_t)cap) != cudaSuccess) {
        cudaGetLastError();
        set_error("voxel map: out of device memory");
        return LATENTAM_ERR_OUT_OF_MEMORY;
    }
    cudaMemset(mark, 0, sizeof(int32_t) * (size_t)cap);
    if (m->epoch_mark) {
        cudaMemcpy(mark, m->epoch_mark, sizeof(int32_t) * (size_t)m->count, cudaMemcpyDeviceToDevice);
        cudaFree(m->epoch_mark);
    }
    m->epoch_mark = mark;
    m->capacity = cap;
    return LATENTAM_OK;
}

latentam_status grow_local(latentam_map* m, int which, int64_t need, int64_t keep) {
    if (need <= m->loc_capacity[which]) return LATENTAM_OK;
    const int64_t cap = std::max<int64_t>(need, 2 * m->loc_capacity[which]);
    cudaDeviceSynchronize();
    Rows old = m->loc[which];
    LAT_TRY(alloc_rows(m->loc[which], cap, m->d, true, &old, keep));
    m->loc_capacity[which] = cap;
    return LATENTAM_OK;
}

latentam_status grow_scratch(latentam_map* m, int64_t n) {
    if (n <= m->scratch_n) return LATENTAM_OK;
    const int64_t cap = std::max<int64_t>(n, 2 * m->scratch_n);
    cudaDeviceSynchronize();
    if (m->slot) cudaFree(m->slot);
    if (m->flag) cudaFree(m->flag);
    if (m->pos) cudaFree(m->pos);
    m->slot = nullptr, m->flag = m->pos = nullptr;
    if (cudaMalloc(&m->slot, sizeof(int32_t) * (size_t)cap) != cudaSuccess ||
        cudaMalloc(&m->flag, sizeof(uint32_t) * (size_t)cap) != cudaSuccess ||
        cudaMalloc(&m->pos, sizeof(uint32_t) * (size_t)cap) != cudaSuccess) {
        cudaGetLastError();
        set_error("voxel map: out of device memory for scratch");
        return LATENTAM_ERR_OUT_OF_MEMORY;
    }
    m->scratch_n = cap;
    return LATENTAM_OK;
}

// ---- device arithmetic (every rounding explicit: the oracle takes the same decisions) -------

__device__ __forceinline__ int slot_of(float x, float y, float z, float s_v, int table_log2) {
    const int64_t vx = (int64_t)floorf(__fdiv_rn(x, s_v)), vy = (int64_t)floorf(__fdiv_rn(y, s_v)),
                  vz = (int64_t)floorf(__fdiv_rn(z, s_v));
    const uint64_t h = ((uint64_t)vx * 73856093ull) ^ ((uint64_t)vy * 19349663ull) ^ ((uint64_t)vz * 83492791ull);
    return (int)(h & ((1ull << table_log2) - 1ull));
}

__device__ __forceinline__ bool in_radius(const float* p, float cx, float cy, float cz, float r2) {
    const float dx = __fsub_rn(p[0], cx), dy = __fsub_rn(p[1], cy), dz = __fsub_rn(p[2], cz);
    const float s = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
    return s <= r2;
}

__device__ __forceinline__ void copy_row(const Rows& s, int64_t i, const Rows& t, int64_t j, int d) {
    for (int k = 0; k < 3; ++k) t.means[3 * j + k] = s.means[3 * i + k];
    for (int k = 0; k < 4; ++k) t.quats[4 * j + k] = s.quats[4 * i + k];
    for (int k = 0; k < 3; ++k) t.scales[3 * j + k] = s.scales[3 * i + k];
    t.opac[j] = s.opac[i];
    for (int k = 0; k < d; ++k) t.f[(size_t)d * j + k] = s.f[(size_t)d * i + k];
}

// Candidates: rows whose slot is empty (and, with gidx, that have no global entry yet) claim it.
__global__ void insert_claim(int64_t n, const float* __restrict__ means, const int32_t* __restrict__ gidx,
                             float s_v, int table_log2, const int32_t* __restrict__ table, int32_t* claim,
                             int32_t* __restrict__ slot, uint32_t* __restrict__ cand) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int s = -1;
    uint32_t c = 0;
    if (!gidx || gidx[i] < 0) {
        s = slot_of(means[3 * i], means[3 * i + 1], means[3 * i + 2], s_v, table_log2);
        if (table[s] < 0) {
            c = 1;
            atomicMin(claim + s, (int)i);
        }
    }
    slot[i] = s;
    cand[i] = c;
}

// win[i] = candidate i holds the lowest claim of its slot (written over cand).
__global__ void insert_win(int64_t n, const int32_t* __restrict__ slot, const int32_t* __restrict__ claim,
                           uint32_t* cand) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (cand[i]) cand[i] = claim[slot[i]] == (int32_t)i ? 1u : 2u;  // 1 = won, 2 = lost
}

// Winners take index base + pos[i] and their slot; every claim is released.
__global__ void insert_commit(int64_t n, Rows src, int d, const int32_t* __restrict__ slot,
                              const uint32_t* __restrict__ win, const uint32_t* __restrict__ pos, int64_t base,
                              int32_t* table, int32_t* claim, Rows dst, int32_t* __restrict__ out_index,
                              int32_t* __restrict__ gidx_out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t w = win[i];
    int32_t idx = -1;
    if (w) claim[slot[i]] = INT_MAX;
    if (w == 1) {
        idx = (int32_t)(base + pos[i]);
        table[slot[i]] = idx;
        copy_row(src, i, dst, idx, d);
        if (gidx_out) gidx_out[i] = idx;
    }
    if (out_index) out_index[i] = idx;
}

// flags of a 0/1 predicate: win[i] = 1 for winners only (losers 2 -> 0) before the scan.
__global__ void winners_only(int64_t n, const uint32_t* __restrict__ cand, uint32_t* __restrict__ flag) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) flag[i] = cand[i] == 1 ? 1u : 0u;
}

__global__ void write_back_rows(int64_t n, Rows local, int d, Rows global) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t g = local.gidx[i];
    if (g >= 0) copy_row(local, i, global, g, d);
}

__global__ void keep_flags(int64_t n, Rows local, float cx, float cy, float cz, float r2, int32_t* epoch_mark,
                           int32_t epoch, uint32_t* __restrict__ keep) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const bool k = in_radius(local.means + 3 * i, cx, cy, cz, r2);
    keep[i] = k ? 1u : 0u;
    if (k && local.gidx[i] >= 0) epoch_mark[local.gidx[i]] = epoch;
}

__global__ void compact_local(int64_t n, Rows src, int d, const uint32_t* __restrict__ keep,
                              const uint32_t* __restrict__ pos, Rows dst) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !keep[i]) return;
    const int64_t j = pos[i];
    copy_row(src, i, dst, j, d);
    for (int k = 0; k < d; ++k) {
        dst.m_f[(size_t)d * j + k] = src.m_f[(size_t)d * i + k];
        dst.v_f[(size_t)d * j + k] = src.v_f[(size_t)d * i + k];
    }
    dst.gidx[j] = src.gidx[i];
}

__global__ void select_global(int64_t g0, int64_t n, const float* __restrict__ means, float cx, float cy, float cz,
                              float r2, const int32_t* __restrict__ epoch_mark, int32_t epoch,
                              uint32_t* __restrict__ sel) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t g = g0 + i;
    sel[i] = (in_radius(means + 3 * g, cx, cy, cz, r2) && epoch_mark[g] != epoch) ? 1u : 0u;
}

__global__ void append_global(int64_t g0, int64_t n, Rows global, int d, const uint32_t* __restrict__ sel,
                              const uint32_t* __restrict__ pos, int64_t base, Rows dst) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !sel[i]) return;
    const int64_t g = g0 + i, j = base + pos[i];
    copy_row(global, g, dst, j, d);
    for (int k = 0; k < d; ++k) dst.m_f[(size_t)d * j + k] = dst.v_f[(size_t)d * j + k] = 0.f;
    dst.gidx[j] = (int32_t)g;
}

unsigned blocks(int64_t n) { return (unsigned)((n + kMapThreads - 1) / kMapThreads); }

latentam_status read_total(latentam_map* m, cudaStream_t st, uint32_t* out) {
    cudaError_t e = cudaMemcpyAsync(out, m->total, sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_error(e, "voxel map: read count");
    return LATENTAM_OK;
}

// Insert-if-free of n rows of `src` (rows with gidx >= 0 skipped when gidx is given); the
// winners' new indices go to out_index (all rows, -1 for the others) and/or gidx.
latentam_status insert_rows(latentam_ctx* ctx, latentam_map* m, int64_t n, const Rows& src, int32_t* gidx,
                            int32_t* out_index, int64_t* n_inserted, cudaStream_t st) {
    if (n_inserted) *n_inserted = 0;
    if (n <= 0) return LATENTAM_OK;
    if (n > kScanChunk) {
        set_error("voxel map: at most %lld Gaussians per insertion", (long long)kScanChunk);
        return LATENTAM_ERR_UNSUPPORTED_SHAPE;
    }
    LAT_TRY(grow_global(m, m->count + n));
    LAT_TRY(grow_scratch(m, n));
    insert_claim<<<blocks(n), kMapThreads, 0, st>>>(n, src.means, gidx, m->voxel_size, m->table_log2, m->table,
                                                    m->claim, m->slot, m->flag);
    LAT_CHECK_LAUNCH("insert_claim");
    insert_win<<<blocks(n), kMapThreads, 0, st>>>(n, m->slot, m->claim, m->flag);
    LAT_CHECK_LAUNCH("insert_win");
    uint32_t* won = m->pos;  // the 0/1 winner flags, scanned in place into positions
    winners_only<<<blocks(n), kMapThreads, 0, st>>>(n, m->flag, won);
    LAT_CHECK_LAUNCH("winners_only");
    LAT_TRY(scan_exclusive_u32(ctx, won, won, n, m->total, st));
    insert_commit<<<blocks(n), kMapThreads, 0, st>>>(n, src, m->d, m->slot, m->flag, won, m->count, m->table,
                                                     m->claim, m->g, out_index, gidx);
    LAT_CHECK_LAUNCH("insert_commit");
    uint32_t added = 0;
    LAT_TRY(read_total(m, st, &added));
    m->count += added;
    if (n_inserted) *n_inserted = added;
    return LATENTAM_OK;
}

Rows gaussian_rows(const latentam_gaussians& g, const float* f) {
    Rows r{};
    r.means = const_cast<float*>(g.means);
    r.quats = const_cast<float*>(g.quats);
    r.scales = const_cast<float*>(g.scales);
    r.opac = const_cast<float*>(g.opacities);
    r.f = const_cast<float*>(f);
    return r;
}

void fill_local(const latentam_map* m, latentam_map_local* out) {
    const Rows& r = m->loc[m->cur];
    *out = latentam_map_local{r.means, r.quats, r.scales, r.opac, r.f, r.m_f, r.v_f, r.gidx, m->local_count};
}

latentam_status enter_map(latentam_ctx* ctx, latentam_map* m) {
    if (!ctx || !m) {
        set_error("null context or map");
        return LATENTAM_ERR_INVALID_ARG;
    }
    if (m->device != ctx->device) {
        set_error("the map lives on device %d, the context on %d", m->device, ctx->device);
        return LATENTAM_ERR_INVALID_ARG;
    }
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_error(e, "cudaSetDevice");
    return LATENTAM_OK;
}

}  // namespace

extern "C" {

latentam_status latentam_map_create(latentam_ctx* ctx, int32_t d, int32_t table_log2, float voxel_size,
                                    int64_t capacity, int32_t host_store, latentam_map** out) {
    if (!ctx || !out) {
        set_error("null context or output");
        return LATENTAM_ERR_INVALID_ARG;
    }
    *out = nullptr;
    if (d < 1 || d > 256 || table_log2 < 4 || table_log2 > 30 || !(voxel_size > 0.f) || capacity < 0) {
        set_error("voxel map: d=%d table_log2=%d voxel_size=%g capacity=%lld out of range", d, table_log2,
                  (double)voxel_size, (long long)capacity);
        return LATENTAM_ERR_INVALID_ARG;
    }
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_error(e, "cudaSetDevice");
    latentam_map* m = new latentam_map();
    memset(m, 0, sizeof(*m));
    m->device = ctx->device;
    m->d = d;
    m->table_log2 = table_log2;
    m->voxel_size = voxel_size;
    m->host_store = host_store != 0;
    m->epoch = 0;
    const size_t T = (size_t)1 << table_log2;
    bool ok = cudaMalloc(&m->table, sizeof(int32_t) * T) == cudaSuccess &&
              cudaMalloc(&m->claim, sizeof(int32_t) * T) == cudaSuccess &&
              cudaMalloc(&m->total, sizeof(uint32_t) * 2) == cudaSuccess;
    if (ok) ok = cudaMemset(m->table, 0xff, sizeof(int32_t) * T) == cudaSuccess;  // -1
    if (ok) {
        // INT_MAX in every claim: fill through a host pattern once
        int32_t* h = static_cast<int32_t*>(malloc(sizeof(int32_t) * std::min<size_t>(T, 1 << 20)));
        ok = h != nullptr;
        if (ok) {
            const size_t chunk = std::min<size_t>(T, 1 << 20);
            for (size_t i = 0; i < chunk; ++i) h[i] = INT_MAX;
            for (size_t o = 0; ok && o < T; o += chunk)
                ok = cudaMemcpy(m->claim + o, h, sizeof(int32_t) * std::min(chunk, T - o), cudaMemcpyHostToDevice) ==
                     cudaSuccess;
            free(h);
        }
    }
    latentam_status s = ok ? LATENTAM_OK : LATENTAM_ERR_OUT_OF_MEMORY;
    if (s == LATENTAM_OK) s = grow_global(m, std::max<int64_t>(capacity, 1024));
    if (s == LATENTAM_OK) s = grow_local(m, 0, 1024, 0);
    if (s == LATENTAM_OK) s = grow_local(m, 1, 1024, 0);
    if (s != LATENTAM_OK) {
        cudaGetLastError();
        latentam_map_destroy(m);
        if (s == LATENTAM_ERR_OUT_OF_MEMORY) set_error("voxel map: out of device memory");
        return s;
    }
    *out = m;
    return LATENTAM_OK;
}

latentam_status latentam_map_destroy(latentam_map* m) {
    if (!m) return LATENTAM_OK;
    cudaSetDevice(m->device);
    cudaDeviceSynchronize();
    free_rows(m->g);
    free_rows(m->loc[0]);
    free_rows(m->loc[1]);
    for (void* p : {(void*)m->table, (void*)m->claim, (void*)m->epoch_mark, (void*)m->slot, (void*)m->flag,
                    (void*)m->pos, (void*)m->total})
        if (p) cudaFree(p);
    delete m;
    return LATENTAM_OK;
}

latentam_status latentam_map_insert(latentam_ctx* ctx, latentam_map* m, const latentam_gaussians* g, const float* f,
                                    int32_t* out_index, int64_t* n_inserted, latentam_stream stream) {
    LAT_TRY(enter_map(ctx, m));
    if (!g || g->n < 0 || (g->n > 0 && (!g->means || !g->quats || !g->scales || !g->opacities || !f))) {
        set_error("null or negative Gaussian input");
        return LATENTAM_ERR_INVALID_ARG;
    }
    return insert_rows(ctx, m, g->n, gaussian_rows(*g, f), nullptr, out_index, n_inserted, (cudaStream_t)stream);
}

latentam_status latentam_map_add_local(latentam_ctx* ctx, latentam_map* m, const latentam_gaussians* g,
                                       const float* f, latentam_stream stream) {
    LAT_TRY(enter_map(ctx, m));
    if (!g || g->n < 0 || (g->n > 0 && (!g->means || !g->quats || !g->scales || !g->opacities || !f))) {
        set_error("null or negative Gaussian input");
        return LATENTAM_ERR_INVALID_ARG;
    }
    const int64_t n = g->n;
    if (n == 0) return LATENTAM_OK;
    cudaStream_t st = (cudaStream_t)stream;
    cudaStreamSynchronize(st);
    LAT_TRY(grow_local(m, m->cur, m->local_count + n, m->local_count));
    const Rows& L = m->loc[m->cur];
    const int64_t o = m->local_count;
    const int d = m->d;
    struct Cp {
        float* dst;
        const float* src;
        int w;
    } cps[] = {{L.means + 3 * o, g->means, 3}, {L.quats + 4 * o, g->quats, 4}, {L.scales + 3 * o, g->scales, 3},
               {L.opac + o, g->opacities, 1}, {L.f + (size_t)d * o, f, d}};
    for (auto& c : cps) {
        cudaError_t e = cudaMemcpyAsync(c.dst, c.src, sizeof(float) * (size_t)n * c.w, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return cuda_error(e, "voxel map: add local");
    }
    cudaError_t e = cudaMemsetAsync(L.m_f + (size_t)d * o, 0, sizeof(float) * (size_t)n * d, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(L.v_f + (size_t)d * o, 0, sizeof(float) * (size_t)n * d, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(L.gidx + o, 0xff, sizeof(int32_t) * (size_t)n, st);  // -1
    if (e != cudaSuccess) return cuda_error(e, "voxel map: add local");
    m->local_count += n;
    return LATENTAM_OK;
}

latentam_status latentam_map_sync(latentam_ctx* ctx, latentam_map* m, const float* centre, float radius,
                                  latentam_map_local* local_out, latentam_stream stream) {
    LAT_TRY(enter_map(ctx, m));
    if (!centre || !(radius >= 0.f)) {
        set_error("null centre or negative radius");
        return LATENTAM_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int d = m->d;
    const int64_t nl = m->local_count;
    // Local -> Global: known Gaussians overwrite their entries, new ones are inserted if free
    if (nl > 0) {
        write_back_rows<<<blocks(nl), kMapThreads, 0, st>>>(nl, m->loc[m->cur], d, m->g);
        LAT_CHECK_LAUNCH("write_back_rows");
        Rows src = m->loc[m->cur];
        LAT_TRY(insert_rows(ctx, m, nl, src, src.gidx, nullptr, nullptr, st));
    }
    // Global -> Local: prune, mark, select, then compact and append into the other buffer
    const float cx = centre[0], cy = centre[1], cz = centre[2];
    const float r2 = radius * radius;
    m->epoch += 1;
    LAT_TRY(grow_scratch(m, std::max<int64_t>(nl, std::min<int64_t>(m->count, kScanChunk))));
    uint32_t kept = 0;
    if (nl > 0) {
        keep_flags<<<blocks(nl), kMapThreads, 0, st>>>(nl, m->loc[m->cur], cx, cy, cz, r2, m->epoch_mark, m->epoch,
                                                       m->flag);
        LAT_CHECK_LAUNCH("keep_flags");
        LAT_TRY(scan_exclusive_u32(ctx, m->flag, m->pos, nl, m->total, st));
        LAT_TRY(read_total(m, st, &kept));
        const int other = m->cur ^ 1;
        LAT_TRY(grow_local(m, other, kept, 0));
        compact_local<<<blocks(nl), kMapThreads, 0, st>>>(nl, m->loc[m->cur], d, m->flag, m->pos, m->loc[other]);
        LAT_CHECK_LAUNCH("compact_local");
    }
    int64_t n_new = kept;
    const int other = m->cur ^ 1;
    for (int64_t g0 = 0; g0 < m->count; g0 += kScanChunk) {
        const int64_t n = std::min<int64_t>(kScanChunk, m->count - g0);
        select_global<<<blocks(n), kMapThreads, 0, st>>>(g0, n, m->g.means, cx, cy, cz, r2, m->epoch_mark, m->epoch,
                                                         m->flag);
        LAT_CHECK_LAUNCH("select_global");
        LAT_TRY(scan_exclusive_u32(ctx, m->flag, m->pos, n, m->total, st));
        uint32_t sel = 0;
        LAT_TRY(read_total(m, st, &sel));
        if (sel == 0) continue;
        LAT_TRY(grow_local(m, other, n_new + sel, n_new));
        append_global<<<blocks(n), kMapThreads, 0, st>>>(g0, n, m->g, d, m->flag, m->pos, n_new, m->loc[other]);
        LAT_CHECK_LAUNCH("append_global");
        n_new += sel;
    }
    m->cur = other;
    m->local_count = n_new;
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_error(e, "voxel map: sync");
    if (local_out) fill_local(m, local_out);
    return LATENTAM_OK;
}

latentam_status latentam_map_local_view(latentam_map* m, latentam_map_local* out) {
    if (!m || !out) {
        set_error("null map or output");
        return LATENTAM_ERR_INVALID_ARG;
    }
    fill_local(m, out);
    return LATENTAM_OK;
}

latentam_status latentam_map_global_view(latentam_map* m, latentam_map_global* out) {
    if (!m || !out) {
        set_error("null map or output");
        return LATENTAM_ERR_INVALID_ARG;
    }
    *out = latentam_map_global{m->g.means, m->g.quats, m->g.scales, m->g.opac, m->g.f, m->table, m->count,
                               (int64_t)1 << m->table_log2};
    return LATENTAM_OK;
}

}  // extern "C"
