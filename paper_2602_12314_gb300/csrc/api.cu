// C ABI of include/latentam.h: argument validation, the context and its workspace, and the
// composition of the kernels into the calls of the latent-feature optimisation step.
#include <math.h>

#include <cmath>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>

#include "internal.cuh"

namespace lat {

static thread_local char g_err[512] = "";
static std::atomic<int64_t> g_launches{0};

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

// Instantiated graphs of the step's iteration, keyed by every pointer, shape and scalar the
// iteration bakes into its launches (and the workspace generation).
struct GraphKey {
    static constexpr int kMax = 1280;  // a batch of 32 frames with masks needs about 1100
    uint64_t v[kMax];
    int n = 0;
    bool overflow = false;  // a key that did not fit never matches (no graph)
    void add(uint64_t x) {
        if (n < kMax)
            v[n++] = x;
        else
            overflow = true;
    }
    void addp(const void* p) { add(reinterpret_cast<uint64_t>(p)); }
    void addf(float f) {
        uint32_t u;
        memcpy(&u, &f, 4);
        add(u);
    }
    void add_camera(const latentam_camera& c) {
        for (int i = 0; i < 9; ++i) addf(c.R[i]);
        for (int i = 0; i < 3; ++i) addf(c.t[i]);
        for (float f : {c.fx, c.fy, c.cx, c.cy, c.z_near}) addf(f);
        add((uint64_t)c.width);
        add((uint64_t)c.height);
    }
    bool operator==(const GraphKey& o) const {
        return !overflow && !o.overflow && n == o.n && memcmp(v, o.v, sizeof(uint64_t) * n) == 0;
    }
};
struct GraphCache {
    // a batch of up to LATENTAM_MAX_BATCH keyframes bins each frame in two captured phases
    static constexpr int kSlots = 2 * LATENTAM_MAX_BATCH + 8;
    GraphKey key[kSlots];
    cudaGraphExec_t exec[kSlots] = {};
    int64_t launches[kSlots] = {};
    int used = 0, next = 0;
    GraphKey warm[kSlots];  // configurations run once eagerly (their workspaces are sized)
    int warm_used = 0, warm_next = 0;
    GraphKey failed[kSlots];  // configurations whose capture failed: always eager
    int failed_used = 0, failed_next = 0;
    static int find(const GraphKey* arr, int used, const GraphKey& k) {
        for (int i = 0; i < used; ++i)
            if (arr[i] == k) return i;
        return -1;
    }
    static void put(GraphKey* arr, int& used, int& next, const GraphKey& k) {
        arr[next] = k;
        next = (next + 1) % kSlots;
        if (used < kSlots) ++used;
    }
    void clear() {
        for (int i = 0; i < kSlots; ++i)
            if (exec[i]) cudaGraphExecDestroy(exec[i]);
        *this = GraphCache();
    }
};

int64_t launch_count_now() { return g_launches.load(std::memory_order_relaxed); }
void launch_count_add(int64_t k);

latentam_status cached_launch(latentam_ctx* ctx, const uint64_t* words, int n, cudaStream_t st,
                              const std::function<latentam_status(cudaStream_t)>& fn) {
    if (!ctx->use_graphs || ctx->profiling || !ctx->sort_graphs) return fn(st);
    GraphKey key;
    for (int i = 0; i < n; ++i) key.add(words[i]);
    if (key.overflow) return fn(st);
    GraphCache& gc = *ctx->sort_graphs;
    int slot = GraphCache::find(gc.key, gc.used, key);
    if (slot < 0) {
        if (GraphCache::find(gc.failed, gc.failed_used, key) >= 0) return fn(st);
        if (GraphCache::find(gc.warm, gc.warm_used, key) < 0) {
            GraphCache::put(gc.warm, gc.warm_used, gc.warm_next, key);
            return fn(st);
        }
        // second sighting: capture, instantiate, then replay below
        cudaGraph_t graph = nullptr;
        const int64_t l0 = launch_count_now();
        cudaError_t e = cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal);
        latentam_status cs = e == cudaSuccess ? fn(ctx->cap_stream) : LATENTAM_ERR_CUDA;
        cudaError_t e2 = e == cudaSuccess ? cudaStreamEndCapture(ctx->cap_stream, &graph) : e;
        const int64_t captured = launch_count_now() - l0;
        launch_count_add(-captured);  // nothing ran yet
        cudaGraphExec_t exec = nullptr;
        if (cs == LATENTAM_OK && e2 == cudaSuccess && graph && cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess) {
            slot = gc.next;
            if (gc.exec[slot]) {
                cudaStreamSynchronize(st);
                cudaGraphExecDestroy(gc.exec[slot]);
            }
            gc.exec[slot] = exec;
            gc.key[slot] = key;
            gc.launches[slot] = captured;
            gc.next = (gc.next + 1) % GraphCache::kSlots;
            if (gc.used < GraphCache::kSlots) ++gc.used;
        } else {
            (void)cudaGetLastError();
            GraphCache::put(gc.failed, gc.failed_used, gc.failed_next, key);
            if (graph) cudaGraphDestroy(graph);
            return fn(st);
        }
        if (graph) cudaGraphDestroy(graph);
    }
    cudaError_t e = cudaGraphLaunch(gc.exec[slot], st);
    if (e != cudaSuccess) return cuda_error(e, "graph launch");
    launch_count_add(gc.launches[slot]);
    return LATENTAM_OK;
}
void launch_count_add(int64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

latentam_status cuda_error(cudaError_t e, const char* what) {
    set_error("%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
    return LATENTAM_ERR_CUDA;
}

void* ws(latentam_ctx* ctx, Slot s, size_t bytes) {
    if (bytes == 0) bytes = 256;
    if (ctx->slot_bytes[s] >= bytes) return ctx->slot_ptr[s];
    ++ctx->ws_generation;  // captured graphs that name the old buffer are stale now
    size_t nb = std::max(bytes, ctx->slot_bytes[s] + ctx->slot_bytes[s] / 4);
    nb = (nb + 4095) & ~(size_t)4095;
    if (ctx->slot_ptr[s]) {
        // work already enqueued may still read the old buffer
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) {
            cuda_error(e, "workspace regrow sync");
            return nullptr;
        }
        cudaFree(ctx->slot_ptr[s]);
        ctx->slot_ptr[s] = nullptr;
        ctx->slot_bytes[s] = 0;
    }
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, nb);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        set_error("workspace allocation of %zu bytes failed: %s", nb, cudaGetErrorString(e));
        return nullptr;
    }
    if (s == WS_COUNTERS) {
        // the counters carry an error word across calls: it starts clear
        e = cudaMemset(p, 0, nb);
        if (e != cudaSuccess) {
            cudaFree(p);
            cuda_error(e, "clear the counters");
            return nullptr;
        }
    }
    ctx->slot_ptr[s] = p;
    ctx->slot_bytes[s] = nb;
    return p;
}

// cp with the launch order of its tiles (computed from the frame's bins into the order slot at
// `offset` tiles); the per-tile kernels then start the longest tile lists first.
latentam_status ordered(latentam_ctx* ctx, CamParams* cp, const latentam_bins& bins, size_t offset, size_t total,
                        cudaStream_t st) {
    int32_t* order = static_cast<int32_t*>(ws(ctx, WS_TILE_ORDER, sizeof(int32_t) * total));
    if (!order) return LATENTAM_ERR_OUT_OF_MEMORY;
    LAT_TRY(launch_tile_order(*cp, bins, order + offset, st));
    cp->tile_order = order + offset;
    return LATENTAM_OK;
}

void* frame_ws(latentam_ctx* ctx, int idx, size_t bytes) {
    if (bytes == 0) bytes = 256;
    if (ctx->frame_bytes[idx] >= bytes) return ctx->frame_ptr[idx];
    ++ctx->ws_generation;
    size_t nb = std::max(bytes, ctx->frame_bytes[idx] + ctx->frame_bytes[idx] / 4);
    nb = (nb + 4095) & ~(size_t)4095;
    if (ctx->frame_ptr[idx]) {
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) {
            cuda_error(e, "frame workspace regrow sync");
            return nullptr;
        }
        cudaFree(ctx->frame_ptr[idx]);
        ctx->frame_ptr[idx] = nullptr;
        ctx->frame_bytes[idx] = 0;
    }
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, nb);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        set_error("frame workspace allocation of %zu bytes failed: %s", nb, cudaGetErrorString(e));
        return nullptr;
    }
    ctx->frame_ptr[idx] = p;
    ctx->frame_bytes[idx] = nb;
    return p;
}

static void prof_fold(latentam_ctx* ctx, int stage) {
    StageProfile& P = ctx->prof[stage];
    for (int i = 0; i < P.used; ++i) {
        float ms = 0.f;
        if (cudaEventSynchronize(P.ev[2 * i + 1]) == cudaSuccess &&
            cudaEventElapsedTime(&ms, P.ev[2 * i], P.ev[2 * i + 1]) == cudaSuccess)
            P.acc_ms += ms;
        P.count += 1;
    }
    (void)cudaGetLastError();
    P.used = 0;
}

int prof_begin(latentam_ctx* ctx, int stage, cudaStream_t st) {
    StageProfile& P = ctx->prof[stage];
    if (P.used == kProfPairs) prof_fold(ctx, stage);
    const int i = P.used;
    while (P.created < 2 * (i + 1)) {
        if (cudaEventCreate(&P.ev[P.created]) != cudaSuccess) {
            (void)cudaGetLastError();
            return -1;
        }
        ++P.created;
    }
    if (cudaEventRecord(P.ev[2 * i], st) != cudaSuccess) {
        (void)cudaGetLastError();
        return -1;
    }
    P.used = i + 1;
    return i;
}

void prof_end(latentam_ctx* ctx, int stage, int idx, cudaStream_t st) {
    if (cudaEventRecord(ctx->prof[stage].ev[2 * idx + 1], st) != cudaSuccess) (void)cudaGetLastError();
}

}  // namespace lat

using namespace lat;

namespace {

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

latentam_status enter(latentam_ctx* ctx) {
    g_err[0] = '\0';
    if (!ctx) {
        set_error("null context");
        return LATENTAM_ERR_INVALID_ARG;
    }
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_error(e, "cudaSetDevice");
    return LATENTAM_OK;
}

// The loss parts of a step into loss_host (synchronises `st`), then the context's sticky
// device flags: a tensor-core wait that gave up -> TIMEOUT; a non-finite loss or a non-finite
// gradient fed to Adam -> NOT_FINITE.  Reported flags are cleared.
latentam_status read_loss(latentam_ctx* ctx, const double* lp, double* loss_host, cudaStream_t st) {
    cudaError_t e = cudaMemcpyAsync(loss_host, lp, sizeof(double) * LATENTAM_LOSS_PARTS, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_error(e, "copy loss");
    int* flags = reinterpret_cast<int*>(ctx->host_counts) + 4;
    e = cudaMemcpyAsync(flags, ctx->dev_flags, 2 * sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_error(e, "copy device flags");
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_error(e, "synchronise step");
    const bool timeout = flags[0] != 0, grad_bad = flags[1] != 0;
    if (timeout || grad_bad) {
        e = cudaMemsetAsync(ctx->dev_flags, 0, 2 * sizeof(int), st);
        if (e != cudaSuccess) return cuda_error(e, "clear device flags");
    }
    if (timeout) {
        set_error("a bounded wait of a tensor-core decode kernel gave up (the loss is NaN)");
        return LATENTAM_ERR_TIMEOUT;
    }
    if (grad_bad || !std::isfinite(loss_host[3])) {
        set_error("non-finite %s (loss %g)", grad_bad ? "gradient met the Adam update" : "loss", loss_host[3]);
        return LATENTAM_ERR_NOT_FINITE;
    }
    return LATENTAM_OK;
}

// The precision forms of the decode.  FP32: the split tensor-core form (every FP32 operand a hi /
// lo pair of BF16 terms, three MMAs per product, FP32 accumulation) where its shapes allow
// (M, D <= 1024), else the FMA-pipe kernels; FP32_FMA: the FMA-pipe kernels at every shape.
bool known_prec(latentam_precision p) {
    return p == LATENTAM_PREC_FP32 || p == LATENTAM_PREC_BF16 || p == LATENTAM_PREC_FP8 || p == LATENTAM_PREC_FP32_FMA;
}

latentam_status run_decode_loss_bwd(latentam_ctx* ctx, const DecodeArgs& a, latentam_precision prec, cudaStream_t st) {
    if (prec == LATENTAM_PREC_FP32 && decode_split_supported(a.d, a.M, a.D)) return decode_loss_bwd_split(ctx, a, st);
    if (prec == LATENTAM_PREC_FP32 || prec == LATENTAM_PREC_FP32_FMA) return decode_loss_bwd_f32(ctx, a, st);
    if (prec == LATENTAM_PREC_BF16 || prec == LATENTAM_PREC_FP8)
        return decode_loss_bwd_bf16(ctx, a, st, prec == LATENTAM_PREC_FP8);
    set_error("unknown precision %d", prec);
    return LATENTAM_ERR_INVALID_ARG;
}

latentam_status run_decode_fwd(latentam_ctx* ctx, const float* Q, int64_t n, int d, const float* K, const float* V,
                               int M, int D, float c, latentam_precision prec, float* F_hat, float* row_stats,
                               cudaStream_t st) {
    if (prec == LATENTAM_PREC_FP32 && decode_split_supported(d, M, D))
        return decode_fwd_split(ctx, Q, n, d, K, V, M, D, c, F_hat, row_stats, st);
    if (prec == LATENTAM_PREC_FP32 || prec == LATENTAM_PREC_FP32_FMA)
        return decode_fwd_f32(ctx, Q, n, d, K, V, M, D, c, F_hat, row_stats, st);
    if (prec == LATENTAM_PREC_BF16 || prec == LATENTAM_PREC_FP8)
        return decode_fwd_bf16(ctx, Q, n, d, K, V, M, D, c, F_hat, row_stats, st, prec == LATENTAM_PREC_FP8);
    set_error("unknown precision %d", prec);
    return LATENTAM_ERR_INVALID_ARG;
}

latentam_status check_camera(const latentam_camera* cam) {
    if (!cam) {
        set_error("null camera");
        return LATENTAM_ERR_INVALID_ARG;
    }
    if (cam->width < 1 || cam->height < 1 || cam->width > 16384 || cam->height > 16384) {
        set_error("image %dx%d outside 1..16384", cam->width, cam->height);
        return LATENTAM_ERR_UNSUPPORTED_SHAPE;
    }
    if (!(cam->fx > 0.f) || !(cam->fy > 0.f) || !(cam->z_near > 0.f)) {
        set_error("camera needs fx, fy, z_near > 0");
        return LATENTAM_ERR_INVALID_ARG;
    }
    return LATENTAM_OK;
}

latentam_status check_d(int d) {
    if (d != 16 && d != 32 && d != 64) {
        set_error("query dimension d=%d not in {16, 32, 64}", d);
        return LATENTAM_ERR_UNSUPPORTED_SHAPE;
    }
    return LATENTAM_OK;
}

latentam_status check_dict(int M, int D) {
    if (M < 32 || M > 1024 || M % 32 != 0) {
        set_error("dictionary size M=%d must be a multiple of 32 in [32, 1024]", M);
        return LATENTAM_ERR_UNSUPPORTED_SHAPE;
    }
    if (D < 128 || D > 2048 || D % 128 != 0) {
        set_error("value dimension D=%d must be a multiple of 128 in [128, 2048]", D);
        return LATENTAM_ERR_UNSUPPORTED_SHAPE;
    }
    return LATENTAM_OK;
}

#define REQUIRE(cond, ...)                       \
    do {                                         \
        if (!(cond)) {                           \
            set_error(__VA_ARGS__);              \
            return LATENTAM_ERR_INVALID_ARG;     \
        }                                        \
    } while (0)

latentam_status check_projected(const latentam_projected* p, int64_t n) {
    REQUIRE(p, "null projection");
    if (n == 0) return LATENTAM_OK;  // empty sets may carry null buffers
    REQUIRE(p->xy && p->conic_opacity && p->depth && p->rect && p->tiles_touched, "incomplete projection buffers");
    REQUIRE(aligned16(p->conic_opacity) && aligned16(p->rect) && (reinterpret_cast<uintptr_t>(p->xy) & 7u) == 0,
            "projection buffers must be 16-byte aligned");
    return LATENTAM_OK;
}

latentam_status check_bins(const latentam_bins* b, bool need_pairs) {
    REQUIRE(b && b->tile_ranges && aligned16(b->tile_ranges), "tile_ranges missing or not 16-byte aligned");
    REQUIRE(b->capacity >= 0, "negative pair capacity");
    if (need_pairs) REQUIRE(b->num_pairs >= 0 && b->num_pairs <= b->capacity, "bins hold no sorted pairs");
    REQUIRE(b->pair_ids || b->capacity == 0, "pair_ids missing");
    return LATENTAM_OK;
}

float logit_scale(const latentam_loss_cfg* cfg, int d) {
    return (cfg && cfg->logit_scale > 0.f) ? cfg->logit_scale : 1.0f / sqrtf((float)d);
}

}  // namespace

namespace {

// Runs `iters` iterations of `iteration(stream, render, step_dev)`.  With `graphable`, a
// configuration seen once before (its workspaces sized) is captured as one iteration on the
// context's stream and replayed; the Adam step then comes from ctx->step_dev.
template <class Iteration>
latentam_status run_iterations(latentam_ctx* ctx, bool graphable, const GraphKey& key, int iters, bool learn_f,
                               latentam_adam_cfg* adam, cudaStream_t st, Iteration&& iteration) {
    int gslot = -1;
    if (graphable && !key.overflow) {
        GraphCache& gc = *ctx->graphs;
        gslot = GraphCache::find(gc.key, gc.used, key);
        const bool failed = GraphCache::find(gc.failed, gc.failed_used, key) >= 0;
        if (gslot < 0 && !failed && GraphCache::find(gc.warm, gc.warm_used, key) >= 0) {
            cudaGraph_t graph = nullptr;
            const int64_t l0 = launch_count_now();
            cudaError_t e = cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal);
            latentam_status cs = e == cudaSuccess ? iteration(ctx->cap_stream, true, ctx->step_dev) : LATENTAM_ERR_CUDA;
            cudaError_t e2 = e == cudaSuccess ? cudaStreamEndCapture(ctx->cap_stream, &graph) : e;
            const int64_t captured = launch_count_now() - l0;
            launch_count_add(-captured);  // nothing ran yet
            cudaGraphExec_t exec = nullptr;
            if (cs == LATENTAM_OK && e2 == cudaSuccess && graph &&
                cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess) {
                const int slot = gc.next;
                if (gc.exec[slot]) {
                    cudaStreamSynchronize(st);  // a replay of the graph being dropped may be queued
                    cudaGraphExecDestroy(gc.exec[slot]);
                }
                gc.exec[slot] = exec;
                gc.key[slot] = key;
                gc.launches[slot] = captured;
                gc.next = (gc.next + 1) % GraphCache::kSlots;
                if (gc.used < GraphCache::kSlots) ++gc.used;
                gslot = slot;
            } else {
                (void)cudaGetLastError();
                GraphCache::put(gc.failed, gc.failed_used, gc.failed_next, key);
            }
            if (graph) cudaGraphDestroy(graph);
        } else if (gslot < 0 && !failed) {
            GraphCache::put(gc.warm, gc.warm_used, gc.warm_next, key);
        }
    }
    if (gslot >= 0) {
        GraphCache& gc = *ctx->graphs;
        LAT_TRY(launch_step_set(ctx->step_dev, adam->step - 1, st));
        for (int it = 0; it < iters; ++it) {
            cudaError_t e = cudaGraphLaunch(gc.exec[gslot], st);
            if (e != cudaSuccess) return cuda_error(e, "step graph launch");
            launch_count_add(gc.launches[gslot]);
        }
        adam->step += iters;
        return LATENTAM_OK;
    }
    for (int it = 0; it < iters; ++it) {
        LAT_TRY(iteration(st, it == 0 || learn_f, nullptr));
        adam->step += 1;
    }
    return LATENTAM_OK;
}

}  // namespace

extern "C" {

int32_t latentam_version(void) { return LATENTAM_ABI_VERSION; }

int64_t latentam_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

const char* latentam_last_error(void) { return g_err; }

int32_t latentam_num_tiles(const latentam_camera* cam) {
    if (!cam || cam->width < 1 || cam->height < 1) return 0;
    return ((cam->width + kTile - 1) / kTile) * ((cam->height + kTile - 1) / kTile);
}

latentam_status latentam_ctx_create(int32_t device, latentam_ctx** out) {
    g_err[0] = '\0';
    if (!out) {
        set_error("null output pointer");
        return LATENTAM_ERR_INVALID_ARG;
    }
    *out = nullptr;
    int count = 0;
    cudaError_t e = cudaGetDeviceCount(&count);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetDeviceCount");
    if (device < 0 || device >= count) {
        set_error("device %d not present (%d devices)", device, count);
        return LATENTAM_ERR_CUDA;
    }
    cudaDeviceProp prop;
    e = cudaGetDeviceProperties(&prop, device);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetDeviceProperties");
    if (!(prop.major == 10 && prop.minor == 3)) {
        set_error("device %d is sm_%d%d; this library is built for sm_103a (GB300) only", device, prop.major,
                  prop.minor);
        return LATENTAM_ERR_CUDA;
    }
    latentam_ctx* c = new (std::nothrow) latentam_ctx;
    if (!c) {
        set_error("host allocation failed");
        return LATENTAM_ERR_OUT_OF_MEMORY;
    }
    memset(c, 0, sizeof(*c));
    c->device = device;
    c->num_sms = prop.multiProcessorCount;
    c->cc_major = prop.major;
    c->cc_minor = prop.minor;
    c->use_graphs = 1;
    c->autotune = 1;
    c->graphs = new (std::nothrow) GraphCache();
    c->sort_graphs = new (std::nothrow) GraphCache();
    e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&c->step_dev, sizeof(int));
    if (e == cudaSuccess) e = cudaHostAlloc(reinterpret_cast<void**>(&c->host_counts),
                                                  sizeof(uint32_t) * (8 + 4 * LATENTAM_MAX_BATCH), cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaMalloc(&c->dev_flags, 4 * sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(c->dev_flags, 0, 4 * sizeof(int));
    if (e != cudaSuccess || !c->graphs || !c->sort_graphs) {
        latentam_ctx_destroy(c);
        if (e != cudaSuccess) return cuda_error(e, "context stream / counter");
        set_error("host allocation failed");
        return LATENTAM_ERR_OUT_OF_MEMORY;
    }
    // the allocation-free decode's static scratch: its address, resolved once per context with
    // the device current (this also loads the module that holds it)
    const latentam_status ss = decode_noalloc_setup(c);
    if (ss != LATENTAM_OK) {
        latentam_ctx_destroy(c);
        return ss;
    }
    *out = c;
    return LATENTAM_OK;
}

latentam_status latentam_ctx_destroy(latentam_ctx* ctx) {
    g_err[0] = '\0';
    if (!ctx) return LATENTAM_OK;
    cudaSetDevice(ctx->device);
    cudaError_t e = cudaDeviceSynchronize();
    for (int s = 0; s < WS_NUM_SLOTS; ++s)
        if (ctx->slot_ptr[s]) cudaFree(ctx->slot_ptr[s]);
    for (int s = 0; s < LATENTAM_NUM_STAGES; ++s)
        for (int i = 0; i < ctx->prof[s].created; ++i) cudaEventDestroy(ctx->prof[s].ev[i]);
    for (int i = 0; i < 8 * LATENTAM_MAX_BATCH; ++i)
        if (ctx->frame_ptr[i]) cudaFree(ctx->frame_ptr[i]);
    if (ctx->bin_streams_ready) {
        for (cudaStream_t b : ctx->bin_streams) cudaStreamDestroy(b);
        for (cudaEvent_t v : ctx->bin_events) cudaEventDestroy(v);
        for (cudaEvent_t v : ctx->iter_events) cudaEventDestroy(v);
    }
    if (ctx->graphs) {
        ctx->graphs->clear();
        delete ctx->graphs;
    }
    if (ctx->sort_graphs) {
        ctx->sort_graphs->clear();
        delete ctx->sort_graphs;
    }
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    if (ctx->step_dev) cudaFree(ctx->step_dev);
    if (ctx->host_counts) cudaFreeHost(ctx->host_counts);
    if (ctx->dev_flags) cudaFree(ctx->dev_flags);
    delete ctx;
    if (e != cudaSuccess) return cuda_error(e, "synchronise before destroy");
    return LATENTAM_OK;
}

latentam_status latentam_graphs_enable(latentam_ctx* ctx, int32_t enable) {
    LAT_TRY(enter(ctx));
    ctx->use_graphs = enable != 0;
    if (!enable) {
        cudaError_t e = cudaDeviceSynchronize();
        ctx->graphs->clear();
        ctx->sort_graphs->clear();
        if (e != cudaSuccess) return cuda_error(e, "synchronise before dropping graphs");
    }
    return LATENTAM_OK;
}

latentam_status latentam_test_wait_timeout(latentam_ctx* ctx, int32_t which) {
    LAT_TRY(enter(ctx));
    if (which == 0) {
        ctx->test_stall_sort = 1;
        return LATENTAM_OK;
    }
    if (which == 1) {
        // what a tensor-core kernel's bounded wait leaves behind when it gives up
        const int one = 1;
        cudaError_t e = cudaMemcpy(ctx->dev_flags, &one, sizeof(int), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_error(e, "raise the tensor-core wait flag");
        return LATENTAM_OK;
    }
    set_error("unknown wait %d (0: radix look-back of the next binning, 1: tensor-core flag)", which);
    return LATENTAM_ERR_INVALID_ARG;
}

latentam_status latentam_autotune_enable(latentam_ctx* ctx, int32_t enable) {
    LAT_TRY(enter(ctx));
    ctx->autotune = enable != 0;
    if (!enable) ctx->tune_used = ctx->tune_next = 0;
    return LATENTAM_OK;
}

latentam_status latentam_autotune_query(latentam_ctx* ctx, int32_t i, latentam_tune_choice* out, int32_t* count) {
    LAT_TRY(enter(ctx));
    if (!count) {
        set_error("count must not be NULL");
        return LATENTAM_ERR_INVALID_ARG;
    }
    *count = ctx->tune_used;
    if (!out) return LATENTAM_OK;
    if (i < 0 || i >= ctx->tune_used) {
        set_error("autotuner choice %d out of range (%d held)", i, ctx->tune_used);
        return LATENTAM_ERR_INVALID_ARG;
    }
    const auto& t = ctx->tune[i];
    *out = latentam_tune_choice{t.n, t.M, t.D, t.which, t.shape, t.z, t.ms};
    return LATENTAM_OK;
}

latentam_status latentam_profile_enable(latentam_ctx* ctx, int32_t enable) {
    LAT_TRY(enter(ctx));
    ctx->profiling = enable != 0;
    return LATENTAM_OK;
}

latentam_status latentam_profile_read(latentam_ctx* ctx, double* ms, int64_t* counts, int32_t reset) {
    LAT_TRY(enter(ctx));
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_error(e, "profile synchronise");
    for (int s = 0; s < LATENTAM_NUM_STAGES; ++s) {
        prof_fold(ctx, s);
        if (ms) ms[s] = ctx->prof[s].acc_ms;
        if (counts) counts[s] = ctx->prof[s].count;
        if (reset) {
            ctx->prof[s].acc_ms = 0.0;
            ctx->prof[s].count = 0;
        }
    }
    return LATENTAM_OK;
}

latentam_status latentam_project(latentam_ctx* ctx, const latentam_gaussians* g, const latentam_camera* cam,
                                 const latentam_projected* out, latentam_stream stream) {
    LAT_TRY(enter(ctx));
    LAT_TRY(check_camera(cam));
    REQUIRE(g && g->n >= 0, "bad Gaussian set");
    LAT_TRY(check_projected(out, g->n));
    if (g->n > 0) REQUIRE(g->means && g->quats && g->scales && g->opacities, "null Gaussian attribute");
    StageTimer tm(ctx, LATENTAM_STAGE_PROJECT, (cudaStream_t)stream);
    return launch_project(*g, cam_params(*cam), *out, (cudaStream_t)stream);
}

latentam_status latentam_sort(latentam_ctx* ctx, int32_t n, const latentam_projected* proj,
                              const latentam_camera* cam, latentam_bins* bins, latentam_stream stream) {
    LAT_TRY(enter(ctx));
    LAT_TRY(check_camera(cam));
    REQUIRE(n >= 0, "negative Gaussian count");
    LAT_TRY(check_projected(proj, n));
    LAT_TRY(check_bins(bins, false));
    StageTimer tm(ctx, LATENTAM_STAGE_SORT, (cudaStream_t)stream);
    return bin_and_sort(ctx, n, *proj, cam_params(*cam), bins, (cudaStream_t)stream);
}

latentam_status latentam_render_fwd(latentam_ctx* ctx, int32_t n, const latentam_projected* proj,
                                    const latentam_camera* cam, const latentam_bins* bins, const float* f, int32_t d,
                                    float* Q, float* T_final, int32_t* n_contrib, latentam_stream stream) {
    LAT_TRY(enter(ctx));
    LAT_TRY(check_camera(cam));
    LAT_TRY(check_d(d));
    LAT_TRY(check_projected(proj, n));
    LAT_TRY(check_bins(bins, true));
    REQUIRE(n >= 0 && (n == 0 || f), "bad queries");
    REQUIRE(Q && T_final && n_contrib, "null output");
    REQUIRE(aligned16(f) && aligned16(Q), "f and Q must be 16-byte aligned");
    StageTimer tm(ctx, LATENTAM_STAGE_RENDER_FWD, (cudaStream_t)stream);
    CamParams cp = cam_params(*cam);
    const size_t tiles = (size_t)cp.tiles_x * cp.tiles_y;
    LAT_TRY(ordered(ctx, &cp, *bins, 0, tiles, (cudaStream_t)stream));
    return launch_render_fwd(cp, *proj, *bins, f, d, Q, T_final, n_contrib, (cudaStream_t)stream);
}

latentam_status latentam_render_bwd(latentam_ctx* ctx, int32_t n, const latentam_projected* proj,
                                    const latentam_camera* cam, const latentam_bins* bins, const int32_t* n_contrib,
                                    const float* dQ, int32_t d, float* df, latentam_stream stream) {
    LAT_TRY(enter(ctx));
    LAT_TRY(check_camera(cam));
    LAT_TRY(check_d(d));
    LAT_TRY(check_projected(proj, n));
    LAT_TRY(check_bins(bins, true));
    REQUIRE(n >= 0 && n_contrib && dQ && (df || n == 0), "null argument");
    REQUIRE(aligned16(dQ), "dQ must be 16-byte aligned");
    if (n == 0) return LATENTAM_OK;
    StageTimer tm(ctx, LATENTAM_STAGE_RENDER_BWD, (cudaStream_t)stream);
    CamParams cp = cam_params(*cam);
    const size_t tiles = (size_t)cp.tiles_x * cp.tiles_y;
    LAT_TRY(ordered(ctx, &cp, *bins, 0, tiles, (cudaStream_t)stream));
    return launch_render_bwd(cp, *proj, *bins, n_contrib, dQ, d, df, n, (cudaStream_t)stream);
}

latentam_status latentam_decode_fwd(latentam_ctx* ctx, const float* Q, int64_t n, int32_t d, const float* K,
                                    const float* V, int32_t M, int32_t D, float logit_scale_, latentam_precision prec,
                                    float* F_hat, float* row_stats, latentam_stream stream) {
    LAT_TRY(enter(ctx));
    LAT_TRY(check_d(d));
    LAT_TRY(check_dict(M, D));
    REQUIRE(n >= 0 && (n == 0 || Q) && K && V, "null argument");
    REQUIRE(aligned16(Q) && aligned16(V) && aligned16(F_hat), "Q, V, F_hat must be 16-byte aligned");
    const float c = logit_scale_ > 0.f ? logit_scale_ : 1.0f / sqrtf((float)d);
    StageTimer tm(ctx, LATENTAM_STAGE_DECODE, (cudaStream_t)stream);
    return run_decode_fwd(ctx, Q, n, d, K, V, M, D, c, prec, F_hat, row_stats, (cudaStream_t)stream);
}

latentam_status latentam_decode_loss_bwd(latentam_ctx* ctx, const float* Q, int64_t n, int32_t d, const float* K,
                                         const float* V, const float* V0, int32_t M, int32_t D, const void* F,
                                         latentam_dtype F_dtype, const uint8_t* mask, const latentam_loss_cfg* cfg,
                                         latentam_precision prec, double* loss_parts, float* dQ, float* dK, float* dV,
                                         latentam_stream stream) {
    LAT_TRY(enter(ctx));
    LAT_TRY(check_d(d));
    LAT_TRY(check_dict(M, D));
    REQUIRE(cfg && loss_parts, "null config or loss output");
    REQUIRE(n >= 0 && (n == 0 || (Q && F)) && K && V && V0, "null argument");
    REQUIRE(F_dtype == LATENTAM_DTYPE_F32 || F_dtype == LATENTAM_DTYPE_BF16, "unknown target dtype %d", F_dtype);
    REQUIRE(aligned16(Q) && aligned16(V) && aligned16(V0) && aligned16(F) && aligned16(dQ) && aligned16(dV),
            "Q, V, V0, F, dQ, dV must be 16-byte aligned");
    DecodeArgs a;
    a.Q = Q;
    a.n = n;
    a.d = d;
    a.K = K;
    a.V = V;
    a.V0 = V0;
    a.M = M;
    a.D = D;
    a.c = logit_scale(cfg, d);
    a.F = F;
    a.F_dtype = F_dtype;
    a.mask = mask;
    a.cfg = *cfg;
    a.loss_parts = loss_parts;
    a.dQ = dQ;
    a.dK = dK;
    a.dV = dV;
    StageTimer tm(ctx, LATENTAM_STAGE_DECODE, (cudaStream_t)stream);
    return run_decode_loss_bwd(ctx, a, prec, (cudaStream_t)stream);
}

namespace {

latentam_status paper_buffers(latentam_ctx* ctx, int64_t n, int ds, int M, int df, lat::PaperBuffers* b) {
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t nn = (size_t)std::max<int64_t>(n, 1), f = sizeof(float);
    size_t off[9], o = 0;
    off[0] = o, o += up(f * M * ds);    // K
    off[1] = o, o += up(f * M);         // nrm
    off[2] = o, o += up(f * ds * ds);   // G
    off[3] = o, o += up(f * nn * ds);   // Q'
    off[4] = o, o += up(f * nn);        // r
    off[5] = o, o += up(f * nn * ds);   // dQ'
    off[6] = o, o += up(f * M * ds);    // dK
    off[7] = o, o += up(f * M * df);    // dV
    off[8] = o, o += up(f * ds * ds);   // C
    char* base = static_cast<char*>(lat::ws(ctx, lat::WS_PAPER, o));
    if (!base) return LATENTAM_ERR_OUT_OF_MEMORY;
    float** dst[9] = {&b->K, &b->nrm, &b->G, &b->Qp, &b->r, &b->dQp, &b->dK, &b->dV, &b->Cm};
    for (int i = 0; i < 9; ++i) *dst[i] = reinterpret_cast<float*>(base + off[i]);
    return LATENTAM_OK;
}

latentam_status check_paper(int64_t n, int ds, const float* Q, const float* W, const float* D, int M, int df,
                            float tau) {
    LAT_TRY(check_d(ds));
    LAT_TRY(check_dict(M, df));
    REQUIRE(n >= 0 && (n == 0 || Q) && W && D, "null argument");
    REQUIRE(aligned16(Q) && aligned16(W) && aligned16(D), "Q, W, D must be 16-byte aligned");
    REQUIRE(tau > 0.f && isfinite(tau), "temperature tau=%g must be positive and finite", (double)tau);
    return LATENTAM_OK;
}

}  // namespace

latentam_status latentam_decode_fwd_paper(latentam_ctx* ctx, const float* Q, int64_t n, int32_t ds, const float* W,
                                          const float* D, int32_t M, int32_t df, float tau, latentam_precision prec,
                                          float* F_hat, float* row_stats, latentam_stream stream) {
    LAT_TRY(enter(ctx));
    LAT_TRY(check_paper(n, ds, Q, W, D, M, df, tau));
    REQUIRE(aligned16(F_hat), "F_hat must be 16-byte aligned");
    REQUIRE(known_prec(prec), "unknown precision %d", prec);
    lat::PaperBuffers b;
    LAT_TRY(paper_buffers(ctx, n, ds, M, df, &b));
    const lat::PaperArgs a{Q, n, ds, W, D, M, df};
    cudaStream_t st = (cudaStream_t)stream;
    StageTimer tm(ctx, LATENTAM_STAGE_DECODE, st);
    LAT_TRY(lat::paper_prepare(ctx, a, b, st));
    return run_decode_fwd(ctx, b.Qp, n, ds, b.K, D, M, df, 1.0f / tau, prec, F_hat, row_stats, st);
}

latentam_status latentam_decode_loss_bwd_paper(latentam_ctx* ctx, const float* Q, int64_t n, int32_t ds,
                                               const float* W, const float* D, const float* D0, int32_t M,
                                               int32_t df, float tau, const void* F, latentam_dtype F_dtype,
                                               const uint8_t* mask, const latentam_loss_cfg* cfg,
                                               latentam_precision prec, double* loss_parts, float* dQ, float* dW,
                                               float* dD, latentam_stream stream) {
    LAT_TRY(enter(ctx));
    LAT_TRY(check_paper(n, ds, Q, W, D, M, df, tau));
    REQUIRE(cfg && loss_parts && D0 && (n == 0 || F), "null argument");
    REQUIRE(F_dtype == LATENTAM_DTYPE_F32 || F_dtype == LATENTAM_DTYPE_BF16, "unknown target dtype %d", F_dtype);
    REQUIRE(aligned16(D0) && aligned16(F) && aligned16(dQ) && aligned16(dW) && aligned16(dD),
            "D0, F, dQ, dW, dD must be 16-byte aligned");
    REQUIRE(known_prec(prec), "unknown precision %d", prec);
    lat::PaperBuffers b;
    LAT_TRY(paper_buffers(ctx, n, ds, M, df, &b));
    const lat::PaperArgs pa{Q, n, ds, W, D, M, df};
    cudaStream_t st = (cudaStream_t)stream;
    StageTimer tm(ctx, LATENTAM_STAGE_DECODE, st);
    LAT_TRY(lat::paper_prepare(ctx, pa, b, st));
    DecodeArgs a;
    a.Q = b.Qp;
    a.n = n;
    a.d = ds;
    a.K = b.K;
    a.V = D;
    a.V0 = D0;
    a.M = M;
    a.D = df;
    a.c = 1.0f / tau;
    a.F = F;
    a.F_dtype = F_dtype;
    a.mask = mask;
    a.cfg = *cfg;
    a.loss_parts = loss_parts;
    a.dQ = (dQ || dW) ? b.dQp : nullptr;  // dW needs dQ' for the query-norm term
    a.dK = b.dK;
    a.dV = b.dV;
    LAT_TRY(run_decode_loss_bwd(ctx, a, prec, st));
    return lat::paper_chain(ctx, pa, b, dQ, dW, dD, st);
}

latentam_status latentam_decode_loss_bwd_noalloc(latentam_ctx* ctx, const float* Q, int64_t n, int32_t d,
                                                 const float* K, const float* V, const float* V0, int32_t M, int32_t D,
                                                 const void* F, latentam_dtype F_dtype, const uint8_t* mask,
                                                 const latentam_loss_cfg* cfg, double* loss_parts, float* dQ,
                                                 float* dK, float* dV, latentam_stream stream) {
    LAT_TRY(enter(ctx));
    LAT_TRY(check_d(d));
    LAT_TRY(check_dict(M, D));
    REQUIRE(cfg && loss_parts, "null config or loss output");
    REQUIRE(n >= 0 && (n == 0 || (Q && F)) && K && V && V0, "null argument");
    REQUIRE(F_dtype == LATENTAM_DTYPE_F32 || F_dtype == LATENTAM_DTYPE_BF16, "unknown target dtype %d", F_dtype);
    REQUIRE(aligned16(Q) && aligned16(V) && aligned16(V0) && aligned16(F) && aligned16(dQ) && aligned16(dV),
            "Q, V, V0, F, dQ, dV must be 16-byte aligned");
    DecodeArgs a;
    a.Q = Q;
    a.n = n;
    a.d = d;
    a.K = K;
    a.V = V;
    a.V0 = V0;
    a.M = M;
    a.D = D;
    a.c = logit_scale(cfg, d);
    a.F = F;
    a.F_dtype = F_dtype;
    a.mask = mask;
    a.cfg = *cfg;
    a.loss_parts = loss_parts;
    a.dQ = dQ;
    a.dK = dK;
    a.dV = dV;
    return decode_loss_bwd_f32_noalloc(ctx, a, (cudaStream_t)stream);
}

latentam_status latentam_backward(latentam_ctx* ctx, int32_t n, const latentam_projected* proj,
                                  const latentam_camera* cam, const latentam_bins* bins, const int32_t* n_contrib,
                                  const float* Q, int32_t d, const float* K, const float* V, const float* V0,
                                  int32_t M, int32_t D, const void* F, latentam_dtype F_dtype, const uint8_t* mask,
                                  const latentam_loss_cfg* cfg, latentam_precision prec, double* loss_parts,
                                  float* dQ_scratch, float* df, float* dK, float* dV, latentam_stream stream) {
    LAT_TRY(enter(ctx));
    LAT_TRY(check_camera(cam));
    REQUIRE(dQ_scratch || !df, "df needs dQ_scratch");
    const int64_t npix = (int64_t)cam->width * cam->height;
    LAT_TRY(latentam_decode_loss_bwd(ctx, Q, npix, d, K, V, V0, M, D, F, F_dtype, mask, cfg, prec, loss_parts,
                                     df ? dQ_scratch : nullptr, dK, dV, stream));
    if (!df) return LATENTAM_OK;
    return latentam_render_bwd(ctx, n, proj, cam, bins, n_contrib, dQ_scratch, d, df, stream);
}

namespace {

latentam_status check_masks(int32_t S, int64_t E, int64_t npix, int d, const int32_t* off, const int32_t* pix) {
    LAT_TRY(check_d(d));
    REQUIRE(S >= 0 && E >= 0 && npix >= 0, "negative mask count, entry count or pixel count");
    REQUIRE(E <= INT32_MAX, "n_entries=%lld exceeds the int32 offsets", (long long)E);
    REQUIRE(S == 0 || off, "null mask offsets");
    REQUIRE(E == 0 || pix, "null mask pixels");
    return LATENTAM_OK;
}

// The plan of a mask set in the context's WS_MASKS slot, followed by `extra` bytes.
latentam_status mask_plan(latentam_ctx* ctx, const int32_t* off, const int32_t* pix, int64_t E, int32_t S,
                          int64_t npix, int d, size_t extra, MaskPlan* p, char** extra_ptr) {
    const size_t pb = (mask_plan_bytes(S, E, d) + 255) & ~(size_t)255;
    char* base = static_cast<char*>(ws(ctx, WS_MASKS, pb + extra));
    if (!base) return LATENTAM_ERR_OUT_OF_MEMORY;
    mask_plan_carve(base, off, pix, E, S, npix, d, p);
    if (extra_ptr) *extra_ptr = base + pb;
    return LATENTAM_OK;
}

}  // namespace

latentam_status latentam_pool_queries(latentam_ctx* ctx, const float* Q, int64_t npix, int32_t d,
                                      const int32_t* mask_offsets, const int32_t* mask_pixels, int64_t n_entries,
                                      int32_t S, float* Qm, latentam_stream stream) {
    LAT_TRY(enter(ctx));
    LAT_TRY(check_masks(S, n_entries, npix, d, mask_offsets, mask_pixels));
    REQUIRE((npix == 0 || Q) && (S == 0 || Qm), "null Q or Qm");
    REQUIRE(aligned16(Q) && aligned16(Qm), "Q, Qm must be 16-byte aligned");
    MaskPlan p;
    LAT_TRY(mask_plan(ctx, mask_offsets, mask_pixels, n_entries, S, npix, d, 0, &p, nullptr));
    cudaStream_t st = (cudaStream_t)stream;
    LAT_TRY(launch_mask_plan(p, st));
    return launch_pool_fwd(p, Q, d, Qm, st);
}

latentam_status latentam_pool_queries_bwd(latentam_ctx* ctx, const float* dQm, int32_t S, int32_t d,
                                          const int32_t* mask_offsets, const int32_t* mask_pixels, int64_t n_entries,
                                          int64_t npix, float* dQ, latentam_stream stream) {
    LAT_TRY(enter(ctx));
    LAT_TRY(check_masks(S, n_entries, npix, d, mask_offsets, mask_pixels));
    REQUIRE((S == 0 || dQm) && (npix == 0 || dQ), "null dQm or dQ");
    REQUIRE(aligned16(dQm) && aligned16(dQ), "dQm, dQ must be 16-byte aligned");
    MaskPlan p;
    LAT_TRY(mask_plan(ctx, mask_offsets, mask_pixels, n_entries, S, npix, d, 0, &p, nullptr));
    cudaStream_t st = (cudaStream_t)stream;
    LAT_TRY(launch_mask_plan(p, st));
    return launch_pool_bwd(p, dQm, d, dQ, st);
}

latentam_status latentam_stream_kmeans(latentam_ctx* ctx, const float* F, int64_t n, int32_t D,
                                       const uint8_t* valid, const int32_t* init_idx, int32_t k_micro,
                                       int32_t iters_local, int32_t iters_global, float* centres, float* weights,
                                       int32_t K, float* micro_centres, float* micro_weights, int32_t* micro_assign,
                                       int32_t* point_assign, latentam_stream stream) {
    LAT_TRY(enter(ctx));
    REQUIRE(F && init_idx && centres && weights, "null argument");
    if (!(n >= 1 && k_micro >= 1 && k_micro <= 32 && k_micro <= n && K >= 1 && K <= 8192 && D >= 4 && D % 4 == 0 &&
          D <= 1024)) {
        set_error("stream_kmeans: unsupported shape n=%lld D=%d k_micro=%d K=%d", (long long)n, D, k_micro, K);
        return LATENTAM_ERR_UNSUPPORTED_SHAPE;
    }
    REQUIRE(iters_local >= 1 && iters_global >= 1, "iteration counts must be >= 1");
    REQUIRE(aligned16(F) && aligned16(centres) && aligned16(micro_centres), "F and centres must be 16-byte aligned");
    KMeansArgs a{F, n, D, valid, init_idx, k_micro, iters_local, iters_global, centres, weights, K,
                 micro_centres, micro_weights, micro_assign, point_assign};
    return stream_kmeans(ctx, a, (cudaStream_t)stream);
}

latentam_status latentam_adam(latentam_ctx* ctx, int32_t count, float* const* params, const float* const* grads,
                              float* const* m, float* const* v, const int64_t* sizes, const float* lrs,
                              const latentam_adam_cfg* cfg, latentam_stream stream) {
    LAT_TRY(enter(ctx));
    REQUIRE(cfg && count >= 0 && (count == 0 || (params && grads && m && v && sizes && lrs)), "null argument");
    AdamTensor t[8];
    REQUIRE(count <= 8, "at most 8 tensors per call");
    for (int k = 0; k < count; ++k) {
        REQUIRE(sizes[k] >= 0 && (sizes[k] == 0 || (params[k] && grads[k] && m[k] && v[k])), "bad tensor %d", k);
        t[k] = AdamTensor{params[k], grads[k], m[k], v[k], sizes[k], lrs[k]};
    }
    StageTimer tm(ctx, LATENTAM_STAGE_ADAM, (cudaStream_t)stream);
    return launch_adam(ctx, t, count, cfg->beta1, cfg->beta2, cfg->eps, cfg->step, (cudaStream_t)stream);
}

latentam_status latentam_backward_full(latentam_ctx* ctx, const latentam_gaussians* g, const float* colours,
                                       const float* f, int32_t d, const latentam_camera* cam, const float* K,
                                       const float* V, const float* V0, int32_t M, int32_t D, const void* F,
                                       latentam_dtype F_dtype, const uint8_t* mask, const float* image,
                                       const float* depth, const latentam_loss_cfg* cfg,
                                       const latentam_image_cfg* icfg, latentam_precision prec, double* loss_parts,
                                       float* d_means, float* d_quats, float* d_scales, float* d_opacities,
                                       float* d_colours, float* df, float* dK, float* dV, latentam_stream stream) {
    LAT_TRY(enter(ctx));
    REQUIRE(g && cam && cfg && icfg && loss_parts, "null argument");
    LAT_TRY(check_camera(cam));
    LAT_TRY(check_d(d));
    LAT_TRY(check_dict(M, D));
    const int N = g->n;
    REQUIRE(N >= 0, "negative Gaussian count");
    REQUIRE(K && V && V0 && image && depth && F && dK && dV, "null dictionary, target or gradient");
    if (N > 0)
        REQUIRE(g->means && g->quats && g->scales && g->opacities && colours && f && d_means && d_quats &&
                    d_scales && d_opacities && d_colours && df,
                "null Gaussian attribute or gradient");
    REQUIRE(aligned16(f) && aligned16(df), "f and df must be 16-byte aligned");
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t npix = (int64_t)cam->width * cam->height;
    const int64_t tiles = latentam_num_tiles(cam);
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    // projection and bins in the step's buffers
    const size_t o_xy = 0, o_co = o_xy + up(8 * (size_t)N), o_dp = o_co + up(16 * (size_t)N),
                 o_rc = o_dp + up(4 * (size_t)N), o_tt = o_rc + up(16 * (size_t)N), o_tr = o_tt + up(4 * (size_t)N),
                 o_end = o_tr + up(8 * (size_t)tiles);
    char* pb = static_cast<char*>(ws(ctx, WS_STEP_PROJ, o_end));
    if (!pb) return LATENTAM_ERR_OUT_OF_MEMORY;
    latentam_projected proj{reinterpret_cast<float*>(pb + o_xy), reinterpret_cast<float*>(pb + o_co),
                            reinterpret_cast<float*>(pb + o_dp), reinterpret_cast<int32_t*>(pb + o_rc),
                            reinterpret_cast<int32_t*>(pb + o_tt)};
    latentam_bins bins{};
    bins.tile_ranges = reinterpret_cast<int32_t*>(pb + o_tr);
    bins.pair_ids = static_cast<int32_t*>(ctx->slot_ptr[WS_STEP_PAIRS]);
    bins.capacity = (int64_t)(ctx->slot_bytes[WS_STEP_PAIRS] / sizeof(int32_t));
    CamParams cp = cam_params(*cam);
    {
        StageTimer tm(ctx, LATENTAM_STAGE_PROJECT, st);
        LAT_TRY(launch_project(*g, cp, proj, st));
    }
    latentam_status s;
    {
        StageTimer tm(ctx, LATENTAM_STAGE_SORT, st);
        s = bin_and_sort(ctx, N, proj, cp, &bins, st);
        if (s == LATENTAM_ERR_CAPACITY) {
            bins.pair_ids = static_cast<int32_t*>(ws(ctx, WS_STEP_PAIRS, sizeof(int32_t) * (size_t)bins.num_pairs));
            if (!bins.pair_ids) return LATENTAM_ERR_OUT_OF_MEMORY;
            bins.capacity = bins.num_pairs;
            s = bin_and_sort(ctx, N, proj, cp, &bins, st);
        }
        if (s == LATENTAM_OK) s = ordered(ctx, &cp, bins, 0, (size_t)tiles, st);
    }
    LAT_TRY(s);
    // images, their gradients and the screen-space gradients
    const size_t nn = (size_t)std::max<int64_t>(npix, 1);
    const size_t i_q = 0, i_c = i_q + up(4 * nn * d), i_z = i_c + up(12 * nn), i_t = i_z + up(4 * nn),
                 i_n = i_t + up(4 * nn), i_dq = i_n + up(4 * nn), i_dc = i_dq + up(4 * nn * d),
                 i_dz = i_dc + up(12 * nn), i_g = i_dz + up(4 * nn),
                 i_end = i_g + up(32 * (size_t)std::max(N, 1));
    char* ib = static_cast<char*>(ws(ctx, WS_FULL_IMG, i_end));
    if (!ib) return LATENTAM_ERR_OUT_OF_MEMORY;
    float* Q = reinterpret_cast<float*>(ib + i_q);
    float* C = reinterpret_cast<float*>(ib + i_c);
    float* Z = reinterpret_cast<float*>(ib + i_z);
    float* T = reinterpret_cast<float*>(ib + i_t);
    int32_t* nc = reinterpret_cast<int32_t*>(ib + i_n);
    float* dQ = reinterpret_cast<float*>(ib + i_dq);
    float* dC = reinterpret_cast<float*>(ib + i_dc);
    float* dZ = reinterpret_cast<float*>(ib + i_dz);
    float* dgeo = reinterpret_cast<float*>(ib + i_g);
    {
        StageTimer tm(ctx, LATENTAM_STAGE_RENDER_FWD, st);
        LAT_TRY(launch_render_full(cp, proj, bins, f, d, colours, Q, C, Z, T, nc, st));
    }
    LAT_TRY(latentam_decode_loss_bwd(ctx, Q, npix, d, K, V, V0, M, D, F, F_dtype, mask, cfg, prec, loss_parts, dQ,
                                     dK, dV, stream));
    // the image losses and the geometry backward count as the render backward stage
    StageTimer tm(ctx, LATENTAM_STAGE_RENDER_BWD, st);
    LAT_TRY(launch_image_loss(ctx, C, Z, image, depth, cam->width, cam->height, *icfg, loss_parts, dC, dZ, st));
    if (N == 0) return LATENTAM_OK;
    LAT_TRY(launch_render_bwd_full(cp, proj, bins, f, d, colours, nc, Q, C, Z, dQ, dC, dZ, df, d_colours, dgeo, N,
                                   st));
    return launch_project_bwd(*g, cp, dgeo, d_means, d_quats, d_scales, d_opacities, st);
}

// The side streams and events of concurrent batch binning and of the render backward branch of
// an iteration (created once per context).
latentam_status bin_streams(latentam_ctx* ctx) {
    if (ctx->bin_streams_ready) return LATENTAM_OK;
    cudaStream_t sides[8] = {};
    cudaEvent_t bev[9] = {}, iev[2] = {};
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < 8 && e == cudaSuccess; ++i) e = cudaStreamCreateWithFlags(&sides[i], cudaStreamNonBlocking);
    for (int i = 0; i < 9 && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&bev[i], cudaEventDisableTiming);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&iev[i], cudaEventDisableTiming);
    if (e != cudaSuccess) {  // release what was created
        for (cudaStream_t x : sides)
            if (x) cudaStreamDestroy(x);
        for (cudaEvent_t x : bev)
            if (x) cudaEventDestroy(x);
        for (cudaEvent_t x : iev)
            if (x) cudaEventDestroy(x);
        return cuda_error(e, "side streams");
    }
    for (int i = 0; i < 8; ++i) ctx->bin_streams[i] = sides[i];
    for (int i = 0; i < 9; ++i) ctx->bin_events[i] = bev[i];
    for (int i = 0; i < 2; ++i) ctx->iter_events[i] = iev[i];
    ctx->bin_streams_ready = 1;
    return LATENTAM_OK;
}

// The render backward of an iteration as a branch of its own: `body` runs on a side stream that
// waits for everything enqueued on `s` so far (the decode up to its final dQ); join_branch makes `s`
// wait for the branch.  Inside a stream capture the branch becomes parallel graph nodes, so the
// render backward overlaps the decode's pixel reductions of dV and dK.
latentam_status fork_branch(latentam_ctx* ctx, cudaStream_t s,
                            const std::function<latentam_status(cudaStream_t)>& body) {
    LAT_TRY(bin_streams(ctx));
    cudaStream_t side = ctx->bin_streams[0];
    cudaError_t e = cudaEventRecord(ctx->iter_events[0], s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(side, ctx->iter_events[0], 0);
    if (e != cudaSuccess) return cuda_error(e, "fork the render backward");
    const latentam_status r = body(side);
    e = cudaEventRecord(ctx->iter_events[1], side);
    if (e != cudaSuccess) return cuda_error(e, "end the render backward branch");
    return r;
}
latentam_status join_branch(latentam_ctx* ctx, cudaStream_t s) {
    cudaError_t e = cudaStreamWaitEvent(s, ctx->iter_events[1], 0);
    return e == cudaSuccess ? LATENTAM_OK : cuda_error(e, "join the render backward");
}

latentam_status latentam_step(latentam_ctx* ctx, const latentam_frame* frame, latentam_params* params,
                              const latentam_loss_cfg* cfg, latentam_adam_cfg* adam, int32_t iters, int32_t learn_f,
                              latentam_precision prec, double* loss_host, latentam_stream stream) {
    LAT_TRY(enter(ctx));
    REQUIRE(frame && params && cfg && adam && iters >= 0, "null argument");
    LAT_TRY(check_camera(&frame->camera));
    LAT_TRY(check_d(params->d));
    LAT_TRY(check_dict(params->M, params->D));
    const latentam_gaussians& g = frame->gaussians;
    REQUIRE(g.n >= 0, "negative Gaussian count");
    REQUIRE(params->f && params->K && params->V && params->V0 && params->m_K && params->v_K && params->m_V &&
                params->v_V && (!learn_f || (params->m_f && params->v_f)),
            "null parameter or moment");
    cudaStream_t st = (cudaStream_t)stream;
    const int d = params->d, M = params->M, D = params->D;
    const float tau = params->tau;
    REQUIRE(tau >= 0.f && isfinite(tau), "tau=%g must be 0 (free keys) or positive", (double)tau);
    const bool paper = tau > 0.f;
    const int64_t ksize = paper ? (int64_t)d * D : (int64_t)M * d;  // K holds W (d x D) in the paper form
    const int N = g.n;
    const latentam_camera& cam = frame->camera;
    const int64_t npix = (int64_t)cam.width * cam.height;
    const int64_t tiles = latentam_num_tiles(&cam);

    // projection + bins in the context's own buffers (256-byte aligned sub-buffers)
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t o_xy = 0, o_co = o_xy + up(8 * (size_t)N), o_dp = o_co + up(16 * (size_t)N),
                 o_rc = o_dp + up(4 * (size_t)N), o_tt = o_rc + up(16 * (size_t)N), o_tr = o_tt + up(4 * (size_t)N),
                 o_end = o_tr + up(8 * (size_t)tiles);
    char* pb = static_cast<char*>(ws(ctx, WS_STEP_PROJ, o_end));
    if (!pb) return LATENTAM_ERR_OUT_OF_MEMORY;
    latentam_projected proj{reinterpret_cast<float*>(pb + o_xy), reinterpret_cast<float*>(pb + o_co),
                            reinterpret_cast<float*>(pb + o_dp), reinterpret_cast<int32_t*>(pb + o_rc),
                            reinterpret_cast<int32_t*>(pb + o_tt)};
    latentam_bins bins{};
    bins.tile_ranges = reinterpret_cast<int32_t*>(pb + o_tr);
    bins.pair_ids = static_cast<int32_t*>(ctx->slot_ptr[WS_STEP_PAIRS]);
    bins.capacity = (int64_t)(ctx->slot_bytes[WS_STEP_PAIRS] / sizeof(int32_t));
    if (N > 0) REQUIRE(g.means && g.quats && g.scales && g.opacities, "null Gaussian attribute");
    {
        StageTimer tm(ctx, LATENTAM_STAGE_PROJECT, st);
        LAT_TRY(launch_project(g, cam_params(cam), proj, st));
    }
    latentam_status s;
    {
        StageTimer tm(ctx, LATENTAM_STAGE_SORT, st);
        s = bin_and_sort(ctx, N, proj, cam_params(cam), &bins, st);
    }
    if (s == LATENTAM_ERR_CAPACITY) {
        bins.pair_ids = static_cast<int32_t*>(ws(ctx, WS_STEP_PAIRS, sizeof(int32_t) * (size_t)bins.num_pairs));
        if (!bins.pair_ids) return LATENTAM_ERR_OUT_OF_MEMORY;
        bins.capacity = bins.num_pairs;
        // the projection buffers are intact; only the binning is redone
        pb = static_cast<char*>(ctx->slot_ptr[WS_STEP_PROJ]);
        StageTimer tm(ctx, LATENTAM_STAGE_SORT, st);
        s = bin_and_sort(ctx, N, proj, cam_params(cam), &bins, st);
    }
    LAT_TRY(s);

    // images and gradients
    const size_t i_q = 0, i_t = i_q + up(4 * (size_t)npix * d), i_n = i_t + up(4 * (size_t)npix),
                 i_dq = i_n + up(4 * (size_t)npix), i_end = i_dq + up(4 * (size_t)npix * d);
    char* ib = static_cast<char*>(ws(ctx, WS_STEP_IMG, i_end));
    const size_t g_df = 0, g_dk = g_df + up(4 * (size_t)N * d), g_dv = g_dk + up(4 * (size_t)ksize),
                 g_lp = g_dv + up(4 * (size_t)M * D), g_end = g_lp + up(8 * LATENTAM_LOSS_PARTS);
    char* gb = static_cast<char*>(ws(ctx, WS_STEP_GRAD, g_end));
    if (!ib || !gb) return LATENTAM_ERR_OUT_OF_MEMORY;
    float* Q = reinterpret_cast<float*>(ib + i_q);
    float* T = reinterpret_cast<float*>(ib + i_t);
    int32_t* nc = reinterpret_cast<int32_t*>(ib + i_n);
    float* dQ = reinterpret_cast<float*>(ib + i_dq);
    float* df = reinterpret_cast<float*>(gb + g_df);
    float* dK = reinterpret_cast<float*>(gb + g_dk);
    float* dV = reinterpret_cast<float*>(gb + g_dv);
    double* lp = reinterpret_cast<double*>(gb + g_lp);
    CamParams cp = cam_params(cam);
    {
        StageTimer tm(ctx, LATENTAM_STAGE_SORT, st);
        LAT_TRY(ordered(ctx, &cp, bins, 0, (size_t)cp.tiles_x * cp.tiles_y, st));
    }
    // mask-pooled targets: the plan of the mask set (once per call) and the pooled queries
    const int32_t S = frame->n_masks;
    const bool pooled = S > 0;
    MaskPlan plan{};
    float *Qm = nullptr, *dQm = nullptr;
    if (pooled) {
        LAT_TRY(check_masks(S, frame->n_mask_entries, npix, d, frame->mask_offsets, frame->mask_pixels));
        const size_t qb = up(4 * (size_t)S * d);
        char* xb = nullptr;
        LAT_TRY(mask_plan(ctx, frame->mask_offsets, frame->mask_pixels, frame->n_mask_entries, S, npix, d, 2 * qb,
                          &plan, &xb));
        Qm = reinterpret_cast<float*>(xb);
        dQm = reinterpret_cast<float*>(xb + qb);
        LAT_TRY(launch_mask_plan(plan, st));
    }
    const float* Qdec = pooled ? Qm : Q;
    const int64_t ndec = pooled ? (int64_t)S : npix;
    // one iteration on stream `s`: render (and pool), decode + loss + backward, render backward
    // (through the pooling's adjoint), Adam (with the step read from step_dev when it is set:
    // graph replays)
    auto iteration = [&](cudaStream_t s, bool render, const int* step_dev) -> latentam_status {
        if (render) {
            StageTimer tm(ctx, LATENTAM_STAGE_RENDER_FWD, s);
            LAT_TRY(launch_render_fwd(cp, proj, bins, params->f, d, Q, T, nc, s));
            if (pooled) LAT_TRY(launch_pool_fwd(plan, Q, d, Qm, s));
        }
        float* dQd = learn_f ? (pooled ? dQm : dQ) : nullptr;
        auto render_bwd = [&](cudaStream_t b) -> latentam_status {
            StageTimer tm(ctx, LATENTAM_STAGE_RENDER_BWD, b);
            if (pooled) LAT_TRY(launch_pool_bwd(plan, dQm, d, dQ, b));
            return launch_render_bwd(cp, proj, bins, nc, dQ, d, df, N, b);
        };
        // the render backward needs only dQ: it branches off once the decode has made it final
        const std::function<latentam_status(cudaStream_t)> fork = [&](cudaStream_t ds) {
            return fork_branch(ctx, ds, render_bwd);
        };
        // (not under the stage timers: each stage is then timed on its own)
        const bool branch = learn_f && N > 0 && !paper && !ctx->profiling;
        ctx->after_dq = branch ? &fork : nullptr;
        ctx->after_dq_called = 0;
        latentam_status sd;
        if (paper)
            sd = latentam_decode_loss_bwd_paper(ctx, Qdec, ndec, d, params->K, params->V, params->V0, M, D, tau,
                                                frame->F, frame->F_dtype, frame->mask, cfg, prec, lp, dQd, dK, dV, s);
        else
            sd = latentam_decode_loss_bwd(ctx, Qdec, ndec, d, params->K, params->V, params->V0, M, D, frame->F,
                                          frame->F_dtype, frame->mask, cfg, prec, lp, dQd, dK, dV, s);
        ctx->after_dq = nullptr;
        const bool joined = ctx->after_dq_called != 0;
        if (joined) LAT_TRY(join_branch(ctx, s));  // joined even when the decode failed after the fork
        LAT_TRY(sd);
        if (learn_f && N > 0 && !joined) LAT_TRY(render_bwd(s));
        AdamTensor t[3];
        int cnt = 0;
        if (learn_f) t[cnt++] = AdamTensor{params->f, df, params->m_f, params->v_f, (int64_t)N * d, adam->lr_f};
        t[cnt++] = AdamTensor{params->K, dK, params->m_K, params->v_K, ksize, adam->lr_dict};
        t[cnt++] = AdamTensor{params->V, dV, params->m_V, params->v_V, (int64_t)M * D, adam->lr_dict};
        StageTimer tm(ctx, LATENTAM_STAGE_ADAM, s);
        if (step_dev) LAT_TRY(launch_step_advance(const_cast<int*>(step_dev), s));
        return launch_adam(ctx, t, cnt, adam->beta1, adam->beta2, adam->eps, adam->step, s, step_dev);
    };
    // Stage I iterations (all of them render) replay one captured graph
    GraphKey key;
    const bool graphable = ctx->use_graphs && learn_f && !ctx->profiling && iters > 0;
    if (graphable) {
        const void* ptrs[] = {params->f, params->K, params->V, params->V0, params->m_f, params->v_f, params->m_K,
                              params->v_K, params->m_V, params->v_V, frame->F, frame->mask, Q, T, nc, dQ, df, dK,
                              dV, lp, proj.xy, proj.conic_opacity, bins.pair_ids, bins.tile_ranges, st,
                              frame->mask_offsets, frame->mask_pixels, Qm, dQm, plan.chunk_start};
        for (const void* p : ptrs) key.addp(p);
        const int64_t ints[] = {N, d, M, D, (int64_t)bins.num_pairs, (int64_t)frame->F_dtype, (int64_t)prec,
                                (int64_t)ctx->ws_generation, (int64_t)S, frame->n_mask_entries};
        for (int64_t x : ints) key.add((uint64_t)x);
        key.add_camera(cam);
        for (float f : {cfg->lambda_f, cfg->lambda_cos, cfg->lambda_2, cfg->lambda_D, cfg->delta, cfg->logit_scale,
                        adam->lr_f, adam->lr_dict, adam->beta1, adam->beta2, adam->eps, tau})
            key.addf(f);
    }
    LAT_TRY(run_iterations(ctx, graphable, key, iters, learn_f != 0, adam, st, iteration));
    if (loss_host) LAT_TRY(read_loss(ctx, lp, loss_host, st));
    return LATENTAM_OK;
}

}  // extern "C"

namespace {

struct FrameState {
    latentam_projected proj;
    latentam_bins bins;
    CamParams cam;
    int64_t pix_off;  // first row of this frame in the stacked images
    int group;        // index of its distinct query array
};

struct QueryGroup {
    float *f, *m, *v, *df;
    int32_t n;
};

}  // namespace

extern "C" latentam_status latentam_step_batch(latentam_ctx* ctx, const latentam_batch_frame* frames,
                                               int32_t n_frames, const void* F, latentam_dtype F_dtype,
                                               const uint8_t* mask, latentam_dictionary* dict,
                                               const latentam_loss_cfg* cfg, latentam_adam_cfg* adam, int32_t iters,
                                               int32_t learn_f, latentam_precision prec, double* loss_host,
                                               latentam_stream stream) {
    LAT_TRY(enter(ctx));
    REQUIRE(frames && dict && cfg && adam && iters >= 0, "null argument");
    REQUIRE(n_frames >= 1 && n_frames <= LATENTAM_MAX_BATCH, "n_frames=%d outside 1..%d", n_frames,
            LATENTAM_MAX_BATCH);
    LAT_TRY(check_d(dict->d));
    LAT_TRY(check_dict(dict->M, dict->D));
    REQUIRE(dict->K && dict->V && dict->V0 && dict->m_K && dict->v_K && dict->m_V && dict->v_V,
            "null dictionary tensor or moment");
    REQUIRE(F && (F_dtype == LATENTAM_DTYPE_F32 || F_dtype == LATENTAM_DTYPE_BF16), "bad targets");
    cudaStream_t st = (cudaStream_t)stream;
    const int d = dict->d, M = dict->M, D = dict->D;
    const float tau = dict->tau;
    REQUIRE(tau >= 0.f && isfinite(tau), "tau=%g must be 0 (free keys) or positive", (double)tau);
    const bool paper = tau > 0.f;
    const int64_t ksize = paper ? (int64_t)d * D : (int64_t)M * d;  // K holds W (d x D) in the paper form
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };

    // distinct query arrays (frames of one map share them)
    FrameState fs[LATENTAM_MAX_BATCH];
    QueryGroup groups[LATENTAM_MAX_BATCH];
    int n_groups = 0;
    int64_t total_pix = 0;
    for (int k = 0; k < n_frames; ++k) {
        const latentam_batch_frame& fr = frames[k];
        LAT_TRY(check_camera(&fr.camera));
        REQUIRE(fr.gaussians.n >= 0 && fr.f && (!learn_f || (fr.m_f && fr.v_f)), "frame %d: bad queries", k);
        if (fr.gaussians.n > 0)
            REQUIRE(fr.gaussians.means && fr.gaussians.quats && fr.gaussians.scales && fr.gaussians.opacities,
                    "frame %d: null Gaussian attribute", k);
        REQUIRE(aligned16(fr.f), "frame %d: f must be 16-byte aligned", k);
        int gidx = -1;
        for (int u = 0; u < n_groups; ++u)
            if (groups[u].f == fr.f) gidx = u;
        if (gidx < 0) {
            gidx = n_groups++;
            groups[gidx] = QueryGroup{fr.f, fr.m_f, fr.v_f, nullptr, fr.gaussians.n};
        } else {
            REQUIRE(groups[gidx].n == fr.gaussians.n && groups[gidx].m == fr.m_f && groups[gidx].v == fr.v_f,
                    "frames sharing f must share N and the Adam moments");
        }
        fs[k].group = gidx;
        fs[k].pix_off = total_pix;
        total_pix += (int64_t)fr.camera.width * fr.camera.height;
    }

    // projection and binning of every frame (once; the geometry is fixed during the step): the
    // pair counts of all frames, one host synchronisation, then each frame's pairs, sort and
    // ranges (binning slot k per frame, its scan offsets at offs + off_at[k])
    size_t off_at[LATENTAM_MAX_BATCH + 1];
    off_at[0] = 0;
    bool any_gauss = false;
    for (int k = 0; k < n_frames; ++k) {
        off_at[k + 1] = off_at[k] + (((size_t)frames[k].gaussians.n + 1 + 63) & ~(size_t)63);
        any_gauss = any_gauss || frames[k].gaussians.n > 0;
    }
    uint32_t* offs = static_cast<uint32_t*>(ws(ctx, WS_OFFSETS, sizeof(uint32_t) * off_at[n_frames]));
    if (!offs) return LATENTAM_ERR_OUT_OF_MEMORY;
    for (int k = 0; k < n_frames; ++k) {
        const latentam_batch_frame& fr = frames[k];
        const int N = fr.gaussians.n;
        const int64_t tiles = latentam_num_tiles(&fr.camera);
        const size_t o_xy = 0, o_co = o_xy + up(8 * (size_t)N), o_dp = o_co + up(16 * (size_t)N),
                     o_rc = o_dp + up(4 * (size_t)N), o_tt = o_rc + up(16 * (size_t)N),
                     o_tr = o_tt + up(4 * (size_t)N), o_end = o_tr + up(8 * (size_t)tiles);
        char* pb = static_cast<char*>(frame_ws(ctx, 2 * k, o_end));
        if (!pb) return LATENTAM_ERR_OUT_OF_MEMORY;
        fs[k].proj = latentam_projected{reinterpret_cast<float*>(pb + o_xy), reinterpret_cast<float*>(pb + o_co),
                                        reinterpret_cast<float*>(pb + o_dp), reinterpret_cast<int32_t*>(pb + o_rc),
                                        reinterpret_cast<int32_t*>(pb + o_tt)};
        fs[k].cam = cam_params(fr.camera);
        latentam_bins& bins = fs[k].bins;
        bins = latentam_bins{};
        bins.tile_ranges = reinterpret_cast<int32_t*>(pb + o_tr);
        bins.pair_ids = static_cast<int32_t*>(ctx->frame_ptr[2 * k + 1]);
        bins.capacity = (int64_t)(ctx->frame_bytes[2 * k + 1] / sizeof(int32_t));
    }
    {
        // the keyframes are projected and binned at the same time, keyframe k on side stream
        // k % 8 (each binning slot has its own scratch), between a fork from and a join back into
        // the step's stream (timed as the sort stage: the projection of a batch is part of it)
        StageTimer tm(ctx, LATENTAM_STAGE_SORT, st);
        const int nside = n_frames > 1 ? std::min(n_frames, 8) : 0;
        if (nside > 0) {
            LAT_TRY(bin_streams(ctx));
            cudaError_t e = cudaEventRecord(ctx->bin_events[0], st);
            for (int i = 0; i < nside && e == cudaSuccess; ++i)
                e = cudaStreamWaitEvent(ctx->bin_streams[i], ctx->bin_events[0], 0);
            if (e != cudaSuccess) return cuda_error(e, "fork the binning streams");
        }
        auto sk = [&](int k) { return nside > 0 ? ctx->bin_streams[k % nside] : st; };
        // every wait below that returns early still joins the side streams into the step's stream
        auto join = [&]() -> latentam_status {
            cudaError_t e = cudaSuccess;
            for (int i = 0; i < nside && e == cudaSuccess; ++i) {
                e = cudaEventRecord(ctx->bin_events[1 + i], ctx->bin_streams[i]);
                if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ctx->bin_events[1 + i], 0);
            }
            return e == cudaSuccess ? LATENTAM_OK : cuda_error(e, "join the binning streams");
        };
        latentam_status s = LATENTAM_OK;
        for (int k = 0; k < n_frames && s == LATENTAM_OK; ++k) {
            s = launch_project(frames[k].gaussians, fs[k].cam, fs[k].proj, sk(k));
            if (s == LATENTAM_OK)
                s = bin_count(ctx, frames[k].gaussians.n, fs[k].proj, fs[k].cam, &fs[k].bins, offs + off_at[k], k,
                              sk(k));
        }
        if (s == LATENTAM_OK && any_gauss) {
            cudaError_t e = cudaSuccess;
            for (int i = 0; i < std::max(nside, 1) && e == cudaSuccess; ++i) e = cudaStreamSynchronize(sk(i));
            if (e != cudaSuccess) s = cuda_error(e, "sync for the pair counts");
        }
        for (int k = 0; k < n_frames && s == LATENTAM_OK; ++k) {
            const int N = frames[k].gaussians.n;
            latentam_bins& bins = fs[k].bins;
            s = bin_finish(ctx, N, fs[k].proj, fs[k].cam, &bins, offs + off_at[k], k, sk(k));
            if (s == LATENTAM_ERR_CAPACITY) {
                bins.pair_ids =
                    static_cast<int32_t*>(frame_ws(ctx, 2 * k + 1, sizeof(int32_t) * (size_t)bins.num_pairs));
                if (!bins.pair_ids) s = LATENTAM_ERR_OUT_OF_MEMORY;
                if (s != LATENTAM_ERR_OUT_OF_MEMORY) {
                    bins.capacity = bins.num_pairs;
                    s = bin_finish(ctx, N, fs[k].proj, fs[k].cam, &bins, offs + off_at[k], k, sk(k));
                }
            }
        }
        const latentam_status sj = join();
        LAT_TRY(s);
        LAT_TRY(sj);
    }
    // one work list over the tiles of every frame, longest lists first, and the two work tickets
    // of the persistent render launches
    int total_tiles = 0;
    for (int k = 0; k < n_frames; ++k) total_tiles += fs[k].cam.tiles_x * fs[k].cam.tiles_y;
    int32_t* work = static_cast<int32_t*>(ws(ctx, WS_TILE_ORDER, sizeof(int32_t) * ((size_t)total_tiles + 64)));
    if (!work) return LATENTAM_ERR_OUT_OF_MEMORY;
    int* tickets = work + ((total_tiles + 31) / 32) * 32;  // [0] forward, [1] backward

    // stacked images, per-group query gradients, dictionary gradients
    const size_t i_q = 0, i_t = i_q + up(4 * (size_t)total_pix * d), i_n = i_t + up(4 * (size_t)total_pix),
                 i_dq = i_n + up(4 * (size_t)total_pix), i_end = i_dq + up(4 * (size_t)total_pix * d);
    char* ib = static_cast<char*>(ws(ctx, WS_STEP_IMG, i_end));
    // mask-pooled batch: one plan per frame, the pooled rows of every frame stacked in order
    bool pooled = false;
    for (int k = 0; k < n_frames; ++k) pooled = pooled || frames[k].n_masks > 0;
    MaskPlan plans[LATENTAM_MAX_BATCH];
    int64_t row_off[LATENTAM_MAX_BATCH + 1];
    row_off[0] = 0;
    float *Qm = nullptr, *dQm = nullptr;
    if (pooled) {
        size_t pbytes[LATENTAM_MAX_BATCH], tot = 0;
        for (int k = 0; k < n_frames; ++k) {
            const latentam_batch_frame& fr = frames[k];
            const int64_t np_k = (int64_t)fr.camera.width * fr.camera.height;
            LAT_TRY(check_masks(fr.n_masks, fr.n_mask_entries, np_k, d, fr.mask_offsets, fr.mask_pixels));
            pbytes[k] = up(mask_plan_bytes(fr.n_masks, fr.n_mask_entries, d));
            tot += pbytes[k];
            row_off[k + 1] = row_off[k] + fr.n_masks;
        }
        const size_t qb = up(4 * (size_t)row_off[n_frames] * d);
        char* mb = static_cast<char*>(ws(ctx, WS_MASKS, tot + 2 * qb));
        if (!mb) return LATENTAM_ERR_OUT_OF_MEMORY;
        size_t o = 0;
        for (int k = 0; k < n_frames; ++k) {
            const latentam_batch_frame& fr = frames[k];
            mask_plan_carve(mb + o, fr.mask_offsets, fr.mask_pixels, fr.n_mask_entries, fr.n_masks,
                            (int64_t)fr.camera.width * fr.camera.height, d, &plans[k]);
            o += pbytes[k];
            LAT_TRY(launch_mask_plan(plans[k], st));
        }
        Qm = reinterpret_cast<float*>(mb + o);
        dQm = reinterpret_cast<float*>(mb + o + qb);
    }
    const int64_t ndec = pooled ? row_off[n_frames] : total_pix;
    size_t g_end = 0;
    size_t g_df[LATENTAM_MAX_BATCH];
    for (int u = 0; u < n_groups; ++u) {
        g_df[u] = g_end;
        g_end += up(4 * (size_t)groups[u].n * d);
    }
    const size_t g_dk = g_end, g_dv = g_dk + up(4 * (size_t)ksize), g_lp = g_dv + up(4 * (size_t)M * D);
    g_end = g_lp + up(8 * LATENTAM_LOSS_PARTS);
    char* gb = static_cast<char*>(ws(ctx, WS_STEP_GRAD, g_end));
    if (!ib || !gb) return LATENTAM_ERR_OUT_OF_MEMORY;
    float* Q = reinterpret_cast<float*>(ib + i_q);
    float* T = reinterpret_cast<float*>(ib + i_t);
    int32_t* nc = reinterpret_cast<int32_t*>(ib + i_n);
    float* dQ = reinterpret_cast<float*>(ib + i_dq);
    for (int u = 0; u < n_groups; ++u) groups[u].df = reinterpret_cast<float*>(gb + g_df[u]);
    float* dK = reinterpret_cast<float*>(gb + g_dk);
    float* dV = reinterpret_cast<float*>(gb + g_dv);
    double* lp = reinterpret_cast<double*>(gb + g_lp);
    BatchJobs jobs{};
    jobs.n = n_frames;
    for (int k = 0; k < n_frames; ++k) {
        const CamParams& cp = fs[k].cam;
        jobs.fr[k] = TileJob{0,
                             cp.tiles_x,
                             cp.W,
                             cp.H,
                             reinterpret_cast<const int2*>(fs[k].bins.tile_ranges),
                             fs[k].bins.pair_ids,
                             reinterpret_cast<const float2*>(fs[k].proj.xy),
                             reinterpret_cast<const float4*>(fs[k].proj.conic_opacity),
                             reinterpret_cast<const float4*>(frames[k].f),
                             reinterpret_cast<float4*>(Q + fs[k].pix_off * d),
                             T + fs[k].pix_off,
                             nc + fs[k].pix_off,
                             reinterpret_cast<const float4*>(dQ + fs[k].pix_off * d),
                             groups[fs[k].group].df};
    }
    {
        StageTimer tm(ctx, LATENTAM_STAGE_SORT, st);
        LAT_TRY(launch_batch_order(jobs, work, st));
    }

    auto iteration = [&](cudaStream_t s, bool render, const int* step_dev) -> latentam_status {
        if (render) {
            StageTimer tm(ctx, LATENTAM_STAGE_RENDER_FWD, s);
            LAT_TRY(launch_render_fwd_batch(jobs, d, work, total_tiles, tickets, s));
            for (int k = 0; pooled && k < n_frames; ++k)
                LAT_TRY(launch_pool_fwd(plans[k], Q + fs[k].pix_off * d, d, Qm + row_off[k] * d, s));
        }
        float* dQd = learn_f ? (pooled ? dQm : dQ) : nullptr;
        auto render_bwd = [&](cudaStream_t b) -> latentam_status {
            StageTimer tm(ctx, LATENTAM_STAGE_RENDER_BWD, b);
            for (int u = 0; u < n_groups; ++u) {
                cudaError_t e = cudaMemsetAsync(groups[u].df, 0, sizeof(float) * (size_t)groups[u].n * d, b);
                if (e != cudaSuccess) return cuda_error(e, "memset df");
            }
            for (int k = 0; pooled && k < n_frames; ++k)
                LAT_TRY(launch_pool_bwd(plans[k], dQm + row_off[k] * d, d, dQ + fs[k].pix_off * d, b));
            return launch_render_bwd_batch(jobs, d, work, total_tiles, tickets + 1, b);
        };
        // the render backward needs only dQ: it branches off once the decode has made it final
        const std::function<latentam_status(cudaStream_t)> fork = [&](cudaStream_t ds) {
            return fork_branch(ctx, ds, render_bwd);
        };
        ctx->after_dq = learn_f && !paper && !ctx->profiling ? &fork : nullptr;  // (see latentam_step)
        ctx->after_dq_called = 0;
        latentam_status sd;
        if (paper)
            sd = latentam_decode_loss_bwd_paper(ctx, pooled ? Qm : Q, ndec, d, dict->K, dict->V, dict->V0, M, D, tau,
                                                F, F_dtype, mask, cfg, prec, lp, dQd, dK, dV, s);
        else
            sd = latentam_decode_loss_bwd(ctx, pooled ? Qm : Q, ndec, d, dict->K, dict->V, dict->V0, M, D, F,
                                          F_dtype, mask, cfg, prec, lp, dQd, dK, dV, s);
        ctx->after_dq = nullptr;
        const bool joined = ctx->after_dq_called != 0;
        if (joined) LAT_TRY(join_branch(ctx, s));  // joined even when the decode failed after the fork
        LAT_TRY(sd);
        if (learn_f && !joined) LAT_TRY(render_bwd(s));
        StageTimer tm(ctx, LATENTAM_STAGE_ADAM, s);
        if (step_dev) LAT_TRY(launch_step_advance(const_cast<int*>(step_dev), s));
        AdamTensor t[8];
        int cnt = 0;
        t[cnt++] = AdamTensor{dict->K, dK, dict->m_K, dict->v_K, ksize, adam->lr_dict};
        t[cnt++] = AdamTensor{dict->V, dV, dict->m_V, dict->v_V, (int64_t)M * D, adam->lr_dict};
        for (int u = 0; learn_f && u < n_groups; ++u) {
            if (cnt == 8) {
                LAT_TRY(launch_adam(ctx, t, cnt, adam->beta1, adam->beta2, adam->eps, adam->step, s, step_dev));
                cnt = 0;
            }
            t[cnt++] = AdamTensor{groups[u].f, groups[u].df, groups[u].m, groups[u].v, (int64_t)groups[u].n * d,
                                  adam->lr_f};
        }
        return launch_adam(ctx, t, cnt, adam->beta1, adam->beta2, adam->eps, adam->step, s, step_dev);
    };
    GraphKey key;
    const bool graphable = ctx->use_graphs && learn_f && !ctx->profiling && iters > 0;
    if (graphable) {
        const void* ptrs[] = {dict->K, dict->V, dict->V0, dict->m_K, dict->v_K, dict->m_V, dict->v_V, F, mask,
                              Q, T, nc, dQ, dK, dV, lp, st, Qm, dQm};
        for (const void* p : ptrs) key.addp(p);
        const int64_t ints[] = {n_frames, n_groups, d, M, D, (int64_t)F_dtype, (int64_t)prec,
                                (int64_t)ctx->ws_generation};
        key.addf(tau);
        for (int64_t x : ints) key.add((uint64_t)x);
        for (int k = 0; k < n_frames; ++k) {
            const latentam_batch_frame& fr = frames[k];
            for (const void* p : {(const void*)fr.f, (const void*)fr.m_f, (const void*)fr.v_f,
                                  (const void*)fs[k].proj.xy, (const void*)fs[k].bins.pair_ids,
                                  (const void*)fs[k].bins.tile_ranges})
                key.addp(p);
            key.add((uint64_t)fr.gaussians.n);
            key.add((uint64_t)fs[k].bins.num_pairs);
            key.add_camera(fr.camera);
            key.addp(fr.mask_offsets);
            key.addp(fr.mask_pixels);
            key.addp(pooled ? plans[k].chunk_start : nullptr);
            key.add((uint64_t)fr.n_mask_entries);
            key.add((uint64_t)fr.n_masks);
        }
        for (int u = 0; u < n_groups; ++u) key.addp(groups[u].df);
        for (float f : {cfg->lambda_f, cfg->lambda_cos, cfg->lambda_2, cfg->lambda_D, cfg->delta, cfg->logit_scale,
                        adam->lr_f, adam->lr_dict, adam->beta1, adam->beta2, adam->eps})
            key.addf(f);
    }
    LAT_TRY(run_iterations(ctx, graphable, key, iters, learn_f != 0, adam, st, iteration));
    if (loss_host) LAT_TRY(read_loss(ctx, lp, loss_host, st));
    return LATENTAM_OK;
}
