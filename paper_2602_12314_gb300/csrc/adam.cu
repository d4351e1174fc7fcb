// Adam update of several tensors in one launch (the optimiser of the latent step; the paper
// gives only lr = 0.01 for the dictionary, Sec. IV-A).  Each tensor gets a share of the
// blocks in proportion to its size and is streamed as float4.
#include <math.h>

#include <algorithm>

#include "internal.cuh"

namespace lat {
namespace {

constexpr int kMaxTensors = 8;

struct AdamBatch {
    AdamTensor t[kMaxTensors];
    int block_start[kMaxTensors + 1];  // first block of each tensor
    int count;
    float beta1, beta2, eps, inv_bc1, inv_bc2;  // inverse bias corrections 1 / (1 - beta^step)
    const int* step_dev;                        // when set: the step is read here (graph replays)
    int* nonfinite;                             // raised (sticky) when a gradient entry is not finite
};

__device__ __forceinline__ void adam_one(float& p, float g, float& m, float& v, float lr, const AdamBatch& b,
                                         float inv_bc1, float inv_bc2) {
    m = b.beta1 * m + (1.0f - b.beta1) * g;
    v = b.beta2 * v + (1.0f - b.beta2) * g * g;
    const float mh = m * inv_bc1, vh = v * inv_bc2;
    p -= lr * mh / (sqrtf(vh) + b.eps);
}

// Each tensor owns a contiguous range of blocks (block_start); a block streams its share of
// the tensor as float4 when the tensor's arrays are 16-byte aligned, element-wise otherwise.
__global__ void __launch_bounds__(256) adam_kernel(AdamBatch b) {
    float inv_bc1 = b.inv_bc1, inv_bc2 = b.inv_bc2;
    if (b.step_dev) {
        // 1 - beta^t = -expm1(t ln beta), free of the cancellation of 1 - powf(beta, t)
        const float t = (float)*b.step_dev;
        inv_bc1 = -1.0f / expm1f(t * logf(b.beta1));
        inv_bc2 = -1.0f / expm1f(t * logf(b.beta2));
    }
    int k = 0;
    while (k + 1 < b.count && (int)blockIdx.x >= b.block_start[k + 1]) ++k;
    const AdamTensor& T = b.t[k];
    const int nblk = b.block_start[k + 1] - b.block_start[k];
    const int64_t tid = (int64_t)(blockIdx.x - b.block_start[k]) * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)nblk * blockDim.x;
    const bool vec = ((reinterpret_cast<uintptr_t>(T.p) | reinterpret_cast<uintptr_t>(T.g) |
                       reinterpret_cast<uintptr_t>(T.m) | reinterpret_cast<uintptr_t>(T.v)) & 15u) == 0;
    int64_t done = 0;
    bool bad = false;
    if (vec) {
        const int64_t n4 = T.n / 4;
        float4* p4 = reinterpret_cast<float4*>(T.p);
        const float4* g4 = reinterpret_cast<const float4*>(T.g);
        float4* m4 = reinterpret_cast<float4*>(T.m);
        float4* v4 = reinterpret_cast<float4*>(T.v);
        for (int64_t i = tid; i < n4; i += stride) {
            float4 p = p4[i], m = m4[i], v = v4[i];
            const float4 g = g4[i];
            bad |= !(isfinite(g.x) && isfinite(g.y) && isfinite(g.z) && isfinite(g.w));
            adam_one(p.x, g.x, m.x, v.x, T.lr, b, inv_bc1, inv_bc2);
            adam_one(p.y, g.y, m.y, v.y, T.lr, b, inv_bc1, inv_bc2);
            adam_one(p.z, g.z, m.z, v.z, T.lr, b, inv_bc1, inv_bc2);
            adam_one(p.w, g.w, m.w, v.w, T.lr, b, inv_bc1, inv_bc2);
            p4[i] = p;
            m4[i] = m;
            v4[i] = v;
        }
        done = n4 * 4;
    }
    for (int64_t i = done + tid; i < T.n; i += stride) {
        float p = T.p[i], m = T.m[i], v = T.v[i];
        bad |= !isfinite(T.g[i]);
        adam_one(p, T.g[i], m, v, T.lr, b, inv_bc1, inv_bc2);
        T.p[i] = p;
        T.m[i] = m;
        T.v[i] = v;
    }
    if (bad && b.nonfinite) atomicExch(b.nonfinite, 1);
}

// The Adam step counter of graph replays: advanced by one on the device before each update.
__global__ void step_advance(int* step) { *step += 1; }
__global__ void step_set(int* step, int v) { *step = v; }

}  // namespace

latentam_status launch_step_set(int* step_dev, int value, cudaStream_t st) {
    step_set<<<1, 1, 0, st>>>(step_dev, value);
    LAT_CHECK_LAUNCH("step_set");
    return LATENTAM_OK;
}

latentam_status launch_step_advance(int* step_dev, cudaStream_t st) {
    step_advance<<<1, 1, 0, st>>>(step_dev);
    LAT_CHECK_LAUNCH("step_advance");
    return LATENTAM_OK;
}

latentam_status launch_adam(latentam_ctx* ctx, const AdamTensor* t, int count, float beta1, float beta2, float eps,
                            int step, cudaStream_t st, const int* step_dev) {
    if (count <= 0) return LATENTAM_OK;
    if (count > kMaxTensors) {
        set_error("at most %d tensors per Adam launch", kMaxTensors);
        return LATENTAM_ERR_INVALID_ARG;
    }
    if (!step_dev && step < 1) {
        set_error("Adam step must be >= 1 (got %d)", step);
        return LATENTAM_ERR_INVALID_ARG;
    }
    AdamBatch b{};
    b.count = count;
    b.beta1 = beta1;
    b.beta2 = beta2;
    b.eps = eps;
    b.inv_bc1 = (float)(1.0 / (1.0 - pow((double)beta1, (double)step)));
    b.inv_bc2 = (float)(1.0 / (1.0 - pow((double)beta2, (double)step)));
    b.step_dev = step_dev;
    b.nonfinite = ctx->dev_flags ? ctx->dev_flags + 1 : nullptr;
    // blocks in proportion to the tensor sizes (at least one each), about 4 waves in total
    int64_t total = 0;
    for (int k = 0; k < count; ++k) {
        b.t[k] = t[k];
        total += t[k].n;
    }
    if (total == 0) return LATENTAM_OK;
    const int64_t budget = 4LL * ctx->num_sms * 8;
    b.block_start[0] = 0;
    for (int k = 0; k < count; ++k) {
        const int64_t want = (t[k].n / 4 + 255) / 256;
        int64_t nb = std::max<int64_t>(1, std::min<int64_t>(want, (budget * t[k].n + total - 1) / total));
        b.block_start[k + 1] = b.block_start[k] + (int)nb;
    }
    adam_kernel<<<(unsigned)b.block_start[count], 256, 0, st>>>(b);
    LAT_CHECK_LAUNCH("adam_kernel");
    return LATENTAM_OK;
}

}  // namespace lat
