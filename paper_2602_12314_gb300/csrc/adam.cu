// Adam update of several tensors in one launch (the optimiser of the latent step; the paper
// gives only lr = 0.01 for the dictionary, Sec. IV-A).  Grid-stride over the concatenation
// of the tensors, float4 where the sizes allow.
#include <math.h>

#include "internal.cuh"

namespace lat {
namespace {

constexpr int kMaxTensors = 8;

struct AdamBatch {
    AdamTensor t[kMaxTensors];
    int64_t start[kMaxTensors + 1];  // prefix sums of sizes
    int count;
    float beta1, beta2, eps, bc1, bc2;
};

__device__ __forceinline__ void adam_one(float& p, float g, float& m, float& v, float lr, const AdamBatch& b) {
    m = b.beta1 * m + (1.0f - b.beta1) * g;
    v = b.beta2 * v + (1.0f - b.beta2) * g * g;
    const float mh = m / b.bc1, vh = v / b.bc2;
    p -= lr * mh / (sqrtf(vh) + b.eps);
}

__global__ void __launch_bounds__(256) adam_kernel(AdamBatch b) {
    const int64_t total = b.start[b.count];
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        int k = 0;
        while (k + 1 < b.count && e >= b.start[k + 1]) ++k;
        const int64_t i = e - b.start[k];
        const AdamTensor& T = b.t[k];
        float p = T.p[i], m = T.m[i], v = T.v[i];
        adam_one(p, T.g[i], m, v, T.lr, b);
        T.p[i] = p;
        T.m[i] = m;
        T.v[i] = v;
    }
}

}  // namespace

latentam_status launch_adam(latentam_ctx* ctx, const AdamTensor* t, int count, float beta1, float beta2, float eps,
                            int step, cudaStream_t st) {
    if (count <= 0) return LATENTAM_OK;
    if (count > kMaxTensors) {
        set_error("at most %d tensors per Adam launch", kMaxTensors);
        return LATENTAM_ERR_INVALID_ARG;
    }
    if (step < 1) {
        set_error("Adam step must be >= 1 (got %d)", step);
        return LATENTAM_ERR_INVALID_ARG;
    }
    AdamBatch b{};
    b.count = count;
    b.beta1 = beta1;
    b.beta2 = beta2;
    b.eps = eps;
    b.bc1 = (float)(1.0 - pow((double)beta1, (double)step));
    b.bc2 = (float)(1.0 - pow((double)beta2, (double)step));
    b.start[0] = 0;
    for (int k = 0; k < count; ++k) {
        b.t[k] = t[k];
        b.start[k + 1] = b.start[k] + t[k].n;
    }
    const int64_t total = b.start[count];
    if (total == 0) return LATENTAM_OK;
    const int64_t want = (total + 255) / 256;
    const unsigned blocks = (unsigned)(want < 8LL * ctx->num_sms ? want : 8LL * ctx->num_sms);
    adam_kernel<<<blocks, 256, 0, st>>>(b);
    LAT_CHECK_LAUNCH("adam_kernel");
    return LATENTAM_OK;
}

}  // namespace lat
