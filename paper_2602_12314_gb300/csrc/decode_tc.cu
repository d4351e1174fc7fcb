// Tensor-core (tcgen05) form of the dictionary decode: BF16 operands, FP32 accumulation.
#include "internal.cuh"

namespace lat {

latentam_status decode_loss_bwd_bf16(latentam_ctx*, const DecodeArgs&, cudaStream_t) {
    set_error("BF16 decode not available in this build");
    return LATENTAM_ERR_UNSUPPORTED_SHAPE;
}

latentam_status decode_fwd_bf16(latentam_ctx*, const float*, int64_t, int, const float*, const float*, int, int, float,
                                float*, float*, cudaStream_t) {
    set_error("BF16 decode not available in this build");
    return LATENTAM_ERR_UNSUPPORTED_SHAPE;
}

}  // namespace lat
