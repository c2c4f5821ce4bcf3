// mlp_tc.cu -- BF16 tensor-core (tcgen05) form of the RPNN forward.
#include <cuda_bf16.h>

#include "common.cuh"

namespace rpnn {

rpnn_status mlp_build_bf16_image(Ctx& c, cudaStream_t s) {
    (void)c; (void)s;
    return RPNN_OK;
}

rpnn_status mlp_forward_bf16(Ctx& c, const void* desc_bf16, int64_t q, const int* q_dev, float* out,
                             cudaStream_t s) {
    (void)c; (void)desc_bf16; (void)q; (void)q_dev; (void)out; (void)s;
    set_error("the BF16 tensor-core network is not available in this build");
    return RPNN_ERR_UNSUPPORTED;
}

}  // namespace rpnn
