// S2, BF16 tensor-core variant (placeholder until the tcgen05 kernel lands).
#include "nvgs_internal.cuh"

namespace nvgs {

size_t mlp_tc_weight_bytes() { return 16; }
void mlp_tc_pack_weights(const float*, uint8_t* out) { for (int k = 0; k < 16; k++) out[k] = 0; }

cudaError_t launch_mlp_tc(const uint2*, uint32_t, const FrameInst*, const AssetDev*, const int64_t*,
                          float, uint32_t*, float*, int, cudaStream_t, LaunchLog*) {
    return cudaErrorNotSupported;
}

}  // namespace nvgs
