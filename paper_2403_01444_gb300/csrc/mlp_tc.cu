// BF16 tensor-core (tcgen05) MLP of the transformation cache -- placeholder
// until the tcgen05 kernels land; the FP32 SIMT path serves meanwhile.
#include "ntc.cuh"

namespace gs3 {

gs_status mlp_tc_fwd(const void *, int, int64_t, const gs_mlp *, float *, cudaStream_t)
{
    set_error("ntc_mlp_fwd: BF16 tensor-core path not built");
    return GS_ERR_INVALID_ARG;
}

gs_status mlp_tc_bwd(const void *, int, int64_t, const gs_mlp *, const float *, const float *,
                     float *, float *, cudaStream_t)
{
    set_error("ntc_mlp_bwd: BF16 tensor-core path not built");
    return GS_ERR_INVALID_ARG;
}

}  // namespace gs3
