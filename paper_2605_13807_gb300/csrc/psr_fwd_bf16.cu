// tcgen05 forward (placeholder until the tensor-core kernel lands).
#include "psr_internal.cuh"

namespace psr {
size_t bf16_packed_bytes() { return 0; }
cudaError_t launch_pack_theta_bf16(const float *, const ThetaLayout &, void *, cudaStream_t) {
    return cudaErrorNotSupported;
}
cudaError_t launch_fwd_bf16(const FwdJobs &, const void *, const float *, const F32Layout &, int,
                            cudaStream_t) {
    return cudaErrorNotSupported;
}
}  // namespace psr
