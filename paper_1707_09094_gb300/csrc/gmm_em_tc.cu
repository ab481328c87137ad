// Tensor-core (tcgen05) fused EM pass -- placeholder until the kernel lands.
#include "gmm_internal.cuh"

namespace gmm {
bool em_tc_supported(int32_t, int32_t) { return false; }
int em_tc_grid(int sms) { return sms; }
cudaError_t launch_em_pass_tc(const EmPassArgs &, int32_t, int32_t, cudaStream_t) { return cudaErrorNotSupported; }
}  // namespace gmm
