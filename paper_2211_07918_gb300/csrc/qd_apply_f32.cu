// complex64 (FP32 arithmetic) instantiations of the per-gate kernels.
#include "qd_apply.cuh"

namespace qd {
cudaError_t launch_gate_f32(const GatePlan &g, void *psi, int sm_count, cudaStream_t s) {
    return launch_gate_t<float>(g, psi, sm_count, s);
}
}  // namespace qd
