// complex128 (FP64 arithmetic) instantiations of the per-gate kernels.
#include "qd_apply.cuh"

namespace qd {
cudaError_t launch_gate_f64(const GatePlan &g, void *psi, int sm_count, cudaStream_t s) {
    return launch_gate_t<double>(g, psi, sm_count, s);
}
}  // namespace qd
