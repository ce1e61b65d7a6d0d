// Tensor-core fused-block kernel (qd_tc.cu).
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "qd_plan.h"

namespace qd {

// Smallest and largest block dimension the tensor-core kernel is used for.
constexpr int kTcMinD = 9;
constexpr int kTcMaxD = 64;

// Padded dimension of a block: D rounded up to a multiple of 8 (16 above 32).
int tc_padded_dim(int D);
// Bytes of the three BF16 matrix terms of a block with padded dimension Dp.
size_t tc_terms_bytes(int Dp);
// Pack the real embedding of the D x D complex matrix U (interleaved, FP64)
// into three BF16 terms (host), in the kernel's shared-memory layout.
void tc_pack_terms(const double *U, int D, int Dp, uint16_t *out);
int tc_smem_bytes(int Dp);
// Launch one block (g.mode == Mode::Tensor) on a complex64 state.
cudaError_t launch_block_tc(const GatePlan &g, void *psi, int sm_count, int32_t *err, cudaStream_t s);

}  // namespace qd
