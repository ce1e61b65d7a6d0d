// The paper's execution model as a comparison path (qd_kron.cu): moments,
// Kronecker-product operators, GEMM chain, GEMV (QuDiet Sec. 3.5-3.6).
#pragma once
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "qd_fuse.h"

namespace qd {

constexpr int64_t kKronMaxN = 4096;  // largest register of this path (three N x N complex128 operators)
constexpr int kKronMaxQudits = 16;

// Moment index of every gate (the first moment after the last one that holds
// a gate on any of its acting qudits) and the number of moments.
std::vector<int> pack_moments(int n, const std::vector<FuseGate> &gates, int *n_moments);

// Apply the gates to psi (N amplitudes, prec 1 = complex64, 2 = complex128)
// through the moment operators; synchronises the stream.
cudaError_t run_moments(void *psi, int prec, int64_t N, int n, const int32_t *dims, const std::vector<FuseGate> &gates,
                        int *n_moments, cudaStream_t s);

}  // namespace qd
