// Diagonal-run kernels (qd_diag.cu): one pass for a run of diagonal gates.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "qd_common.cuh"

namespace qd {

constexpr uint64_t kDiagTableMax = uint64_t(1) << 24;  // table entries (256 MiB at 16 bytes)
constexpr int kDiagMaxRange = 24;                       // qudits of the covered range
constexpr int kDiagMaxActing = 16;                      // acting qudits of one gate

// The contiguous qudit range [qa, qa + nr) a diagonal run covers: dims in order.
struct DiagRange {
    int32_t nr;
    int32_t d[kDiagMaxRange];
};

// One gate of the run: acting qudits as positions in the range (first = most
// significant local digit) and the offset of its diagonal in the pool.
struct DiagGateDesc {
    int32_t nq;
    int32_t q[kDiagMaxActing];
    int64_t off;
};

// tab[k], k < TS = prod rg.d: product of the gates' diagonal entries at the
// digits of k (prec 1: float4 hi.x, hi.y, lo.x, lo.y; prec 2: double2).
cudaError_t diag_table_build(void *tab, int prec, uint64_t TS, const DiagRange &rg, const DiagGateDesc *gates_dev,
                             int32_t ngates, const double2 *pool_dev, int sm_count, cudaStream_t s);

// psi[i] *= tab[(i / s_qa) mod TS] for every i < N (wide: 64-bit index
// arithmetic below 2^31 amplitudes too).
cudaError_t diag_table_apply(void *psi, int prec, uint64_t N, uint64_t s_qa, uint64_t TS, const void *tab,
                             int sm_count, cudaStream_t s, bool wide = false);

}  // namespace qd
