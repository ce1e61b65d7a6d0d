// Ket readout launcher (qd_ket.cu).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace qd {

// Number of compaction chunks of a state of N amplitudes: counts needs
// ket_chunks(N) entries, offsets ket_chunks(N) + 1.
uint64_t ket_chunks(uint64_t N);

// Entries i with |psi_i|^2 > threshold (FP64), ascending: the first cap of
// them go to idx_out[] and val_out[] (method 0: re, im per entry; 1: the
// probability); offsets[ket_chunks(N)] receives the total count.
cudaError_t ket_select(const void *psi, int prec, uint64_t N, double threshold, int method, int64_t cap,
                       int64_t *counts, int64_t *offsets, int64_t *idx_out, double *val_out, int sm_count,
                       cudaStream_t s);

}  // namespace qd
