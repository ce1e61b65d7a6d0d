// Initialisation and FP64 readout launchers (qd_reduce.cu).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "qd_common.cuh"

namespace qd {

// psi = |idx> : zero every amplitude, set psi[idx] = 1.  prec: 1 = c64, 2 = c128.
cudaError_t init_basis(void *psi, int prec, uint64_t N, uint64_t idx, int sm_count, cudaStream_t s);

// Number of partial-sum blocks the norm kernels use (part must hold
// nslices * reduce_blocks(sm_count) doubles).
int reduce_blocks(int sm_count);

// out_dev[y] = sum over r < M of |psi[expand(r, ex) + y * slice_stride]|^2 for
// y < nslices (FP64).  ex.n == 0 and nslices == 1 gives the squared norm.
cudaError_t slice_norms(const void *psi, int prec, uint64_t M, const Expand64 &ex, uint64_t slice_stride, int nslices,
                        double *part, int nb, double *out_dev, cudaStream_t s);

// out_dev[0..1] = <a|b> = sum conj(a_i) b_i (FP64), for states of equal length
// (precisions may differ).  part holds 2 * nb doubles.
cudaError_t overlap(const void *a, int prec_a, const void *b, int prec_b, uint64_t N, double *part, int nb,
                    double *out_dev, cudaStream_t s);

// p[i] = |psi_i|^2 (FP64).
cudaError_t probabilities(const void *psi, int prec, uint64_t N, double *out, int sm_count, cudaStream_t s);

// Inclusive prefix sums of |psi_i|^2 (FP64).  chunk_sums must hold
// cdf_chunks(N) + 1 doubles; on return chunk_sums[cdf_chunks(N)] is the total.
uint64_t cdf_chunks(uint64_t N);
cudaError_t cdf(const void *psi, int prec, uint64_t N, double *chunk_sums, double *out, cudaStream_t s);

// out[s] = smallest i with cdf[i] > u_s * cdf[N-1]; u_s from u_dev, or from
// Philox4x64-10 (counter (s,0,0,0), key (seed,0)) when u_dev is null.
cudaError_t sample(const double *cdf_dev, uint64_t N, const double *u_dev, uint64_t seed, int64_t shots,
                   int64_t *out_dev, int sm_count, cudaStream_t s);

}  // namespace qd
