// Ket readout (QuDiet Sec. 3.8 OutputType / OutputMethod; Sec. 3.9 prints
// the basis states of nonzero probability with their amplitudes): the basis
// indices i with |psi_i|^2 > threshold, in ascending order, with their
// amplitudes or probabilities, found by a stream compaction on the device.
//
// Three launches: per-chunk counts of the kept entries, one exclusive scan of
// the counts, and a write pass in which every chunk re-evaluates the same
// FP64 test and places its entries at its scanned offset (entries beyond the
// caller's capacity are counted but not written).
#include <cstdint>
#include <cuda_runtime.h>

#include "qd_common.cuh"
#include "qd_ket.h"

namespace qd {

namespace {

constexpr int kKetBlock = 256;
constexpr int kKetPer = 16;                            // consecutive amplitudes per thread
constexpr uint64_t kKetChunk = kKetBlock * kKetPer;    // amplitudes per chunk

template <typename T>
__device__ __forceinline__ double kprob(const v2<T> a) {
    const double x = (double)a.x, y = (double)a.y;
    return fma(x, x, y * y);
}

// Exclusive prefix of v over the block (thread order); *total gets the sum.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t *sh, uint32_t *total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    __syncthreads();
    if (lane == 31) sh[w] = x;
    __syncthreads();
    if (w == 0) {
        const int nw = blockDim.x >> 5;
        uint32_t s = lane < nw ? sh[lane] : 0u;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < nw) sh[lane] = s;  // inclusive prefix of warp totals
    }
    __syncthreads();
    const uint32_t before = (w > 0 ? sh[w - 1] : 0u) + x - v;
    *total = sh[(blockDim.x >> 5) - 1];
    return before;
}

template <typename T>
__global__ void __launch_bounds__(kKetBlock) k_ket_count(const v2<T> *__restrict__ psi, uint64_t N, double thr,
                                                         uint64_t nchunks, int64_t *__restrict__ counts) {
    __shared__ uint32_t sh[32];
    for (uint64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
        const uint64_t i0 = c * kKetChunk + (uint64_t)threadIdx.x * kKetPer;
        uint32_t n = 0;
#pragma unroll 4
        for (int k = 0; k < kKetPer; ++k) {
            const uint64_t i = i0 + k;
            if (i < N && kprob<T>(psi[i]) > thr) ++n;
        }
        uint32_t tot = 0;
        block_excl_scan(n, sh, &tot);
        if (threadIdx.x == 0) counts[c] = (int64_t)tot;
        __syncthreads();
    }
}

// One block: offsets[c] = sum of counts[0..c), offsets[nchunks] = total.
__global__ void __launch_bounds__(1024) k_ket_scan(const int64_t *__restrict__ counts, uint64_t nchunks,
                                                   int64_t *__restrict__ offsets) {
    __shared__ int64_t sh[32];
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (uint64_t base = 0; base < nchunks; base += blockDim.x) {
        const uint64_t c = base + threadIdx.x;
        const int64_t v = c < nchunks ? counts[c] : 0;
        int64_t x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) sh[w] = x;
        __syncthreads();
        if (w == 0) {
            int64_t s = sh[lane];
            for (int o = 1; o < 32; o <<= 1) {
                const int64_t y = __shfl_up_sync(0xffffffffu, s, o);
                if (lane >= o) s += y;
            }
            sh[lane] = s;
        }
        __syncthreads();
        const int64_t excl = carry + (w > 0 ? sh[w - 1] : 0) + x - v;
        if (c < nchunks) offsets[c] = excl;
        __syncthreads();
        if (threadIdx.x == 0) carry += sh[31];
        __syncthreads();
    }
    if (threadIdx.x == 0) offsets[nchunks] = carry;
}

template <typename T>
__global__ void __launch_bounds__(kKetBlock) k_ket_write(const v2<T> *__restrict__ psi, uint64_t N, double thr,
                                                         uint64_t nchunks, const int64_t *__restrict__ offsets,
                                                         int64_t cap, int method, int64_t *__restrict__ idx_out,
                                                         double *__restrict__ val_out) {
    __shared__ uint32_t sh[32];
    for (uint64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
        const int64_t base = offsets[c];
        if (base >= cap) continue;  // uniform across the block: nothing of this chunk fits
        const uint64_t i0 = c * kKetChunk + (uint64_t)threadIdx.x * kKetPer;
        uint32_t n = 0;
        for (int k = 0; k < kKetPer; ++k) {
            const uint64_t i = i0 + k;
            if (i < N && kprob<T>(psi[i]) > thr) ++n;
        }
        uint32_t tot = 0;
        int64_t o = base + (int64_t)block_excl_scan(n, sh, &tot);
        for (int k = 0; k < kKetPer && o < cap; ++k) {
            const uint64_t i = i0 + k;
            if (i >= N) break;
            const v2<T> a = psi[i];
            const double p = kprob<T>(a);
            if (p > thr) {
                idx_out[o] = (int64_t)i;
                if (method == 0) {
                    val_out[2 * o] = (double)a.x;
                    val_out[2 * o + 1] = (double)a.y;
                } else {
                    val_out[o] = p;
                }
                ++o;
            }
        }
        __syncthreads();
    }
}

int ket_grid(uint64_t nchunks, int sm_count) {
    const uint64_t cap = (uint64_t)sm_count * 8;
    return (int)(nchunks < cap ? nchunks : cap);
}

}  // namespace

uint64_t ket_chunks(uint64_t N) { return (N + kKetChunk - 1) / kKetChunk; }

cudaError_t ket_select(const void *psi, int prec, uint64_t N, double threshold, int method, int64_t cap,
                       int64_t *counts, int64_t *offsets, int64_t *idx_out, double *val_out, int sm_count,
                       cudaStream_t s) {
    const uint64_t nch = ket_chunks(N);
    const int grid = ket_grid(nch, sm_count);
    if (prec == 1)
        k_ket_count<float><<<grid, kKetBlock, 0, s>>>(static_cast<const float2 *>(psi), N, threshold, nch, counts);
    else
        k_ket_count<double><<<grid, kKetBlock, 0, s>>>(static_cast<const double2 *>(psi), N, threshold, nch, counts);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_ket_scan<<<1, 1024, 0, s>>>(counts, nch, offsets);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (cap > 0) {
        if (prec == 1)
            k_ket_write<float><<<grid, kKetBlock, 0, s>>>(static_cast<const float2 *>(psi), N, threshold, nch, offsets,
                                                          cap, method, idx_out, val_out);
        else
            k_ket_write<double><<<grid, kKetBlock, 0, s>>>(static_cast<const double2 *>(psi), N, threshold, nch,
                                                           offsets, cap, method, idx_out, val_out);
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace qd
