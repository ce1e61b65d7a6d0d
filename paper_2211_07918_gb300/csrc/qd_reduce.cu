// Register initialisation and FP64 readout kernels (QuDiet Sec. 3.2
// init_states; Sec. 3.8 output as amplitudes or probabilities), plus the
// measurement-sampling extension (prefix sums of probabilities and inverse-CDF
// draws from a counter-based generator).
//
// Every reduction accumulates in FP64 in a fixed order (per-thread strided
// sums, then a fixed tree), so results are run-to-run deterministic.
#include <cstdint>
#include <cuda_runtime.h>

#include "qd_common.cuh"
#include "qd_reduce.h"

namespace qd {

namespace {

constexpr int kRedBlock = 256;

template <typename T>
__device__ __forceinline__ double prob(const v2<T> a) {
    const double x = (double)a.x, y = (double)a.y;
    return fma(x, x, y * y);
}

__device__ __forceinline__ double block_sum(double v, double *sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    v = 0.0;
    if (w == 0) {
        const int nw = blockDim.x >> 5;
        v = lane < nw ? sh[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    }
    return v;  // valid in thread 0
}

// psi = 0 except psi[idx] = 1.
template <typename T>
__global__ void k_init(v2<T> *psi, uint64_t N, uint64_t idx) {
    const uint64_t step = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += step)
        psi[i] = mk<T>(i == idx ? T(1) : T(0), T(0));
}

// Per-block partial sums of |psi_i|^2 over a grid-stride walk, unrolled by 4
// for memory-level parallelism; slice (blockIdx.y) selects a digit value of
// one qudit through an inserted digit when ex.n > 0 (marginals).
template <typename T>
__global__ void __launch_bounds__(kRedBlock) k_norm_partial(const v2<T> *__restrict__ psi, uint64_t M,
                                                            Expand64 ex, uint64_t slice_stride,
                                                            double *__restrict__ part) {
    __shared__ double sh[32];
    const uint64_t off = (uint64_t)blockIdx.y * slice_stride;
    const uint64_t step = (uint64_t)gridDim.x * blockDim.x;
    double acc = 0.0;
    uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (ex.n == 0) {
        for (; r + 3 * step < M; r += 4 * step) {
            const v2<T> a0 = psi[r], a1 = psi[r + step], a2 = psi[r + 2 * step], a3 = psi[r + 3 * step];
            acc += prob<T>(a0) + prob<T>(a1) + prob<T>(a2) + prob<T>(a3);
        }
        for (; r < M; r += step) acc += prob<T>(psi[r]);
    } else {
        for (; r < M; r += step) acc += prob<T>(psi[expand(r, ex) + off]);
    }
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) part[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = acc;
}

// out[y] = sum over the nb partials of slice y, in index order per thread.
__global__ void k_sum_partials(const double *__restrict__ part, int nb, double *__restrict__ out) {
    __shared__ double sh[32];
    double acc = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) acc += part[(size_t)blockIdx.x * nb + i];
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) out[blockIdx.x] = acc;
}

// Per-block partial sums of conj(a_i) * b_i (FP64), fixed order.
template <typename TA, typename TB>
__global__ void __launch_bounds__(kRedBlock) k_overlap_partial(const v2<TA> *__restrict__ a, const v2<TB> *__restrict__ b,
                                                               uint64_t N, double *__restrict__ part) {
    __shared__ double sh[32];
    const uint64_t step = (uint64_t)gridDim.x * blockDim.x;
    double re = 0.0, im = 0.0;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += step) {
        const v2<TA> x = a[i];
        const v2<TB> y = b[i];
        const double xr = (double)x.x, xi = (double)x.y, yr = (double)y.x, yi = (double)y.y;
        re = fma(xr, yr, fma(xi, yi, re));
        im = fma(xr, yi, fma(-xi, yr, im));
    }
    re = block_sum(re, sh);
    im = block_sum(im, sh);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = re;
        part[2 * blockIdx.x + 1] = im;
    }
}

__global__ void k_sum_pairs(const double *__restrict__ part, int nb, double *__restrict__ out) {
    __shared__ double sh[32];
    double re = 0.0, im = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        re += part[2 * i];
        im += part[2 * i + 1];
    }
    re = block_sum(re, sh);
    im = block_sum(im, sh);
    if (threadIdx.x == 0) {
        out[0] = re;
        out[1] = im;
    }
}

template <typename T>
__global__ void k_probs(const v2<T> *__restrict__ psi, uint64_t N, double *__restrict__ p) {
    const uint64_t step = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += step) p[i] = prob<T>(psi[i]);
}

// ---- prefix sums: chunk sums, scan of chunk sums, scan inside chunks -------
constexpr int kScanBlock = 256;
constexpr int kScanPer = 16;
constexpr int kChunk = kScanBlock * kScanPer;  // 4096 amplitudes per chunk

template <typename T>
__global__ void __launch_bounds__(kScanBlock) k_chunk_sums(const v2<T> *__restrict__ psi, uint64_t N,
                                                           double *__restrict__ sums) {
    __shared__ double sh[32];
    const uint64_t c0 = (uint64_t)blockIdx.x * kChunk;
    double acc = 0.0;
    for (int k = 0; k < kScanPer; ++k) {
        const uint64_t i = c0 + (uint64_t)k * kScanBlock + threadIdx.x;
        if (i < N) acc += prob<T>(psi[i]);
    }
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) sums[blockIdx.x] = acc;
}

// Exclusive scan of nb chunk sums in one block of 1024 threads; thread t owns
// a contiguous run.  Also writes the grand total to sums[nb].
__global__ void __launch_bounds__(1024) k_scan_sums(double *sums, uint64_t nb) {
    __shared__ double sh[1024];
    const uint64_t per = (nb + blockDim.x - 1) / blockDim.x;
    const uint64_t a = threadIdx.x * per, b = (a + per < nb) ? a + per : nb;
    double loc = 0.0;
    for (uint64_t i = a; i < b; ++i) loc += sums[i];
    sh[threadIdx.x] = loc;
    __syncthreads();
    // Hillis-Steele inclusive scan of the 1024 thread totals
    for (int o = 1; o < 1024; o <<= 1) {
        const double v = threadIdx.x >= (unsigned)o ? sh[threadIdx.x - o] : 0.0;
        __syncthreads();
        sh[threadIdx.x] += v;
        __syncthreads();
    }
    double run = threadIdx.x ? sh[threadIdx.x - 1] : 0.0;
    for (uint64_t i = a; i < b; ++i) {
        const double v = sums[i];
        sums[i] = run;
        run += v;
    }
    if (threadIdx.x == blockDim.x - 1) sums[nb] = sh[blockDim.x - 1];
}

// Shared-memory index with one pad entry per kScanPer, so the thread-serial
// pass (thread t owns entries t*kScanPer ...) does not hit one bank.
__device__ __forceinline__ int padx(int e) { return e + e / kScanPer; }

template <typename T>
__global__ void __launch_bounds__(kScanBlock) k_chunk_scan(const v2<T> *__restrict__ psi, uint64_t N,
                                                           const double *__restrict__ offs,
                                                           double *__restrict__ cdf) {
    __shared__ double buf[kChunk + kChunk / kScanPer];
    __shared__ double tot[kScanBlock];
    const uint64_t c0 = (uint64_t)blockIdx.x * kChunk;
    for (int k = 0; k < kScanPer; ++k) {
        const int e = k * kScanBlock + threadIdx.x;
        const uint64_t i = c0 + e;
        buf[padx(e)] = i < N ? prob<T>(psi[i]) : 0.0;
    }
    __syncthreads();
    // each thread scans its kScanPer consecutive entries
    double run = 0.0;
    const int e0 = threadIdx.x * kScanPer;
    for (int k = 0; k < kScanPer; ++k) {
        run += buf[padx(e0 + k)];
        buf[padx(e0 + k)] = run;
    }
    tot[threadIdx.x] = run;
    __syncthreads();
    for (int o = 1; o < kScanBlock; o <<= 1) {
        const double v = threadIdx.x >= (unsigned)o ? tot[threadIdx.x - o] : 0.0;
        __syncthreads();
        tot[threadIdx.x] += v;
        __syncthreads();
    }
    const double add = offs[blockIdx.x] + (threadIdx.x ? tot[threadIdx.x - 1] : 0.0);
    for (int k = 0; k < kScanPer; ++k) buf[padx(e0 + k)] += add;
    __syncthreads();
    for (int k = 0; k < kScanPer; ++k) {
        const int e = k * kScanBlock + threadIdx.x;
        const uint64_t i = c0 + e;
        if (i < N) cdf[i] = buf[padx(e)];
    }
}

// ---- sampling ---------------------------------------------------------------
// Philox4x64-10 (Salmon et al., SC 2011): two 64x64->128 multiplies per round
// with the published multipliers and Weyl key increments.
__device__ __forceinline__ uint64_t philox_word0(uint64_t c0, uint64_t key0) {
    uint64_t c[4] = {c0, 0, 0, 0};
    uint64_t k0 = key0, k1 = 0;
    const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t hi0 = __umul64hi(M0, c[0]), lo0 = M0 * c[0];
        const uint64_t hi1 = __umul64hi(M1, c[2]), lo1 = M1 * c[2];
        const uint64_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
        k0 += W0;
        k1 += W1;
    }
    return c[0];
}

// smallest i with cdf[i] > target (upper bound), N >= 1
__device__ __forceinline__ int64_t upper_bound(const double *cdf, uint64_t N, double target) {
    uint64_t lo = 0, hi = N;  // answer in [lo, hi]
    while (lo < hi) {
        const uint64_t mid = lo + ((hi - lo) >> 1);
        if (cdf[mid] > target) hi = mid;
        else lo = mid + 1;
    }
    return (int64_t)(lo < N ? lo : N - 1);
}

__global__ void k_sample(const double *__restrict__ cdf, uint64_t N, const double *__restrict__ u, uint64_t seed,
                         int64_t shots, int64_t *__restrict__ out) {
    const double total = cdf[N - 1];
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < shots; s += (int64_t)gridDim.x * blockDim.x) {
        double us;
        if (u) {
            us = u[s];
        } else {
            us = (double)(philox_word0((uint64_t)s, seed) >> 11) * (1.0 / 9007199254740992.0);
        }
        out[s] = upper_bound(cdf, N, us * total);
    }
}

int grid_for(uint64_t n, int block, int sm_count, int per_sm) {
    uint64_t g = (n + block - 1) / block;
    const uint64_t cap = (uint64_t)sm_count * per_sm;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

}  // namespace

cudaError_t init_basis(void *psi, int prec, uint64_t N, uint64_t idx, int sm_count, cudaStream_t s) {
    const int g = grid_for(N, 256, sm_count, 8);
    if (prec == 1) k_init<float><<<g, 256, 0, s>>>(static_cast<float2 *>(psi), N, idx);
    else k_init<double><<<g, 256, 0, s>>>(static_cast<double2 *>(psi), N, idx);
    return cudaGetLastError();
}

int reduce_blocks(int sm_count) { return sm_count * 4; }

cudaError_t slice_norms(const void *psi, int prec, uint64_t M, const Expand64 &ex, uint64_t slice_stride, int nslices,
                        double *part, int nb, double *out_dev, cudaStream_t s) {
    dim3 grid(nb, nslices);
    if (prec == 1) k_norm_partial<float><<<grid, kRedBlock, 0, s>>>(static_cast<const float2 *>(psi), M, ex, slice_stride, part);
    else k_norm_partial<double><<<grid, kRedBlock, 0, s>>>(static_cast<const double2 *>(psi), M, ex, slice_stride, part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_sum_partials<<<nslices, 256, 0, s>>>(part, nb, out_dev);
    return cudaGetLastError();
}

cudaError_t probabilities(const void *psi, int prec, uint64_t N, double *out, int sm_count, cudaStream_t s) {
    const int g = grid_for(N, 256, sm_count, 8);
    if (prec == 1) k_probs<float><<<g, 256, 0, s>>>(static_cast<const float2 *>(psi), N, out);
    else k_probs<double><<<g, 256, 0, s>>>(static_cast<const double2 *>(psi), N, out);
    return cudaGetLastError();
}

cudaError_t overlap(const void *a, int prec_a, const void *b, int prec_b, uint64_t N, double *part, int nb,
                    double *out_dev, cudaStream_t s) {
    if (prec_a == 1 && prec_b == 1)
        k_overlap_partial<float, float><<<nb, kRedBlock, 0, s>>>(static_cast<const float2 *>(a), static_cast<const float2 *>(b), N, part);
    else if (prec_a == 1)
        k_overlap_partial<float, double><<<nb, kRedBlock, 0, s>>>(static_cast<const float2 *>(a), static_cast<const double2 *>(b), N, part);
    else if (prec_b == 1)
        k_overlap_partial<double, float><<<nb, kRedBlock, 0, s>>>(static_cast<const double2 *>(a), static_cast<const float2 *>(b), N, part);
    else
        k_overlap_partial<double, double><<<nb, kRedBlock, 0, s>>>(static_cast<const double2 *>(a), static_cast<const double2 *>(b), N, part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_sum_pairs<<<1, 256, 0, s>>>(part, nb, out_dev);
    return cudaGetLastError();
}

uint64_t cdf_chunks(uint64_t N) { return (N + kChunk - 1) / kChunk; }

cudaError_t cdf(const void *psi, int prec, uint64_t N, double *chunk_sums, double *out, cudaStream_t s) {
    const uint64_t nb = cdf_chunks(N);
    if (nb > 0x7fffffffull) return cudaErrorInvalidValue;
    if (prec == 1) k_chunk_sums<float><<<(unsigned)nb, kScanBlock, 0, s>>>(static_cast<const float2 *>(psi), N, chunk_sums);
    else k_chunk_sums<double><<<(unsigned)nb, kScanBlock, 0, s>>>(static_cast<const double2 *>(psi), N, chunk_sums);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_scan_sums<<<1, 1024, 0, s>>>(chunk_sums, nb);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (prec == 1) k_chunk_scan<float><<<(unsigned)nb, kScanBlock, 0, s>>>(static_cast<const float2 *>(psi), N, chunk_sums, out);
    else k_chunk_scan<double><<<(unsigned)nb, kScanBlock, 0, s>>>(static_cast<const double2 *>(psi), N, chunk_sums, out);
    return cudaGetLastError();
}

cudaError_t sample(const double *cdf_dev, uint64_t N, const double *u_dev, uint64_t seed, int64_t shots,
                   int64_t *out_dev, int sm_count, cudaStream_t s) {
    if (shots <= 0) return cudaSuccess;
    const int g = grid_for((uint64_t)shots, 256, sm_count, 4);
    k_sample<<<g, 256, 0, s>>>(cdf_dev, N, u_dev, seed, shots, out_dev);
    return cudaGetLastError();
}

}  // namespace qd
