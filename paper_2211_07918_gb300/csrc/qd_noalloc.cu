// qd_cdf_noalloc: the FP64 prefix sum of |psi_i|^2 for callers that cannot
// allocate device memory.
//
// Some callers of this library may not call cudaMalloc or any routine that
// allocates: code that runs while the application's allocator owns all
// device memory (a framework that reserves the heap up front and hands out
// slices itself), and latency-critical loops where a device allocation is
// not allowed because it can synchronise the device and stall every other
// stream.  qd_cdf allocates the output and its scratch on first use; this
// entry point takes the output buffer from the caller and keeps its scratch
// (the per-chunk partial sums of the scan) in the fixed array below, which
// is part of the library's device image and so needs no allocation.
//
// The array holds kNoAllocChunkSums chunk sums of 4096 amplitudes each (plus
// the grand total), which bounds the state at kNoAllocMaxAmplitudes.  Every
// GPU that loads the library holds the array until the process exits.
#include <cstdint>
#include <mutex>
#include <string>

#include <cuda_runtime.h>

#include "../../include/qudit.h"
#include "qd_reduce.h"

namespace qd {
int set_last_error(int code, const char *msg);  // qd_api.cu: the message qd_last_error() returns
}

namespace {

constexpr int64_t kNoAllocChunkSums = 65536;                 // 512 KiB of FP64
constexpr int64_t kNoAllocChunk = 4096;                      // amplitudes per chunk sum
constexpr int64_t kNoAllocMaxAmplitudes = kNoAllocChunkSums * kNoAllocChunk;  // 2^28
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_chunk_sums[kNoAllocChunkSums + 1];

int noalloc_fail(int code, const std::string &msg) { return qd::set_last_error(code, msg.c_str()); }

// Device address of the scratch array on each device, looked up with that
// device current.  In host code the array's name stands for a host-side
// shadow, not a device address, so it must never be handed to a kernel
// directly.  Only a successful lookup is kept: a failed one (for example a
// first call made during stream capture, or a transient error) is retried by
// the next call instead of failing every later call on that device.
double *g_scratch_ptr[kMaxDevices] = {};
std::mutex g_scratch_mu;

cudaError_t scratch_for(int dev, double **out) {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_chunk_sums);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();  // reset the runtime's last-error state before a later retry
            return e != cudaSuccess ? e : cudaErrorInvalidSymbol;
        }
        g_scratch_ptr[dev] = static_cast<double *>(p);
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" int qd_cdf_noalloc(const void *state, int64_t n_amplitudes, int32_t precision, double *cdf_out,
                              void *stream) {
    if (!state || !cdf_out) return noalloc_fail(QD_ERR_ARG, "qd_cdf_noalloc: null state or output pointer");
    if (precision != QD_C64 && precision != QD_C128)
        return noalloc_fail(QD_ERR_ARG, "qd_cdf_noalloc: precision must be QD_C64 or QD_C128");
    if (n_amplitudes < 1 || n_amplitudes > kNoAllocMaxAmplitudes ||
        qd::cdf_chunks((uint64_t)n_amplitudes) > (uint64_t)kNoAllocChunkSums)
        return noalloc_fail(QD_ERR_DIM, "qd_cdf_noalloc: n_amplitudes must be in [1, 2^28]; the fixed scratch "
                                        "holds 65536 chunk sums of 4096 amplitudes");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return noalloc_fail(QD_ERR_CUDA, std::string("qd_cdf_noalloc: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(QD_ERR_ARG, "qd_cdf_noalloc: device ordinal too large");
    double *scratch = nullptr;
    e = scratch_for(dev, &scratch);
    if (e != cudaSuccess)
        return noalloc_fail(QD_ERR_CUDA, std::string("qd_cdf_noalloc: cudaGetSymbolAddress failed: ") +
                                             cudaGetErrorString(e));
    // Every chunk-sum slot the scan reads is written earlier in the same call
    // (chunk sums, then their exclusive scan, then the per-chunk scans), so
    // what an earlier call left in the array is never read.
    e = qd::cdf(state, precision, (uint64_t)n_amplitudes, scratch, cdf_out,
                static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return noalloc_fail(QD_ERR_CUDA, std::string("qd_cdf_noalloc: ") + cudaGetErrorString(e));
    return QD_OK;
}
