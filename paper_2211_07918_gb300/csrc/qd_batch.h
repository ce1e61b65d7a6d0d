// Batched persistent execution (qd_batch.cu): device-side encoding of
// segments, gates and work items, shared with the host API in qd_api.cu.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "qd_common.cuh"

namespace qd {

constexpr int kBatchMaxD = 25;          // largest target dimension of a batched gate
constexpr uint32_t kBatchMaxTile = 24576;  // largest tile (amplitudes) kept in shared memory

constexpr int kBExMax = 8;              // insertion runs of a tile-local gate (<= 14 local qudits)
constexpr uint32_t kBatchDescBytes = 8192;  // target size of one chunk (a single larger gate is its own chunk)

// Insert-digit expansion with at most kBExMax runs (adjacent removed qudits
// merged into one run).
struct BEx {
    int32_t n;
    int32_t pad;
    FastDiv32 div[kBExMax];
    uint32_t span[kBExMax];
};

__host__ __device__ __forceinline__ uint32_t expand(uint32_t r, const BEx &e) {
#pragma unroll 1
    for (int k = 0; k < e.n; ++k) {
        const uint32_t q = fdiv(r, e.div[k]);
        const uint32_t lo = r - q * e.div[k].d;
        r = q * e.span[k] + lo;
    }
    return r;
}

// One gate in the local index space of its segment's tile (32-bit direct
// geometry): dense (kind 0, D x D coefficients) or a permutation with phases
// (kind 1, D phases).  Coefficients: ncoef FP32 "hi" entries at coef (float2
// offset inside its chunk's coefficient block, even), then ncoef "lo" entries.
struct __align__(16) BGate {
    int32_t kind;
    int32_t D;
    uint32_t R;     // groups in the tile
    uint32_t base;  // control offset in the tile
    uint32_t active, unit;
    uint32_t coef;
    uint32_t ncoef;
    BEx ex;         // group index -> tile-local base
    uint16_t off[kBatchMaxD];
    int8_t src[kBatchMaxD];
};

// Consecutive gates of a segment whose descriptors and coefficients fit
// kBatchDescBytes of shared memory, loaded together.
struct BChunk {
    int32_t gate0, ngates;
    uint32_t coef0;  // float2 offset of the coefficient block (even: 16-byte aligned)
    uint32_t ncoef;  // float2 entries of the block
};

// A segment: consecutive gates of one circuit whose acting qudits all lie in
// a qudit set S.  The register splits into N / T tiles of T = prod_{q in S} d_q
// amplitudes (one tile per assignment of the other qudits).  Tile-local index
// l = j + B h, where j < B runs over the qudits below the lowest qudit missing
// from S (contiguous in the register) and h over the rest of S; the flat
// index is expand(tile, ex) + j + hoff[h].
struct BSeg {
    int32_t chunk0, nchunks;
    uint32_t T, B;
    FastDiv32 divB;
    uint32_t hoff;          // offset of this segment's run table in the run-table arena
    uint32_t ntiles;
    uint32_t pair;          // B even: every run starts at an even arena index (registers start
                            // even), so tiles are gathered as 16-byte amplitude pairs
    uint32_t pad;
    Expand32 ex;            // tile index -> flat base of the tile
};

// One work item: tiles [first, first + count) of segment seg of a circuit,
// started once the circuit's completion counter reaches wait_target (every
// tile of the circuit's earlier segments is done).
struct BItem {
    int32_t circuit;
    int32_t seg;
    uint32_t first, count;
    uint32_t wait_target;
    uint32_t pad;
};

struct BatchLaunch {
    float2 *arena;
    uint64_t total;  // arena amplitudes (every register padded to an even count)
    const uint64_t *offs;
    const uint64_t *basis;
    const BSeg *segs;
    const BChunk *chunks;
    const BGate *gates;
    const float2 *coef;
    const uint32_t *hoff;
    const BItem *items;
    int32_t nitems;
    int32_t ncirc;
    uint32_t *counters;  // [0] queue head, [1 + c] completed tiles of circuit c
    int32_t *err;
    double *probs;
    int sm_count;
    int ctas_per_sm;     // 0: as many as fit
    uint32_t tile_cap;   // largest tile of any segment (shared-memory amplitudes)
    uint32_t desc_bytes; // shared-memory area for one chunk (>= every chunk, multiple of 16)
    uint32_t poll_limit; // polls of a dependent item's wait before it gives up (error word 2)
};

constexpr uint32_t kBatchPollLimit = 1u << 22;  // default: >= 0.5 s of polling

size_t batch_smem_bytes(uint32_t tile_cap, uint32_t desc_bytes);
// Enqueue: reset the counters and every state to its basis state, the
// persistent kernel, and the FP64 probabilities of the whole arena.  When
// ev0/ev1 are given they are recorded around the persistent kernel.
cudaError_t batch_launch(const BatchLaunch &b, cudaStream_t s, cudaEvent_t ev0 = nullptr, cudaEvent_t ev1 = nullptr);
// Resident CTAs per SM of the persistent kernel for a tile capacity.
int batch_occupancy(uint32_t tile_cap, uint32_t desc_bytes);

}  // namespace qd
