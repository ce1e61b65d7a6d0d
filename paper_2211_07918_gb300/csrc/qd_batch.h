// Batched persistent execution (qd_batch.cu): device-side gate encoding and
// launch description shared with the host API in qd_api.cu.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "qd_common.cuh"

namespace qd {

constexpr int kBatchMaxD = 25;  // largest target dimension of a batched gate

// One gate of a batched circuit, 32-bit geometry (direct mode): dense
// (kind 0, D x D coefficients at coef: hi block then lo block) or a
// permutation with phases (kind 1, D phases at coef: hi then lo).
struct BGate {
    int32_t kind;
    int32_t D;
    uint32_t R;     // groups
    uint32_t base;  // control offset
    Expand32 ex;
    uint32_t off[kBatchMaxD];
    int32_t src[kBatchMaxD];
    uint32_t active, unit;
    uint64_t coef;  // offset (float2 units) into the coefficient arena
};

// One work item: a whole small circuit (ngates > 0) or a tile of one gate of
// a large circuit (ngates == 0) that waits for wait_target completed tiles.
struct BItem {
    int32_t circuit;
    int32_t gate;
    int32_t ngates;
    uint32_t first, count;
    uint32_t wait_target;
};

struct BatchLaunch {
    float2 *arena;
    uint64_t total;
    const uint64_t *offs;
    const uint64_t *basis;
    const uint32_t *sizes;
    const BGate *gates;
    const float2 *coef;
    const BItem *items;
    int32_t nitems;
    int32_t ncirc;
    uint32_t *counters;  // [0] queue head, [1 + c] completed tiles of circuit c
    int32_t *err;
    double *probs;
    int sm_count;
    int ctas_per_sm;     // 0: as many as fit
    uint32_t smem_amps;  // largest state kept whole in shared memory
};

size_t batch_smem_bytes(uint32_t smem_amps);
// Enqueue: reset the counters and every state to |0...0>, the persistent
// kernel, and the FP64 probabilities of the whole arena.
// When ev0/ev1 are given they are recorded around the persistent kernel.
cudaError_t batch_launch(const BatchLaunch &b, cudaStream_t s, cudaEvent_t ev0 = nullptr, cudaEvent_t ev1 = nullptr);

}  // namespace qd
