// Batched execution: many independent circuits, each on its own register of
// uneven size (QuDiet Sec. 2.2 registers, Sec. 2.1.2 / 3.4 gates), in one
// persistent kernel launch, captured with the resets and the FP64
// probability readout into one CUDA graph.
//
// Work items, dequeued in order from a global counter by persistent CTAs:
//   * a small circuit (state fits in shared memory): one CTA loads the whole
//     state, applies every gate of the circuit in shared memory and writes it
//     back;
//   * a large circuit: item (gate g, group range) applies gate g to a tile of
//     its groups.  Before starting, the CTA waits until the circuit's
//     completion counter shows every tile of gates < g done; after finishing
//     it adds one to the counter.  Items are queued by gate level, so every
//     item a CTA can wait on was dequeued earlier by a running CTA: the
//     schedule cannot deadlock.  Waits are bounded (polls with __nanosleep);
//     on expiry the CTA records an error in the device error word and skips
//     the item.  State reads bypass L1 (ld.global.cg) so that a CTA never
//     sees a stale copy of another CTA's writes.
// Gates are encoded on the host (qd_batch_set_circuit) as dense D x D (FP32
// hi + lo coefficient pairs, as in the per-gate kernels) or as permutations
// with phases, D <= 25, with 32-bit index geometry (every register holds
// fewer than 2^31 amplitudes).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/qudit.h"
#include "qd_batch.h"
#include "qd_common.cuh"
#include "qd_reduce.h"

namespace qd {

namespace {

constexpr int kBThreads = 256;
constexpr uint32_t kPollLimit = 1u << 22;  // bounded waits on a circuit counter

__device__ __forceinline__ float2 ldcg2(const float2 *p) { return __ldcg(p); }

__device__ __forceinline__ void cmac(float2 &acc, const float2 u, const float2 v) {
    acc.x = fmaf(u.x, v.x, acc.x);
    acc.x = fmaf(-u.y, v.y, acc.x);
    acc.y = fmaf(u.x, v.y, acc.y);
    acc.y = fmaf(u.y, v.x, acc.y);
}

// Load gate g's coefficients into shared memory (all threads).
__device__ __forceinline__ void load_gate(const BGate &G, const float2 *__restrict__ coef, float2 *sU, float2 *sUlo) {
    if (G.kind == 0) {
        const int DD = G.D * G.D;
        for (int i = threadIdx.x; i < DD; i += blockDim.x) {
            sU[i] = coef[G.coef + i];
            sUlo[i] = coef[G.coef + DD + i];
        }
    } else {
        for (int i = threadIdx.x; i < G.D; i += blockDim.x) {
            sU[i] = coef[G.coef + i];
            sUlo[i] = coef[G.coef + G.D + i];
        }
    }
}

// Apply gate G to group r of a state (global when SMEM == false).
template <bool SMEM>
__device__ __forceinline__ void apply_group(const BGate &G, float2 *psi, uint32_t r, const float2 *sU,
                                            const float2 *sUlo) {
    const uint32_t base = expand(r, G.ex) + G.base;
    float2 v[kBatchMaxD];
    if (G.kind == 0) {
#pragma unroll
        for (int j = 0; j < kBatchMaxD; ++j)
            if (j < G.D) v[j] = SMEM ? psi[base + G.off[j]] : ldcg2(psi + base + G.off[j]);
        for (int i = 0; i < G.D; ++i) {
            float2 acc = make_float2(0.f, 0.f);
#pragma unroll
            for (int j = 0; j < kBatchMaxD; ++j)
                if (j < G.D) cmac(acc, sUlo[i * G.D + j], v[j]);
#pragma unroll
            for (int j = 0; j < kBatchMaxD; ++j)
                if (j < G.D) cmac(acc, sU[i * G.D + j], v[j]);
            psi[base + G.off[i]] = acc;
        }
    } else {
#pragma unroll
        for (int i = 0; i < kBatchMaxD; ++i)
            if (i < G.D && ((G.active >> i) & 1u))
                v[i] = SMEM ? psi[base + G.off[G.src[i]]] : ldcg2(psi + base + G.off[G.src[i]]);
#pragma unroll
        for (int i = 0; i < kBatchMaxD; ++i) {
            if (i < G.D && ((G.active >> i) & 1u)) {
                float2 o = v[i];
                if (!((G.unit >> i) & 1u)) {
                    float2 acc = make_float2(0.f, 0.f);
                    cmac(acc, sUlo[i], v[i]);
                    cmac(acc, sU[i], v[i]);
                    o = acc;
                }
                psi[base + G.off[i]] = o;
            }
        }
    }
}

__global__ void __launch_bounds__(kBThreads) k_batch(float2 *__restrict__ arena, const uint64_t *__restrict__ offs,
                                                     const uint32_t *__restrict__ sizes, const BGate *__restrict__ gates,
                                                     const float2 *__restrict__ coef, const BItem *__restrict__ items,
                                                     int32_t nitems, uint32_t *__restrict__ next,
                                                     uint32_t *__restrict__ done, int32_t *__restrict__ err,
                                                     uint32_t smem_amps) {
    extern __shared__ __align__(16) unsigned char smraw[];
    float2 *sU = reinterpret_cast<float2 *>(smraw);
    float2 *sUlo = sU + kBatchMaxD * kBatchMaxD;
    float2 *sstate = sUlo + kBatchMaxD * kBatchMaxD;
    __shared__ int32_t item_id;
    __shared__ int32_t ok;
    for (;;) {
        if (threadIdx.x == 0) item_id = (int32_t)atomicAdd(next, 1u);
        __syncthreads();
        const int32_t id = item_id;
        if (id >= nitems) break;
        const BItem it = items[id];
        float2 *psi = arena + offs[it.circuit];
        if (it.ngates > 0) {
            // ---- small circuit in shared memory
            const uint32_t N = sizes[it.circuit];
            for (uint32_t i = threadIdx.x; i < N; i += blockDim.x) sstate[i] = ldcg2(psi + i);
            for (int g = it.gate; g < it.gate + it.ngates; ++g) {
                const BGate &G = gates[g];
                __syncthreads();
                load_gate(G, coef, sU, sUlo);
                __syncthreads();
                for (uint32_t r = threadIdx.x; r < G.R; r += blockDim.x) apply_group<true>(G, sstate, r, sU, sUlo);
            }
            __syncthreads();
            for (uint32_t i = threadIdx.x; i < N; i += blockDim.x) psi[i] = sstate[i];
            __syncthreads();
            continue;
        }
        // ---- tile of a large circuit's gate: wait for the earlier gates
        if (threadIdx.x == 0) {
            ok = 1;
            const volatile uint32_t *d = done + it.circuit;
            uint32_t polls = 0;
            while (*d < it.wait_target) {
                if (++polls > kPollLimit) {
                    atomicExch(err, 2);
                    ok = 0;
                    break;
                }
                __nanosleep(128);
            }
            __threadfence();
        }
        __syncthreads();
        if (ok) {
            const BGate &G = gates[it.gate];
            load_gate(G, coef, sU, sUlo);
            __syncthreads();
            for (uint32_t r = it.first + threadIdx.x; r < it.first + it.count; r += blockDim.x)
                apply_group<false>(G, psi, r, sU, sUlo);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(done + it.circuit, 1u);
        }
    }
}

// Zero fill of the arena; k_batch_ones then sets each circuit's basis amplitude.
__global__ void k_batch_init(float2 *arena, uint64_t total) {
    const uint64_t step = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += step)
        arena[i] = make_float2(0.f, 0.f);
}

__global__ void k_batch_ones(float2 *arena, const uint64_t *offs, const uint64_t *basis, int32_t ncirc) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncirc; c += gridDim.x * blockDim.x)
        arena[offs[c] + basis[c]] = make_float2(1.f, 0.f);
}

}  // namespace

size_t batch_smem_bytes(uint32_t smem_amps) {
    return (size_t)2 * kBatchMaxD * kBatchMaxD * sizeof(float2) + (size_t)smem_amps * sizeof(float2);
}

cudaError_t batch_launch(const BatchLaunch &b, cudaStream_t s, cudaEvent_t ev0, cudaEvent_t ev1) {
    cudaError_t e = cudaMemsetAsync(b.counters, 0, sizeof(uint32_t) * (1 + (size_t)b.ncirc), s);
    if (e != cudaSuccess) return e;
    k_batch_init<<<b.sm_count * 4, 256, 0, s>>>(b.arena, b.total);
    k_batch_ones<<<(b.ncirc + 255) / 256, 256, 0, s>>>(b.arena, b.offs, b.basis, b.ncirc);
    const size_t smem = batch_smem_bytes(b.smem_amps);
    e = cudaFuncSetAttribute((const void *)k_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (b.nitems == 0) return probabilities(b.arena, 1, b.total, b.probs, b.sm_count, s);
    int occ = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch, kBThreads, smem);
    if (occ < 1) occ = 1;
    const int per_sm = b.ctas_per_sm > 0 && b.ctas_per_sm < occ ? b.ctas_per_sm : occ;
    const int grid = b.sm_count * per_sm;
    if (ev0) cudaEventRecord(ev0, s);
    k_batch<<<grid, kBThreads, smem, s>>>(b.arena, b.offs, b.sizes, b.gates, b.coef, b.items, b.nitems, b.counters,
                                         b.counters + 1, b.err, b.smem_amps);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (ev1) cudaEventRecord(ev1, s);
    return probabilities(b.arena, 1, b.total, b.probs, b.sm_count, s);
}

}  // namespace qd
