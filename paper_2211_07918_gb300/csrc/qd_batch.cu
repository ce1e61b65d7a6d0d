// Batched execution: many independent circuits, each on its own register of
// uneven size (QuDiet Sec. 2.2 registers, Sec. 2.1.2 / 3.4 gates), in one
// persistent kernel launch, captured with the resets and the FP64
// probability readout into one CUDA graph.
//
// Each circuit is cut into segments of consecutive gates whose acting qudits
// fit one shared-memory tile (a circuit small enough is a single segment
// whose one tile is the whole register).  A work item loads tiles of one
// segment from the state into shared memory, applies every gate of the
// segment there (one specialised loop per target dimension) and writes the
// tiles back: one pass over the state per segment rather than per gate.
//
// Persistent CTAs dequeue items in order from a global counter.  An item of
// segment k waits until the circuit's completion counter shows every tile of
// segments < k done, and adds its tiles to the counter when finished.  Every
// item waits only on items queued before it, and a CTA claims its next item
// while it works on the current one (an item of lower index), so the
// lowest-indexed unfinished item always belongs to a CTA whose dependencies
// are complete: the schedule cannot deadlock.  Waits are bounded (polls with
// __nanosleep); on expiry the CTA records an error in the device error word
// and skips the item.  State reads bypass L1 (ld.global.cg) so that a CTA
// never sees a stale copy of another CTA's writes.
#include <algorithm>
#include <cstdint>

#include <cuda_runtime.h>

#include "../../include/qudit.h"
#include "qd_batch.h"
#include "qd_common.cuh"
#include "qd_reduce.h"

namespace qd {

namespace {

constexpr int kBThreads = 128;

// Copy a descriptor from global to shared memory (word by word, all threads).
template <typename T>
__device__ __forceinline__ void copy_desc(T *dst, const T *src) {
    static_assert(sizeof(T) % 4 == 0, "descriptor size");
    const uint32_t *s = reinterpret_cast<const uint32_t *>(src);
    uint32_t *d = reinterpret_cast<uint32_t *>(dst);
    for (int i = threadIdx.x; i < (int)(sizeof(T) / 4); i += blockDim.x) d[i] = __ldg(s + i);
}

// Asynchronous 16-byte global -> shared copies (read-only tables only: the
// copies may be served from L1).
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Issue the copies of one chunk: its gate descriptors, then its coefficients.
__device__ __forceinline__ void load_chunk(const BChunk &ch, const BGate *__restrict__ gates,
                                           const float2 *__restrict__ coef, unsigned char *desc) {
    const uint4 *gsrc = reinterpret_cast<const uint4 *>(gates + ch.gate0);
    uint4 *gdst = reinterpret_cast<uint4 *>(desc);
    const int ng = ch.ngates * (int)(sizeof(BGate) / 16);
    for (int i = threadIdx.x; i < ng; i += blockDim.x) cp_async16(gdst + i, gsrc + i);
    const uint4 *csrc = reinterpret_cast<const uint4 *>(coef + ch.coef0);
    uint4 *cdst = reinterpret_cast<uint4 *>(desc + ch.ngates * sizeof(BGate));
    const int nc = (int)(ch.ncoef / 2);
    for (int i = threadIdx.x; i < nc; i += blockDim.x) cp_async16(cdst + i, csrc + i);
}

// Packed FP32 pairs (Blackwell fma.rn.f32x2: two FMAs, each rounded as fmaf).
typedef unsigned long long f2p;

__device__ __forceinline__ f2p pack2(float a, float b) {
    f2p r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float2 unpack2(f2p r) {
    float a, b;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
    return make_float2(a, b);
}
__device__ __forceinline__ f2p fma2(f2p a, f2p b, f2p c) {
    f2p d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// Coefficients u = hi + lo (FP32 each) are stored as a hi block then a lo
// block.  A dot product sum_j u_j v_j takes every lo term first and then
// every hi term, on one accumulator: the lo sum must be present before the
// hi terms are rounded (added to an already rounded hi sum it is below half
// a unit in the last place and is lost, and the FP32 rounding of U then
// drifts the norm coherently).
__device__ __forceinline__ void cmac(float2 &acc, const float2 u, const float2 v) {
    acc.x = fmaf(u.x, v.x, acc.x);
    acc.x = fmaf(-u.y, v.y, acc.x);
    acc.y = fmaf(u.x, v.y, acc.y);
    acc.y = fmaf(u.y, v.x, acc.y);
}
// In registers, a coefficient is expanded to the pairs (u.x, u.x) and (-u.y,
// u.y) for packed FMAs: with v = (re, im) and vs = (im, re),
// acc += u v is re += u.x re - u.y im, im += u.x im + u.y re, the same
// roundings as cmac.
struct Pk {
    f2p xx, yy;
};
__device__ __forceinline__ Pk pk_coef(const float2 u) { return Pk{pack2(u.x, u.x), pack2(-u.y, u.y)}; }
__device__ __forceinline__ f2p pmac(f2p acc, const Pk &c, f2p v, f2p vs) {
    acc = fma2(c.xx, v, acc);
    return fma2(c.yy, vs, acc);
}

// Dense gate of dimension D on the tile in shared memory; hi, lo: D x D
// coefficient blocks, row-major.  Each specialisation is its own function
// (called once per gate and tile), so that the register demand of the large
// ones stays out of the kernel body.  D <= 3: coefficients held in registers,
// packed FMAs (two groups per iteration for D = 2); D <= 8: rows fully
// unrolled, offsets in registers; larger D: one row at a time (bounded code).
template <int D>
__device__ __noinline__ void dense_tile(const BGate &G, float2 *st, const float2 *hi) {
    const float2 *lo = hi + D * D;
    constexpr bool kSmall = D <= 8;
    uint32_t off[kSmall ? D : 1];
    if (kSmall) {
#pragma unroll
        for (int j = 0; j < D; ++j) off[kSmall ? j : 0] = G.off[j];
    }
#define QD_OFF(j) (kSmall ? off[kSmall ? (j) : 0] : (uint32_t)G.off[j])
    if constexpr (D <= 3) {
        constexpr uint32_t P = D <= 2 ? 2 : 1;
        Pk ch[D * D], cl[D * D];
#pragma unroll
        for (int k = 0; k < D * D; ++k) {
            ch[k] = pk_coef(hi[k]);
            cl[k] = pk_coef(lo[k]);
        }
        for (uint32_t r0 = threadIdx.x; r0 < G.R; r0 += P * blockDim.x) {
            uint32_t base[P];
            bool ok[P];
            f2p v[P][D], vs[P][D];
#pragma unroll
            for (uint32_t p = 0; p < P; ++p) {
                const uint32_t r = r0 + p * blockDim.x;
                ok[p] = r < G.R;
                base[p] = ok[p] ? expand(r, G.ex) + G.base : 0;
#pragma unroll
                for (int j = 0; j < D; ++j) {
                    const float2 a = ok[p] ? st[base[p] + off[j]] : make_float2(0.f, 0.f);
                    v[p][j] = pack2(a.x, a.y);
                    vs[p][j] = pack2(a.y, a.x);
                }
            }
#pragma unroll
            for (int i = 0; i < D; ++i) {
#pragma unroll
                for (uint32_t p = 0; p < P; ++p) {
                    f2p acc = 0ull;
#pragma unroll
                    for (int j = 0; j < D; ++j) acc = pmac(acc, cl[i * D + j], v[p][j], vs[p][j]);
#pragma unroll
                    for (int j = 0; j < D; ++j) acc = pmac(acc, ch[i * D + j], v[p][j], vs[p][j]);
                    if (ok[p]) st[base[p] + off[i]] = unpack2(acc);
                }
            }
        }
    } else {
        for (uint32_t r = threadIdx.x; r < G.R; r += blockDim.x) {
            const uint32_t base = expand(r, G.ex) + G.base;
            float2 v[D];
#pragma unroll
            for (int j = 0; j < D; ++j) v[j] = st[base + QD_OFF(j)];
            if (kSmall) {
#pragma unroll
                for (int i = 0; i < D; ++i) {
                    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
                    for (int j = 0; j < D; ++j) cmac(acc, lo[i * D + j], v[j]);
#pragma unroll
                    for (int j = 0; j < D; ++j) cmac(acc, hi[i * D + j], v[j]);
                    st[base + QD_OFF(i)] = acc;
                }
            } else {
#pragma unroll 1
                for (int i = 0; i < D; ++i) {
                    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
                    for (int j = 0; j < D; ++j) cmac(acc, lo[i * D + j], v[j]);
#pragma unroll
                    for (int j = 0; j < D; ++j) cmac(acc, hi[i * D + j], v[j]);
                    st[base + G.off[i]] = acc;
                }
            }
        }
    }
}

// Permutation with phases of dimension D: out[i] = lam[i] in[src[i]] for the
// active i (lam[i] == 1 exactly where unit bit i is set); hi, lo: D phases.
template <int D>
__device__ __noinline__ void mono_tile(const BGate &G, float2 *st, const float2 *hi) {
    const float2 *lo = hi + D;
    constexpr bool kSmall = D <= 8;
    constexpr bool kRegLam = D <= 5;
    uint32_t off[kSmall ? D : 1], soff[kSmall ? D : 1];  // soff[i] = off[src[i]]
    if (kSmall) {
#pragma unroll
        for (int j = 0; j < D; ++j) {
            off[kSmall ? j : 0] = G.off[j];
            soff[kSmall ? j : 0] = G.off[G.src[j]];
        }
    }
#define QD_SOFF(i) (kSmall ? soff[kSmall ? (i) : 0] : (uint32_t)G.off[G.src[i]])
    const uint32_t active = G.active, unit = G.unit;
    Pk lh[kRegLam ? D : 1], ll[kRegLam ? D : 1];
    if (kRegLam) {
#pragma unroll
        for (int j = 0; j < D; ++j) {
            lh[kRegLam ? j : 0] = pk_coef(hi[j]);
            ll[kRegLam ? j : 0] = pk_coef(lo[j]);
        }
    }
    constexpr uint32_t P = D <= 5 ? 2 : 1;
    for (uint32_t r0 = threadIdx.x; r0 < G.R; r0 += P * blockDim.x) {
        uint32_t base[P];
        bool ok[P];
        float2 v[P][D];
#pragma unroll
        for (uint32_t p = 0; p < P; ++p) {
            const uint32_t r = r0 + p * blockDim.x;
            ok[p] = r < G.R;
            base[p] = ok[p] ? expand(r, G.ex) + G.base : 0;
#pragma unroll
            for (int i = 0; i < D; ++i)
                v[p][i] = (ok[p] && ((active >> i) & 1u)) ? st[base[p] + QD_SOFF(i)] : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (uint32_t p = 0; p < P; ++p) {
#pragma unroll
            for (int i = 0; i < D; ++i) {
                if (ok[p] && ((active >> i) & 1u)) {
                    float2 o = v[p][i];
                    if (!((unit >> i) & 1u)) {
                        if (kRegLam) {
                            const f2p w = pack2(o.x, o.y), ws = pack2(o.y, o.x);
                            o = unpack2(pmac(pmac(0ull, ll[kRegLam ? i : 0], w, ws), lh[kRegLam ? i : 0], w, ws));
                        } else {
                            float2 acc = make_float2(0.f, 0.f);
                            cmac(acc, lo[i], o);
                            cmac(acc, hi[i], o);
                            o = acc;
                        }
                    }
                    st[base[p] + QD_OFF(i)] = o;
                }
            }
        }
    }
}
#undef QD_OFF
#undef QD_SOFF

// Any D <= kBatchMaxD (dimensions that no specialisation covers).
__device__ __noinline__ void generic_tile(const BGate &G, float2 *st, const float2 *hi) {
    const int D = G.D;
    const float2 *lo = hi + G.ncoef;
    for (uint32_t r = threadIdx.x; r < G.R; r += blockDim.x) {
        const uint32_t base = expand(r, G.ex) + G.base;
        float2 v[kBatchMaxD];
        if (G.kind == 0) {
            for (int j = 0; j < D; ++j) v[j] = st[base + G.off[j]];
            for (int i = 0; i < D; ++i) {
                float2 acc = make_float2(0.f, 0.f);
                for (int j = 0; j < D; ++j) cmac(acc, lo[i * D + j], v[j]);
                for (int j = 0; j < D; ++j) cmac(acc, hi[i * D + j], v[j]);
                st[base + G.off[i]] = acc;
            }
        } else {
            for (int i = 0; i < D; ++i)
                if ((G.active >> i) & 1u) v[i] = st[base + G.off[G.src[i]]];
            for (int i = 0; i < D; ++i) {
                if ((G.active >> i) & 1u) {
                    float2 o = v[i];
                    if (!((G.unit >> i) & 1u)) {
                        float2 acc = make_float2(0.f, 0.f);
                        cmac(acc, lo[i], o);
                        cmac(acc, hi[i], o);
                        o = acc;
                    }
                    st[base + G.off[i]] = o;
                }
            }
        }
    }
}

__device__ __forceinline__ void apply_gate(const BGate &G, float2 *st, const float2 *cf) {
#define QD_BATCH_CASE(DD)                         \
    case DD:                                      \
        if (G.kind == 0) dense_tile<DD>(G, st, cf); \
        else mono_tile<DD>(G, st, cf);            \
        break;
    switch (G.D) {
        QD_BATCH_CASE(2)
        QD_BATCH_CASE(3)
        QD_BATCH_CASE(4)
        QD_BATCH_CASE(5)
        QD_BATCH_CASE(6)
        QD_BATCH_CASE(8)
        QD_BATCH_CASE(9)
        QD_BATCH_CASE(10)
        QD_BATCH_CASE(12)
        QD_BATCH_CASE(15)
        QD_BATCH_CASE(16)
        QD_BATCH_CASE(20)
        QD_BATCH_CASE(25)
        default:
            generic_tile(G, st, cf);
    }
#undef QD_BATCH_CASE
}

// State gathers bypass L1 (another CTA may have written the amplitudes).
__device__ __forceinline__ void cp_async_cg16(void *smem, const void *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}

// Gather (LOAD) or scatter one tile between the state and shared memory.
// Paired segments gather 16-byte amplitude pairs asynchronously (the caller
// waits with cp_async_wait_all); otherwise 8 accesses per thread in flight.
template <bool LOAD>
__device__ __forceinline__ void move_tile(float2 *psi, float2 *st, const BSeg &S, uint32_t tb,
                                          const uint32_t *__restrict__ hoff) {
    constexpr int U = 8;
    const uint32_t T = S.T, B = S.B;
    const FastDiv32 divB = S.divB;
    auto flat = [&](uint32_t l) {
        const uint32_t h = fdiv(l, divB);
        return tb + (l - h * B) + __ldg(hoff + h);
    };
    if (LOAD && S.pair) {
        for (uint32_t l = 2 * threadIdx.x; l < T; l += 2 * kBThreads) cp_async_cg16(st + l, psi + flat(l));
        return;
    }
    for (uint32_t l0 = threadIdx.x; l0 < T; l0 += U * kBThreads) {
        if (LOAD) {
            float2 v[U];
#pragma unroll
            for (int k = 0; k < U; ++k)
                if (l0 + k * kBThreads < T) v[k] = __ldcg(psi + flat(l0 + k * kBThreads));
#pragma unroll
            for (int k = 0; k < U; ++k)
                if (l0 + k * kBThreads < T) st[l0 + k * kBThreads] = v[k];
        } else {
#pragma unroll
            for (int k = 0; k < U; ++k)
                if (l0 + k * kBThreads < T) psi[flat(l0 + k * kBThreads)] = st[l0 + k * kBThreads];
        }
    }
}

__global__ void __launch_bounds__(kBThreads, 5)
    k_batch(float2 *__restrict__ arena, const uint64_t *__restrict__ offs, const BSeg *__restrict__ segs,
            const BChunk *__restrict__ chunks, const BGate *__restrict__ gates, const float2 *__restrict__ coef,
            const uint32_t *__restrict__ hofftab, const BItem *__restrict__ items, int32_t nitems,
            uint32_t *__restrict__ next, uint32_t *__restrict__ done, int32_t *__restrict__ err,
            uint32_t desc_bytes, uint32_t poll_limit) {
    extern __shared__ __align__(16) unsigned char smraw[];
    BSeg &S = *reinterpret_cast<BSeg *>(smraw);
    unsigned char *desc = smraw + ((sizeof(BSeg) + 15) / 16) * 16;
    float2 *st = reinterpret_cast<float2 *>(desc + desc_bytes);
    __shared__ BChunk s_ch;
    __shared__ int32_t s_item;
    __shared__ int32_t s_ok;
    int32_t nxt = 0;
    if (threadIdx.x == 0) nxt = (int32_t)atomicAdd(next, 1u);
    for (;;) {
        if (threadIdx.x == 0) s_item = nxt;
        __syncthreads();
        const int32_t id = s_item;
        if (id >= nitems) break;
        const BItem it = items[id];
        if (threadIdx.x == 0) {
            nxt = (int32_t)atomicAdd(next, 1u);  // claim the following item now
            s_ok = 1;
            const volatile uint32_t *d = done + it.circuit;
            uint32_t polls = 0;
            while (*d < it.wait_target) {
                if (++polls > poll_limit) {
                    atomicExch(err, 2);
                    s_ok = 0;
                    break;
                }
                __nanosleep(128);
            }
            __threadfence();
        }
        copy_desc(&S, segs + it.seg);
        __syncthreads();
        if (s_ok) {
            float2 *psi = arena + offs[it.circuit];
            const uint32_t *hoff = hofftab + S.hoff;
            const bool one_chunk = S.nchunks == 1;
            for (uint32_t t = it.first; t < it.first + it.count; ++t) {
                const uint32_t tb = expand(t, S.ex);
                for (int c = 0; c < S.nchunks; ++c) {
                    const bool fresh = !(one_chunk && t > it.first);
                    if (fresh) {
                        if (threadIdx.x == 0) s_ch = chunks[S.chunk0 + c];
                        __syncthreads();
                        load_chunk(s_ch, gates, coef, desc);
                    }
                    if (c == 0) move_tile<true>(psi, st, S, tb, hoff);
                    if (fresh || (c == 0 && S.pair)) cp_async_wait_all();
                    __syncthreads();
                    // s_ch is read once here, before the first gate's barrier: thread 0
                    // rewrites it for the next chunk after the last gate's barrier
                    const int ng = s_ch.ngates;
                    const BGate *sg = reinterpret_cast<const BGate *>(desc);
                    const float2 *sc = reinterpret_cast<const float2 *>(desc + ng * sizeof(BGate));
                    for (int g = 0; g < ng; ++g) {
                        const BGate &G = sg[g];
                        // descriptor sanity: a gate's groups stay inside the tile and its
                        // coefficients inside the chunk (else: error word, gate skipped)
                        if (G.D >= 2 && G.D <= kBatchMaxD && (uint64_t)G.R * (uint32_t)G.D <= S.T &&
                            ng * sizeof(BGate) + (size_t)(G.coef + 2 * G.ncoef) * sizeof(float2) <= desc_bytes)
                            apply_gate(G, st, sc + G.coef);
                        else if (threadIdx.x == 0)
                            atomicExch(err, 3);
                        __syncthreads();
                    }
                }
                move_tile<false>(psi, st, S, tb, hoff);
                __syncthreads();
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(done + it.circuit, it.count);
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

size_t batch_smem_bytes(uint32_t tile_cap, uint32_t desc_bytes) {
    return ((sizeof(BSeg) + 15) / 16) * 16 + desc_bytes + (size_t)tile_cap * sizeof(float2);
}

int batch_occupancy(uint32_t tile_cap, uint32_t desc_bytes) {
    const size_t smem = batch_smem_bytes(tile_cap, desc_bytes);
    if (cudaFuncSetAttribute((const void *)k_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch, kBThreads, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return occ;
}

cudaError_t batch_launch(const BatchLaunch &b, cudaStream_t s, cudaEvent_t ev0, cudaEvent_t ev1) {
    cudaError_t e = cudaMemsetAsync(b.counters, 0, sizeof(uint32_t) * (1 + (size_t)b.ncirc), s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(b.err, 0, sizeof(int32_t), s);  // the error word reports this run only
    if (e != cudaSuccess) return e;
    k_batch_init<<<b.sm_count * 4, 256, 0, s>>>(b.arena, b.total);
    k_batch_ones<<<(b.ncirc + 255) / 256, 256, 0, s>>>(b.arena, b.offs, b.basis, b.ncirc);
    if (b.nitems > 0) {
        const size_t smem = batch_smem_bytes(b.tile_cap, b.desc_bytes);
        const int occ = std::max(1, batch_occupancy(b.tile_cap, b.desc_bytes));
        const int per_sm = b.ctas_per_sm > 0 && b.ctas_per_sm < occ ? b.ctas_per_sm : occ;
        const int grid = b.sm_count * per_sm;
        if (ev0) cudaEventRecord(ev0, s);
        k_batch<<<grid, kBThreads, smem, s>>>(b.arena, b.offs, b.segs, b.chunks, b.gates, b.coef, b.hoff, b.items,
                                             b.nitems, b.counters, b.counters + 1, b.err, b.desc_bytes, b.poll_limit);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        if (ev1) cudaEventRecord(ev1, s);
    } else if (ev0) {
        cudaEventRecord(ev0, s);
        cudaEventRecord(ev1, s);
    }
    return probabilities(b.arena, 1, b.total, b.probs, b.sm_count, s);
}

}  // namespace qd
