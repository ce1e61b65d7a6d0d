// Fused-block apply on the fifth-generation tensor cores (tcgen05, sm_100+).
//
// A fused block is a dense D x D complex matrix U over a set of qudits (the
// FP64 product of a run of gates, QuDiet Sec. 2.1.2 / 3.4 gates).  For every
// group of D amplitudes v (the block's local index, as in the per-gate
// kernels), v <- U v.  Stacking 128 groups as the rows of a matrix X
// (128 x 2D reals, interleaved re/im), the update is one real GEMM
//     Y (128 x 2D) = X (128 x 2D) * B^T,   B = [[Ur, -Ui], [Ui, Ur]] interleaved,
// issued as tcgen05.mma kind::f16 (BF16 inputs, FP32 accumulation in TMEM),
// M = 128 groups, N = K = 2 Dp (Dp = D rounded up to a multiple of 8).
//
// Precision.  The tensor cores round each accumulation step toward zero; a
// rounded running sum loses on average about 0.36 ulp per instruction, always
// toward zero, which shrinks every amplitude coherently (measured: 1 - F =
// 1.5e-6 after one D = 64 block with a hi/lo split).  The kernel therefore
// keeps every partial sum exact (the error-free splitting of Ozaki, Ogita,
// Oishi and Rump, 2012): each state row r is scaled by 2^-e_r (e_r from the
// row maximum) and cut into three 8-bit fixed-point slices
//     x~ = x1 + x2 + x3 + O(2^-27),  x_s = k / 2^(9s-1),  |k| <= 256,
// and each matrix row n likewise with its own 2^-f_n into B1 + B2 + B3.  Every
// slice value is exact in BF16, every product of two slices is a multiple of
// one quantum per significance level, and a level's sum stays below 2^24
// quanta, so the tensor core accumulates it without rounding.  Three TMEM
// accumulators hold the levels 2^0 (x1 B1), 2^-9 (x1 B2 + x2 B1) and 2^-18
// (x1 B3 + x2 B2 + x3 B1); the epilogue adds them in FP32 with
// round-to-nearest and rescales by 2^(e_r + f_n).  The matrix is represented
// to 2^-27 (coherent error ~1e-8 per block), the state to 2^-27 before the
// dropped level-2^-27 products (incoherent).
//
// Shared-memory operands use the no-swizzle K-major canonical layout: core
// matrices of 8 rows x 16 bytes (8 BF16), consecutive along K at 128 B
// (leading byte offset), 8-row groups at K*16 B (stride byte offset).
// One CTA of 128 threads owns a tile of 128 groups per iteration: thread t
// gathers group t, slices it and writes row t of X1..X3; one thread issues
// the MMAs and commits them to an mbarrier; after the (bounded) wait, thread
// t reads TMEM lane t (its group's outputs at the three levels) and scatters
// them back.  Every wait is bounded; on expiry the kernel records an error,
// waits (bounded) for its MMAs, frees its TMEM and returns.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "qd_plan.h"
#include "qd_tc.h"

namespace qd {

namespace {

constexpr int kTcThreads = 128;
constexpr int kTcRows = 128;             // groups per tile (MMA M)
constexpr uint32_t kWaitLimit = 1u << 24;  // bounded mbarrier polls

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of element (row, k) in a K-major no-swizzle tile with K columns
__host__ __device__ __forceinline__ uint32_t cm_off(uint32_t row, uint32_t k, uint32_t K) {
    return (row >> 3) * (K * 16u) + (k >> 3) * 128u + (row & 7u) * 16u + (k & 7u) * 2u;
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version for tcgen05
    // base offset 0, absolute LBO mode 0, layout type 0 = no swizzle
    return d;
}

// Instruction descriptor, kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N and M encoded >>3 and >>4.
__host__ __device__ __forceinline__ uint32_t idesc_bf16(uint32_t M, uint32_t N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t mbar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ bool mbar_wait_bounded(uint32_t mbar, uint32_t parity) {
    for (uint32_t it = 0; it < kWaitLimit; ++it)
        if (mbar_try(mbar, parity)) return true;
    return false;
}

template <int NCOL>
__device__ __forceinline__ void tmem_ld(uint32_t taddr, float *out);

// 16 consecutive columns of this thread's TMEM lane, no wait (the caller
// issues tcgen05.wait::ld once for a batch of loads).
__device__ __forceinline__ void tmem_ld16_nowait(uint32_t taddr, uint32_t *r) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory"); }

template <>
__device__ __forceinline__ void tmem_ld<8>(uint32_t taddr, float *o) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int i = 0; i < 8; ++i) o[i] = __uint_as_float(r[i]);
}

}  // namespace

// Kernel arguments: direct-mode group geometry plus the matrix slices,
// already in the K-major canonical layout (B1 | B2 | B3, each N x K BF16 =
// 2*N*K bytes), followed by the N row scales 2^f_n (float), in global memory.
template <typename I>
struct TcArgs {
    float2 *psi;
    I R;
    ExpandT<I> ex;
    I off[kMaxBlockD];
    int32_t D, Dp;
    const __nv_bfloat16 *terms;
    int32_t *err;
};

// 8-bit fixed-point slices of a value already scaled into [-1, 1]:
// s1 = k1/2^8, s2 = k2/2^17, s3 = k3/2^26 with |k| <= 256 (exact in BF16).
__device__ __forceinline__ void slice3(float v, __nv_bfloat16 &a, __nv_bfloat16 &b, __nv_bfloat16 &c) {
    const float s1 = rintf(v * 256.0f) * (1.0f / 256.0f);
    const float r1 = v - s1;
    const float s2 = rintf(r1 * 131072.0f) * (1.0f / 131072.0f);
    const float r2 = r1 - s2;
    const float s3 = rintf(r2 * 67108864.0f) * (1.0f / 67108864.0f);
    a = __float2bfloat16_rn(s1);
    b = __float2bfloat16_rn(s2);
    c = __float2bfloat16_rn(s3);
}

__device__ __forceinline__ void named_sync(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;\n" ::"r"(id), "r"(nthreads) : "memory");
}

// MAXD: compile-time bound on Dp (16, 32 or 64); the group's values stay in
// registers between the row-maximum pass and the slicing.  SLOTS independent
// 128-row tiles per CTA (2 when the slices fit twice, else 1): slot s uses
// warps 4s..4s+3, its own X slices, mbarrier, named barrier and TMEM columns,
// so one slot's gather overlaps the other's MMAs and epilogue.
template <typename I, int MAXD>
__global__ void __launch_bounds__(kTcThreads *(MAXD <= 32 ? 2 : 1), 1) k_block_tc(const __grid_constant__ TcArgs<I> a) {
    constexpr int SLOTS = MAXD <= 32 ? 2 : 1;
    extern __shared__ __align__(1024) unsigned char sm[];
    const uint32_t K = 2u * (uint32_t)a.Dp;  // = N
    const uint32_t xbytes = kTcRows * K * 2u;  // one state slice (BF16)
    const uint32_t bbytes = K * K * 2u;        // one matrix slice
    unsigned char *B = sm;                     // B1 | B2 | B3 | row scales
    float *bscale = reinterpret_cast<float *>(B + 3u * bbytes);
    const uint32_t bregion = (3u * bbytes + K * 4u + 1023u) & ~1023u;
    __shared__ __align__(8) uint64_t mbar[SLOTS];
    __shared__ uint32_t tmem_base;
    __shared__ int32_t abort_flag[SLOTS];

    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int slot = tid >> 7;       // 128 threads per slot
    const int row = tid & 127;       // group row of this thread within its tile
    unsigned char *X = sm + bregion + (uint32_t)slot * 3u * xbytes;  // X1 | X2 | X3 of this slot
    uint32_t ncols = 32;
    while (ncols < (uint32_t)SLOTS * 3u * K) ncols <<= 1;

    // matrix slices and row scales: global -> shared (16-byte copies)
    {
        const uint4 *src = reinterpret_cast<const uint4 *>(a.terms);
        uint4 *dst = reinterpret_cast<uint4 *>(B);
        const uint32_t n16 = (3u * bbytes + K * 4u + 15u) / 16u;
        for (uint32_t i = tid; i < n16; i += blockDim.x) dst[i] = src[i];
    }
    if (tid < SLOTS) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&mbar[tid])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        abort_flag[tid] = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_base)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t acc = tmem_base + (uint32_t)slot * 3u * K;  // this slot's three level accumulators
    const uint32_t idesc = idesc_bf16(kTcRows, K);
    const uint32_t lbo = 128u, sbo = K * 16u;
    const uint32_t mb = smem_u32(&mbar[slot]);
    const int bar_id = 1 + slot;

    uint32_t phase = 0;
    const I ntiles = (a.R + kTcRows - 1) / kTcRows;
    const I tstride = (I)gridDim.x * SLOTS;
    I tile = (I)blockIdx.x * SLOTS + slot;
    // The amplitudes of the next tile are loaded right after this tile's MMAs
    // are issued, so their latency hides behind the MMAs and the epilogue.
    float2 v[MAXD];
    I base = 0;
    bool valid = false;
    auto gather = [&](I t) {
        const I g = t * kTcRows + row;
        valid = g < a.R;
        base = valid ? expand(g, a.ex) : 0;
#pragma unroll
        for (int j = 0; j < MAXD; ++j) v[j] = (valid && j < a.D) ? a.psi[base + a.off[j]] : make_float2(0.f, 0.f);
    };
    if (tile < ntiles) gather(tile);
    while (tile < ntiles) {
        // ---- row scale 2^-e from the row maximum ...
        float amax = 0.f;
#pragma unroll
        for (int j = 0; j < MAXD; ++j) amax = fmaxf(amax, fmaxf(fabsf(v[j].x), fabsf(v[j].y)));
        int e = 0;
        frexpf(amax, &e);  // amax <= 2^e
        const float inv = ldexpf(1.0f, -e);
        // ... cut every value into three slices, write row `row` of X1..X3
#pragma unroll
        for (int c0 = 0; c0 < MAXD; c0 += 4) {  // 4 amplitudes = 8 BF16 = one 16-byte chunk
            if (c0 < a.Dp) {
                __align__(16) __nv_bfloat16 h1[8], h2[8], h3[8];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    slice3(v[c0 + u].x * inv, h1[2 * u], h2[2 * u], h3[2 * u]);
                    slice3(v[c0 + u].y * inv, h1[2 * u + 1], h2[2 * u + 1], h3[2 * u + 1]);
                }
                const uint32_t o = cm_off((uint32_t)row, (uint32_t)(2 * c0), K);
                *reinterpret_cast<uint4 *>(X + o) = *reinterpret_cast<const uint4 *>(h1);
                *reinterpret_cast<uint4 *>(X + xbytes + o) = *reinterpret_cast<const uint4 *>(h2);
                *reinterpret_cast<uint4 *>(X + 2u * xbytes + o) = *reinterpret_cast<const uint4 *>(h3);
            }
        }
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        named_sync(bar_id, kTcRows);
        // ---- one thread of the slot issues the six slice products into three level accumulators
        if (row == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            const uint32_t x0 = smem_u32(X), b0 = smem_u32(B);
            // (level, x slice, B slice)
            const int pairs[6][3] = {{0, 0, 0}, {1, 0, 1}, {1, 1, 0}, {2, 0, 2}, {2, 1, 1}, {2, 2, 0}};
            const uint32_t ksteps = K / 16u;
#pragma unroll 1
            for (int p = 0; p < 6; ++p) {
                const uint32_t dcol = acc + (uint32_t)pairs[p][0] * K;
                const uint32_t xa = x0 + (uint32_t)pairs[p][1] * xbytes;
                const uint32_t bt = b0 + (uint32_t)pairs[p][2] * bbytes;
                const bool first_of_level = (p == 0 || p == 1 || p == 3);
#pragma unroll 1
                for (uint32_t s = 0; s < ksteps; ++s) {
                    const uint64_t ad = smem_desc(xa + s * 256u, lbo, sbo);
                    const uint64_t bd = smem_desc(bt + s * 256u, lbo, sbo);
                    mma_bf16(dcol, ad, bd, idesc, (first_of_level && s == 0) ? 0u : 1u);
                }
            }
            mma_commit(mb);
        }
        // ---- prefetch the next tile while the MMAs run
        const I base_cur = base;
        const bool valid_cur = valid;
        const I next = tile + tstride;
        if (next < ntiles) gather(next);
        // ---- wait for the MMAs (bounded)
        const bool ok = mbar_wait_bounded(mb, phase);
        phase ^= 1u;
        if (!ok) {
            atomicExch(a.err, 1);
            abort_flag[slot] = 1;
        }
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        named_sync(bar_id, kTcRows);
        if (abort_flag[slot]) {
            // one more bounded wait for the MMAs in flight, then release TMEM
            mbar_wait_bounded(mb, phase ^ 1u);
            break;
        }
        // ---- TMEM lane `row`: levels 2^0, 2^-9, 2^-18 -> outputs -> scatter back
        const uint32_t lane_addr = acc + ((uint32_t)((warp & 3) * 32) << 16);
        const float escale = ldexpf(1.0f, e);
#pragma unroll
        for (int c0 = 0; c0 < MAXD; c0 += 8) {  // 8 amplitudes = 16 columns per level
            if (c0 < a.Dp) {
                uint32_t l0[16], l1[16], l2[16];
                tmem_ld16_nowait(lane_addr + (uint32_t)(2 * c0), l0);
                tmem_ld16_nowait(lane_addr + K + (uint32_t)(2 * c0), l1);
                tmem_ld16_nowait(lane_addr + 2u * K + (uint32_t)(2 * c0), l2);
                tmem_wait_ld();
                if (valid_cur) {
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int j = c0 + u;
                        if (j < a.D) {
                            const int n = 2 * j;
                            const float re = (__uint_as_float(l0[2 * u]) +
                                              (__uint_as_float(l1[2 * u]) + __uint_as_float(l2[2 * u]))) *
                                             (escale * bscale[n]);
                            const float im = (__uint_as_float(l0[2 * u + 1]) +
                                              (__uint_as_float(l1[2 * u + 1]) + __uint_as_float(l2[2 * u + 1]))) *
                                             (escale * bscale[n + 1]);
                            a.psi[base_cur + a.off[j]] = make_float2(re, im);
                        }
                    }
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        named_sync(bar_id, kTcRows);
        tile = next;
    }
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem_base), "r"(ncols)
                     : "memory");
}

// ---------------------------------------------------------------------------
// Warp-specialised variant for Dp <= 32 (the common fused blocks): the three
// steps of a tile run in different warps so that they overlap across tiles.
//   producers (warps 5..12, two groups of 128 rows): gather a tile's groups,
//     slice them into stage s of a 3-stage shared-memory ring, arrive full[s];
//   MMA issuer (warp 4, one lane): wait full[s] and acc_empty[a], issue the
//     six slice products into accumulator slot a of a 2-slot TMEM ring,
//     commit to acc_full[a];
//   epilogue (warps 0..3, one TMEM lane per thread): wait acc_full[a], combine
//     the levels, scatter the outputs, arrive acc_empty[a] and empty[s].
// Tile i of this CTA uses stage i % 3 and slot i % 2; mbarrier phases count
// the reuses.  Every wait is bounded and also gives up when another warp has
// raised the abort flag; the MMA warp waits (bounded) for its last commit
// before TMEM is freed.
// ---------------------------------------------------------------------------
constexpr int kWsStages = 3;
constexpr int kWsSlots = 2;
constexpr int kWsProducerWarps = 8;
constexpr int kWsThreads = 32 * (4 + 1 + kWsProducerWarps);

__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(mbar) : "memory");
}

// Bounded wait that also returns (false) once *abort is set by another warp.
__device__ __forceinline__ bool ws_wait(uint32_t mbar, uint32_t parity, volatile int32_t *abort, int32_t *err) {
    for (uint32_t it = 0; it < kWaitLimit; ++it) {
        if (mbar_try(mbar, parity)) return true;
        if ((it & 255u) == 255u && *abort) return false;
    }
    *abort = 1;
    atomicExch(err, 1);
    return false;
}

template <typename I, int MAXD>
__global__ void __launch_bounds__(kWsThreads, 1) k_block_tc_ws(const __grid_constant__ TcArgs<I> a) {
    extern __shared__ __align__(1024) unsigned char sm[];
    const uint32_t K = 2u * (uint32_t)a.Dp;
    const uint32_t xbytes = kTcRows * K * 2u;
    const uint32_t bbytes = K * K * 2u;
    unsigned char *B = sm;
    float *bscale = reinterpret_cast<float *>(B + 3u * bbytes);
    const uint32_t bregion = (3u * bbytes + K * 4u + 1023u) & ~1023u;
    unsigned char *stages = sm + bregion;  // stage s: X1 | X2 | X3 at s * 3 * xbytes
    __shared__ __align__(8) uint64_t full[kWsStages], empty[kWsStages], acc_full[kWsSlots], acc_empty[kWsSlots];
    __shared__ int32_t erow[kWsStages][kTcRows];
    __shared__ uint32_t tmem_base;
    __shared__ volatile int32_t abort_flag;

    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    uint32_t ncols = 32;
    while (ncols < (uint32_t)kWsSlots * 3u * K) ncols <<= 1;

    {
        const uint4 *src = reinterpret_cast<const uint4 *>(a.terms);
        uint4 *dst = reinterpret_cast<uint4 *>(B);
        const uint32_t n16 = (3u * bbytes + K * 4u + 15u) / 16u;
        for (uint32_t i = tid; i < n16; i += blockDim.x) dst[i] = src[i];
    }
    if (tid == 0) {
        for (int q = 0; q < kWsStages; ++q) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(&full[q])), "r"(kTcRows) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(&empty[q])), "r"(kTcRows) : "memory");
        }
        for (int q = 0; q < kWsSlots; ++q) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&acc_full[q])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(&acc_empty[q])), "r"(kTcRows)
                         : "memory");
        }
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        abort_flag = 0;
    }
    if (warp == 4) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_base)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");

    const I ntiles = (a.R + kTcRows - 1) / kTcRows;
    const I nlocal = (I)blockIdx.x < ntiles ? (ntiles - (I)blockIdx.x + (I)gridDim.x - 1) / (I)gridDim.x : 0;
    const uint32_t tmem = tmem_base;

    if (warp >= 5) {
        // ------------------------------------------------------------ producers
        const int p = tid - 160;
        const int grp = p >> 7, row = p & 127;
        for (I i = (I)grp; i < nlocal; i += 2) {
            const int st = (int)(i % kWsStages);
            const uint32_t use = (uint32_t)(i / kWsStages);
            const I t = (I)blockIdx.x + i * (I)gridDim.x;
            const I g = t * kTcRows + row;
            const bool valid = g < a.R;
            const I base = valid ? expand(g, a.ex) : 0;
            float2 v[MAXD];
#pragma unroll
            for (int j = 0; j < MAXD; ++j)
                v[j] = (valid && j < a.D) ? a.psi[base + a.off[j]] : make_float2(0.f, 0.f);
            float amax = 0.f;
#pragma unroll
            for (int j = 0; j < MAXD; ++j) amax = fmaxf(amax, fmaxf(fabsf(v[j].x), fabsf(v[j].y)));
            int e = 0;
            frexpf(amax, &e);
            const float inv = ldexpf(1.0f, -e);
            if (use >= 1 && !ws_wait(smem_u32(&empty[st]), (use - 1) & 1u, &abort_flag, a.err)) break;
            unsigned char *X = stages + (uint32_t)st * 3u * xbytes;
#pragma unroll
            for (int c0 = 0; c0 < MAXD; c0 += 4) {
                if (c0 < a.Dp) {
                    __align__(16) __nv_bfloat16 h1[8], h2[8], h3[8];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        slice3(v[c0 + u].x * inv, h1[2 * u], h2[2 * u], h3[2 * u]);
                        slice3(v[c0 + u].y * inv, h1[2 * u + 1], h2[2 * u + 1], h3[2 * u + 1]);
                    }
                    const uint32_t o = cm_off((uint32_t)row, (uint32_t)(2 * c0), K);
                    *reinterpret_cast<uint4 *>(X + o) = *reinterpret_cast<const uint4 *>(h1);
                    *reinterpret_cast<uint4 *>(X + xbytes + o) = *reinterpret_cast<const uint4 *>(h2);
                    *reinterpret_cast<uint4 *>(X + 2u * xbytes + o) = *reinterpret_cast<const uint4 *>(h3);
                }
            }
            erow[st][row] = e;
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            mbar_arrive(smem_u32(&full[st]));
        }
    } else if (warp == 4) {
        // ------------------------------------------------------------ MMA issuer
        if ((tid & 31) == 0) {
            const uint32_t idesc = idesc_bf16(kTcRows, K);
            const uint32_t lbo = 128u, sbo = K * 16u;
            const uint32_t b0 = smem_u32(B);
            const int pairs[6][3] = {{0, 0, 0}, {1, 0, 1}, {1, 1, 0}, {2, 0, 2}, {2, 1, 1}, {2, 2, 0}};
            const uint32_t ksteps = K / 16u;
            I issued = 0;
            for (I i = 0; i < nlocal; ++i) {
                const int st = (int)(i % kWsStages), sl = (int)(i & 1);
                if (!ws_wait(smem_u32(&full[st]), (uint32_t)(i / kWsStages) & 1u, &abort_flag, a.err)) break;
                if (i >= 2 && !ws_wait(smem_u32(&acc_empty[sl]), (uint32_t)((i >> 1) - 1) & 1u, &abort_flag, a.err))
                    break;
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                const uint32_t x0 = smem_u32(stages + (uint32_t)st * 3u * xbytes);
                const uint32_t acc = tmem + (uint32_t)sl * 3u * K;
#pragma unroll 1
                for (int pp = 0; pp < 6; ++pp) {
                    const uint32_t dcol = acc + (uint32_t)pairs[pp][0] * K;
                    const uint32_t xa = x0 + (uint32_t)pairs[pp][1] * xbytes;
                    const uint32_t bt = b0 + (uint32_t)pairs[pp][2] * bbytes;
                    const bool first_of_level = (pp == 0 || pp == 1 || pp == 3);
#pragma unroll 1
                    for (uint32_t ks = 0; ks < ksteps; ++ks)
                        mma_bf16(dcol, smem_desc(xa + ks * 256u, lbo, sbo), smem_desc(bt + ks * 256u, lbo, sbo), idesc,
                                 (first_of_level && ks == 0) ? 0u : 1u);
                }
                mma_commit(smem_u32(&acc_full[sl]));
                issued = i + 1;
            }
            // before TMEM is released: the last commit must have completed
            if (issued > 0) {
                const I last = issued - 1;
                const uint32_t mb = smem_u32(&acc_full[last & 1]);
                for (uint32_t it = 0; it < kWaitLimit; ++it)
                    if (mbar_try(mb, (uint32_t)(last >> 1) & 1u)) break;
            }
        }
    } else {
        // ------------------------------------------------------------ epilogue
        const int row = tid;  // TMEM lane of this thread (warps 0..3)
        const float *bs = bscale;
        for (I i = 0; i < nlocal; ++i) {
            const int st = (int)(i % kWsStages), sl = (int)(i & 1);
            if (!ws_wait(smem_u32(&acc_full[sl]), (uint32_t)(i >> 1) & 1u, &abort_flag, a.err)) break;
            // the producers' row scales of this stage (phase already complete)
            if (!ws_wait(smem_u32(&full[st]), (uint32_t)(i / kWsStages) & 1u, &abort_flag, a.err)) break;
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            const int e = erow[st][row];
            const float escale = ldexpf(1.0f, e);
            const I t = (I)blockIdx.x + i * (I)gridDim.x;
            const I g = t * kTcRows + row;
            const bool valid = g < a.R;
            const I base = valid ? expand(g, a.ex) : 0;
            const uint32_t lane_addr = tmem + (uint32_t)sl * 3u * K + ((uint32_t)(warp * 32) << 16);
#pragma unroll
            for (int c0 = 0; c0 < MAXD; c0 += 8) {
                if (c0 < a.Dp) {
                    uint32_t l0[16], l1[16], l2[16];
                    tmem_ld16_nowait(lane_addr + (uint32_t)(2 * c0), l0);
                    tmem_ld16_nowait(lane_addr + K + (uint32_t)(2 * c0), l1);
                    tmem_ld16_nowait(lane_addr + 2u * K + (uint32_t)(2 * c0), l2);
                    tmem_wait_ld();
                    if (valid) {
#pragma unroll
                        for (int u = 0; u < 8; ++u) {
                            const int j = c0 + u;
                            if (j < a.D) {
                                const int n = 2 * j;
                                const float re = (__uint_as_float(l0[2 * u]) +
                                                  (__uint_as_float(l1[2 * u]) + __uint_as_float(l2[2 * u]))) *
                                                 (escale * bs[n]);
                                const float im = (__uint_as_float(l0[2 * u + 1]) +
                                                  (__uint_as_float(l1[2 * u + 1]) + __uint_as_float(l2[2 * u + 1]))) *
                                                 (escale * bs[n + 1]);
                                a.psi[base + a.off[j]] = make_float2(re, im);
                            }
                        }
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
            mbar_arrive(smem_u32(&acc_empty[sl]));
            mbar_arrive(smem_u32(&empty[st]));
        }
    }
    __syncthreads();
    if (warp == 4)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(ncols) : "memory");
}

size_t tc_terms_bytes(int Dp) {
    const size_t K = 2 * (size_t)Dp;
    return (3 * K * K * 2 + K * 4 + 15) / 16 * 16;
}

// Host: the real embedding B (N x K, N = K = 2 Dp) of the D x D complex
// matrix U (interleaved FP64), each row n scaled by 2^-f_n (its maximum
// <= 2^f_n) and cut into three 8-bit fixed-point slices stored as BF16 in the
// kernel's shared-memory layout, followed by the row scales 2^f_n (float).
void tc_pack_terms(const double *U, int D, int Dp, uint16_t *out) {
    const int K = 2 * Dp;
    const size_t term_elems = (size_t)K * K;
    std::memset(out, 0, tc_terms_bytes(Dp));
    auto bf16_bits = [](double x) -> uint16_t {
        // x is a slice value k * 2^-m with |k| <= 256: exact in FP32 and BF16
        const float f = (float)x;
        uint32_t u;
        std::memcpy(&u, &f, 4);
        return (uint16_t)(u >> 16);
    };
    std::vector<double> row((size_t)K);
    float *scales = reinterpret_cast<float *>(out + 3 * term_elems);
    for (int n = 0; n < K; ++n) {
        std::fill(row.begin(), row.end(), 0.0);
        if (n < 2 * D) {
            const int i = n / 2, p = n % 2;
            for (int k = 0; k < D; ++k) {
                const double ur = U[2 * (i * D + k)], ui = U[2 * (i * D + k) + 1];
                // row 2i: (ur, -ui) ; row 2i+1: (ui, ur) on columns (2k, 2k+1)
                row[2 * k] = p == 0 ? ur : ui;
                row[2 * k + 1] = p == 0 ? -ui : ur;
            }
        }
        double mx = 0.0;
        for (double v : row) mx = std::max(mx, std::fabs(v));
        int f = 0;
        std::frexp(mx, &f);  // mx <= 2^f
        scales[n] = (float)std::ldexp(1.0, f);
        for (int kk = 0; kk < K; ++kk) {
            double v = std::ldexp(row[kk], -f);
            const double s1 = std::nearbyint(v * 256.0) / 256.0;
            v -= s1;
            const double s2 = std::nearbyint(v * 131072.0) / 131072.0;
            v -= s2;
            const double s3 = std::nearbyint(v * 67108864.0) / 67108864.0;
            const uint32_t off = cm_off((uint32_t)n, (uint32_t)kk, (uint32_t)K) / 2;
            out[off] = bf16_bits(s1);
            out[term_elems + off] = bf16_bits(s2);
            out[2 * term_elems + off] = bf16_bits(s3);
        }
    }
}

static int tc_slots(int Dp) { return Dp <= 32 ? 2 : 1; }

static int tc_ws_smem_bytes(int Dp) {
    const int K = 2 * Dp;
    const int bregion = (3 * K * K * 2 + K * 4 + 1023) & ~1023;
    return bregion + kWsStages * 3 * kTcRows * K * 2;
}

int tc_smem_bytes(int Dp) {
    const int K = 2 * Dp;
    const int bregion = (3 * K * K * 2 + K * 4 + 1023) & ~1023;
    return bregion + tc_slots(Dp) * 3 * kTcRows * K * 2;
}

template <typename I, int MAXD>
static cudaError_t launch_tc_im(const GatePlan &g, void *psi, int sm_count, int32_t *err, cudaStream_t s) {
    TcArgs<I> a;
    a.psi = static_cast<float2 *>(psi);
    a.R = (I)g.R;
    if constexpr (sizeof(I) == 4) a.ex = narrow(g.ex);
    else a.ex = g.ex;
    for (int j = 0; j < kMaxBlockD; ++j) a.off[j] = j < g.D ? (I)g.off[j] : 0;
    a.D = g.D;
    a.Dp = g.Dp;
    a.terms = static_cast<const __nv_bfloat16 *>(g.tc_terms);
    a.err = err;
    const int smem = tc_smem_bytes(g.Dp);
    const int threads = kTcThreads * tc_slots(g.Dp);
    auto fn = k_block_tc<I, MAXD>;
    cudaError_t e = cudaFuncSetAttribute((const void *)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    int occ = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, threads, smem);
    // TMEM: 512 columns per SM; each CTA holds the next power of two >= slots * 3 N
    int ncols = 32;
    while (ncols < tc_slots(g.Dp) * 3 * 2 * g.Dp) ncols <<= 1;
    const int tmem_cap = 512 / ncols;
    occ = occ < 1 ? 1 : (occ > tmem_cap ? tmem_cap : occ);
    const uint64_t tiles = (g.R + kTcRows - 1) / kTcRows;
    const uint64_t ctas = (tiles + tc_slots(g.Dp) - 1) / tc_slots(g.Dp);
    const uint64_t cap = (uint64_t)sm_count * occ;
    const int grid = (int)(ctas < cap ? ctas : cap);
    if (grid <= 0) return cudaSuccess;
    fn<<<grid, threads, smem, s>>>(a);
    return cudaGetLastError();
}

template <typename I, int MAXD>
static cudaError_t launch_tc_ws(const GatePlan &g, void *psi, int sm_count, int32_t *err, cudaStream_t s) {
    TcArgs<I> a;
    a.psi = static_cast<float2 *>(psi);
    a.R = (I)g.R;
    if constexpr (sizeof(I) == 4) a.ex = narrow(g.ex);
    else a.ex = g.ex;
    for (int j = 0; j < kMaxBlockD; ++j) a.off[j] = j < g.D ? (I)g.off[j] : 0;
    a.D = g.D;
    a.Dp = g.Dp;
    a.terms = static_cast<const __nv_bfloat16 *>(g.tc_terms);
    a.err = err;
    const int smem = tc_ws_smem_bytes(g.Dp);
    auto fn = k_block_tc_ws<I, MAXD>;
    cudaError_t e = cudaFuncSetAttribute((const void *)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    int occ = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kWsThreads, smem);
    int ncols = 32;
    while (ncols < kWsSlots * 3 * 2 * g.Dp) ncols <<= 1;
    const int tmem_cap = 512 / ncols;
    occ = occ < 1 ? 1 : (occ > tmem_cap ? tmem_cap : occ);
    const uint64_t tiles = (g.R + kTcRows - 1) / kTcRows;
    const uint64_t cap = (uint64_t)sm_count * occ;
    const int grid = (int)(tiles < cap ? tiles : cap);
    if (grid <= 0) return cudaSuccess;
    fn<<<grid, kWsThreads, smem, s>>>(a);
    return cudaGetLastError();
}

template <typename I>
static cudaError_t launch_tc_i(const GatePlan &g, void *psi, int sm_count, int32_t *err, cudaStream_t s) {
    if (g.Dp <= 16) return launch_tc_ws<I, 16>(g, psi, sm_count, err, s);
    if (g.Dp <= 32) return launch_tc_ws<I, 32>(g, psi, sm_count, err, s);
    return launch_tc_im<I, 64>(g, psi, sm_count, err, s);
}

cudaError_t launch_block_tc(const GatePlan &g, void *psi, int sm_count, int32_t *err, cudaStream_t s) {
    if (g.N < (uint64_t(1) << 31)) return launch_tc_i<uint32_t>(g, psi, sm_count, err, s);
    return launch_tc_i<uint64_t>(g, psi, sm_count, err, s);
}

}  // namespace qd
