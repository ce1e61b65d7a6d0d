// Fused-block apply on the fifth-generation tensor cores (tcgen05, sm_100+).
//
// A fused block is a dense D x D complex matrix U over a set of qudits (the
// FP64 product of a run of gates, QuDiet Sec. 2.1.2 / 3.4 gates).  For every
// group of D amplitudes v (the block's local index, as in the per-gate
// kernels), v <- U v.  Stacking 128 groups as the rows of a matrix X
// (128 x 2D reals, interleaved re/im), the update is one real GEMM
//     Y (128 x 2D) = X (128 x 2D) * B^T,   B = [[Ur, -Ui], [Ui, Ur]] interleaved,
// issued as tcgen05.mma kind::f16 (BF16 inputs, FP32 accumulation in TMEM)
// with M = 128 groups, K = 2 Dp and N = 2 Dp in one MMA pass (Dp = D rounded
// up to a multiple of 8, or of 16 above 32).
//
// Precision.  The tensor cores round each accumulation step toward zero; a
// rounded running sum of the whole product loses on average about 0.36 ulp
// per instruction, always toward zero, which shrinks every amplitude
// coherently (measured: 1 - F = 1.5e-6 after one D = 64 block with a hi/lo
// split).  The kernel therefore keeps the leading part of every sum exact
// (the error-free splitting of Ozaki, Ogita, Oishi and Rump, 2012): each
// state row r is scaled by 2^-e_r (e_r from the row maximum) and cut into
// 8-bit fixed-point slices
//     x~ = x1 + x2 + x3 + O(2^-27),  x_s = k / 2^(9s-1),  |k| <= 256,
// and each matrix row n likewise with its own 2^-f_n into B1 + B2 + B3.  Every
// slice value is exact in BF16 and every product x1 B1 is a multiple of
// 2^-16 below 1, so the K = 2 Dp <= 128 products of the leading level sum to
// fewer than 2^24 quanta and its accumulator (x1 B1) never rounds.  The
// correction terms of significance 2^-9 and 2^-18 (x1 B2 + x2 B1 + x1 B3 +
// x2 B2 + x3 B1) share a second accumulator.  That one does round toward zero,
// but its value is itself a small correction whose sign is unrelated to the
// output's, so the truncation is about 2^-32 of the output per instruction in
// no preferred direction: no coherent shrink.  The epilogue adds the two
// accumulators in FP32 with round-to-nearest and rescales by 2^(e_r + f_n).
// The matrix is represented to 2^-27 (coherent error ~1e-8 per block); the
// dropped state terms are incoherent, 2^-27 relative.  Two accumulators (not
// one per significance level) leave room in the 512 TMEM columns for two
// accumulator slots at every D up to 64.

// Shared-memory operands use the no-swizzle K-major canonical layout: core
// matrices of 8 rows x 16 bytes (8 BF16), consecutive along K at 128 B
// (leading byte offset), 8-row groups at K*16 B (stride byte offset).
//
// Warp roles (the steps of a tile overlap across tiles):
//   producers (up to D = 32, 8 warps in two groups alternating tiles, one
//     thread per row; above D = 32, 16 warps in one group of four parts;
//     part p holds amplitudes p RA .. (p + 1) RA - 1 of every row):
//     gather a tile's groups, slice them in registers, then (once its part
//     of the stage is free) store the slices of its K part into stage s of
//     a shared-memory ring and arrive full[s][p];
//   MMA issuer (warp 4, one lane): wait full[s][p] and acc_empty[a], issue
//     the slice products into accumulator slot a of a 2-slot TMEM ring one K
//     part at a time, each part of the stage released by its own commit to
//     empty[s][p], and commit to acc_full[a];
//   epilogue (warps 0..3, one TMEM lane per thread): wait acc_full[a], add the
//     two accumulators, scatter the outputs, arrive acc_empty[a].
// A stage is released by a tcgen05.commit to empty[s] once its MMAs have
// completed, so producers fill the next tile while the epilogue drains the
// previous one; the per-row scales of a tile travel to the epilogue through
// their own 2-deep ring (sc_full / sc_empty), which keeps every barrier at
// most one phase ahead of its waiters.
// Tile i uses accumulator slot i % 2 and stage i % STAGES; mbarrier phases
// count the reuses.  Every wait is bounded and also gives up when another
// warp has raised the abort flag (the device error word is set); the MMA
// warp waits (bounded) for its last commit before TMEM is freed.
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

constexpr int kTcRows = 128;               // groups per tile (MMA M)
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

}  // namespace

// Compile-time shape of the kernel for a bound MAXD on Dp.
// Above Dp = 32 three state slices and the three matrix slices fill the
// 227 KB of shared memory with one stage; the producers then load and slice
// the next tile in registers before they wait for that stage, so only the
// shared-memory stores sit between two tiles' MMAs.  (Two state slices would
// fit two stages, but the dropped 2^-18 residual changes every amplitude by a
// random +-2^-18 of its row maximum per block, visible on small registers.)
template <int MAXD> struct TcCfg {
    static constexpr int XS = 3;      // state slices
    static constexpr int NACC = 2;    // accumulators per slot: exact leading level, corrections
    static constexpr int SLOTS = 2;   // TMEM accumulator ring (2 x 2 x 2 Dp <= 512 columns)
    static constexpr int STAGES = MAXD <= 32 ? 3 : 1;   // shared-memory ring
    static constexpr int PW = MAXD <= 32 ? 8 : 16;      // producer warps
    // threads per tile row (the parts of a row, each holding RA amplitudes
    // and writing its own K part of the stage): one up to D = 32 (two
    // producer groups of 4 warps alternate tiles over three stages; two
    // parts of a row measured slower there), four above (21 warps of at most
    // 96 registers: 0.575 -> 0.727 of the copy peak at D = 64)
    static constexpr int TPR = MAXD <= 32 ? 1 : 4;
    static constexpr int NGRP = PW * 32 / (kTcRows * TPR);  // producer groups (alternate tiles)
    // the row-scale ring's slot is tile & 1: with more than two groups two of
    // them would share a slot and wait on phases two apart (parity aliasing)
    static_assert(NGRP >= 1 && NGRP <= 2, "at most two producer groups");
    static constexpr int RA = MAXD / TPR;                   // amplitudes per producer thread
    static constexpr int THREADS = 32 * (5 + PW);
    static constexpr int NPAIRS = 6;
    static constexpr bool PRE = MAXD <= 32;  // slices built before the stage is free
    // A stage is written in TPR K parts, each by the threads that hold its
    // amplitudes and released by the MMAs of that part alone: while some
    // parts' MMAs run, the other parts of the next tile are sliced and
    // stored (with one stage above D = 32, this is the only overlap).
    // Stage-release barriers: tile i's MMAs commit to empty[i % NE]; the
    // writer of tile i waits for tile i - STAGES on empty[(i - STAGES) % NE].
    // With one stage NE = 2 (one barrier per tile parity): should two
    // producer groups share the stage, a group can then never wait on a
    // barrier two phases behind its target, which a single barrier would
    // alias through its parity.
    static constexpr int NE = STAGES == 1 ? 2 : STAGES;
};

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

// Packed FP32 pairs (Blackwell fma.rn.f32x2: two FMAs, each rounded as fmaf);
// the (re, im) parts of an amplitude travel as one pair.
typedef unsigned long long f2p;
__device__ __forceinline__ f2p pk2(float a, float b) {
    f2p r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ f2p fma2(f2p a, f2p b, f2p c) {
    f2p d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
// BF16x2 word of a pair whose parts have at most 8 significant bits: the
// first part (re) in the low half, the second (im) in the high half.  Such
// a float's low 16 bits are zero, so its BF16 value is its high half
// exactly: one byte permute instead of two conversions.
__device__ __forceinline__ uint32_t bf16x2_of(f2p x) {
    uint32_t lo, hi, w;
    asm("mov.b64 {%0, %1}, %2;" : "=r"(lo), "=r"(hi) : "l"(x));
    asm("prmt.b32 %0, %1, %2, 0x7632;" : "=r"(w) : "r"(lo), "r"(hi));
    return w;
}

// The XS slices of one amplitude v = (re, im), already scaled into [-1, 1],
// as BF16x2 words.  Level l rounds the remaining residual to a multiple of
// q_l = 2^-(9l-1): with M = 1.5 * 2^23, fma(r, 1/q_l, M) - M is r / q_l
// rounded to the nearest integer k (|r / q_l| < 2^22, so the sum's unit is
// 1), the slice is k q_l and the next residual r - k q_l is exact (the two
// are within a factor of two, or k = 0).
template <int XS>
__device__ __forceinline__ void slice_amp(f2p v, uint32_t *w) {
    const float M = 12582912.0f;  // 1.5 * 2^23
    const f2p Mp = pk2(M, M), Mn = pk2(-M, -M), one = pk2(1.f, 1.f), zero = 0ull;
    f2p r = v;
#pragma unroll
    for (int l = 0; l < XS; ++l) {
        const float inv_q = l == 0 ? 256.0f : (l == 1 ? 131072.0f : 67108864.0f);
        const float q = 1.0f / inv_q;  // exact power of two
        const f2p k = fma2(fma2(r, pk2(inv_q, inv_q), Mp), one, Mn);
        const f2p sl = fma2(k, pk2(q, q), zero);
        w[l] = bf16x2_of(sl);
        if (l + 1 < XS) r = fma2(k, pk2(-q, -q), r);
    }
}

template <typename I, int MAXD>
__global__ void __launch_bounds__(TcCfg<MAXD>::THREADS, 1) k_block_tc(const __grid_constant__ TcArgs<I> a) {
    using C = TcCfg<MAXD>;
    extern __shared__ __align__(1024) unsigned char sm[];
    const uint32_t K = 2u * (uint32_t)a.Dp;
    const uint32_t Nc = K;  // output columns: N = 2 Dp reals
    const uint32_t xbytes = kTcRows * K * 2u;
    const uint32_t bbytes = K * K * 2u;
    unsigned char *B = sm;
    const float *bscale = reinterpret_cast<const float *>(B + 3u * bbytes);
    const uint32_t bregion = (3u * bbytes + K * 4u + 1023u) & ~1023u;
    unsigned char *stages = sm + bregion;  // stage s: X1 | X2 | X3 at s * XS * xbytes
    // full / empty: one barrier per stage and K part
    __shared__ __align__(8) uint64_t full[C::STAGES * C::TPR], empty[C::NE * C::TPR], acc_full[C::SLOTS],
        acc_empty[C::SLOTS];
    // the parts of a row exchange their maxima through
    // shared memory (a 2-deep ring, one barrier per slot)
    // (a 2-deep ring per producer group: slot 2 grp + (local tile & 1))
    __shared__ __align__(8) uint64_t xm_full[2 * C::NGRP];
    __shared__ float xmax[2 * C::NGRP][C::TPR][kTcRows];
    // row scales of a tile: a 2-deep ring between producers and epilogue
    __shared__ __align__(8) uint64_t sc_full[2], sc_empty[2];
    __shared__ int32_t erow[2][kTcRows];
    __shared__ uint32_t tmem_base;
    __shared__ volatile int32_t abort_flag;

    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    uint32_t ncols = 32;
    while (ncols < (uint32_t)(C::SLOTS * C::NACC) * Nc) ncols <<= 1;

    {
        const uint4 *src = reinterpret_cast<const uint4 *>(a.terms);
        uint4 *dst = reinterpret_cast<uint4 *>(B);
        const uint32_t n16 = (3u * bbytes + K * 4u + 15u) / 16u;
        for (uint32_t i = tid; i < n16; i += blockDim.x) dst[i] = src[i];
    }
    if (tid == 0) {
        for (int q = 0; q < C::STAGES * C::TPR; ++q)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(&full[q])), "r"(kTcRows)
                         : "memory");
        // a stage (half) is free once the MMAs reading it have completed (tcgen05.commit)
        for (int q = 0; q < C::NE * C::TPR; ++q)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&empty[q])) : "memory");
        for (int q = 0; q < 2 * C::NGRP; ++q)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(&xm_full[q])), "r"(C::TPR * kTcRows)
                         : "memory");
        for (int q = 0; q < C::SLOTS; ++q) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&acc_full[q])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(&acc_empty[q])), "r"(kTcRows)
                         : "memory");
        }
        for (int q = 0; q < 2; ++q) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(&sc_full[q])), "r"(kTcRows)
                         : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(&sc_empty[q])), "r"(kTcRows)
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
        constexpr int NGRP = C::NGRP;
        const int p = tid - 160;
        const int grp = p / (kTcRows * C::TPR);
        const int q = p % (kTcRows * C::TPR);
        // this thread's amplitudes: [part RA, (part + 1) RA) of its row; the
        // two parts of the rows are in different warps
        const int row = q % kTcRows, part = q / kTcRows;
        const int j0 = part * C::RA;
        for (I i = (I)grp; i < nlocal; i += NGRP) {
            const int st = (int)(i % C::STAGES);
            const I t = (I)blockIdx.x + i * (I)gridDim.x;
            const I g = t * kTcRows + row;
            const bool valid = g < a.R;
            const I base = valid ? expand(g, a.ex) : 0;
            float2 v[C::RA];
#pragma unroll
            for (int j = 0; j < C::RA; ++j)
                v[j] = (valid && j0 + j < a.D) ? a.psi[base + a.off[j0 + j]] : make_float2(0.f, 0.f);
            if constexpr (!C::PRE) {
                // above D = 32 one producer group serves every tile, so its loads
                // wait out the full memory latency: the same amplitudes of its
                // next tile go into L2 now and the next loads wait for L2 only
                const I gn = g + (I)NGRP * (I)gridDim.x * (I)kTcRows;
                if (i + NGRP < nlocal && gn < a.R) {
                    const I bn = expand(gn, a.ex);
#pragma unroll
                    for (int j = 0; j < C::RA; ++j)
                        if (j0 + j < a.D) asm volatile("prefetch.global.L2 [%0];" ::"l"(a.psi + bn + a.off[j0 + j]));
                }
            }
            float amax = 0.f;
#pragma unroll
            for (int j = 0; j < C::RA; ++j) amax = fmaxf(amax, fmaxf(fabsf(v[j].x), fabsf(v[j].y)));
            if constexpr (C::TPR > 1) {
                // the group's local tile li: slot 2 grp + (li & 1), phase li >> 1.
                // A slot is rewritten two of the group's tiles later, after every
                // thread of the group has passed the exchange in between (and so
                // has read this one)
                const I li = i / (I)NGRP;
                const int xs = 2 * grp + (int)(li & 1);
                xmax[xs][part][row] = amax;
                mbar_arrive(smem_u32(&xm_full[xs]));
                bool okx = ws_wait(smem_u32(&xm_full[xs]), (uint32_t)(li >> 1) & 1u, &abort_flag, a.err);
                okx = __all_sync(0xffffffffu, okx);
                if (!okx) break;
                amax = xmax[xs][0][row];
#pragma unroll
                for (int pp = 1; pp < C::TPR; ++pp) amax = fmaxf(amax, xmax[xs][pp][row]);
            }
            int e = 0;
            frexpf(amax, &e);  // amax <= 2^e
            const f2p inv2 = pk2(ldexpf(1.0f, -e), ldexpf(1.0f, -e));
            // up to D = 32 the slices are built in registers before the stage is
            // free (word [s][j]: slice s of amplitude j0 + j); above, where one
            // thread holds 32 amplitudes and the registers would not hold both,
            // they are built chunk by chunk as they are stored
            uint32_t w[C::PRE ? C::XS : 1][C::PRE ? C::RA : 1];
            if constexpr (C::PRE) {
#pragma unroll
                for (int j = 0; j < C::RA; ++j) {
                    uint32_t ws[3];
                    slice_amp<C::XS>(fma2(pk2(v[j].x, v[j].y), inv2, 0ull), ws);
#pragma unroll
                    for (int s2 = 0; s2 < C::XS; ++s2) w[s2][j] = ws[s2];
                }
            }
            // row scale into the ring slot of this tile (the epilogue has read
            // the scale of tile i - 2 from it)
            {
                const int es = (int)(i & 1);
                const uint32_t euse = (uint32_t)(i >> 1);
                // with several threads per row the warp leaves the loop together
                // (every lane takes the same exits): every lane reaches the vote
                bool ok = euse < 1 || ws_wait(smem_u32(&sc_empty[es]), (euse - 1) & 1u, &abort_flag, a.err);
                if constexpr (C::TPR > 1) ok = __all_sync(0xffffffffu, ok);
                if (!ok) break;
                if (part == 0) {
                    erow[es][row] = e;
                    mbar_arrive(smem_u32(&sc_full[es]));
                }
            }
            bool ok = true;
            if (i >= (I)C::STAGES) {
                const I wt = i - (I)C::STAGES;  // the tile whose MMAs last read this stage (half)
                ok = ws_wait(smem_u32(&empty[(int)(wt % C::NE) * C::TPR + part]), (uint32_t)(wt / C::NE) & 1u,
                             &abort_flag, a.err);
            }
            if constexpr (C::TPR > 1) ok = __all_sync(0xffffffffu, ok);
            if (!ok) break;
            unsigned char *X = stages + (uint32_t)st * C::XS * xbytes;
#pragma unroll
            for (int c0 = 0; c0 < C::RA; c0 += 4) {  // 4 amplitudes = 8 BF16 = one 16-byte chunk per slice
                if (j0 + c0 < a.Dp) {
                    const uint32_t o = cm_off((uint32_t)row, (uint32_t)(2 * (j0 + c0)), K);
                    uint32_t q[C::XS][4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        if constexpr (C::PRE) {
#pragma unroll
                            for (int s2 = 0; s2 < C::XS; ++s2) q[s2][u] = w[s2][c0 + u];
                        } else {
                            uint32_t ws[3];
                            slice_amp<C::XS>(fma2(pk2(v[c0 + u].x, v[c0 + u].y), inv2, 0ull), ws);
#pragma unroll
                            for (int s2 = 0; s2 < C::XS; ++s2) q[s2][u] = ws[s2];
                        }
                    }
#pragma unroll
                    for (int s2 = 0; s2 < C::XS; ++s2)
                        *reinterpret_cast<uint4 *>(X + (uint32_t)s2 * xbytes + o) =
                            make_uint4(q[s2][0], q[s2][1], q[s2][2], q[s2][3]);
                }
            }
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            mbar_arrive(smem_u32(&full[st * C::TPR + part]));
        }
    } else if (warp == 4) {
        // ------------------------------------------------------------ MMA issuer
        if ((tid & 31) == 0) {
            const uint32_t idesc = idesc_bf16(kTcRows, Nc);
            const uint32_t lbo = 128u, sbo = K * 16u;
            const uint32_t b0 = smem_u32(B);
            // (accumulator, x slice, B slice): the exact leading level x1 B1, then
            // every correction pair into the second accumulator; the first pair of
            // each accumulator starts it
            const int pairs[6][3] = {{0, 0, 0}, {1, 0, 1}, {1, 1, 0}, {1, 0, 2}, {1, 1, 1}, {1, 2, 0}};
            const uint32_t ksteps = K / 16u;
            // K steps of the first half: the columns of part 0's amplitudes
            // K steps of each part's columns (2 RA of them): part h writes and
            // releases K steps [h kpart, (h + 1) kpart) of the stage
            const uint32_t kpart = (uint32_t)(2 * C::RA / 16);
            // the most recent commit: once it has arrived, every MMA issued
            // before it has completed
            uint32_t last_mb = 0, last_par = 0;
            bool any = false;
            bool good = true;
            for (I i = 0; i < nlocal && good; ++i) {
                const int st = (int)(i % C::STAGES);
                const uint32_t fpar = (uint32_t)(i / C::STAGES) & 1u;
                if (!ws_wait(smem_u32(&full[st * C::TPR]), fpar, &abort_flag, a.err)) break;
                const int sl = (int)(i % C::SLOTS);
                if (i >= (I)C::SLOTS &&
                    !ws_wait(smem_u32(&acc_empty[sl]), (uint32_t)(i / C::SLOTS - 1) & 1u, &abort_flag, a.err))
                    break;
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                const uint32_t x0 = smem_u32(stages + (uint32_t)st * C::XS * xbytes);
                const uint32_t acc = tmem + (uint32_t)sl * (uint32_t)C::NACC * Nc;
                // the pair table is unrolled into constants; a K step moves both
                // operands by 256 bytes, i.e. 16 in the descriptors' address field
                // (shared addresses stay below 2^18, so the field does not overflow)
#pragma unroll
                for (int h = 0; h < C::TPR; ++h) {
                    const uint32_t k_lo = std::min<uint32_t>((uint32_t)h * kpart, ksteps);
                    const uint32_t k_hi = h + 1 == C::TPR ? ksteps : std::min<uint32_t>((uint32_t)(h + 1) * kpart, ksteps);
                    if (h > 0) {
                        // the next part of the stage, written by its own producer warps
                        if (!ws_wait(smem_u32(&full[st * C::TPR + h]), fpar, &abort_flag, a.err)) {
                            good = false;
                            break;
                        }
                        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                    }
#pragma unroll
                    for (int pp = 0; pp < C::NPAIRS; ++pp) {
                        const uint32_t dcol = acc + (uint32_t)pairs[pp][0] * Nc;
                        const uint32_t xa = x0 + (uint32_t)pairs[pp][1] * xbytes;
                        const uint32_t bt = b0 + (uint32_t)pairs[pp][2] * bbytes;
                        const bool first_of_acc = h == 0 && (pp == 0 || pp == 1);
                        const uint64_t da = smem_desc(xa, lbo, sbo), db = smem_desc(bt, lbo, sbo);
#pragma unroll 1
                        for (uint32_t ks = k_lo; ks < k_hi; ++ks)
                            mma_bf16(dcol, da + (uint64_t)(ks * 16u), db + (uint64_t)(ks * 16u), idesc,
                                     (first_of_acc && ks == 0) ? 0u : 1u);
                    }
                    if (h + 1 == C::TPR) mma_commit(smem_u32(&acc_full[sl]));
                    // this stage (half) is free once its MMAs complete
                    last_mb = smem_u32(&empty[(int)(i % C::NE) * C::TPR + h]);
                    last_par = (uint32_t)(i / C::NE) & 1u;
                    any = true;
                    mma_commit(last_mb);
                }
            }
            // before TMEM and the CTA's shared memory are released: the last commit
            // must have arrived
            if (any)
                for (uint32_t it = 0; it < kWaitLimit; ++it)
                    if (mbar_try(last_mb, last_par)) break;
        }
    } else {
        // ------------------------------------------------------------ epilogue
        const int row = tid;  // TMEM lane of this thread (warps 0..3)
        for (I i = 0; i < nlocal; ++i) {
            // the producers' row scale of this tile
            const int es = (int)(i & 1);
            if (!ws_wait(smem_u32(&sc_full[es]), (uint32_t)(i >> 1) & 1u, &abort_flag, a.err)) break;
            const int e = erow[es][row];
            mbar_arrive(smem_u32(&sc_empty[es]));
            const float escale = ldexpf(1.0f, e);
            const I t = (I)blockIdx.x + i * (I)gridDim.x;
            const I g = t * kTcRows + row;
            const bool valid = g < a.R;
            const I base = valid ? expand(g, a.ex) : 0;
            const int sl = (int)(i % C::SLOTS);
            if (!ws_wait(smem_u32(&acc_full[sl]), (uint32_t)(i / C::SLOTS) & 1u, &abort_flag, a.err)) break;
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            const uint32_t lane_addr = tmem + (uint32_t)sl * (uint32_t)C::NACC * Nc + ((uint32_t)(warp * 32) << 16);
            // 16 amplitudes (32 columns of each accumulator) per TMEM wait: the
            // four loads are in flight together
#pragma unroll
            for (int c0 = 0; c0 < MAXD; c0 += 16) {
                if (c0 < a.Dp) {
                    uint32_t l0[2][16], l1[2][16];
                    tmem_ld16_nowait(lane_addr + (uint32_t)(2 * c0), l0[0]);
                    tmem_ld16_nowait(lane_addr + Nc + (uint32_t)(2 * c0), l1[0]);
                    const bool second = c0 + 8 < a.Dp;
                    if (second) {
                        tmem_ld16_nowait(lane_addr + (uint32_t)(2 * (c0 + 8)), l0[1]);
                        tmem_ld16_nowait(lane_addr + Nc + (uint32_t)(2 * (c0 + 8)), l1[1]);
                    }
                    tmem_wait_ld();
                    if (valid) {
#pragma unroll
                        for (int hh = 0; hh < 2; ++hh) {
#pragma unroll
                            for (int u2 = 0; u2 < 4; ++u2) {
                                if (c0 + 8 * hh + 2 * u2 >= a.D) break;
                                // the column scales of two amplitudes (16-byte aligned, inside
                                // the 2 Dp scales: Dp is even)
                                const float4 bs = *reinterpret_cast<const float4 *>(bscale + 2 * (c0 + 8 * hh + 2 * u2));
#pragma unroll
                                for (int w2 = 0; w2 < 2; ++w2) {
                                    const int uu = 2 * u2 + w2;
                                    const int j = c0 + 8 * hh + uu;
                                    if (j < a.D) {
                                        const float sr = w2 == 0 ? bs.x : bs.z, si = w2 == 0 ? bs.y : bs.w;
                                        const float re =
                                            (__uint_as_float(l0[hh][2 * uu]) + __uint_as_float(l1[hh][2 * uu])) *
                                            (escale * sr);
                                        const float im = (__uint_as_float(l0[hh][2 * uu + 1]) +
                                                          __uint_as_float(l1[hh][2 * uu + 1])) *
                                                         (escale * si);
                                        a.psi[base + a.off[j]] = make_float2(re, im);
                                    }
                                }
                            }
                        }
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
            mbar_arrive(smem_u32(&acc_empty[sl]));
        }
    }
    __syncthreads();
    if (warp == 4)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(ncols) : "memory");
}

int tc_padded_dim(int D) { return D <= 32 ? (D + 7) / 8 * 8 : (D + 15) / 16 * 16; }

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

template <int MAXD>
static int smem_bytes_for(int Dp) {
    using C = TcCfg<MAXD>;
    const int K = 2 * Dp;
    const int bregion = (3 * K * K * 2 + K * 4 + 1023) & ~1023;
    return bregion + C::STAGES * C::XS * kTcRows * K * 2;
}

int tc_smem_bytes(int Dp) {
    if (Dp <= 16) return smem_bytes_for<16>(Dp);
    if (Dp <= 32) return smem_bytes_for<32>(Dp);
    return smem_bytes_for<64>(Dp);
}

template <typename I, int MAXD>
static cudaError_t launch_tc_im(const GatePlan &g, void *psi, int sm_count, int32_t *err, cudaStream_t s) {
    using C = TcCfg<MAXD>;
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
    const int smem = smem_bytes_for<MAXD>(g.Dp);
    auto fn = k_block_tc<I, MAXD>;
    cudaError_t e = cudaFuncSetAttribute((const void *)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    int occ = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, C::THREADS, smem);
    // TMEM: 512 columns per SM; each CTA holds the next power of two >= slots * accumulators * N
    int ncols = 32;
    while (ncols < C::SLOTS * C::NACC * 2 * g.Dp) ncols <<= 1;
    const int tmem_cap = 512 / ncols;
    occ = occ < 1 ? 1 : (occ > tmem_cap ? tmem_cap : occ);
    const uint64_t tiles = (g.R + kTcRows - 1) / kTcRows;
    const uint64_t cap = (uint64_t)sm_count * occ;
    const int grid = (int)(tiles < cap ? tiles : cap);
    if (grid <= 0) return cudaSuccess;
    fn<<<grid, C::THREADS, smem, s>>>(a);
    return cudaGetLastError();
}

template <typename I>
static cudaError_t launch_tc_i(const GatePlan &g, void *psi, int sm_count, int32_t *err, cudaStream_t s) {
    if (g.Dp <= 16) return launch_tc_im<I, 16>(g, psi, sm_count, err, s);
    if (g.Dp <= 32) return launch_tc_im<I, 32>(g, psi, sm_count, err, s);
    return launch_tc_im<I, 64>(g, psi, sm_count, err, s);
}

cudaError_t launch_block_tc(const GatePlan &g, void *psi, int sm_count, int32_t *err, cudaStream_t s) {
    if (!wide_index(g)) return launch_tc_i<uint32_t>(g, psi, sm_count, err, s);
    return launch_tc_i<uint64_t>(g, psi, sm_count, err, s);
}

}  // namespace qd
