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
// Precision (complex64 states, FP32 storage): BF16 keeps 8 mantissa bits, so
// both operands are split into unevaluated sums of BF16 terms: the state
// x = x1 + x2 (|x - x1 - x2| <= 2^-18 |x|, incoherent per amplitude) and the
// matrix B = B1 + B2 + B3 (|B - B1 - B2 - B3| <= 2^-27 |B|).  Four products
// are accumulated: B1 x1 + B2 x1 + B3 x1 + B1 x2.  The matrix applied to the
// dominant part x1 is accurate to 2^-27, so the coherent (same for every
// group) non-unitarity that would make the norm drift over a circuit stays
// ~1e-8 per block; the dropped terms are below 2^-17 of each amplitude and
// incoherent.  This is the split-operand idea of Markidis et al. (2018) and
// Ootomo & Yokota (2022) applied with BF16 terms.
//
// Shared-memory operands use the no-swizzle K-major canonical layout: core
// matrices of 8 rows x 16 bytes (8 BF16), consecutive along K at 128 B
// (leading byte offset), 8-row groups at K*16 B (stride byte offset).
// One CTA of 128 threads owns a tile of 128 groups per iteration: thread t
// gathers group t, splits it to BF16 and writes row t of X1, X2; one thread
// issues the MMAs and commits them to an mbarrier; after the (bounded) wait,
// thread t reads TMEM lane t (its group's 2D outputs) and scatters them back.
// Every wait is bounded; on expiry the kernel records an error, waits (bounded)
// for its MMAs, frees its TMEM and returns.
#include <cstdint>
#include <cstring>
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

// Kernel arguments: direct-mode group geometry plus the three BF16 matrix
// terms, already in the K-major canonical layout (B1 | B2 | B3, each
// N x K BF16 = 2*N*K bytes), in global memory.
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

template <typename I>
__global__ void __launch_bounds__(kTcThreads, 1) k_block_tc(const __grid_constant__ TcArgs<I> a) {
    extern __shared__ __align__(1024) unsigned char sm[];
    const uint32_t K = 2u * (uint32_t)a.Dp;  // = N
    const uint32_t xbytes = kTcRows * K * 2u;  // one state tile (BF16)
    const uint32_t bbytes = K * K * 2u;        // one matrix term
    unsigned char *X1 = sm;
    unsigned char *X2 = X1 + xbytes;
    unsigned char *B = X2 + xbytes;  // B1 | B2 | B3
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    __shared__ int32_t abort_flag;

    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    uint32_t ncols = 32;
    while (ncols < K) ncols <<= 1;

    // matrix terms: global -> shared (16-byte copies)
    {
        const uint4 *src = reinterpret_cast<const uint4 *>(a.terms);
        uint4 *dst = reinterpret_cast<uint4 *>(B);
        for (uint32_t i = tid; i < 3u * bbytes / 16u; i += kTcThreads) dst[i] = src[i];
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&mbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        abort_flag = 0;
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
    const uint32_t tmem = tmem_base;
    const uint32_t idesc = idesc_bf16(kTcRows, K);
    const uint32_t lbo = 128u, sbo = K * 16u;
    const uint32_t mb = smem_u32(&mbar);

    uint32_t phase = 0;
    const I ntiles = (a.R + kTcRows - 1) / kTcRows;
    for (I tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        // ---- gather group tid, split to BF16 hi/lo, write rows of X1, X2
        const I g = tile * kTcRows + tid;
        const bool valid = g < a.R;
        const I base = valid ? expand(g, a.ex) : 0;
        for (int c0 = 0; c0 < a.Dp; c0 += 4) {  // 4 amplitudes = 8 BF16 = one 16-byte chunk
            __align__(16) __nv_bfloat16 h[8], l[8];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int j = c0 + u;
                float2 v = make_float2(0.f, 0.f);
                if (valid && j < a.D) v = a.psi[base + a.off[j]];
                const __nv_bfloat16 hr = __float2bfloat16_rn(v.x), hi = __float2bfloat16_rn(v.y);
                h[2 * u] = hr;
                h[2 * u + 1] = hi;
                l[2 * u] = __float2bfloat16_rn(v.x - __bfloat162float(hr));
                l[2 * u + 1] = __float2bfloat16_rn(v.y - __bfloat162float(hi));
            }
            const uint32_t o = cm_off((uint32_t)tid, (uint32_t)(2 * c0), K);
            *reinterpret_cast<uint4 *>(X1 + o) = *reinterpret_cast<const uint4 *>(h);
            *reinterpret_cast<uint4 *>(X2 + o) = *reinterpret_cast<const uint4 *>(l);
        }
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        __syncthreads();
        // ---- one thread issues B1 x1 + B2 x1 + B3 x1 + B1 x2
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            const uint32_t x1 = smem_u32(X1), x2 = smem_u32(X2), b0 = smem_u32(B);
            uint32_t acc = 0;
            const uint32_t ksteps = K / 16u;
#pragma unroll 1
            for (int term = 0; term < 4; ++term) {
                const uint32_t xa = term < 3 ? x1 : x2;
                const uint32_t bt = b0 + (uint32_t)(term < 3 ? term : 0) * bbytes;
#pragma unroll 1
                for (uint32_t s = 0; s < ksteps; ++s) {
                    const uint64_t ad = smem_desc(xa + s * 256u, lbo, sbo);
                    const uint64_t bd = smem_desc(bt + s * 256u, lbo, sbo);
                    mma_bf16(tmem, ad, bd, idesc, acc);
                    acc = 1;
                }
            }
            mma_commit(mb);
        }
        // ---- wait for the MMAs (bounded)
        const bool ok = mbar_wait_bounded(mb, phase);
        phase ^= 1u;
        if (!ok) {
            atomicExch(a.err, 1);
            abort_flag = 1;
        }
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        __syncthreads();
        if (abort_flag) {
            // one more bounded wait for the MMAs in flight, then release TMEM
            mbar_wait_bounded(mb, phase ^ 1u);
            break;
        }
        // ---- TMEM lane tid -> this group's 2D outputs -> scatter back
        const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
        for (int c0 = 0; c0 < a.Dp; c0 += 4) {
            float o[8];
            tmem_ld<8>(lane_addr + (uint32_t)(2 * c0), o);
            if (valid) {
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int j = c0 + u;
                    if (j < a.D) a.psi[base + a.off[j]] = make_float2(o[2 * u], o[2 * u + 1]);
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        __syncthreads();
    }
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(ncols) : "memory");
}

size_t tc_terms_bytes(int Dp) { return (size_t)3 * (2 * Dp) * (2 * Dp) * 2; }

// Host: the real embedding B (N x K, N = K = 2 Dp) of the D x D complex
// matrix U, split into three BF16 terms in the K-major canonical layout.
void tc_pack_terms(const double *U, int D, int Dp, uint16_t *out) {
    const int K = 2 * Dp;
    const size_t term_elems = (size_t)K * K;
    for (size_t i = 0; i < 3 * term_elems; ++i) out[i] = 0;
    auto bf16_bits = [](double x) -> uint16_t {
        // round-to-nearest-even of the FP32 value, as __float2bfloat16_rn
        const float f = (float)x;
        uint32_t u;
        std::memcpy(&u, &f, 4);
        if ((u & 0x7fffffffu) > 0x7f800000u) return 0x7fc0;
        const uint32_t lsb = (u >> 16) & 1u;
        u += 0x7fffu + lsb;
        return (uint16_t)(u >> 16);
    };
    auto bf16_val = [](uint16_t b) -> double {
        uint32_t u = (uint32_t)b << 16;
        float f;
        std::memcpy(&f, &u, 4);
        return (double)f;
    };
    for (int i = 0; i < D; ++i)
        for (int k = 0; k < D; ++k) {
            const double ur = U[2 * (i * D + k)], ui = U[2 * (i * D + k) + 1];
            // rows n = 2i (re), 2i+1 (im); columns 2k (x_re), 2k+1 (x_im)
            const double e[2][2] = {{ur, -ui}, {ui, ur}};
            for (int p = 0; p < 2; ++p)
                for (int q = 0; q < 2; ++q) {
                    double rem = e[p][q];
                    const uint32_t n = 2 * i + p, kk = 2 * k + q;
                    const uint32_t off = cm_off(n, kk, (uint32_t)K) / 2;
                    for (int t = 0; t < 3; ++t) {
                        const uint16_t b = bf16_bits(rem);
                        out[t * term_elems + off] = b;
                        rem -= bf16_val(b);
                    }
                }
        }
}

int tc_smem_bytes(int Dp) {
    const int K = 2 * Dp;
    return kTcRows * K * 2 * 2 + 3 * K * K * 2;
}

template <typename I>
static cudaError_t launch_tc_i(const GatePlan &g, void *psi, int sm_count, int32_t *err, cudaStream_t s) {
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
    auto fn = k_block_tc<I>;
    cudaError_t e = cudaFuncSetAttribute((const void *)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    int occ = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kTcThreads, smem);
    // TMEM: 512 columns per SM; each CTA holds at most 128
    occ = occ < 1 ? 1 : (occ > 4 ? 4 : occ);
    const uint64_t tiles = (g.R + kTcRows - 1) / kTcRows;
    const uint64_t cap = (uint64_t)sm_count * occ;
    const int grid = (int)(tiles < cap ? tiles : cap);
    if (grid <= 0) return cudaSuccess;
    fn<<<grid, kTcThreads, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_block_tc(const GatePlan &g, void *psi, int sm_count, int32_t *err, cudaStream_t s) {
    if (g.N < (uint64_t(1) << 31)) return launch_tc_i<uint32_t>(g, psi, sm_count, err, s);
    return launch_tc_i<uint64_t>(g, psi, sm_count, err, s);
}

}  // namespace qd
