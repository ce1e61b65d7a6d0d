// Diagonal runs: a run of consecutive diagonal gates (phase gates Z_d,
// controlled phases such as those of a d-ary QFT, diagonal user gates;
// QuDiet Sec. 2.1.2 and 3.4), on any number of qudits, applied in one pass.
// Diagonal gates commute, so their product is one diagonal; it depends only
// on the digits of the qudits the run touches.  Over the contiguous qudit
// range [qa, qb] that covers them, the product is a table T of
// TS = s_{qb+1} / s_qa entries, and amplitude i is multiplied by
// T[(i / s_qa) mod TS].  The table is built on the device in FP64 from the
// gates' own diagonals, then kept as FP32 hi + lo pairs (complex64 states,
// the same coefficient precision as the per-gate kernels) or FP64.
#include <cstdint>
#include <cuda_runtime.h>

#include "qd_diag.h"

namespace qd {

namespace {

constexpr int kDiagBlock = 256;

// T[k] for k in [0, TS): the FP64 product of every gate's diagonal entry at
// the digits of k (qudit qa + m has digit (k / w_m) mod d_m, w_m = prod_{p<m} d_p).
template <typename Out>
__global__ void k_diag_build(Out *__restrict__ tab, uint64_t TS, DiagRange rg, const DiagGateDesc *__restrict__ gates,
                             int32_t ngates, const double2 *__restrict__ pool) {
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < TS;
         k += (uint64_t)gridDim.x * blockDim.x) {
        int32_t dig[kDiagMaxRange];
        uint64_t r = k;
        for (int m = 0; m < rg.nr; ++m) {
            dig[m] = (int32_t)(r % (uint64_t)rg.d[m]);
            r /= (uint64_t)rg.d[m];
        }
        double re = 1.0, im = 0.0;
        for (int g = 0; g < ngates; ++g) {
            const DiagGateDesc &dg = gates[g];
            int32_t loc = 0;
            for (int m = 0; m < dg.nq; ++m) loc = loc * rg.d[dg.q[m]] + dig[dg.q[m]];
            const double2 u = pool[dg.off + loc];
            const double nr = re * u.x - im * u.y, ni = re * u.y + im * u.x;
            re = nr;
            im = ni;
        }
        if constexpr (sizeof(Out) == 16 && sizeof(((Out *)0)->x) == 4) {
            // complex64: hi + lo pair of each part
            const float hr = (float)re, hi_ = (float)im;
            tab[k] = Out{hr, hi_, (float)(re - (double)hr), (float)(im - (double)hi_)};
        } else {
            tab[k] = Out{re, im};
        }
    }
}

template <typename I> struct DivOf;
template <> struct DivOf<uint32_t> { using type = FastDiv32; };
template <> struct DivOf<uint64_t> { using type = FastDiv64; };

// psi[i] *= T[(i / s_qa) mod TS]; a warp takes a chunk of 128 consecutive
// amplitudes per iteration, lane l the amplitudes l, l + 32, l + 64, l + 96
// of it (every access coalesced, four loads issued first).  complex64:
// (lo * v) + hi * v, lo first.
template <typename I>
__device__ __forceinline__ I diag_chunk0() {
    return ((I)blockIdx.x * blockDim.x + (threadIdx.x & ~31u)) * 4 + (threadIdx.x & 31u);
}

template <typename I>
__global__ void __launch_bounds__(kDiagBlock) k_diag_apply_f32(float2 *__restrict__ psi, I N,
                                                               typename DivOf<I>::type divA,
                                                               typename DivOf<I>::type divT,
                                                               const float4 *__restrict__ tab) {
    const I step = (I)gridDim.x * blockDim.x * 4;
    for (I i0 = diag_chunk0<I>(); i0 < N; i0 += step) {
        float2 v[4];
        float4 t[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const I i = i0 + 32 * u;
            if (i < N) {
                v[u] = psi[i];
                const I q = fdiv(i, divA);
                const I k = q - fdiv(q, divT) * (I)divT.d;
                t[u] = __ldg(&tab[k]);
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const I i = i0 + 32 * u;
            if (i < N) {
                float re = fmaf(t[u].z, v[u].x, -t[u].w * v[u].y);
                float im = fmaf(t[u].z, v[u].y, t[u].w * v[u].x);
                re = fmaf(t[u].x, v[u].x, fmaf(-t[u].y, v[u].y, re));
                im = fmaf(t[u].x, v[u].y, fmaf(t[u].y, v[u].x, im));
                psi[i] = make_float2(re, im);
            }
        }
    }
}

template <typename I>
__global__ void __launch_bounds__(kDiagBlock) k_diag_apply_f64(double2 *__restrict__ psi, I N,
                                                               typename DivOf<I>::type divA,
                                                               typename DivOf<I>::type divT,
                                                               const double2 *__restrict__ tab) {
    const I step = (I)gridDim.x * blockDim.x * 4;
    for (I i0 = diag_chunk0<I>(); i0 < N; i0 += step) {
        double2 v[4], t[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const I i = i0 + 32 * u;
            if (i < N) {
                v[u] = psi[i];
                const I q = fdiv(i, divA);
                const I k = q - fdiv(q, divT) * (I)divT.d;
                t[u] = __ldg(&tab[k]);
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const I i = i0 + 32 * u;
            if (i < N) psi[i] = make_double2(fma(t[u].x, v[u].x, -t[u].y * v[u].y), fma(t[u].x, v[u].y, t[u].y * v[u].x));
        }
    }
}

int grid_for(uint64_t work, int per_thread, int sm_count) {
    const uint64_t need = (work + (uint64_t)kDiagBlock * per_thread - 1) / ((uint64_t)kDiagBlock * per_thread);
    const uint64_t cap = (uint64_t)sm_count * 8;
    return (int)(need < cap ? need : cap);
}

}  // namespace

cudaError_t diag_table_build(void *tab, int prec, uint64_t TS, const DiagRange &rg, const DiagGateDesc *gates_dev,
                             int32_t ngates, const double2 *pool_dev, int sm_count, cudaStream_t s) {
    const int grid = grid_for(TS, 1, sm_count);
    if (grid <= 0) return cudaSuccess;
    if (prec == 1)
        k_diag_build<float4><<<grid, kDiagBlock, 0, s>>>(static_cast<float4 *>(tab), TS, rg, gates_dev, ngates,
                                                         pool_dev);
    else
        k_diag_build<double2><<<grid, kDiagBlock, 0, s>>>(static_cast<double2 *>(tab), TS, rg, gates_dev, ngates,
                                                          pool_dev);
    return cudaGetLastError();
}

cudaError_t diag_table_apply(void *psi, int prec, uint64_t N, uint64_t s_qa, uint64_t TS, const void *tab,
                             int sm_count, cudaStream_t s, bool wide) {
    const int grid = grid_for(N, 4, sm_count);
    if (grid <= 0) return cudaSuccess;
    if (N < (uint64_t(1) << 31) && !wide) {
        const FastDiv32 a = make_fastdiv32((uint32_t)s_qa), t = make_fastdiv32((uint32_t)TS);
        if (prec == 1)
            k_diag_apply_f32<uint32_t><<<grid, kDiagBlock, 0, s>>>(static_cast<float2 *>(psi), (uint32_t)N, a, t,
                                                                   static_cast<const float4 *>(tab));
        else
            k_diag_apply_f64<uint32_t><<<grid, kDiagBlock, 0, s>>>(static_cast<double2 *>(psi), (uint32_t)N, a, t,
                                                                   static_cast<const double2 *>(tab));
    } else {
        const FastDiv64 a = make_fastdiv64(s_qa), t = make_fastdiv64(TS);
        if (prec == 1)
            k_diag_apply_f32<uint64_t><<<grid, kDiagBlock, 0, s>>>(static_cast<float2 *>(psi), N, a, t,
                                                                   static_cast<const float4 *>(tab));
        else
            k_diag_apply_f64<uint64_t><<<grid, kDiagBlock, 0, s>>>(static_cast<double2 *>(psi), N, a, t,
                                                                   static_cast<const double2 *>(tab));
    }
    return cudaGetLastError();
}

}  // namespace qd
