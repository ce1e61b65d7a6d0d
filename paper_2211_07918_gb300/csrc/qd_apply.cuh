// Per-gate in-place apply kernels (QuDiet Sec. 2.1.2 gates, Sec. 3.4 user
// gates), instantiated for FP32 (complex64) and FP64 (complex128) states.
//
// A gate with targets T (D = prod d_t local states) and controls C at levels
// l_c maps, for every group r over the remaining qudits, the D amplitudes
//   v_j = psi[base(r) + off_j],   base(r) = insert_digits(r) + sum_c l_c s_c,
// to U v (dense) or to out_i = lam_i v_src(i) (diagonal / permutation with
// phases: "mono").  Amplitudes outside the selected control slice are never
// touched.
//
// Two memory schemes:
//   direct  one thread per group, loads straight from HBM.  Used when every
//           target and control has a flat stride >= 32, so that a warp's 32
//           consecutive groups read 32 consecutive amplitudes per member.
//   tile    a CTA stages DH chunks of B contiguous amplitudes (B = s_m covers
//           all low-stride targets and controls) in shared memory with
//           coalesced loads, applies the gate to the groups inside the tile,
//           and writes the chunks back.
#pragma once
#include <algorithm>

#include "qd_plan.h"

namespace qd {

template <typename T>
__device__ __forceinline__ void cmac(v2<T> &acc, const v2<T> u, const v2<T> v) {
    acc.x = fma(u.x, v.x, acc.x);
    acc.x = fma(-u.y, v.y, acc.x);
    acc.y = fma(u.x, v.y, acc.y);
    acc.y = fma(u.y, v.x, acc.y);
}

template <typename T>
__device__ __forceinline__ v2<T> cmul(const v2<T> u, const v2<T> v) {
    v2<T> r;
    r.x = fma(u.x, v.x, -u.y * v.y);
    r.y = fma(u.x, v.y, u.y * v.x);
    return r;
}

// ------------------------------------------------------------ argument blocks
// MD is the compile-time member bound; EX says D == MD exactly.

template <typename T, int MD>
struct DenseDirectArgs {
    v2<T> *psi;
    uint64_t R, base;
    int32_t D;
    Expand64 ex;
    int64_t off[MD];
    v2<T> U[MD * MD];  // row-major, zero-padded to MD x MD
};

template <typename T, int MD>
struct MonoDirectArgs {
    v2<T> *psi;
    uint64_t R, base;
    uint32_t active, unit;
    Expand64 ex;
    int64_t off[MD];     // destination offsets
    int64_t offsrc[MD];  // off[src[i]]
    v2<T> lam[MD];
};

struct TileGeo {
    uint64_t R_tiles, base_hi;
    uint32_t B, DH, tpc, G_in, lo_off, pad;
    FastDiv32 divB, divG;
    Expand64 ex_hi;
    Expand32 ex_lo;
};

template <typename T, int MD>
struct DenseTileArgs {
    v2<T> *psi;
    int32_t D;
    TileGeo t;
    int64_t offH[MD];
    int32_t smoff[MD];
    v2<T> U[MD * MD];
};

template <typename T, int MD>
struct MonoTileArgs {
    v2<T> *psi;
    uint32_t active, unit;
    TileGeo t;
    int64_t offH[MD];
    int32_t smoff[MD];
    int32_t smoffsrc[MD];
    v2<T> lam[MD];
};

// ------------------------------------------------------------ direct kernels

template <typename T, int MD, bool EX>
__global__ void __launch_bounds__(256) k_dense_direct(const __grid_constant__ DenseDirectArgs<T, MD> a) {
    const int D = EX ? MD : a.D;
    const uint64_t step = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r < a.R; r += step) {
        const uint64_t base = expand(r, a.ex) + a.base;
        v2<T> v[MD];
#pragma unroll
        for (int j = 0; j < MD; ++j) v[j] = (EX || j < D) ? a.psi[base + a.off[j]] : mk<T>(T(0), T(0));
#pragma unroll
        for (int i = 0; i < MD; ++i) {
            if (EX || i < D) {
                v2<T> acc = mk<T>(T(0), T(0));
#pragma unroll
                for (int j = 0; j < MD; ++j) cmac<T>(acc, a.U[i * MD + j], v[j]);
                a.psi[base + a.off[i]] = acc;
            }
        }
    }
}

template <typename T, int MD>
__global__ void __launch_bounds__(256) k_mono_direct(const __grid_constant__ MonoDirectArgs<T, MD> a) {
    const uint64_t step = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r < a.R; r += step) {
        const uint64_t base = expand(r, a.ex) + a.base;
        v2<T> w[MD];
#pragma unroll
        for (int i = 0; i < MD; ++i)
            if ((a.active >> i) & 1u) w[i] = a.psi[base + a.offsrc[i]];
#pragma unroll
        for (int i = 0; i < MD; ++i)
            if ((a.active >> i) & 1u) a.psi[base + a.off[i]] = ((a.unit >> i) & 1u) ? w[i] : cmul<T>(a.lam[i], w[i]);
    }
}

// -------------------------------------------------------------- tile kernels

// Dynamic shared memory: chunk bases (uint64, tpc*DH) then the tile data.
template <typename T>
__device__ __forceinline__ v2<T> *tile_data(unsigned char *raw, uint32_t nchunks) {
    size_t off = ((size_t)nchunks * sizeof(uint64_t) + 15) & ~size_t(15);
    return reinterpret_cast<v2<T> *>(raw + off);
}

template <typename T, int MD>
__device__ __forceinline__ void tile_load(const TileGeo &t, const int64_t *offH, v2<T> *psi, uint64_t tile0,
                                          uint32_t nt, uint64_t *cbase, v2<T> *sm) {
    const uint32_t nch = nt * t.DH;
    for (uint32_t c = threadIdx.x; c < nch; c += blockDim.x) {
        const uint32_t u = c / t.DH;
        const uint32_t h = c - u * t.DH;
        cbase[c] = expand(tile0 + u, t.ex_hi) * t.B + t.base_hi + offH[h];
    }
    __syncthreads();
    const uint32_t E = nch * t.B;
    for (uint32_t f = threadIdx.x; f < E; f += blockDim.x) {
        const uint32_t c = fdiv(f, t.divB);
        sm[f] = psi[cbase[c] + (f - c * t.B)];
    }
    __syncthreads();
}

template <typename T>
__device__ __forceinline__ void tile_store(const TileGeo &t, v2<T> *psi, uint32_t nt, const uint64_t *cbase,
                                           const v2<T> *sm) {
    const uint32_t E = nt * t.DH * t.B;
    for (uint32_t f = threadIdx.x; f < E; f += blockDim.x) {
        const uint32_t c = fdiv(f, t.divB);
        psi[cbase[c] + (f - c * t.B)] = sm[f];
    }
}

template <typename T, int MD, bool EX>
__global__ void __launch_bounds__(256) k_dense_tile(const __grid_constant__ DenseTileArgs<T, MD> a) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const TileGeo &t = a.t;
    const int D = EX ? MD : a.D;
    uint64_t *cbase = reinterpret_cast<uint64_t *>(smraw);
    v2<T> *sm = tile_data<T>(smraw, t.tpc * t.DH);
    const uint32_t tileE = t.DH * t.B;
    for (uint64_t tile0 = (uint64_t)blockIdx.x * t.tpc; tile0 < t.R_tiles; tile0 += (uint64_t)gridDim.x * t.tpc) {
        const uint64_t left = t.R_tiles - tile0;
        const uint32_t nt = left < (uint64_t)t.tpc ? (uint32_t)left : t.tpc;
        tile_load<T, MD>(t, a.offH, a.psi, tile0, nt, cbase, sm);
        const uint32_t G = nt * t.G_in;
        for (uint32_t gi = threadIdx.x; gi < G; gi += blockDim.x) {
            const uint32_t u = fdiv(gi, t.divG);
            const uint32_t eb = u * tileE + expand(gi - u * t.G_in, t.ex_lo) + t.lo_off;
            v2<T> v[MD];
#pragma unroll
            for (int j = 0; j < MD; ++j) v[j] = (EX || j < D) ? sm[eb + a.smoff[j]] : mk<T>(T(0), T(0));
#pragma unroll
            for (int i = 0; i < MD; ++i) {
                if (EX || i < D) {
                    v2<T> acc = mk<T>(T(0), T(0));
#pragma unroll
                    for (int j = 0; j < MD; ++j) cmac<T>(acc, a.U[i * MD + j], v[j]);
                    sm[eb + a.smoff[i]] = acc;
                }
            }
        }
        __syncthreads();
        tile_store<T>(t, a.psi, nt, cbase, sm);
        __syncthreads();
    }
}

template <typename T, int MD>
__global__ void __launch_bounds__(256) k_mono_tile(const __grid_constant__ MonoTileArgs<T, MD> a) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const TileGeo &t = a.t;
    uint64_t *cbase = reinterpret_cast<uint64_t *>(smraw);
    v2<T> *sm = tile_data<T>(smraw, t.tpc * t.DH);
    const uint32_t tileE = t.DH * t.B;
    for (uint64_t tile0 = (uint64_t)blockIdx.x * t.tpc; tile0 < t.R_tiles; tile0 += (uint64_t)gridDim.x * t.tpc) {
        const uint64_t left = t.R_tiles - tile0;
        const uint32_t nt = left < (uint64_t)t.tpc ? (uint32_t)left : t.tpc;
        tile_load<T, MD>(t, a.offH, a.psi, tile0, nt, cbase, sm);
        const uint32_t G = nt * t.G_in;
        for (uint32_t gi = threadIdx.x; gi < G; gi += blockDim.x) {
            const uint32_t u = fdiv(gi, t.divG);
            const uint32_t eb = u * tileE + expand(gi - u * t.G_in, t.ex_lo) + t.lo_off;
            v2<T> w[MD];
#pragma unroll
            for (int i = 0; i < MD; ++i)
                if ((a.active >> i) & 1u) w[i] = sm[eb + a.smoffsrc[i]];
#pragma unroll
            for (int i = 0; i < MD; ++i)
                if ((a.active >> i) & 1u) sm[eb + a.smoff[i]] = ((a.unit >> i) & 1u) ? w[i] : cmul<T>(a.lam[i], w[i]);
        }
        __syncthreads();
        tile_store<T>(t, a.psi, nt, cbase, sm);
        __syncthreads();
    }
}

// ------------------------------------------------------------------ launchers

int occupancy_blocks(const void *fn, int block, size_t smem);  // cached, in qd_api.cu

inline size_t tile_smem_bytes(const GatePlan &g, size_t elem) {
    const size_t nch = (size_t)g.tpc * g.DH;
    return ((nch * sizeof(uint64_t) + 15) & ~size_t(15)) + nch * g.B * elem;
}

template <typename T>
inline void fill_tilegeo(TileGeo &t, const GatePlan &g) {
    t.R_tiles = g.R_tiles;
    t.base_hi = g.base_off_hi;
    t.B = g.B;
    t.DH = g.DH;
    t.tpc = g.tpc;
    t.G_in = g.G_in;
    t.lo_off = g.lo_off;
    t.pad = 0;
    t.divB = g.divB;
    t.divG = g.divG;
    t.ex_hi = g.ex_hi;
    t.ex_lo = g.ex_lo;
}

template <typename T, int MD, bool EX>
cudaError_t launch_dense(const GatePlan &g, void *psi, int sm_count, cudaStream_t s) {
    constexpr int kBlock = 256;
    if (g.mode == Mode::Direct) {
        DenseDirectArgs<T, MD> a;
        a.psi = static_cast<v2<T> *>(psi);
        a.R = g.R;
        a.base = g.base_off;
        a.D = g.D;
        a.ex = g.ex;
        for (int j = 0; j < MD; ++j) a.off[j] = j < g.D ? g.off[j] : 0;
        for (int i = 0; i < MD; ++i)
            for (int j = 0; j < MD; ++j)
                a.U[i * MD + j] = (i < g.D && j < g.D) ? mk<T>((T)g.U[2 * (i * g.D + j)], (T)g.U[2 * (i * g.D + j) + 1])
                                                       : mk<T>(T(0), T(0));
        auto fn = k_dense_direct<T, MD, EX>;
        const int occ = occupancy_blocks((const void *)fn, kBlock, 0);
        const uint64_t need = (g.R + kBlock - 1) / kBlock;
        const int grid = (int)std::min<uint64_t>(need, (uint64_t)sm_count * occ);
        if (grid <= 0) return cudaSuccess;
        fn<<<grid, kBlock, 0, s>>>(a);
        return cudaGetLastError();
    }
    DenseTileArgs<T, MD> a;
    a.psi = static_cast<v2<T> *>(psi);
    a.D = g.D;
    fill_tilegeo<T>(a.t, g);
    for (int j = 0; j < MD; ++j) {
        a.offH[j] = j < (int)g.DH ? g.offH[j] : 0;
        a.smoff[j] = j < g.D ? g.smoff[j] : 0;
    }
    for (int i = 0; i < MD; ++i)
        for (int j = 0; j < MD; ++j)
            a.U[i * MD + j] = (i < g.D && j < g.D) ? mk<T>((T)g.U[2 * (i * g.D + j)], (T)g.U[2 * (i * g.D + j) + 1])
                                                   : mk<T>(T(0), T(0));
    auto fn = k_dense_tile<T, MD, EX>;
    const size_t smem = tile_smem_bytes(g, sizeof(v2<T>));
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute((const void *)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const int occ = occupancy_blocks((const void *)fn, kBlock, smem);
    const uint64_t need = (g.R_tiles + g.tpc - 1) / g.tpc;
    const int grid = (int)std::min<uint64_t>(need, (uint64_t)sm_count * std::max(occ, 1));
    if (grid <= 0) return cudaSuccess;
    fn<<<grid, kBlock, smem, s>>>(a);
    return cudaGetLastError();
}

template <typename T, int MD>
cudaError_t launch_mono(const GatePlan &g, void *psi, int sm_count, cudaStream_t s) {
    constexpr int kBlock = 256;
    if (g.mode == Mode::Direct) {
        MonoDirectArgs<T, MD> a;
        a.psi = static_cast<v2<T> *>(psi);
        a.R = g.R;
        a.base = g.base_off;
        a.active = g.active;
        a.unit = g.unit;
        a.ex = g.ex;
        for (int i = 0; i < MD; ++i) {
            const bool in = i < g.D;
            a.off[i] = in ? g.off[i] : 0;
            a.offsrc[i] = in ? g.off[g.src[i]] : 0;
            a.lam[i] = in ? mk<T>((T)g.lam[2 * i], (T)g.lam[2 * i + 1]) : mk<T>(T(1), T(0));
        }
        auto fn = k_mono_direct<T, MD>;
        const int occ = occupancy_blocks((const void *)fn, kBlock, 0);
        const uint64_t need = (g.R + kBlock - 1) / kBlock;
        const int grid = (int)std::min<uint64_t>(need, (uint64_t)sm_count * occ);
        if (grid <= 0) return cudaSuccess;
        fn<<<grid, kBlock, 0, s>>>(a);
        return cudaGetLastError();
    }
    MonoTileArgs<T, MD> a;
    a.psi = static_cast<v2<T> *>(psi);
    a.active = g.active;
    a.unit = g.unit;
    fill_tilegeo<T>(a.t, g);
    for (int i = 0; i < MD; ++i) {
        const bool in = i < g.D;
        a.offH[i] = i < (int)g.DH ? g.offH[i] : 0;
        a.smoff[i] = in ? g.smoff[i] : 0;
        a.smoffsrc[i] = in ? g.smoff[g.src[i]] : 0;
        a.lam[i] = in ? mk<T>((T)g.lam[2 * i], (T)g.lam[2 * i + 1]) : mk<T>(T(1), T(0));
    }
    auto fn = k_mono_tile<T, MD>;
    const size_t smem = tile_smem_bytes(g, sizeof(v2<T>));
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute((const void *)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    const int occ = occupancy_blocks((const void *)fn, kBlock, smem);
    const uint64_t need = (g.R_tiles + g.tpc - 1) / g.tpc;
    const int grid = (int)std::min<uint64_t>(need, (uint64_t)sm_count * std::max(occ, 1));
    if (grid <= 0) return cudaSuccess;
    fn<<<grid, kBlock, smem, s>>>(a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_gate_t(const GatePlan &g, void *psi, int sm_count, cudaStream_t s) {
    if (g.kind == Kind::Mono) {
        if (g.D <= 4) return launch_mono<T, 4>(g, psi, sm_count, s);
        if (g.D <= 8) return launch_mono<T, 8>(g, psi, sm_count, s);
        if (g.D <= 16) return launch_mono<T, 16>(g, psi, sm_count, s);
        return launch_mono<T, 32>(g, psi, sm_count, s);
    }
    switch (g.D) {
        case 2: return launch_dense<T, 2, true>(g, psi, sm_count, s);
        case 3: return launch_dense<T, 3, true>(g, psi, sm_count, s);
        case 4: return launch_dense<T, 4, true>(g, psi, sm_count, s);
        case 5: return launch_dense<T, 5, true>(g, psi, sm_count, s);
        case 6: return launch_dense<T, 6, true>(g, psi, sm_count, s);
        case 8: return launch_dense<T, 8, true>(g, psi, sm_count, s);
        case 9: return launch_dense<T, 9, true>(g, psi, sm_count, s);
        default: break;
    }
    if (g.D <= 16) return launch_dense<T, 16, false>(g, psi, sm_count, s);
    return launch_dense<T, 32, false>(g, psi, sm_count, s);
}

}  // namespace qd
