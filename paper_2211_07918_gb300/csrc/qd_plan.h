// Host-side description of one prepared gate launch (precision independent).
// Built by the planner in qd_api.cu, consumed by the per-precision launchers.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "qd_common.cuh"

namespace qd {

enum class Mode : int32_t { Direct = 0, Tile = 1, Tensor = 2, Table = 3 };
enum class Kind : int32_t { Dense = 0, Mono = 1 };

// Largest number of amplitudes a tile-mode CTA stages in shared memory per
// iteration, and the hard cap when the block length must be raised to reach
// a coalescing width.
constexpr uint32_t kTileBudget = 2048;
constexpr uint32_t kTileHardMax = 8192;
// Default stride threshold of tile mode: a gate whose lowest target or control
// stride is below it is staged through shared memory.  Measured on GB300 the
// direct kernel is faster for every stride (L1 absorbs the short strided
// runs), so the default is 0 (never tile); QD_TILE_STRIDE in the environment
// or qd_set_tuning(QD_TUNE_TILE_STRIDE) per register override it.
constexpr int64_t kLowStride = 0;

struct GatePlan {
    Mode mode = Mode::Direct;
    Kind kind = Kind::Dense;
    int32_t D = 0;
    uint64_t N = 0;  // register size (selects 32- or 64-bit index arithmetic)
    bool wide = false;  // 64-bit index arithmetic below 2^31 too (QD_TUNE_INDEX64)
    bool pow2 = false;  // every qudit dimension of the register is a power of two

    // --- direct mode: one thread per group --------------------------------
    uint64_t R = 0;          // number of groups
    uint64_t base_off = 0;   // sum over controls of level * stride
    Expand64 ex{};           // group index -> flat base
    int64_t off[kMaxBlockD] = {};  // flat offset of local index j

    // --- tile mode: a CTA stages DH chunks of B contiguous amplitudes -------
    uint64_t R_tiles = 0;      // number of tiles
    uint64_t base_off_hi = 0;  // controls at or above the block, level * stride
    Expand64 ex_hi{};          // tile index -> flat tile base (already scaled by B)
    uint32_t B = 0;            // block length (amplitudes), = s_m
    uint32_t DH = 0;           // combinations of the targets at or above the block
    uint32_t tpc = 0;          // tiles per CTA iteration
    uint32_t G_in = 0;         // groups per tile
    FastDiv32 divB{};          // element index -> chunk
    FastDiv32 divG{};          // group index -> tile
    Expand32 ex_lo{};          // in-tile group index -> position inside the block
    uint32_t lo_off = 0;       // controls below the block, level * stride
    int64_t offH[kMaxBlockD] = {};  // flat offset of chunk h
    int32_t smoff[kMaxBlockD] = {}; // shared-memory offset of local index j in a tile

    // --- numerics (FP64, rounded to the state precision at launch) ---------
    double U[2 * kMaxD * kMaxD] = {};  // dense: row-major D x D (re, im)
    int32_t src[kMaxD] = {};           // mono: out[i] = lam[i] * in[src[i]]
    double lam[2 * kMaxD] = {};

    // --- tensor mode: fused block on tcgen05 (complex64 states) -------------
    int32_t Dp = 0;                    // D rounded up to a multiple of 8
    const void *tc_terms = nullptr;    // device: three BF16 terms of the real embedding
    // --- table mode: a run of diagonal gates (psi[i] *= tab[(i / tab_div) mod tab_size])
    uint64_t tab_div = 0;
    uint64_t tab_size = 0;
    const void *tab = nullptr;         // device table (float4 hi/lo or double2 entries)

    uint32_t active = 0;               // mono: bit i set if out[i] != in[i]
    uint32_t unit = 0;                 // mono: bit i set if lam[i] == 1 exactly

    // --- accounting --------------------------------------------------------
    double alg_bytes = 0;  // algorithmic HBM bytes of one launch
};

// 64-bit index kernels: registers of 2^31 amplitudes or more (FastDiv32's
// dividend bound), or any register when asked for.  A register whose
// dimensions are all powers of two keeps 32-bit indices up to 2^32
// amplitudes: every index is below 2^32, and FastDiv32 by a power of two
// (m = 2^31, a shift of n * 2^31 < 2^63) is exact for every 32-bit n.
inline bool wide_index(const GatePlan &g) {
    if (g.wide) return true;
    if (g.N < (uint64_t(1) << 31)) return false;
    return !(g.pow2 && g.N <= (uint64_t(1) << 32));
}

// Per-precision launchers (qd_apply_f32.cu / qd_apply_f64.cu).
cudaError_t launch_gate_f32(const GatePlan &g, void *psi, int sm_count, cudaStream_t s);
cudaError_t launch_gate_f64(const GatePlan &g, void *psi, int sm_count, cudaStream_t s);

}  // namespace qd
