// Per-gate in-place apply kernels (QuDiet Sec. 2.1.2 gates, Sec. 3.4 user
// gates), instantiated for FP32 (complex64) and FP64 (complex128) states and
// for 32- or 64-bit index arithmetic.
//
// A gate with targets T (D = prod d_t local states) and controls C at levels
// l_c maps, for every group r over the remaining qudits, the D amplitudes
//   v_j = psi[base(r) + off_j],   base(r) = insert_digits(r) + sum_c l_c s_c,
// to U v (dense) or to out_i = lam_i v_src(i) (diagonal / permutation with
// phases: "mono").  Amplitudes outside the selected control slice are never
// touched.
//
// Two memory schemes:
//   direct  one thread per group, loads straight from global memory.  Used
//           when every target and control has a flat stride >= the planner's
//           threshold, so that a warp's 32 consecutive groups read runs of
//           consecutive amplitudes for each member.
//   tile    a CTA stages DH chunks of B contiguous amplitudes (B = s_m covers
//           all low-stride targets and controls) in shared memory with
//           asynchronous copies, applies the gate to the groups inside the
//           tile, and writes the chunks back with coalesced stores.
#pragma once
#include <algorithm>
#include <cstring>
#include <type_traits>

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

// complex64 states carry every gate coefficient as an unevaluated pair of
// floats c = hi + lo (|lo| <= ulp(hi)/2).  Rounding the coefficients to one
// float would make the applied matrix non-unitary by ~1e-7 in the same way
// for every group of the register, a coherent norm drift that adds up over a
// circuit; with the pair the coefficient error is ~1e-14 and what remains is
// the incoherent per-amplitude rounding of FP32 arithmetic.
template <typename T> constexpr bool kSplit = std::is_same<T, float>::value;
template <typename T> __host__ __device__ constexpr int split_len(int n) { return kSplit<T> ? n : 1; }

template <typename T>
__device__ __forceinline__ v2<T> cmul_split(const v2<T> hi, const v2<T> lo, const v2<T> v) {
    if constexpr (kSplit<T>) {
        v2<T> r = cmul<T>(lo, v);
        r.x = fma(hi.x, v.x, fma(-hi.y, v.y, r.x));
        r.y = fma(hi.x, v.y, fma(hi.y, v.x, r.y));
        return r;
    } else {
        return cmul<T>(hi, v);
    }
}

// Packed FP32 pairs (fma.rn.f32x2: two FMAs, each rounded as fmaf).  A
// coefficient u is carried as the pairs (u.x, u.x) and (-u.y, u.y); with
// v = (re, im) and vs = (im, re), acc += u v is two packed FMAs with the
// roundings of cmac<float>.
typedef unsigned long long f2p;
__device__ __forceinline__ f2p pk_fma(f2p a, f2p b, f2p c) {
    f2p d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f2p pk_pack(float a, float b) {
    f2p r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float2 pk_unpack(f2p r) {
    float a, b;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
    return make_float2(a, b);
}
inline unsigned long long pk_host(float a, float b) {
    unsigned int ua, ub;
    std::memcpy(&ua, &a, 4);
    std::memcpy(&ub, &b, 4);
    return (unsigned long long)ua | ((unsigned long long)ub << 32);
}
// Dense complex64 gates of up to 4 x 4, and of 9 x 9 (two qutrits: 72 FP32
// FMAs per amplitude, which unpacked did not hide under the memory pass;
// measured 0.59-0.64 -> 0.73-0.78 of the copy peak), use the packed path
// (8 x 8 measured slower packed).
template <typename T, int MD> constexpr bool kPacked = kSplit<T> && (MD <= 4 || MD == 9);
// Kernels with a contiguous-members path (complex64, even member bound):
// a gate on the lowest qudits, whose group is D consecutive amplitudes
// starting at a multiple of D, reads and writes 16-byte amplitude pairs.
template <typename T, int MD> constexpr bool kVecPairs = kSplit<T> && MD % 2 == 0 && MD <= 16;

template <typename T>
inline void split_coef(double re, double im, v2<T> &hi, v2<T> &lo) {
    hi = mk<T>((T)re, (T)im);
    lo = mk<T>((T)(re - (double)hi.x), (T)(im - (double)hi.y));
}

// ------------------------------------------------------------ argument blocks
// MD is the compile-time member bound; EX says D == MD exactly; I is the index
// type.

template <typename T, typename I, int MD>
struct DenseDirectArgs {
    v2<T> *psi;
    I R, base;
    int32_t D;
    int32_t contig;  // members at offsets 0..D-1 (D == MD): 16-byte amplitude-pair accesses
    ExpandT<I> ex;
    I off[MD];
    v2<T> U[MD * MD];  // row-major, zero-padded to MD x MD
    v2<T> Ulo[split_len<T>(MD * MD)];
    // packed path: per coefficient lo (x,x), lo (-y,y), hi (x,x), hi (-y,y)
    unsigned long long Pk[kPacked<T, MD> ? 4 * MD * MD : 1];
};

template <typename T, typename I, int MD>
struct MonoDirectArgs {
    v2<T> *psi;
    I R, base;
    uint32_t active, unit;
    ExpandT<I> ex;
    I off[MD];     // destination offsets
    I offsrc[MD];  // off[src[i]]
    v2<T> lam[MD];
    v2<T> lamlo[split_len<T>(MD)];
};

template <typename I>
struct TileGeo {
    I R_tiles, base_hi;
    uint32_t B, DH, tpc, G_in, lo_off, pad;
    FastDiv32 divB, divG;
    ExpandT<I> ex_hi;
    Expand32 ex_lo;
};

template <typename T, typename I, int MD>
struct DenseTileArgs {
    v2<T> *psi;
    int32_t D;
    TileGeo<I> t;
    I offH[MD];
    int32_t smoff[MD];
    v2<T> U[MD * MD];
    v2<T> Ulo[split_len<T>(MD * MD)];
};

template <typename T, typename I, int MD>
struct MonoTileArgs {
    v2<T> *psi;
    uint32_t active, unit;
    TileGeo<I> t;
    I offH[MD];
    int32_t smoff[MD];
    int32_t smoffsrc[MD];
    v2<T> lam[MD];
    v2<T> lamlo[split_len<T>(MD)];
};

// ------------------------------------------------------------ direct kernels

// Groups per thread per iteration: loads of all of them are issued before any
// arithmetic, for memory-level parallelism (bounded by register pressure).
// A permutation or diagonal gate moves few amplitudes per group (a qubit
// phase touches one), so its kernel takes more groups per iteration.
template <typename T, typename I, int MD>
__host__ __device__ constexpr int direct_unroll() {
    return (MD * (int)sizeof(v2<T>)) <= 32 ? 2 : 1;
}
template <typename T, typename I, int MD>
__host__ __device__ constexpr int mono_unroll() {
    return MD <= 2 ? 4 : (MD <= 4 ? 2 : 1);
}
// Resident CTAs of 256 threads the register budget must allow (the memory
// parallelism of these kernels is the loads all their threads have in
// flight): for complex64, 4 (64 registers) where that costs no spills, 3 for
// the 8-member dense kernel and the largest mono bucket, 2 for the largest
// dense; complex128 (bound by FP64 arithmetic) is left unconstrained.
template <typename T, int MD, bool DENSE>
__host__ __device__ constexpr int direct_min_blocks() {
    return !kSplit<T> ? 1 : MD >= 32 ? (DENSE ? 2 : 3) : (DENSE && MD == 8 ? 3 : 4);
}

template <typename T, typename I, int MD, bool EX>
__global__ void __launch_bounds__(256, (direct_min_blocks<T, MD, true>())) k_dense_direct(const __grid_constant__ DenseDirectArgs<T, I, MD> a) {
    constexpr int UN = direct_unroll<T, I, MD>();
    const int D = EX ? MD : a.D;
    const I step = (I)gridDim.x * blockDim.x;
    for (I r0 = (I)blockIdx.x * blockDim.x + threadIdx.x; r0 < a.R; r0 += UN * step) {
        I base[UN];
        bool ok[UN];
        v2<T> v[UN][MD];
#pragma unroll
        for (int u = 0; u < UN; ++u) {
            const I r = r0 + u * step;
            ok[u] = r < a.R;
            base[u] = ok[u] ? expand(r, a.ex) + a.base : 0;
        }
        const bool pairs = kVecPairs<T, MD> && a.contig;
#pragma unroll
        for (int u = 0; u < UN; ++u) {
            if constexpr (kVecPairs<T, MD>) {
                if (pairs) {
                    const float4 *p = reinterpret_cast<const float4 *>(a.psi + base[u]);
#pragma unroll
                    for (int h = 0; h < MD / 2; ++h) {
                        const float4 q = ok[u] ? p[h] : make_float4(0.f, 0.f, 0.f, 0.f);
                        v[u][2 * h] = mk<T>(q.x, q.y);
                        v[u][2 * h + 1] = mk<T>(q.z, q.w);
                    }
                    continue;
                }
            }
#pragma unroll
            for (int j = 0; j < MD; ++j)
                v[u][j] = (ok[u] && (EX || j < D)) ? a.psi[base[u] + a.off[j]] : mk<T>(T(0), T(0));
        }
        // output i of group u: with amplitude pairs, odd outputs store the pair
        v2<T> prev = mk<T>(T(0), T(0));
        auto put = [&](int u, int i, const v2<T> o) {
            if constexpr (kVecPairs<T, MD>) {
                if (pairs) {
                    if (i & 1)
                        reinterpret_cast<float4 *>(a.psi + base[u])[i / 2] = make_float4(prev.x, prev.y, o.x, o.y);
                    else
                        prev = o;
                    return;
                }
            }
            a.psi[base[u] + a.off[i]] = o;
        };
        if constexpr (kPacked<T, MD>) {
            // lo terms first, then hi terms (as below), two lanes per FMA
#pragma unroll
            for (int u = 0; u < UN; ++u) {
                if (!ok[u]) continue;
                f2p pv[MD], ps[MD];
#pragma unroll
                for (int j = 0; j < MD; ++j) {
                    pv[j] = pk_pack(v[u][j].x, v[u][j].y);
                    ps[j] = pk_pack(v[u][j].y, v[u][j].x);
                }
#pragma unroll
                for (int i = 0; i < MD; ++i) {
                    if (EX || i < D) {
                        f2p acc = 0ull;
#pragma unroll
                        for (int j = 0; j < MD; ++j) {
                            acc = pk_fma(a.Pk[4 * (i * MD + j) + 0], pv[j], acc);
                            acc = pk_fma(a.Pk[4 * (i * MD + j) + 1], ps[j], acc);
                        }
#pragma unroll
                        for (int j = 0; j < MD; ++j) {
                            acc = pk_fma(a.Pk[4 * (i * MD + j) + 2], pv[j], acc);
                            acc = pk_fma(a.Pk[4 * (i * MD + j) + 3], ps[j], acc);
                        }
                        const float2 o = pk_unpack(acc);
                        put(u, i, mk<T>(o.x, o.y));
                    }
                }
            }
        } else {
#pragma unroll
        for (int u = 0; u < UN; ++u) {
            if (!ok[u]) continue;
#pragma unroll
            for (int i = 0; i < MD; ++i) {
                if (EX || i < D) {
                    v2<T> acc = mk<T>(T(0), T(0));
                    if constexpr (kSplit<T>) {
#pragma unroll
                        for (int j = 0; j < MD; ++j) cmac<T>(acc, a.Ulo[i * MD + j], v[u][j]);
                    }
#pragma unroll
                    for (int j = 0; j < MD; ++j) cmac<T>(acc, a.U[i * MD + j], v[u][j]);
                    put(u, i, acc);
                }
            }
        }
        }
    }
}

template <typename T, typename I, int MD>
__global__ void __launch_bounds__(256, (direct_min_blocks<T, MD, false>())) k_mono_direct(const __grid_constant__ MonoDirectArgs<T, I, MD> a) {
    constexpr int UN = mono_unroll<T, I, MD>();
    const I step = (I)gridDim.x * blockDim.x;
    for (I r0 = (I)blockIdx.x * blockDim.x + threadIdx.x; r0 < a.R; r0 += UN * step) {
        I base[UN];
        bool ok[UN];
        v2<T> w[UN][MD];
#pragma unroll
        for (int u = 0; u < UN; ++u) {
            const I r = r0 + u * step;
            ok[u] = r < a.R;
            base[u] = ok[u] ? expand(r, a.ex) + a.base : 0;
        }
#pragma unroll
        for (int u = 0; u < UN; ++u)
#pragma unroll
            for (int i = 0; i < MD; ++i)
                if (ok[u] && ((a.active >> i) & 1u)) w[u][i] = a.psi[base[u] + a.offsrc[i]];
#pragma unroll
        for (int u = 0; u < UN; ++u)
#pragma unroll
            for (int i = 0; i < MD; ++i)
                if (ok[u] && ((a.active >> i) & 1u))
                    a.psi[base[u] + a.off[i]] =
                        ((a.unit >> i) & 1u) ? w[u][i] : cmul_split<T>(a.lam[i], a.lamlo[kSplit<T> ? i : 0], w[u][i]);
    }
}

// Dense gate followed by a run of diagonal gates, one pass: out = U v for
// every group, then each output amplitude at flat index i is multiplied by
// the run's table entry T[(i / s_qa) mod TS] (the product of the run's
// diagonals; complex64 entries as FP32 hi + lo, applied lo first).
template <typename I> struct DivOfI;
template <> struct DivOfI<uint32_t> { using type = FastDiv32; };
template <> struct DivOfI<uint64_t> { using type = FastDiv64; };

template <typename T> struct TabEntry;
template <> struct TabEntry<float> { using type = float4; };
template <> struct TabEntry<double> { using type = double2; };

template <typename T, typename I, int MD>
struct DenseTableArgs {
    DenseDirectArgs<T, I, MD> d;
    typename DivOfI<I>::type divA, divT;  // by s_qa and by TS
    uint32_t oq[MD];  // (off_j / s_qa) mod TS
    I thr[MD];        // s_qa - off_j mod s_qa: member j's carry iff b mod s_qa >= thr_j
    uint32_t carry;   // some off_j is not a multiple of s_qa
    uint32_t tsmask;  // TS - 1 when TS is a power of two, else 0
    const typename TabEntry<T>::type *tab;
};

template <typename T>
__device__ __forceinline__ v2<T> times_entry(const v2<T> o, const typename TabEntry<T>::type t) {
    if constexpr (kSplit<T>) {
        return cmul_split<T>(mk<T>(t.x, t.y), mk<T>(t.z, t.w), o);
    } else {
        return cmul<T>(mk<T>(t.x, t.y), o);
    }
}

// Two groups per thread per iteration for up to four members.  The table
// index of member j of a group at base b is, with b = qb s_qa + rb,
// (qb + off_j / s_qa + [rb + off_j mod s_qa >= s_qa]) mod TS (< 2^24): two
// divisions per group instead of two per member (none when every member
// offset is a multiple of s_qa, a mask when TS is a power of two).  The table entries of a
// group's outputs are loaded before the first of them is stored (a load
// after a store to the state could not be moved above it, and each output
// would wait out its own table latency): all of them for up to four
// members, pairs above (register budget).  The kernel is bound by the loads
// its resident threads keep in flight, so complex64 keeps 4 CTAs of 256
// threads per SM (64 registers; a group's table position is computed after
// its member loads are issued, which keeps it within them).
template <typename T, typename I, int MD>
__host__ __device__ constexpr int table_min_blocks() {
    return kSplit<T> ? 4 : direct_min_blocks<T, MD, true>();
}

template <typename T, typename I, int MD, bool EX>
__global__ void __launch_bounds__(256, (table_min_blocks<T, I, MD>()))
    k_dense_table(const __grid_constant__ DenseTableArgs<T, I, MD> a) {
    constexpr int UN = MD <= 4 ? 2 : 1;
    constexpr int TB = MD <= 4 ? MD : 2;  // outputs whose entries are loaded together
    using Entry = typename TabEntry<T>::type;
    const int D = EX ? MD : a.d.D;
    const I step = (I)gridDim.x * blockDim.x;
    const I sA = (I)a.divA.d;
    const uint32_t TS = (uint32_t)a.divT.d;
    for (I r0 = (I)blockIdx.x * blockDim.x + threadIdx.x; r0 < a.d.R; r0 += UN * step) {
        I base[UN];
        bool ok[UN];
        v2<T> v[UN][MD];
#pragma unroll
        for (int u = 0; u < UN; ++u) {
            const I r = r0 + u * step;
            ok[u] = r < a.d.R;
            base[u] = ok[u] ? expand(r, a.d.ex) + a.d.base : 0;
        }
#pragma unroll
        for (int u = 0; u < UN; ++u)
#pragma unroll
            for (int j = 0; j < MD; ++j)
                v[u][j] = (ok[u] && (EX || j < D)) ? a.d.psi[base[u] + a.d.off[j]] : mk<T>(T(0), T(0));
#pragma unroll
        for (int u = 0; u < UN; ++u) {
            if (!ok[u]) continue;
            // the group's table position (while its member loads are in flight)
            const I qb = fdiv(base[u], a.divA);
            const uint32_t kb = a.tsmask ? (uint32_t)qb & a.tsmask : (uint32_t)(qb - fdiv(qb, a.divT) * (I)TS);
#pragma unroll
            for (int c0 = 0; c0 < MD; c0 += TB) {
                Entry t[TB];
#pragma unroll
                for (int c = 0; c < TB; ++c) {
                    const int i = c0 + c;
                    if (EX || i < D) {
                        uint32_t k = kb + a.oq[i];  // < 2 TS
                        if (a.carry && base[u] - qb * sA >= a.thr[i]) ++k;
                        if (a.tsmask) {
                            k &= a.tsmask;
                        } else {
                            if (k >= TS) k -= TS;
                            if (k >= TS) k -= TS;
                        }
                        t[c] = __ldg(&a.tab[k]);
                    }
                }
#pragma unroll
                for (int c = 0; c < TB; ++c) {
                    const int i = c0 + c;
                    if (!(EX || i < D)) continue;
                    v2<T> acc = mk<T>(T(0), T(0));
                    if constexpr (kPacked<T, MD>) {
                        // lo terms first, then hi terms, two lanes per FMA
                        f2p pa = 0ull;
#pragma unroll
                        for (int j = 0; j < MD; ++j) {
                            pa = pk_fma(a.d.Pk[4 * (i * MD + j) + 0], pk_pack(v[u][j].x, v[u][j].y), pa);
                            pa = pk_fma(a.d.Pk[4 * (i * MD + j) + 1], pk_pack(v[u][j].y, v[u][j].x), pa);
                        }
#pragma unroll
                        for (int j = 0; j < MD; ++j) {
                            pa = pk_fma(a.d.Pk[4 * (i * MD + j) + 2], pk_pack(v[u][j].x, v[u][j].y), pa);
                            pa = pk_fma(a.d.Pk[4 * (i * MD + j) + 3], pk_pack(v[u][j].y, v[u][j].x), pa);
                        }
                        const float2 o = pk_unpack(pa);
                        acc = mk<T>(o.x, o.y);
                    } else {
                        if constexpr (kSplit<T>) {
#pragma unroll
                            for (int j = 0; j < MD; ++j) cmac<T>(acc, a.d.Ulo[i * MD + j], v[u][j]);
                        }
#pragma unroll
                        for (int j = 0; j < MD; ++j) cmac<T>(acc, a.d.U[i * MD + j], v[u][j]);
                    }
                    a.d.psi[base[u] + a.d.off[i]] = times_entry<T>(acc, t[c]);
                }
            }
        }
    }
}

// -------------------------------------------------------------- tile kernels

// Dynamic shared memory: chunk bases (I, tpc*DH entries) then the tile data.
template <typename T, typename I>
__device__ __forceinline__ v2<T> *tile_data(unsigned char *raw, uint32_t nchunks) {
    size_t off = ((size_t)nchunks * sizeof(I) + 15) & ~size_t(15);
    return reinterpret_cast<v2<T> *>(raw + off);
}

// Asynchronous global->shared copy of one amplitude (sm_80+ cp.async; 8-byte
// copies go through L1, 16-byte copies bypass it).
template <typename T>
__device__ __forceinline__ void cp_async_amp(v2<T> *dst, const v2<T> *src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    if constexpr (sizeof(v2<T>) == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

template <typename T, typename I, int MD>
__device__ __forceinline__ void tile_load(const TileGeo<I> &t, const I *offH, v2<T> *psi, I tile0, uint32_t nt,
                                          I *cbase, v2<T> *sm) {
    const uint32_t nch = nt * t.DH;
    for (uint32_t c = threadIdx.x; c < nch; c += blockDim.x) {
        const uint32_t u = c / t.DH;
        const uint32_t h = c - u * t.DH;
        cbase[c] = expand((I)(tile0 + u), t.ex_hi) * t.B + t.base_hi + offH[h];
    }
    __syncthreads();
    const uint32_t E = nch * t.B;
    for (uint32_t f = threadIdx.x; f < E; f += blockDim.x) {
        const uint32_t c = fdiv(f, t.divB);
        cp_async_amp<T>(sm + f, psi + cbase[c] + (f - c * t.B));
    }
    cp_async_wait_all();
    __syncthreads();
}

template <typename T, typename I>
__device__ __forceinline__ void tile_store(const TileGeo<I> &t, v2<T> *psi, uint32_t nt, const I *cbase,
                                           const v2<T> *sm) {
    const uint32_t E = nt * t.DH * t.B;
    for (uint32_t f = threadIdx.x; f < E; f += blockDim.x) {
        const uint32_t c = fdiv(f, t.divB);
        psi[cbase[c] + (f - c * t.B)] = sm[f];
    }
}

template <typename T, typename I, int MD, bool EX>
__global__ void __launch_bounds__(256) k_dense_tile(const __grid_constant__ DenseTileArgs<T, I, MD> a) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const TileGeo<I> &t = a.t;
    const int D = EX ? MD : a.D;
    I *cbase = reinterpret_cast<I *>(smraw);
    v2<T> *sm = tile_data<T, I>(smraw, t.tpc * t.DH);
    const uint32_t tileE = t.DH * t.B;
    for (I tile0 = (I)blockIdx.x * t.tpc; tile0 < t.R_tiles; tile0 += (I)gridDim.x * t.tpc) {
        const I left = t.R_tiles - tile0;
        const uint32_t nt = left < (I)t.tpc ? (uint32_t)left : t.tpc;
        tile_load<T, I, MD>(t, a.offH, a.psi, tile0, nt, cbase, sm);
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
                    if constexpr (kSplit<T>) {
#pragma unroll
                        for (int j = 0; j < MD; ++j) cmac<T>(acc, a.Ulo[i * MD + j], v[j]);
                    }
#pragma unroll
                    for (int j = 0; j < MD; ++j) cmac<T>(acc, a.U[i * MD + j], v[j]);
                    sm[eb + a.smoff[i]] = acc;
                }
            }
        }
        __syncthreads();
        tile_store<T, I>(t, a.psi, nt, cbase, sm);
        __syncthreads();
    }
}

template <typename T, typename I, int MD>
__global__ void __launch_bounds__(256) k_mono_tile(const __grid_constant__ MonoTileArgs<T, I, MD> a) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const TileGeo<I> &t = a.t;
    I *cbase = reinterpret_cast<I *>(smraw);
    v2<T> *sm = tile_data<T, I>(smraw, t.tpc * t.DH);
    const uint32_t tileE = t.DH * t.B;
    for (I tile0 = (I)blockIdx.x * t.tpc; tile0 < t.R_tiles; tile0 += (I)gridDim.x * t.tpc) {
        const I left = t.R_tiles - tile0;
        const uint32_t nt = left < (I)t.tpc ? (uint32_t)left : t.tpc;
        tile_load<T, I, MD>(t, a.offH, a.psi, tile0, nt, cbase, sm);
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
                if ((a.active >> i) & 1u)
                    sm[eb + a.smoff[i]] =
                        ((a.unit >> i) & 1u) ? w[i] : cmul_split<T>(a.lam[i], a.lamlo[kSplit<T> ? i : 0], w[i]);
        }
        __syncthreads();
        tile_store<T, I>(t, a.psi, nt, cbase, sm);
        __syncthreads();
    }
}

// ------------------------------------------------------------------ launchers

int occupancy_blocks(const void *fn, int block, size_t smem);  // cached, in qd_api.cu

template <typename I>
inline size_t tile_smem_bytes(const GatePlan &g, size_t elem) {
    const size_t nch = (size_t)g.tpc * g.DH;
    return ((nch * sizeof(I) + 15) & ~size_t(15)) + nch * g.B * elem;
}

template <typename I>
inline ExpandT<I> expand_for(const Expand64 &e) {
    if constexpr (sizeof(I) == 4) return narrow(e);
    else return e;
}

template <typename I>
inline void fill_tilegeo(TileGeo<I> &t, const GatePlan &g) {
    t.R_tiles = (I)g.R_tiles;
    t.base_hi = (I)g.base_off_hi;
    t.B = g.B;
    t.DH = g.DH;
    t.tpc = g.tpc;
    t.G_in = g.G_in;
    t.lo_off = g.lo_off;
    t.pad = 0;
    t.divB = g.divB;
    t.divG = g.divG;
    t.ex_hi = expand_for<I>(g.ex_hi);
    t.ex_lo = g.ex_lo;
}

template <typename T, int MD>
inline void fill_matrix(v2<T> *U, v2<T> *Ulo, const GatePlan &g) {
    for (int i = 0; i < MD; ++i)
        for (int j = 0; j < MD; ++j) {
            v2<T> hi = mk<T>(T(0), T(0)), lo = hi;
            if (i < g.D && j < g.D) split_coef<T>(g.U[2 * (i * g.D + j)], g.U[2 * (i * g.D + j) + 1], hi, lo);
            U[i * MD + j] = hi;
            if constexpr (kSplit<T>) Ulo[i * MD + j] = lo;
        }
    if constexpr (!kSplit<T>) Ulo[0] = mk<T>(T(0), T(0));
}

// Packed coefficient pairs of a dense matrix (complex64, MD <= 4), from the
// hi / lo entries fill_matrix wrote.
template <typename T, typename I, int MD>
inline void fill_packed(DenseDirectArgs<T, I, MD> &a) {
    if constexpr (kPacked<T, MD>) {
        for (int k = 0; k < MD * MD; ++k) {
            const float hx = (float)a.U[k].x, hy = (float)a.U[k].y;
            const float lx = (float)a.Ulo[k].x, ly = (float)a.Ulo[k].y;
            a.Pk[4 * k + 0] = pk_host(lx, lx);
            a.Pk[4 * k + 1] = pk_host(-ly, ly);
            a.Pk[4 * k + 2] = pk_host(hx, hx);
            a.Pk[4 * k + 3] = pk_host(-hy, hy);
        }
    } else {
        a.Pk[0] = 0;
    }
}

template <typename T, int MD>
inline void fill_lam(v2<T> *lam, v2<T> *lamlo, const GatePlan &g) {
    for (int i = 0; i < MD; ++i) {
        v2<T> hi = mk<T>(T(1), T(0)), lo = mk<T>(T(0), T(0));
        if (i < g.D) split_coef<T>(g.lam[2 * i], g.lam[2 * i + 1], hi, lo);
        lam[i] = hi;
        if constexpr (kSplit<T>) lamlo[i] = lo;
    }
    if constexpr (!kSplit<T>) lamlo[0] = mk<T>(T(0), T(0));
}

template <typename F>
inline cudaError_t set_smem(F fn, size_t smem) {
    if (smem > 48 * 1024)
        return cudaFuncSetAttribute((const void *)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return cudaSuccess;
}

constexpr int kBlock = 256;

inline int grid_of(uint64_t work_items, uint64_t per_block, int sm_count, int occ) {
    const uint64_t need = (work_items + per_block - 1) / per_block;
    return (int)std::min<uint64_t>(need, (uint64_t)sm_count * std::max(occ, 1));
}

template <typename T, typename I, int MD, bool EX>
cudaError_t launch_dense(const GatePlan &g, void *psi, int sm_count, cudaStream_t s) {
    if (g.mode == Mode::Direct) {
        DenseDirectArgs<T, I, MD> a;
        a.psi = static_cast<v2<T> *>(psi);
        a.R = (I)g.R;
        a.base = (I)g.base_off;
        a.D = g.D;
        a.ex = expand_for<I>(g.ex);
        for (int j = 0; j < MD; ++j) a.off[j] = j < g.D ? (I)g.off[j] : 0;
        fill_matrix<T, MD>(a.U, a.Ulo, g);
        a.contig = 0;
        if constexpr (kVecPairs<T, MD>) {
            // a group of D == MD consecutive amplitudes (the gate acts on the
            // lowest qudits): relabel the local basis in address order (rows
            // and columns of U alike) and move amplitude pairs
            int perm[MD];
            bool contig = g.D == MD;
            for (int j = 0; j < MD && contig; ++j) {
                perm[j] = -1;
                for (int m = 0; m < MD; ++m)
                    if (g.off[m] == j) perm[j] = m;
                contig = perm[j] >= 0;
            }
            if (contig) {
                v2<T> U2[MD * MD], L2[MD * MD];
                for (int i = 0; i < MD; ++i)
                    for (int j = 0; j < MD; ++j) {
                        U2[i * MD + j] = a.U[perm[i] * MD + perm[j]];
                        L2[i * MD + j] = a.Ulo[perm[i] * MD + perm[j]];
                    }
                for (int k = 0; k < MD * MD; ++k) {
                    a.U[k] = U2[k];
                    a.Ulo[k] = L2[k];
                }
                for (int j = 0; j < MD; ++j) a.off[j] = (I)j;
                a.contig = 1;
            }
        }
        fill_packed<T, I, MD>(a);
        auto fn = k_dense_direct<T, I, MD, EX>;
        const int grid = grid_of(g.R, kBlock, sm_count, occupancy_blocks((const void *)fn, kBlock, 0));
        if (grid <= 0) return cudaSuccess;
        fn<<<grid, kBlock, 0, s>>>(a);
        return cudaGetLastError();
    }
    DenseTileArgs<T, I, MD> a;
    a.psi = static_cast<v2<T> *>(psi);
    a.D = g.D;
    fill_tilegeo<I>(a.t, g);
    for (int j = 0; j < MD; ++j) {
        a.offH[j] = j < (int)g.DH ? (I)g.offH[j] : 0;
        a.smoff[j] = j < g.D ? g.smoff[j] : 0;
    }
    fill_matrix<T, MD>(a.U, a.Ulo, g);
    auto fn = k_dense_tile<T, I, MD, EX>;
    const size_t smem = tile_smem_bytes<I>(g, sizeof(v2<T>));
    cudaError_t e = set_smem(fn, smem);
    if (e != cudaSuccess) return e;
    const int grid = grid_of(g.R_tiles, g.tpc, sm_count, occupancy_blocks((const void *)fn, kBlock, smem));
    if (grid <= 0) return cudaSuccess;
    fn<<<grid, kBlock, smem, s>>>(a);
    return cudaGetLastError();
}

// A permutation with phases whose moved members are few (a fused Toffoli
// rung moves 2 of its 16): only the active members enter the kernel, as a
// list of at most MD, so the kernel of that bound runs with its groups per
// thread (4 for two members): more loads in flight for the same groups.
template <typename T, typename I, int MD>
cudaError_t launch_mono_compact(const GatePlan &g, void *psi, int sm_count, cudaStream_t s) {
    MonoDirectArgs<T, I, MD> a;
    a.psi = static_cast<v2<T> *>(psi);
    a.R = (I)g.R;
    a.base = (I)g.base_off;
    a.ex = expand_for<I>(g.ex);
    int na = 0;
    uint32_t unit = 0;
    for (int i = 0; i < g.D && na < MD; ++i) {
        if (!((g.active >> i) & 1u)) continue;
        a.off[na] = (I)g.off[i];
        a.offsrc[na] = (I)g.off[g.src[i]];
        v2<T> hi, lo;
        split_coef<T>(g.lam[2 * i], g.lam[2 * i + 1], hi, lo);
        a.lam[na] = hi;
        if constexpr (kSplit<T>) a.lamlo[na] = lo;
        if ((g.unit >> i) & 1u) unit |= 1u << na;
        ++na;
    }
    for (int k = na; k < MD; ++k) {
        a.off[k] = 0;
        a.offsrc[k] = 0;
        a.lam[k] = mk<T>(T(1), T(0));
        if constexpr (kSplit<T>) a.lamlo[k] = mk<T>(T(0), T(0));
    }
    if constexpr (!kSplit<T>) a.lamlo[0] = mk<T>(T(0), T(0));
    a.active = (1u << na) - 1u;
    a.unit = unit;
    auto fn = k_mono_direct<T, I, MD>;
    const int grid = grid_of(g.R, kBlock, sm_count, occupancy_blocks((const void *)fn, kBlock, 0));
    if (grid <= 0) return cudaSuccess;
    fn<<<grid, kBlock, 0, s>>>(a);
    return cudaGetLastError();
}

template <typename T, typename I, int MD>
cudaError_t launch_mono(const GatePlan &g, void *psi, int sm_count, cudaStream_t s) {
    if (g.mode == Mode::Direct) {
        MonoDirectArgs<T, I, MD> a;
        a.psi = static_cast<v2<T> *>(psi);
        a.R = (I)g.R;
        a.base = (I)g.base_off;
        a.active = g.active;
        a.unit = g.unit;
        a.ex = expand_for<I>(g.ex);
        for (int i = 0; i < MD; ++i) {
            const bool in = i < g.D;
            a.off[i] = in ? (I)g.off[i] : 0;
            a.offsrc[i] = in ? (I)g.off[g.src[i]] : 0;
        }
        fill_lam<T, MD>(a.lam, a.lamlo, g);
        auto fn = k_mono_direct<T, I, MD>;
        const int grid = grid_of(g.R, kBlock, sm_count, occupancy_blocks((const void *)fn, kBlock, 0));
        if (grid <= 0) return cudaSuccess;
        fn<<<grid, kBlock, 0, s>>>(a);
        return cudaGetLastError();
    }
    MonoTileArgs<T, I, MD> a;
    a.psi = static_cast<v2<T> *>(psi);
    a.active = g.active;
    a.unit = g.unit;
    fill_tilegeo<I>(a.t, g);
    for (int i = 0; i < MD; ++i) {
        const bool in = i < g.D;
        a.offH[i] = i < (int)g.DH ? (I)g.offH[i] : 0;
        a.smoff[i] = in ? g.smoff[i] : 0;
        a.smoffsrc[i] = in ? g.smoff[g.src[i]] : 0;
    }
    fill_lam<T, MD>(a.lam, a.lamlo, g);
    auto fn = k_mono_tile<T, I, MD>;
    const size_t smem = tile_smem_bytes<I>(g, sizeof(v2<T>));
    cudaError_t e = set_smem(fn, smem);
    if (e != cudaSuccess) return e;
    const int grid = grid_of(g.R_tiles, g.tpc, sm_count, occupancy_blocks((const void *)fn, kBlock, smem));
    if (grid <= 0) return cudaSuccess;
    fn<<<grid, kBlock, smem, s>>>(a);
    return cudaGetLastError();
}

template <typename T, typename I, int MD, bool EX>
cudaError_t launch_dense_table(const GatePlan &g, void *psi, int sm_count, cudaStream_t s) {
    DenseTableArgs<T, I, MD> a;
    a.d.psi = static_cast<v2<T> *>(psi);
    a.d.R = (I)g.R;
    a.d.base = (I)g.base_off;
    a.d.D = g.D;
    a.d.contig = 0;
    a.d.ex = expand_for<I>(g.ex);
    for (int j = 0; j < MD; ++j) a.d.off[j] = j < g.D ? (I)g.off[j] : 0;
    fill_matrix<T, MD>(a.d.U, a.d.Ulo, g);
    fill_packed<T, I, MD>(a.d);
    if constexpr (sizeof(I) == 4) {
        a.divA = make_fastdiv32((uint32_t)g.tab_div);
        a.divT = make_fastdiv32((uint32_t)g.tab_size);
    } else {
        a.divA = make_fastdiv64(g.tab_div);
        a.divT = make_fastdiv64(g.tab_size);
    }
    a.carry = 0;
    for (int j = 0; j < MD; ++j) {
        const uint64_t o = j < g.D ? (uint64_t)g.off[j] : 0;
        a.oq[j] = (uint32_t)((o / g.tab_div) % g.tab_size);
        a.thr[j] = (I)(g.tab_div - o % g.tab_div);
        if (o % g.tab_div) a.carry = 1;
    }
    a.tsmask = (g.tab_size & (g.tab_size - 1)) == 0 ? (uint32_t)(g.tab_size - 1) : 0u;
    a.tab = static_cast<const typename TabEntry<T>::type *>(g.tab);
    auto fn = k_dense_table<T, I, MD, EX>;
    const int grid = grid_of(g.R, kBlock, sm_count, occupancy_blocks((const void *)fn, kBlock, 0));
    if (grid <= 0) return cudaSuccess;
    fn<<<grid, kBlock, 0, s>>>(a);
    return cudaGetLastError();
}

template <typename T, typename I>
cudaError_t launch_gate_ti(const GatePlan &g, void *psi, int sm_count, cudaStream_t s) {
    if (g.tab) {  // dense part + diagonal-run table (D <= 16, direct geometry)
        switch (g.D) {
            case 2: return launch_dense_table<T, I, 2, true>(g, psi, sm_count, s);
            case 3: return launch_dense_table<T, I, 3, true>(g, psi, sm_count, s);
            case 4: return launch_dense_table<T, I, 4, true>(g, psi, sm_count, s);
            default: break;
        }
        if (g.D <= 8) return launch_dense_table<T, I, 8, false>(g, psi, sm_count, s);
        return launch_dense_table<T, I, 16, false>(g, psi, sm_count, s);
    }
    if (g.kind == Kind::Mono) {
        if (g.mode == Mode::Direct && g.D > 4) {
            const int na = __builtin_popcount(g.active & (g.D >= 32 ? 0xffffffffu : ((1u << g.D) - 1u)));
            if (na <= 2) return launch_mono_compact<T, I, 2>(g, psi, sm_count, s);
            if (na <= 4) return launch_mono_compact<T, I, 4>(g, psi, sm_count, s);
        }
        if (g.D <= 2) return launch_mono<T, I, 2>(g, psi, sm_count, s);
        if (g.D <= 4) return launch_mono<T, I, 4>(g, psi, sm_count, s);
        if (g.D <= 8) return launch_mono<T, I, 8>(g, psi, sm_count, s);
        if (g.D <= 16) return launch_mono<T, I, 16>(g, psi, sm_count, s);
        return launch_mono<T, I, 32>(g, psi, sm_count, s);
    }
    switch (g.D) {
        case 2: return launch_dense<T, I, 2, true>(g, psi, sm_count, s);
        case 3: return launch_dense<T, I, 3, true>(g, psi, sm_count, s);
        case 4: return launch_dense<T, I, 4, true>(g, psi, sm_count, s);
        case 5: return launch_dense<T, I, 5, true>(g, psi, sm_count, s);
        case 6: return launch_dense<T, I, 6, true>(g, psi, sm_count, s);
        case 8: return launch_dense<T, I, 8, true>(g, psi, sm_count, s);
        case 9: return launch_dense<T, I, 9, true>(g, psi, sm_count, s);
        default: break;
    }
    if (g.D <= 16) return launch_dense<T, I, 16, false>(g, psi, sm_count, s);
    return launch_dense<T, I, 32, false>(g, psi, sm_count, s);
}

template <typename T>
cudaError_t launch_gate_t(const GatePlan &g, void *psi, int sm_count, cudaStream_t s) {
    if (!wide_index(g)) return launch_gate_ti<T, uint32_t>(g, psi, sm_count, s);
    return launch_gate_ti<T, uint64_t>(g, psi, sm_count, s);
}

}  // namespace qd
