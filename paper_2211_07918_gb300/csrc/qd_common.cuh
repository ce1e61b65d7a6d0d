// Shared device/host definitions of libqudit: complex vector types, invariant
// integer division, and the mixed-radix "insert digits" expansion that maps a
// compressed group index onto the flat amplitude index.
//
// Mixed-radix convention (QuDiet Sec. 3.2): qudit 0 is the least significant
// digit, s_q = prod_{p<q} d_p, amplitude index i = sum_q x_q s_q.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace qd {

constexpr int kMaxIns = 16;   // targets + controls a gate may remove from the index space
constexpr int kMaxD = 32;     // largest target-space dimension of a per-gate kernel
constexpr int kMaxBlockD = 64;  // largest dimension of a fused block (tensor-core kernel)

template <typename T> struct V2;
template <> struct V2<float> { using type = float2; };
template <> struct V2<double> { using type = double2; };
template <typename T> using v2 = typename V2<T>::type;

template <typename T>
__host__ __device__ __forceinline__ v2<T> mk(T a, T b) { v2<T> r; r.x = a; r.y = b; return r; }

// ---------------------------------------------------------------------------
// Division by a run-time invariant divisor (Granlund & Montgomery, "Division
// by invariant integers using multiplication", PLDI 1994, Thm 4.2): for
// 0 <= n < 2^P and l = ceil(log2 d), m = ceil(2^(P+l) / d) gives
// floor(n / d) = floor(m n / 2^(P+l)).
// ---------------------------------------------------------------------------

// Dividends below 2^41 (N <= 2^40 amplitudes); m < 2^42; 128-bit product.
struct FastDiv64 {
    uint64_t d;
    uint64_t m;
    uint32_t sh;
    uint32_t p2;  // log2(d) + 1 when d is a power of two (a shift), else 0
};

inline FastDiv64 make_fastdiv64(uint64_t d) {
    FastDiv64 f{};
    f.d = d;
    uint32_t l = 0;
    while ((uint64_t(1) << l) < d) ++l;
    const uint32_t P = 41;
    f.sh = P + l;
    // m = ceil(2^(P+l) / d) computed with 128-bit arithmetic
    unsigned __int128 num = (unsigned __int128)1 << f.sh;
    unsigned __int128 m = (num + d - 1) / d;
    f.m = (uint64_t)m;
    f.p2 = (d & (d - 1)) == 0 ? l + 1 : 0;
    return f;
}

__host__ __device__ __forceinline__ uint64_t mulhi64(uint64_t a, uint64_t b) {
#ifdef __CUDA_ARCH__
    return __umul64hi(a, b);
#else
    return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

// A power-of-two divisor (every stride of a register of qubits and
// ququarts) is a shift; the test is uniform across a launch.
__host__ __device__ __forceinline__ uint64_t fdiv(uint64_t n, const FastDiv64 &f) {
    if (f.p2) return n >> (f.p2 - 1);
    const uint64_t hi = mulhi64(n, f.m);
    const uint64_t lo = n * f.m;
    return f.sh >= 64 ? (hi >> (f.sh - 64)) : ((hi << (64 - f.sh)) | (lo >> f.sh));
}

// Dividends below 2^31; m < 2^32.
struct FastDiv32 {
    uint32_t d;
    uint32_t m;
    uint32_t sh;
    uint32_t pad;
};

inline FastDiv32 make_fastdiv32(uint32_t d) {
    FastDiv32 f{};
    f.d = d;
    uint32_t l = 0;
    while ((uint64_t(1) << l) < d) ++l;
    f.sh = 31 + l;
    uint64_t num = uint64_t(1) << f.sh;
    f.m = (uint32_t)((num + d - 1) / d);
    return f;
}

__host__ __device__ __forceinline__ uint32_t fdiv(uint32_t n, const FastDiv32 &f) {
    return (uint32_t)(((uint64_t)n * f.m) >> f.sh);
}

// ---------------------------------------------------------------------------
// Insert-digit expansion.  A gate removes some qudits from the index space
// (its targets, whose digits the group enumerates, and its controls, whose
// digits are fixed).  Groups are numbered by the compressed index r over the
// remaining qudits.  Inserting a zero digit at each removed qudit, in
// ascending stride order, maps r to the flat index of the group's base:
//   lo = r mod s_p;  r = (r div s_p) * (s_p d_p) + lo.
// After the first k insertions the digits below the k-th removed qudit are in
// the flat layout, so s_p is always the flat stride.
// ---------------------------------------------------------------------------
struct Expand64 {
    int32_t n;
    int32_t pad;
    FastDiv64 div[kMaxIns];
    uint64_t span[kMaxIns];
};

// The loops run over the insertions actually present (e.n is uniform across
// a launch): a loop unrolled to kMaxIns with a predicate per step would issue
// every predicated-off step as well.
__host__ __device__ __forceinline__ uint64_t expand(uint64_t r, const Expand64 &e) {
#pragma unroll 1
    for (int k = 0; k < e.n; ++k) {
        const uint64_t q = fdiv(r, e.div[k]);
        const uint64_t lo = r - q * e.div[k].d;
        r = q * e.span[k] + lo;
    }
    return r;
}

struct Expand32 {
    int32_t n;
    int32_t pad;
    FastDiv32 div[kMaxIns];
    uint32_t span[kMaxIns];
};

__host__ __device__ __forceinline__ uint32_t expand(uint32_t r, const Expand32 &e) {
#pragma unroll 1
    for (int k = 0; k < e.n; ++k) {
        const uint32_t q = fdiv(r, e.div[k]);
        const uint32_t lo = r - q * e.div[k].d;
        r = q * e.span[k] + lo;
    }
    return r;
}

// Index width of a launch: 32-bit arithmetic when every index of the register
// is below 2^31 (FastDiv32's dividend bound), 64-bit otherwise.
template <typename I> struct ExpandOf;
template <> struct ExpandOf<uint32_t> { using type = Expand32; };
template <> struct ExpandOf<uint64_t> { using type = Expand64; };

template <typename I> using ExpandT = typename ExpandOf<I>::type;

inline Expand32 narrow(const Expand64 &e) {
    Expand32 r{};
    r.n = e.n;
    for (int k = 0; k < e.n; ++k) {
        r.div[k] = make_fastdiv32((uint32_t)e.div[k].d);
        r.span[k] = (uint32_t)e.span[k];
    }
    return r;
}

}  // namespace qd
