// The paper's own execution model (QuDiet Sec. 3.5 Moment, Sec. 3.6
// OperatorFlow), kept as an in-repo comparison with the in-place stride
// apply: gates are packed into moments, every moment becomes the full
// N x N Kronecker-product operator (identity on the qudits no gate of the
// moment touches), the moment operators are multiplied from the last moment
// down to the first (GEMM chain) and the product is applied to the initial
// state (GEMV).  All arithmetic is complex128 (FP64) on the device; the
// operators take N^2 entries each, so this path is for small registers only.
//
// Moment packing (Sec. 3.5): a gate goes into the first moment after the last
// moment holding a gate on any of its qudits (targets and controls), which is
// the result of the paper's rule of replacing identities of immediate
// predecessor moments until a gate or the initial state is met.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>

#include <cuda_runtime.h>

#include "qd_kron.h"

namespace qd {

namespace {

constexpr int kKronMaxActing = kKronMaxQudits;  // acting qudits of one gate (targets + controls)

struct KronGate {
    int32_t nq;                       // acting qudits
    int32_t q[kKronMaxActing];        // acting qudits, first = most significant local digit
    int32_t Dact;
    int64_t moff;                     // offset of its Dact x Dact matrix in the matrix pool (complex entries)
};

// K[i][j] = prod over the moment's gates of M_g[loc_g(i)][loc_g(j)] when the
// digits of i and j agree on every qudit no gate of the moment acts on, else 0.
__global__ void k_kron_moment(double2 *__restrict__ K, int64_t N, int32_t n, const int32_t *__restrict__ dims,
                              uint64_t free_mask, const KronGate *__restrict__ gates, int32_t ngates,
                              const double2 *__restrict__ pool) {
    const int64_t total = N * N;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / N, j = e - (e / N) * N;
        int32_t di[kKronMaxQudits], dj[kKronMaxQudits];
        int64_t a = i, b = j;
        bool same = true;
        for (int q = 0; q < n; ++q) {
            di[q] = (int32_t)(a % dims[q]);
            dj[q] = (int32_t)(b % dims[q]);
            a /= dims[q];
            b /= dims[q];
            if (((free_mask >> q) & 1u) && di[q] != dj[q]) same = false;
        }
        double2 v = make_double2(same ? 1.0 : 0.0, 0.0);
        for (int g = 0; g < ngates && same; ++g) {
            const KronGate &kg = gates[g];
            int32_t li = 0, lj = 0;
            for (int m = 0; m < kg.nq; ++m) {
                li = li * dims[kg.q[m]] + di[kg.q[m]];
                lj = lj * dims[kg.q[m]] + dj[kg.q[m]];
            }
            const double2 u = pool[kg.moff + (int64_t)li * kg.Dact + lj];
            v = make_double2(v.x * u.x - v.y * u.y, v.x * u.y + v.y * u.x);
        }
        K[e] = v;
    }
}

// C = A B for N x N complex128 row-major matrices: 16 x 16 output tiles, one
// output per thread, K staged through shared memory in 16-wide slabs.
__global__ void k_zgemm(const double2 *__restrict__ A, const double2 *__restrict__ B, double2 *__restrict__ C,
                        int64_t N) {
    __shared__ double2 As[16][16], Bs[16][16];
    const int64_t row = (int64_t)blockIdx.y * 16 + threadIdx.y, col = (int64_t)blockIdx.x * 16 + threadIdx.x;
    double re = 0.0, im = 0.0;
    for (int64_t k0 = 0; k0 < N; k0 += 16) {
        As[threadIdx.y][threadIdx.x] = (row < N && k0 + threadIdx.x < N) ? A[row * N + k0 + threadIdx.x]
                                                                         : make_double2(0.0, 0.0);
        Bs[threadIdx.y][threadIdx.x] = (k0 + threadIdx.y < N && col < N) ? B[(k0 + threadIdx.y) * N + col]
                                                                         : make_double2(0.0, 0.0);
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const double2 a = As[threadIdx.y][k], b = Bs[k][threadIdx.x];
            re = fma(a.x, b.x, fma(-a.y, b.y, re));
            im = fma(a.x, b.y, fma(a.y, b.x, im));
        }
        __syncthreads();
    }
    if (row < N && col < N) C[row * N + col] = make_double2(re, im);
}

// y = A x (complex128), one row per thread.
__global__ void k_zgemv(const double2 *__restrict__ A, const double2 *__restrict__ x, double2 *__restrict__ y,
                        int64_t N) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= N) return;
    double re = 0.0, im = 0.0;
    for (int64_t k = 0; k < N; ++k) {
        const double2 a = A[r * N + k], b = x[k];
        re = fma(a.x, b.x, fma(-a.y, b.y, re));
        im = fma(a.x, b.y, fma(a.y, b.x, im));
    }
    y[r] = make_double2(re, im);
}

__global__ void k_widen(const float2 *__restrict__ in, double2 *__restrict__ out, int64_t N) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) out[i] = make_double2((double)in[i].x, (double)in[i].y);
}

__global__ void k_narrow(const double2 *__restrict__ in, float2 *__restrict__ out, int64_t N) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) out[i] = make_float2((float)in[i].x, (float)in[i].y);
}

}  // namespace

std::vector<int> pack_moments(int n, const std::vector<FuseGate> &gates, int *n_moments) {
    std::vector<int> last(n, -1), moment(gates.size(), 0);
    int count = 0;
    for (size_t g = 0; g < gates.size(); ++g) {
        int m = 0;
        for (int q : gates[g].acting) m = std::max(m, last[q] + 1);
        moment[g] = m;
        for (int q : gates[g].acting) last[q] = m;
        count = std::max(count, m + 1);
    }
    if (n_moments) *n_moments = count;
    return moment;
}

cudaError_t run_moments(void *psi, int prec, int64_t N, int n, const int32_t *dims,
                        const std::vector<FuseGate> &gates, int *n_moments, cudaStream_t s) {
    int nm = 0;
    const std::vector<int> moment = pack_moments(n, gates, &nm);
    if (n_moments) *n_moments = nm;
    const size_t NN = (size_t)N * (size_t)N;
    double2 *acc = nullptr, *K = nullptr, *tmp = nullptr, *x = nullptr, *y = nullptr, *pool = nullptr;
    int32_t *ddims = nullptr;
    KronGate *dgates = nullptr;
    cudaError_t e = cudaSuccess;
    auto done = [&](cudaError_t r) {
        cudaStreamSynchronize(s);
        for (void *p : {(void *)acc, (void *)K, (void *)tmp, (void *)x, (void *)y, (void *)pool, (void *)ddims,
                        (void *)dgates})
            if (p) cudaFree(p);
        return r;
    };
    // matrix pool and per-moment gate descriptors (host), uploaded once
    std::vector<double2> hpool;
    std::vector<KronGate> hg(gates.size());
    for (size_t g = 0; g < gates.size(); ++g) {
        KronGate &kg = hg[g];
        std::memset(&kg, 0, sizeof(kg));
        kg.nq = (int32_t)gates[g].acting.size();
        for (int m = 0; m < kg.nq; ++m) kg.q[m] = gates[g].acting[m];
        kg.Dact = gates[g].Dact;
        kg.moff = (int64_t)hpool.size();
        for (int64_t k = 0; k < (int64_t)gates[g].Dact * gates[g].Dact; ++k)
            hpool.push_back(make_double2(gates[g].M[2 * k], gates[g].M[2 * k + 1]));
    }
    // gates grouped by moment, in moment order
    std::vector<KronGate> byMoment;
    std::vector<int> start(nm + 1, 0);
    for (int m = 0; m < nm; ++m) {
        start[m] = (int)byMoment.size();
        for (size_t g = 0; g < gates.size(); ++g)
            if (moment[g] == m) byMoment.push_back(hg[g]);
    }
    start[nm] = (int)byMoment.size();
    if ((e = cudaMalloc(&x, sizeof(double2) * N)) != cudaSuccess) return done(e);
    if ((e = cudaMalloc(&y, sizeof(double2) * N)) != cudaSuccess) return done(e);
    if (prec == 1) {
        k_widen<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(static_cast<const float2 *>(psi), x, N);
    } else {
        e = cudaMemcpyAsync(x, psi, sizeof(double2) * N, cudaMemcpyDeviceToDevice, s);
    }
    if (e != cudaSuccess || (e = cudaGetLastError()) != cudaSuccess) return done(e);
    if (nm > 0) {
        if ((e = cudaMalloc(&acc, sizeof(double2) * NN)) != cudaSuccess) return done(e);
        if ((e = cudaMalloc(&K, sizeof(double2) * NN)) != cudaSuccess) return done(e);
        if ((e = cudaMalloc(&tmp, sizeof(double2) * NN)) != cudaSuccess) return done(e);
        if ((e = cudaMalloc(&pool, sizeof(double2) * std::max<size_t>(hpool.size(), 1))) != cudaSuccess) return done(e);
        if ((e = cudaMalloc(&ddims, sizeof(int32_t) * n)) != cudaSuccess) return done(e);
        if ((e = cudaMalloc(&dgates, sizeof(KronGate) * std::max<size_t>(byMoment.size(), 1))) != cudaSuccess)
            return done(e);
        if (!hpool.empty() &&
            (e = cudaMemcpyAsync(pool, hpool.data(), sizeof(double2) * hpool.size(), cudaMemcpyHostToDevice, s)) !=
                cudaSuccess)
            return done(e);
        if ((e = cudaMemcpyAsync(ddims, dims, sizeof(int32_t) * n, cudaMemcpyHostToDevice, s)) != cudaSuccess)
            return done(e);
        if (!byMoment.empty() && (e = cudaMemcpyAsync(dgates, byMoment.data(), sizeof(KronGate) * byMoment.size(),
                                                      cudaMemcpyHostToDevice, s)) != cudaSuccess)
            return done(e);
        const unsigned kgrid = (unsigned)std::min<size_t>((NN + 255) / 256, 65535u * 8);
        const dim3 gblk(16, 16), ggrid((unsigned)((N + 15) / 16), (unsigned)((N + 15) / 16));
        // OperatorFlow evaluated from the last moment down to the first
        for (int m = nm - 1; m >= 0; --m) {
            uint64_t free_mask = (n >= 64) ? ~0ull : ((1ull << n) - 1);
            for (int g = start[m]; g < start[m + 1]; ++g)
                for (int k = 0; k < byMoment[g].nq; ++k) free_mask &= ~(1ull << byMoment[g].q[k]);
            double2 *dst = (m == nm - 1) ? acc : K;
            k_kron_moment<<<kgrid, 256, 0, s>>>(dst, N, n, ddims, free_mask, dgates + start[m], start[m + 1] - start[m],
                                                pool);
            if ((e = cudaGetLastError()) != cudaSuccess) return done(e);
            if (m < nm - 1) {
                k_zgemm<<<ggrid, gblk, 0, s>>>(acc, K, tmp, N);
                if ((e = cudaGetLastError()) != cudaSuccess) return done(e);
                std::swap(acc, tmp);
            }
        }
        k_zgemv<<<(unsigned)((N + 127) / 128), 128, 0, s>>>(acc, x, y, N);
        if ((e = cudaGetLastError()) != cudaSuccess) return done(e);
    } else {
        std::swap(x, y);
    }
    if (prec == 1) {
        k_narrow<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(y, static_cast<float2 *>(psi), N);
        e = cudaGetLastError();
    } else {
        e = cudaMemcpyAsync(psi, y, sizeof(double2) * N, cudaMemcpyDeviceToDevice, s);
    }
    return done(e);
}

}  // namespace qd
