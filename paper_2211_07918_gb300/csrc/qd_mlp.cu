// Learned cost model: a multilayer perceptron 12 -> 64 -> 64 -> 64 -> 1 with
// ReLU hidden units, predicting log(launch time in microseconds) from the
// launch features of a candidate fused block or gate (qd_fuse.h).  The
// planner evaluates every candidate segment of a circuit in one batched
// inference launch and runs its segmentation search on the predictions.
//
// Training runs on the GPU with these kernels only: forward (FP32 master
// weights, activations kept for the backward pass), mean-squared-error loss,
// backward (per-block partial gradients, then a fixed-order reduction), and
// Adam.  Inference uses FP16 copies of the weights with FP32 accumulation.
//
// Parameter vector layout (floats): W1 (12x64, row = input), b1 (64),
// W2 (64x64), b2 (64), W3 (64x64), b3 (64), W4 (64), b4 (1); 9,217 values.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "../../include/qudit.h"
#include "qd_mlp.h"

namespace qd {
int set_last_error(int code, const char *msg);
}

namespace {

constexpr int IN = qd::kMlpIn, H = qd::kMlpHidden;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + IN * H, OFF_W2 = OFF_B1 + H, OFF_B2 = OFF_W2 + H * H,
              OFF_W3 = OFF_B2 + H, OFF_B3 = OFF_W3 + H * H, OFF_W4 = OFF_B3 + H, OFF_B4 = OFF_W4 + H,
              NPARAM = OFF_B4 + 1;
static_assert(NPARAM == qd::kMlpParams, "parameter count");

constexpr int kTile = 32;  // samples per CTA

// Forward pass for a tile of samples: thread j owns hidden unit j (64
// threads); inputs, weights and activations in shared memory.  W is FP32 or
// FP16.  Saves pre-activations (z1..z3) when `save` is set.
template <typename W>
__global__ void __launch_bounds__(H) k_mlp_forward(const W *__restrict__ p, const float *__restrict__ x, int n,
                                                   float *__restrict__ y, float *__restrict__ save) {
    __shared__ float in[kTile][IN];
    __shared__ float h[2][kTile][H];
    const int j = threadIdx.x;
    const int s0 = blockIdx.x * kTile;
    for (int e = j; e < kTile * IN; e += H) {
        const int s = e / IN, f = e % IN;
        in[s][f] = (s0 + s < n) ? x[(size_t)(s0 + s) * IN + f] : 0.f;
    }
    __syncthreads();
    auto wv = [&](int idx) { return (float)p[idx]; };
    // layer 1
    for (int s = 0; s < kTile; ++s) {
        float z = wv(OFF_B1 + j);
        for (int i = 0; i < IN; ++i) z = fmaf(in[s][i], wv(OFF_W1 + i * H + j), z);
        if (save && s0 + s < n) save[((size_t)(s0 + s) * 3 + 0) * H + j] = z;
        h[0][s][j] = fmaxf(z, 0.f);
    }
    __syncthreads();
    // layers 2 and 3
    for (int l = 0; l < 2; ++l) {
        const int ow = l == 0 ? OFF_W2 : OFF_W3, ob = l == 0 ? OFF_B2 : OFF_B3;
        const int src = l & 1, dst = src ^ 1;
        for (int s = 0; s < kTile; ++s) {
            float z = wv(ob + j);
            for (int i = 0; i < H; ++i) z = fmaf(h[src][s][i], wv(ow + i * H + j), z);
            if (save && s0 + s < n) save[((size_t)(s0 + s) * 3 + 1 + l) * H + j] = z;
            h[dst][s][j] = fmaxf(z, 0.f);
        }
        __syncthreads();
    }
    // output: h[0] holds layer-3 activations
    if (j < kTile && s0 + j < n) {
        float z = wv(OFF_B4);
        for (int i = 0; i < H; ++i) z = fmaf(h[0][j][i], wv(OFF_W4 + i), z);
        y[s0 + j] = z;
    }
}

// g[s] = 2 (y[s] - t[s]) / n ; loss partials per block
__global__ void k_mse(const float *__restrict__ y, const float *__restrict__ t, int n, float *__restrict__ g,
                      double *__restrict__ loss) {
    __shared__ double sh[256];
    double acc = 0.0;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        const float d = y[s] - t[s];
        g[s] = 2.f * d / (float)n;
        acc += (double)d * d;
    }
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) loss[blockIdx.x] = sh[0];
}

// Backward pass for a tile of samples, writing this block's gradient partial
// (NPARAM floats) to part[blockIdx.x].  Uses the pre-activations saved by the
// forward pass; recomputes activations from them.
__global__ void __launch_bounds__(H) k_mlp_backward(const float *__restrict__ p, const float *__restrict__ x, int n,
                                                    const float *__restrict__ save, const float *__restrict__ g,
                                                    float *__restrict__ part) {
    __shared__ float in[kTile][IN];
    __shared__ float a[3][kTile][H];   // activations after each hidden layer
    __shared__ float d[2][kTile][H];   // dL/dz of the current and previous layer
    __shared__ float go[kTile];
    const int j = threadIdx.x;
    const int s0 = blockIdx.x * kTile;
    float *gp = part + (size_t)blockIdx.x * NPARAM;
    for (int e = j; e < kTile * IN; e += H) {
        const int s = e / IN, f = e % IN;
        in[s][f] = (s0 + s < n) ? x[(size_t)(s0 + s) * IN + f] : 0.f;
    }
    for (int s = 0; s < kTile; ++s)
        for (int l = 0; l < 3; ++l)
            a[l][s][j] = (s0 + s < n) ? fmaxf(save[((size_t)(s0 + s) * 3 + l) * H + j], 0.f) : 0.f;
    if (j < kTile) go[j] = (s0 + j < n) ? g[s0 + j] : 0.f;
    __syncthreads();
    // output layer: dW4[j] = sum_s a3[s][j] go[s]; db4 = sum_s go[s]
    {
        float acc = 0.f;
        for (int s = 0; s < kTile; ++s) acc = fmaf(a[2][s][j], go[s], acc);
        gp[OFF_W4 + j] = acc;
        if (j == 0) {
            float b = 0.f;
            for (int s = 0; s < kTile; ++s) b += go[s];
            gp[OFF_B4] = b;
        }
        // dz3 = go * W4[j] * relu'(z3)
        for (int s = 0; s < kTile; ++s) d[0][s][j] = a[2][s][j] > 0.f ? go[s] * p[OFF_W4 + j] : 0.f;
    }
    __syncthreads();
    // hidden layers 3 and 2: weights W3 (from a2), W2 (from a1)
    for (int l = 2; l >= 1; --l) {
        const int ow = l == 2 ? OFF_W3 : OFF_W2, ob = l == 2 ? OFF_B3 : OFF_B2;
        const int cur = (2 - l) & 1, nxt = cur ^ 1;
        // dW[i][j] for this thread's column j, i over the 64 inputs a[l-1]
        for (int i = 0; i < H; ++i) {
            float acc = 0.f;
            for (int s = 0; s < kTile; ++s) acc = fmaf(a[l - 1][s][i], d[cur][s][j], acc);
            gp[ow + i * H + j] = acc;
        }
        {
            float b = 0.f;
            for (int s = 0; s < kTile; ++s) b += d[cur][s][j];
            gp[ob + j] = b;
        }
        // dz of the layer below (unit j): sum_k d[cur][s][k] W[j][k] * relu'(z)
        for (int s = 0; s < kTile; ++s) {
            float acc = 0.f;
            for (int k = 0; k < H; ++k) acc = fmaf(d[cur][s][k], p[ow + j * H + k], acc);
            d[nxt][s][j] = a[l - 1][s][j] > 0.f ? acc : 0.f;
        }
        __syncthreads();
    }
    // first layer: dz1 sits in d[0] after two swaps
    for (int i = 0; i < IN; ++i) {
        float acc = 0.f;
        for (int s = 0; s < kTile; ++s) acc = fmaf(in[s][i], d[0][s][j], acc);
        gp[OFF_W1 + i * H + j] = acc;
    }
    {
        float b = 0.f;
        for (int s = 0; s < kTile; ++s) b += d[0][s][j];
        gp[OFF_B1 + j] = b;
    }
}

// grad[k] = sum over blocks of part[b][k], fixed order
__global__ void k_reduce_grad(const float *__restrict__ part, int nb, float *__restrict__ grad) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < NPARAM; k += gridDim.x * blockDim.x) {
        float acc = 0.f;
        for (int b = 0; b < nb; ++b) acc += part[(size_t)b * NPARAM + k];
        grad[k] = acc;
    }
}

// Adam (Kingma & Ba, 2015) with bias correction, then the FP16 inference copy.
__global__ void k_adam(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, __half *__restrict__ p16, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < NPARAM; k += gridDim.x * blockDim.x) {
        const float gk = g[k];
        const float mk = b1 * m[k] + (1.f - b1) * gk;
        const float vk = b2 * v[k] + (1.f - b2) * gk * gk;
        m[k] = mk;
        v[k] = vk;
        const float upd = lr * (mk / c1) / (sqrtf(vk / c2) + eps);
        p[k] -= upd;
        p16[k] = __float2half_rn(p[k]);
    }
}

__global__ void k_to_half(const float *__restrict__ p, __half *__restrict__ p16) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < NPARAM; k += gridDim.x * blockDim.x)
        p16[k] = __float2half_rn(p[k]);
}

}  // namespace

struct qd_model {
    float *p = nullptr;    // device FP32 master weights
    __half *p16 = nullptr; // device FP16 inference weights
    float *m = nullptr, *v = nullptr, *grad = nullptr;
    float mean[IN] = {}, stdv[IN] = {};
    float y_mean = 0.f, y_std = 1.f;
    int64_t steps = 0;
    ~qd_model() {
        cudaFree(p);
        cudaFree(p16);
        cudaFree(m);
        cudaFree(v);
        cudaFree(grad);
    }
};

namespace {
int mfail(int code, const std::string &msg) { return qd::set_last_error(code, msg.c_str()); }
#define MLP_CUDA(call)                                                                                      \
    do {                                                                                                    \
        cudaError_t _e = (call);                                                                            \
        if (_e != cudaSuccess) return mfail(QD_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(_e)); \
    } while (0)

struct DevBuf {
    void *ptr = nullptr;
    ~DevBuf() { cudaFree(ptr); }
    template <typename T> T *as() { return static_cast<T *>(ptr); }
};

// Normalised copy of features (host) for the model.
std::vector<float> normalise(const qd_model *m, const float *X, int n) {
    std::vector<float> out((size_t)n * IN);
    for (int s = 0; s < n; ++s)
        for (int f = 0; f < IN; ++f) out[(size_t)s * IN + f] = (X[(size_t)s * IN + f] - m->mean[f]) / m->stdv[f];
    return out;
}
}  // namespace

extern "C" {

int qd_model_create(qd_model **out) {
    if (!out) return mfail(QD_ERR_ARG, "null output");
    qd_model *m = new qd_model();
    if (cudaMalloc(&m->p, NPARAM * 4) != cudaSuccess || cudaMalloc(&m->p16, NPARAM * 2) != cudaSuccess ||
        cudaMalloc(&m->m, NPARAM * 4) != cudaSuccess || cudaMalloc(&m->v, NPARAM * 4) != cudaSuccess ||
        cudaMalloc(&m->grad, NPARAM * 4) != cudaSuccess) {
        cudaGetLastError();
        delete m;
        return mfail(QD_ERR_OOM, "model allocation failed");
    }
    cudaMemset(m->m, 0, NPARAM * 4);
    cudaMemset(m->v, 0, NPARAM * 4);
    for (int f = 0; f < IN; ++f) m->stdv[f] = 1.f;
    *out = m;
    return QD_OK;
}

int qd_model_destroy(qd_model *m) {
    delete m;
    return QD_OK;
}

int qd_model_set(qd_model *m, const float *params, const float *feat_mean, const float *feat_std, float y_mean,
                 float y_std) {
    if (!m || !params) return mfail(QD_ERR_ARG, "null model or parameters");
    MLP_CUDA(cudaMemcpy(m->p, params, NPARAM * 4, cudaMemcpyHostToDevice));
    k_to_half<<<8, 256>>>(m->p, m->p16);
    MLP_CUDA(cudaGetLastError());
    MLP_CUDA(cudaDeviceSynchronize());
    for (int f = 0; f < IN; ++f) {
        m->mean[f] = feat_mean ? feat_mean[f] : 0.f;
        m->stdv[f] = feat_std ? (feat_std[f] > 0.f ? feat_std[f] : 1.f) : 1.f;
    }
    m->y_mean = y_mean;
    m->y_std = y_std > 0.f ? y_std : 1.f;
    MLP_CUDA(cudaMemset(m->m, 0, NPARAM * 4));
    MLP_CUDA(cudaMemset(m->v, 0, NPARAM * 4));
    m->steps = 0;
    return QD_OK;
}

int qd_model_get(const qd_model *m, float *params, float *feat_mean, float *feat_std, float *y_mean, float *y_std) {
    if (!m) return mfail(QD_ERR_ARG, "null model");
    if (params) MLP_CUDA(cudaMemcpy(params, m->p, NPARAM * 4, cudaMemcpyDeviceToHost));
    for (int f = 0; f < IN; ++f) {
        if (feat_mean) feat_mean[f] = m->mean[f];
        if (feat_std) feat_std[f] = m->stdv[f];
    }
    if (y_mean) *y_mean = m->y_mean;
    if (y_std) *y_std = m->y_std;
    return QD_OK;
}

// Raw network on already-normalised inputs: y[n] (FP32 weights when fp16 == 0).
int qd_model_forward_raw(qd_model *m, const float *Xn, int32_t n, float *y, int32_t fp16) {
    if (!m || !Xn || !y || n < 0) return mfail(QD_ERR_ARG, "bad forward arguments");
    if (n == 0) return QD_OK;
    DevBuf dx, dy;
    MLP_CUDA(cudaMalloc(&dx.ptr, (size_t)n * IN * 4));
    MLP_CUDA(cudaMalloc(&dy.ptr, (size_t)n * 4));
    MLP_CUDA(cudaMemcpy(dx.ptr, Xn, (size_t)n * IN * 4, cudaMemcpyHostToDevice));
    const int nb = (n + kTile - 1) / kTile;
    if (fp16) k_mlp_forward<__half><<<nb, H>>>(m->p16, dx.as<float>(), n, dy.as<float>(), nullptr);
    else k_mlp_forward<float><<<nb, H>>>(m->p, dx.as<float>(), n, dy.as<float>(), nullptr);
    MLP_CUDA(cudaGetLastError());
    MLP_CUDA(cudaMemcpy(y, dy.ptr, (size_t)n * 4, cudaMemcpyDeviceToHost));
    return QD_OK;
}

// Loss (mean squared error) and its gradient for already-normalised data,
// computed by the forward and backward kernels with FP32 weights.
int qd_model_grad_raw(qd_model *m, const float *Xn, const float *t, int32_t n, double *loss, float *grad) {
    if (!m || !Xn || !t || n < 1) return mfail(QD_ERR_ARG, "bad gradient arguments");
    const int nb = (n + kTile - 1) / kTile;
    DevBuf dx, dt, dy, dg, dsave, dpart, dloss;
    MLP_CUDA(cudaMalloc(&dx.ptr, (size_t)n * IN * 4));
    MLP_CUDA(cudaMalloc(&dt.ptr, (size_t)n * 4));
    MLP_CUDA(cudaMalloc(&dy.ptr, (size_t)n * 4));
    MLP_CUDA(cudaMalloc(&dg.ptr, (size_t)n * 4));
    MLP_CUDA(cudaMalloc(&dsave.ptr, (size_t)n * 3 * H * 4));
    MLP_CUDA(cudaMalloc(&dpart.ptr, (size_t)nb * NPARAM * 4));
    MLP_CUDA(cudaMalloc(&dloss.ptr, 64 * 8));
    MLP_CUDA(cudaMemcpy(dx.ptr, Xn, (size_t)n * IN * 4, cudaMemcpyHostToDevice));
    MLP_CUDA(cudaMemcpy(dt.ptr, t, (size_t)n * 4, cudaMemcpyHostToDevice));
    k_mlp_forward<float><<<nb, H>>>(m->p, dx.as<float>(), n, dy.as<float>(), dsave.as<float>());
    k_mse<<<64, 256>>>(dy.as<float>(), dt.as<float>(), n, dg.as<float>(), dloss.as<double>());
    k_mlp_backward<<<nb, H>>>(m->p, dx.as<float>(), n, dsave.as<float>(), dg.as<float>(), dpart.as<float>());
    k_reduce_grad<<<(NPARAM + 255) / 256, 256>>>(dpart.as<float>(), nb, m->grad);
    MLP_CUDA(cudaGetLastError());
    if (grad) MLP_CUDA(cudaMemcpy(grad, m->grad, NPARAM * 4, cudaMemcpyDeviceToHost));
    double lp[64];
    MLP_CUDA(cudaMemcpy(lp, dloss.ptr, sizeof(lp), cudaMemcpyDeviceToHost));
    double s = 0.0;
    for (double v : lp) s += v;
    if (loss) *loss = s / n;
    return QD_OK;
}

int qd_model_train(qd_model *m, const float *X, const float *y, int32_t n, int32_t epochs, int32_t batch, float lr,
                   uint64_t seed, double *final_loss) {
    if (!m || !X || !y || n < 2 || epochs < 1 || batch < 1) return mfail(QD_ERR_ARG, "bad training arguments");
    // feature and target statistics
    for (int f = 0; f < IN; ++f) {
        double mu = 0, s2 = 0;
        for (int s = 0; s < n; ++s) mu += X[(size_t)s * IN + f];
        mu /= n;
        for (int s = 0; s < n; ++s) s2 += (X[(size_t)s * IN + f] - mu) * (X[(size_t)s * IN + f] - mu);
        m->mean[f] = (float)mu;
        m->stdv[f] = s2 > 0 ? (float)std::sqrt(s2 / n) : 1.f;
    }
    double ym = 0, ys = 0;
    for (int s = 0; s < n; ++s) ym += y[s];
    ym /= n;
    for (int s = 0; s < n; ++s) ys += (y[s] - ym) * (y[s] - ym);
    m->y_mean = (float)ym;
    m->y_std = ys > 0 ? (float)std::sqrt(ys / n) : 1.f;
    std::vector<float> Xn = normalise(m, X, n), tn((size_t)n);
    for (int s = 0; s < n; ++s) tn[s] = (y[s] - m->y_mean) / m->y_std;
    // He-style initialisation from a seeded generator (splitmix64)
    std::vector<float> p0(NPARAM, 0.f);
    uint64_t st = seed;
    auto rnd = [&]() {
        st += 0x9E3779B97F4A7C15ull;
        uint64_t z = st;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        return ((z >> 11) * (1.0 / 9007199254740992.0)) * 2.0 - 1.0;  // uniform [-1, 1)
    };
    auto init = [&](int off, int fan_in, int count) {
        const double a = std::sqrt(6.0 / fan_in);
        for (int k = 0; k < count; ++k) p0[off + k] = (float)(a * rnd());
    };
    init(OFF_W1, IN, IN * H);
    init(OFF_W2, H, H * H);
    init(OFF_W3, H, H * H);
    init(OFF_W4, H, H);
    MLP_CUDA(cudaMemcpy(m->p, p0.data(), NPARAM * 4, cudaMemcpyHostToDevice));
    MLP_CUDA(cudaMemset(m->m, 0, NPARAM * 4));
    MLP_CUDA(cudaMemset(m->v, 0, NPARAM * 4));
    m->steps = 0;
    // device copies of the whole training set
    const int bmax = batch < n ? batch : n;
    const int nbmax = (bmax + kTile - 1) / kTile;
    DevBuf dX, dT, dy, dg, dsave, dpart, dloss;
    MLP_CUDA(cudaMalloc(&dX.ptr, (size_t)n * IN * 4));
    MLP_CUDA(cudaMalloc(&dT.ptr, (size_t)n * 4));
    MLP_CUDA(cudaMalloc(&dy.ptr, (size_t)bmax * 4));
    MLP_CUDA(cudaMalloc(&dg.ptr, (size_t)bmax * 4));
    MLP_CUDA(cudaMalloc(&dsave.ptr, (size_t)bmax * 3 * H * 4));
    MLP_CUDA(cudaMalloc(&dpart.ptr, (size_t)nbmax * NPARAM * 4));
    MLP_CUDA(cudaMalloc(&dloss.ptr, 64 * 8));
    // shuffled order per epoch (host), samples copied contiguously per batch
    std::vector<int> order(n);
    for (int s = 0; s < n; ++s) order[s] = s;
    std::vector<float> bx((size_t)n * IN), bt((size_t)n);
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    double last = 0.0;
    for (int ep = 0; ep < epochs; ++ep) {
        for (int s = n - 1; s > 0; --s) {
            const int r = (int)((rnd() * 0.5 + 0.5) * (s + 1)) % (s + 1);
            std::swap(order[s], order[r]);
        }
        for (int s = 0; s < n; ++s) {
            std::memcpy(&bx[(size_t)s * IN], &Xn[(size_t)order[s] * IN], IN * 4);
            bt[s] = tn[order[s]];
        }
        MLP_CUDA(cudaMemcpy(dX.ptr, bx.data(), (size_t)n * IN * 4, cudaMemcpyHostToDevice));
        MLP_CUDA(cudaMemcpy(dT.ptr, bt.data(), (size_t)n * 4, cudaMemcpyHostToDevice));
        for (int b0 = 0; b0 < n; b0 += bmax) {
            const int nb = (n - b0) < bmax ? (n - b0) : bmax;
            const int blocks = (nb + kTile - 1) / kTile;
            const float *xb = dX.as<float>() + (size_t)b0 * IN;
            const float *tb = dT.as<float>() + b0;
            k_mlp_forward<float><<<blocks, H>>>(m->p, xb, nb, dy.as<float>(), dsave.as<float>());
            k_mse<<<64, 256>>>(dy.as<float>(), tb, nb, dg.as<float>(), dloss.as<double>());
            k_mlp_backward<<<blocks, H>>>(m->p, xb, nb, dsave.as<float>(), dg.as<float>(), dpart.as<float>());
            k_reduce_grad<<<(NPARAM + 255) / 256, 256>>>(dpart.as<float>(), blocks, m->grad);
            ++m->steps;
            const float c1 = 1.f - std::pow(b1, (float)m->steps), c2 = 1.f - std::pow(b2, (float)m->steps);
            k_adam<<<(NPARAM + 255) / 256, 256>>>(m->p, m->grad, m->m, m->v, m->p16, lr, b1, b2, eps, c1, c2);
        }
        MLP_CUDA(cudaGetLastError());
    }
    // final loss over the whole set (normalised units)
    {
        double loss = 0;
        std::vector<float> pred((size_t)n);
        int rc = qd_model_forward_raw(m, Xn.data(), n, pred.data(), 0);
        if (rc) return rc;
        for (int s = 0; s < n; ++s) loss += (double)(pred[s] - tn[s]) * (pred[s] - tn[s]);
        last = loss / n;
    }
    k_to_half<<<8, 256>>>(m->p, m->p16);
    MLP_CUDA(cudaGetLastError());
    MLP_CUDA(cudaDeviceSynchronize());
    if (final_loss) *final_loss = last;
    return QD_OK;
}

int qd_model_predict(qd_model *m, const float *X, int32_t n, float *y) {
    if (!m || !X || !y || n < 0) return mfail(QD_ERR_ARG, "bad predict arguments");
    if (n == 0) return QD_OK;
    std::vector<float> Xn = normalise(m, X, n);
    int rc = qd_model_forward_raw(m, Xn.data(), n, y, 1);
    if (rc) return rc;
    for (int s = 0; s < n; ++s) y[s] = y[s] * m->y_std + m->y_mean;
    return QD_OK;
}

}  // extern "C"
