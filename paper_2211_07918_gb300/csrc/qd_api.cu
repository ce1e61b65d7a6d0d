// libqudit C ABI: registers, gate planning and launch, circuits, readout.
//
// Gate definitions follow QuDiet (arXiv 2211.07918) Sec. 2.1.2: generalized
// NOT X^d_{+a}, phase shift Z_d with w = exp(2 pi i/d), generalized Hadamard
// F_d[j][k] = w^{jk}/sqrt(d), and controlled versions that fire on a control
// level (d_c - 1 for C_{X,d}, C^n_{X,d}; any chosen level after Fig. 1).
// Registers follow Sec. 2.2 / Sec. 3.2: N = prod d_q, qudit 0 least
// significant, initial basis levels.
#include <algorithm>
#include <complex>
#include <array>
#include <atomic>
#include <chrono>
#include <thread>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "../../include/qudit.h"
#include "../../include/qudit_debug.h"
#include "qd_batch.h"
#include "qd_fuse.h"
#include "qd_mlp.h"
#include "qd_plan.h"
#include "qd_reduce.h"
#include "qd_ket.h"
#include "qd_kron.h"
#include "qd_diag.h"
#include "qd_tc.h"

using namespace qd;

// ------------------------------------------------------------------ errors

namespace {
thread_local std::string g_last_error;

int fail(int code, const std::string &msg) {
    g_last_error = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char *where) {
    return fail(QD_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}
}  // namespace

#define QD_CUDA(call)                                        \
    do {                                                     \
        cudaError_t _e = (call);                             \
        if (_e != cudaSuccess) return cuda_fail(_e, #call);  \
    } while (0)

// ---------------------------------------------------------------- register

struct qd_reg {
    int32_t n = 0;
    int32_t dims[QD_MAX_QUDITS] = {};
    int64_t s[QD_MAX_QUDITS + 1] = {};  // s[q] = prod_{p<q} d_p, s[n] = N
    int64_t N = 0;
    int32_t prec = QD_C64;
    size_t esize = 8;
    void *psi = nullptr;
    bool owns = false;
    cudaStream_t stream = nullptr;
    int device = 0;
    int sm_count = 0;
    double *red = nullptr;  // reduction partials + results
    size_t red_cap = 0;     // doubles
    double *cdf = nullptr;  // lazily allocated N doubles
    double *cdf_chunks = nullptr;
    int32_t *dev_err = nullptr;
    int64_t tile_stride = -1;  // -1: process default
    int32_t fuse_kmax = 3;     // largest number of qudits of a fused block
    int32_t index64 = 0;       // 64-bit index kernels below 2^31 amplitudes too
    int32_t fuse_dmax = -1;    // largest dimension of a fused block (-1: 64 for c64, 32 for c128)
    int32_t tc_min_d = 0;      // complex64 fused blocks of D >= this on the tensor cores (0: the cost model decides)
    qd_model *model = nullptr; // learned cost model for QD_PLAN_LEARNED
    bool measured = false;     // measurement flag set: later gates are ignored (Sec. 3.4)
};

struct qd_plan {
    qd_reg *reg = nullptr;
    std::vector<GatePlan> gates;
    int32_t blocks = 0;
    void *tc_buf = nullptr;  // device: BF16 terms of every tensor-core block
    void *tab_buf = nullptr; // device: tables of every diagonal run
    bool profile = false;
    std::vector<cudaEvent_t> events;  // launches + 1 when profiling
    bool use_graph = true;            // capture on first run, replay afterwards
    std::atomic<int> gate_open{1};    // profiling: holds the stream until every launch is enqueued
    bool measure_after = false;       // the gate list ended with the measurement flag
    cudaGraphExec_t exec = nullptr;   // captured launches (non-default streams)
    void drop_graph() {
        if (exec) cudaGraphExecDestroy(exec);
        exec = nullptr;
    }
    ~qd_plan() {
        drop_graph();
        for (cudaEvent_t e : events) cudaEventDestroy(e);
        if (tc_buf) cudaFree(tc_buf);
        if (tab_buf) cudaFree(tab_buf);
    }
};

namespace qd {
int set_last_error(int code, const char *msg) { return fail(code, msg); }

int occupancy_blocks(const void *fn, int block, size_t smem) {
    static std::mutex mu;
    static std::map<std::pair<const void *, size_t>, int> cache;
    std::lock_guard<std::mutex> lk(mu);
    auto key = std::make_pair(fn, smem);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, block, smem) != cudaSuccess || nb < 1) nb = 1;
    cache[key] = nb;
    return nb;
}
}  // namespace qd

namespace {

int reg_ok(const qd_reg *r) {
    if (!r) return fail(QD_ERR_ARG, "null register");
    return QD_OK;
}

// Every qudit dimension a power of two (so every stride and every divisor a
// gate's kernel takes is one).
bool all_pow2(const qd_reg *r) {
    for (int q = 0; q < r->n; ++q)
        if (r->dims[q] & (r->dims[q] - 1)) return false;
    return true;
}

cudaError_t launch_plan(const qd_reg *r, const GatePlan &g) {
    if (g.mode == Mode::Tensor) return launch_block_tc(g, r->psi, r->sm_count, r->dev_err, r->stream);
    if (g.mode == Mode::Table)
        return diag_table_apply(r->psi, r->prec, (uint64_t)r->N, g.tab_div, g.tab_size, g.tab, r->sm_count, r->stream,
                                g.wide);
    if (r->prec == QD_C64) return launch_gate_f32(g, r->psi, r->sm_count, r->stream);
    return launch_gate_f64(g, r->psi, r->sm_count, r->stream);
}

// ---- gate matrices (Sec. 2.1.2), FP64 -----------------------------------

// w^m for w = exp(2 pi i / d); exponent reduced mod d first, quarter turns exact.
void omega(int d, long long m, double *re, double *im) {
    m %= d;
    if (m < 0) m += d;
    if ((4 * m) % d == 0) {
        static const double tr[4] = {1, 0, -1, 0}, ti[4] = {0, 1, 0, -1};
        const int q = (int)((4 * m) / d);
        *re = tr[q];
        *im = ti[q];
        return;
    }
    const double t = 2.0 * M_PI * (double)m / (double)d;
    *re = std::cos(t);
    *im = std::sin(t);
}

std::vector<double> mat_x(int d, int a) {  // column x -> row (x+a) mod d
    std::vector<double> m(2 * d * d, 0.0);
    for (int x = 0; x < d; ++x) m[2 * (((x + a) % d) * d + x)] = 1.0;
    return m;
}

std::vector<double> mat_z(int d, int p) {
    std::vector<double> m(2 * d * d, 0.0);
    for (int j = 0; j < d; ++j) omega(d, (long long)p * j, &m[2 * (j * d + j)], &m[2 * (j * d + j) + 1]);
    return m;
}

std::vector<double> mat_f(int d) {
    std::vector<double> m(2 * d * d, 0.0);
    const double sc = 1.0 / std::sqrt((double)d);
    for (int j = 0; j < d; ++j)
        for (int k = 0; k < d; ++k) {
            double re, im;
            omega(d, (long long)j * k, &re, &im);
            m[2 * (j * d + k)] = re * sc;
            m[2 * (j * d + k) + 1] = im * sc;
        }
    return m;
}

// ---- validation -----------------------------------------------------------

struct Acting {
    int k = 0, nc = 0;
    int t[QD_MAX_TARGETS];
    int c[QD_MAX_CONTROLS];
    int lv[QD_MAX_CONTROLS];
    int D = 1;
};

int validate(const qd_reg *r, const int32_t *targets, int32_t k, const int32_t *controls, const int32_t *levels,
             int32_t nc, Acting &a) {
    if (!targets || k < 1 || k > QD_MAX_TARGETS) return fail(QD_ERR_ARG, "need 1..QD_MAX_TARGETS targets");
    if (nc < 0 || nc > QD_MAX_CONTROLS || (nc > 0 && !controls)) return fail(QD_ERR_ARG, "bad control list");
    bool used[QD_MAX_QUDITS] = {};
    a.k = k;
    a.nc = nc;
    a.D = 1;
    for (int m = 0; m < k; ++m) {
        const int q = targets[m];
        if (q < 0 || q >= r->n) return fail(QD_ERR_ARG, "target out of range");
        if (used[q]) return fail(QD_ERR_OVERLAP, "repeated target");
        used[q] = true;
        a.t[m] = q;
        a.D *= r->dims[q];
        if (a.D > QD_MAX_D) return fail(QD_ERR_DIM, "target space larger than QD_MAX_D");
    }
    for (int m = 0; m < nc; ++m) {
        const int q = controls[m];
        if (q < 0 || q >= r->n) return fail(QD_ERR_ARG, "control out of range");
        if (used[q]) return fail(QD_ERR_OVERLAP, "control repeats a target or control");
        used[q] = true;
        int l = levels ? levels[m] : -1;
        if (l < 0) l = r->dims[q] - 1;
        if (l >= r->dims[q]) return fail(QD_ERR_ARG, "control level out of range");
        a.c[m] = q;
        a.lv[m] = l;
    }
    return QD_OK;
}

// ---- planning of one gate ---------------------------------------------------

void set_expand64(Expand64 &e, const std::vector<std::pair<int64_t, int64_t>> &stride_dim) {
    e = Expand64{};
    e.n = (int32_t)stride_dim.size();
    for (size_t i = 0; i < stride_dim.size(); ++i) {
        e.div[i] = make_fastdiv64((uint64_t)stride_dim[i].first);
        e.span[i] = (uint64_t)(stride_dim[i].first * stride_dim[i].second);
    }
}

void set_expand32(Expand32 &e, const std::vector<std::pair<int64_t, int64_t>> &stride_dim) {
    e = Expand32{};
    e.n = (int32_t)stride_dim.size();
    for (size_t i = 0; i < stride_dim.size(); ++i) {
        e.div[i] = make_fastdiv32((uint32_t)stride_dim[i].first);
        e.span[i] = (uint32_t)(stride_dim[i].first * stride_dim[i].second);
    }
}

// Classify M (D x D, interleaved complex): returns true and fills src/lam if
// every row and every column has exactly one nonzero entry.
bool classify_mono(const double *M, int D, GatePlan &g) {
    std::vector<int> colcount(D, 0);
    for (int i = 0; i < D; ++i) {
        int nz = -1, cnt = 0;
        for (int j = 0; j < D; ++j) {
            const double re = M[2 * (i * D + j)], im = M[2 * (i * D + j) + 1];
            if (re != 0.0 || im != 0.0) {
                ++cnt;
                nz = j;
            }
        }
        if (cnt != 1) return false;
        if (++colcount[nz] > 1) return false;
        g.src[i] = nz;
        g.lam[2 * i] = M[2 * (i * D + nz)];
        g.lam[2 * i + 1] = M[2 * (i * D + nz) + 1];
    }
    g.active = 0;
    g.unit = 0;
    for (int i = 0; i < D; ++i) {
        const bool one = g.lam[2 * i] == 1.0 && g.lam[2 * i + 1] == 0.0;
        if (one) g.unit |= 1u << i;
        if (g.src[i] != i || !one) g.active |= 1u << i;
    }
    return true;
}

// Build the launch plan of one gate: matrix M over the targets (first listed
// most significant), controls at levels.  Returns QD_OK; sets *noop when the
// gate is the identity.
int plan_gate(const qd_reg *r, const double *M, const Acting &a, bool diag_only, GatePlan &g, bool *noop,
              bool force_dense = false) {
    *noop = false;
    g = GatePlan{};
    const int D = a.D;
    g.D = D;
    g.N = (uint64_t)r->N;
    g.wide = r->index64 != 0;
    g.pow2 = all_pow2(r);
    // matrix / classification
    if (force_dense) {  // the dense kernels, whatever the matrix (a dense part with a table epilogue)
        g.kind = Kind::Dense;
        std::memcpy(g.U, M, sizeof(double) * 2 * D * D);
    } else if (diag_only) {
        for (int i = 0; i < D; ++i) {
            g.src[i] = i;
            g.lam[2 * i] = M[2 * i];
            g.lam[2 * i + 1] = M[2 * i + 1];
        }
        g.active = g.unit = 0;
        for (int i = 0; i < D; ++i) {
            const bool one = g.lam[2 * i] == 1.0 && g.lam[2 * i + 1] == 0.0;
            if (one) g.unit |= 1u << i;
            else g.active |= 1u << i;
        }
        g.kind = Kind::Mono;
    } else if (classify_mono(M, D, g)) {
        g.kind = Kind::Mono;
    } else {
        g.kind = Kind::Dense;
        std::memcpy(g.U, M, sizeof(double) * 2 * D * D);
    }
    if (g.kind == Kind::Mono && g.active == 0) {
        *noop = true;
        return QD_OK;
    }

    const int n = r->n;
    const int64_t *s = r->s;
    bool is_t[QD_MAX_QUDITS] = {}, is_c[QD_MAX_QUDITS] = {};
    int level[QD_MAX_QUDITS] = {};
    for (int m = 0; m < a.k; ++m) is_t[a.t[m]] = true;
    for (int m = 0; m < a.nc; ++m) {
        is_c[a.c[m]] = true;
        level[a.c[m]] = a.lv[m];
    }
    int64_t cprod = 1;
    for (int m = 0; m < a.nc; ++m) cprod *= r->dims[a.c[m]];

    // flat offset of local index j: digits of j in the target radices, first target most significant
    for (int j = 0; j < D; ++j) {
        int rem = j;
        int64_t o = 0;
        for (int m = a.k - 1; m >= 0; --m) {
            const int t = a.t[m];
            o += (int64_t)(rem % r->dims[t]) * s[t];
            rem /= r->dims[t];
        }
        g.off[j] = o;
    }
    int64_t min_stride = r->N;
    for (int q = 0; q < n; ++q)
        if (is_t[q] || is_c[q]) min_stride = std::min<int64_t>(min_stride, s[q]);

    const int64_t touched = r->N / cprod;  // amplitudes in the selected control slice
    if (g.kind == Kind::Dense) g.alg_bytes = 2.0 * (double)touched * (double)r->esize;
    else g.alg_bytes = 2.0 * (double)(touched / D) * __builtin_popcount(g.active) * (double)r->esize;

    static const int64_t default_low_stride = [] {
        const char *v = std::getenv("QD_TILE_STRIDE");
        return v ? (int64_t)std::atoll(v) : kLowStride;
    }();
    const int64_t low_stride = r->tile_stride >= 0 ? r->tile_stride : default_low_stride;
    // direct geometry (always computed: it is the fallback of tile mode)
    {
        g.mode = Mode::Direct;
        g.R = (uint64_t)(r->N / (D * cprod));
        std::vector<std::pair<int64_t, int64_t>> ins;
        uint64_t base = 0;
        for (int q = 0; q < n; ++q)
            if (is_t[q] || is_c[q]) {
                ins.push_back({s[q], r->dims[q]});
                if (is_c[q]) base += (uint64_t)level[q] * (uint64_t)s[q];
            }
        set_expand64(g.ex, ins);
        g.base_off = base;
    }
    if (min_stride >= low_stride) return QD_OK;

    // ---- tile mode (falls back to direct when the tile would not fit) ----
    int m = 0;
    for (int q = 0; q < n; ++q)
        if ((is_t[q] || is_c[q]) && s[q] < low_stride) m = q + 1;
    auto DH_of = [&](int mm) {
        int64_t dh = 1;
        for (int q = mm; q < n; ++q)
            if (is_t[q]) dh *= r->dims[q];
        return dh;
    };
    int64_t B = s[m];
    int64_t DH = DH_of(m);
    while (m < n) {
        const int q = m;
        const int64_t d = r->dims[q];
        if (is_t[q]) {
            B *= d;
            DH /= d;
            ++m;
            continue;
        }
        if (is_c[q]) break;
        const int64_t grown = B * d * DH;
        if (grown <= (int64_t)kTileBudget || (B < kLowStride && grown <= (int64_t)kTileHardMax)) {
            B *= d;
            ++m;
            continue;
        }
        break;
    }
    if (B * DH > (int64_t)kTileHardMax) return QD_OK;  // stays in direct mode
    g.mode = Mode::Tile;
    g.B = (uint32_t)B;
    g.DH = (uint32_t)DH;
    // high (>= m) removed digits: expansion over block-level strides s_q / B
    std::vector<std::pair<int64_t, int64_t>> hi, lo;
    uint64_t base_hi = 0;
    uint32_t lo_off = 0;
    int64_t chi = 1, clo = 1, DL = 1;
    for (int q = 0; q < n; ++q) {
        if (!(is_t[q] || is_c[q])) continue;
        if (q >= m) {
            hi.push_back({s[q] / B, r->dims[q]});
            if (is_c[q]) {
                base_hi += (uint64_t)level[q] * (uint64_t)s[q];
                chi *= r->dims[q];
            }
        } else {
            lo.push_back({s[q], r->dims[q]});
            if (is_c[q]) {
                lo_off += (uint32_t)(level[q] * s[q]);
                clo *= r->dims[q];
            } else {
                DL *= r->dims[q];
            }
        }
    }
    set_expand64(g.ex_hi, hi);
    set_expand32(g.ex_lo, lo);
    g.base_off_hi = base_hi;
    g.lo_off = lo_off;
    g.R_tiles = (uint64_t)((r->N / B) / (DH * chi));
    g.G_in = (uint32_t)(B / (DL * clo));
    g.tpc = (uint32_t)std::max<int64_t>(1, (int64_t)kTileBudget / (DH * B));
    if ((uint64_t)g.tpc > g.R_tiles) g.tpc = (uint32_t)std::max<uint64_t>(1, g.R_tiles);
    g.divB = make_fastdiv32(g.B);
    g.divG = make_fastdiv32(g.G_in);
    // chunk offsets: high targets in list order, first listed most significant
    int th[QD_MAX_TARGETS], nth = 0;
    for (int mm = 0; mm < a.k; ++mm)
        if (a.t[mm] >= m) th[nth++] = a.t[mm];
    for (int h = 0; h < (int)DH; ++h) {
        int rem = h;
        int64_t o = 0;
        for (int i = nth - 1; i >= 0; --i) {
            o += (int64_t)(rem % r->dims[th[i]]) * s[th[i]];
            rem /= r->dims[th[i]];
        }
        g.offH[h] = o;
    }
    // shared-memory offsets of local index j: chunk index (high digits) * B + low offset
    for (int j = 0; j < D; ++j) {
        int rem = j;
        int64_t h = 0, hmul = 1, offl = 0;
        for (int mm = a.k - 1; mm >= 0; --mm) {
            const int t = a.t[mm];
            const int x = rem % r->dims[t];
            rem /= r->dims[t];
            if (t >= m) {
                h += x * hmul;
                hmul *= r->dims[t];
            } else {
                offl += (int64_t)x * s[t];
            }
        }
        g.smoff[j] = (int32_t)(h * B + offl);
    }
    return QD_OK;
}

int gate_matrix(const qd_reg *r, const qd_gate *gt, const Acting &a, std::vector<double> &M, bool *diag) {
    *diag = false;
    switch (gt->kind) {
        case QD_GATE_X: {
            if (a.k != 1) return fail(QD_ERR_ARG, "X acts on one qudit");
            const int d = r->dims[a.t[0]];
            if (gt->param < 1 || gt->param > d - 1) return fail(QD_ERR_ARG, "X shift must be in [1, d-1]");
            M = mat_x(d, gt->param);
            return QD_OK;
        }
        case QD_GATE_Z:
            if (a.k != 1) return fail(QD_ERR_ARG, "Z acts on one qudit");
            M = mat_z(r->dims[a.t[0]], gt->param);
            return QD_OK;
        case QD_GATE_H:
            if (a.k != 1) return fail(QD_ERR_ARG, "H acts on one qudit");
            M = mat_f(r->dims[a.t[0]]);
            return QD_OK;
        case QD_GATE_U:
            if (!gt->matrix) return fail(QD_ERR_ARG, "U gate without matrix");
            M.assign(gt->matrix, gt->matrix + 2 * a.D * a.D);
            return QD_OK;
        case QD_GATE_DIAG:
            if (!gt->matrix) return fail(QD_ERR_ARG, "DIAG gate without entries");
            M.assign(gt->matrix, gt->matrix + 2 * a.D);
            *diag = true;
            return QD_OK;
        default:
            return fail(QD_ERR_ARG, "unknown gate kind");
    }
}

int prepare_gate(const qd_reg *r, const qd_gate *gt, GatePlan &g, bool *noop) {
    if (!gt) return fail(QD_ERR_ARG, "null gate");
    Acting a;
    int rc = validate(r, gt->targets, gt->k, gt->controls, gt->ctrl_levels, gt->nc, a);
    if (rc) return rc;
    std::vector<double> M;
    bool diag = false;
    if ((rc = gate_matrix(r, gt, a, M, &diag))) return rc;
    return plan_gate(r, M.data(), a, diag, g, noop);
}

int apply_record(qd_reg *r, const qd_gate *gt) {
    if (gt->kind == QD_GATE_MEASURE) {  // the flag that ends the circuit (Sec. 3.4)
        r->measured = true;
        return QD_OK;
    }
    if (r->measured) return QD_OK;  // a gate after the measurement flag is ignored
    GatePlan g;
    bool noop = false;
    int rc = prepare_gate(r, gt, g, &noop);
    if (rc) return rc;
    if (noop) return QD_OK;
    cudaError_t e = launch_plan(r, g);
    if (e != cudaSuccess) return cuda_fail(e, "gate launch");
    return QD_OK;
}

qd_gate make_record(int kind, const int32_t *targets, int32_t k, const int32_t *controls, const int32_t *levels,
                    int32_t nc, int32_t param, const double *matrix) {
    qd_gate g;
    std::memset(&g, 0, sizeof(g));
    g.kind = kind;
    g.k = k;
    for (int i = 0; i < k && i < QD_MAX_TARGETS; ++i) g.targets[i] = targets[i];
    g.nc = nc;
    for (int i = 0; i < nc && i < QD_MAX_CONTROLS; ++i) {
        g.controls[i] = controls[i];
        g.ctrl_levels[i] = levels ? levels[i] : -1;
    }
    g.param = param;
    g.matrix = matrix;
    return g;
}

int ensure_red(qd_reg *r, size_t doubles) {
    if (r->red_cap >= doubles) return QD_OK;
    if (r->red) cudaFree(r->red);
    r->red = nullptr;
    r->red_cap = 0;
    if (cudaMalloc(&r->red, doubles * sizeof(double)) != cudaSuccess)
        return fail(QD_ERR_OOM, "reduction scratch allocation failed");
    r->red_cap = doubles;
    return QD_OK;
}

int ensure_cdf(qd_reg *r) {
    if (r->cdf) return QD_OK;
    const size_t nch = cdf_chunks((uint64_t)r->N) + 1;
    if (cudaMalloc(&r->cdf, (size_t)r->N * sizeof(double)) != cudaSuccess) {
        r->cdf = nullptr;
        return fail(QD_ERR_OOM, "CDF buffer allocation failed");
    }
    if (cudaMalloc(&r->cdf_chunks, nch * sizeof(double)) != cudaSuccess) {
        cudaFree(r->cdf);
        r->cdf = nullptr;
        r->cdf_chunks = nullptr;
        return fail(QD_ERR_OOM, "CDF chunk allocation failed");
    }
    return QD_OK;
}

int compute_cdf(qd_reg *r) {
    int rc = ensure_cdf(r);
    if (rc) return rc;
    QD_CUDA(cdf(r->psi, r->prec, (uint64_t)r->N, r->cdf_chunks, r->cdf, r->stream));
    return QD_OK;
}

}  // namespace

// ====================================================================== ABI

extern "C" {

const char *qd_strerror(int code) {
    switch (code) {
        case QD_OK: return "ok";
        case QD_ERR_ARG: return "invalid argument";
        case QD_ERR_DIM: return "dimension out of range";
        case QD_ERR_OVERLAP: return "overlapping qudits";
        case QD_ERR_OOM: return "out of memory";
        case QD_ERR_CUDA: return "CUDA error";
        case QD_ERR_TIMEOUT: return "device wait timed out";
        case QD_ERR_DEVICE: return "device reported an error";
        case QD_ERR_UNSUPPORTED: return "unsupported";
        default: return "unknown error";
    }
}

const char *qd_last_error(void) { return g_last_error.c_str(); }

int qd_create(const int32_t *dims, int32_t n, const int32_t *init_levels, int32_t precision, void *dev_buf,
              size_t dev_buf_bytes, void *stream, qd_reg **out) {
    if (!out) return fail(QD_ERR_ARG, "null output handle");
    *out = nullptr;
    if (!dims || n < 1 || n > QD_MAX_QUDITS) return fail(QD_ERR_ARG, "need 1..QD_MAX_QUDITS dims");
    if (precision != QD_C64 && precision != QD_C128) return fail(QD_ERR_ARG, "precision must be QD_C64 or QD_C128");
    int64_t N = 1;
    for (int q = 0; q < n; ++q) {
        if (dims[q] < 2 || dims[q] > 64) return fail(QD_ERR_DIM, "qudit dimension must be in [2, 64]");
        if (N > QD_MAX_AMPLITUDES / dims[q]) return fail(QD_ERR_DIM, "register larger than QD_MAX_AMPLITUDES");
        N *= dims[q];
    }
    int64_t idx = 0;
    {
        int64_t s = 1;
        for (int q = 0; q < n; ++q) {
            const int l = init_levels ? init_levels[q] : 0;
            if (l < 0 || l >= dims[q]) return fail(QD_ERR_ARG, "init level out of range");
            idx += (int64_t)l * s;
            s *= dims[q];
        }
    }
    qd_reg *r = new qd_reg();
    r->n = n;
    int64_t s = 1;
    for (int q = 0; q < n; ++q) {
        r->dims[q] = dims[q];
        r->s[q] = s;
        s *= dims[q];
    }
    r->s[n] = s;
    r->N = N;
    r->prec = precision;
    r->esize = precision == QD_C64 ? 8 : 16;
    r->stream = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaGetDevice(&r->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&r->sm_count, cudaDevAttrMultiProcessorCount, r->device);
    if (e != cudaSuccess) {
        delete r;
        return cuda_fail(e, "device query");
    }
    const size_t bytes = (size_t)N * r->esize;
    if (dev_buf) {
        if (dev_buf_bytes < bytes) {
            delete r;
            return fail(QD_ERR_OOM, "caller buffer smaller than N amplitudes");
        }
        if (reinterpret_cast<uintptr_t>(dev_buf) % 16 != 0) {
            delete r;
            return fail(QD_ERR_ARG, "caller buffer must be 16-byte aligned");
        }
        r->psi = dev_buf;
        r->owns = false;
    } else {
        if (cudaMalloc(&r->psi, bytes) != cudaSuccess) {
            cudaGetLastError();
            delete r;
            return fail(QD_ERR_OOM, "state allocation failed");
        }
        r->owns = true;
    }
    if (cudaMalloc(&r->dev_err, sizeof(int32_t)) != cudaSuccess ||
        cudaMemsetAsync(r->dev_err, 0, sizeof(int32_t), r->stream) != cudaSuccess) {
        cudaGetLastError();
        qd_destroy(r);
        return fail(QD_ERR_OOM, "error word allocation failed");
    }
    int rc = ensure_red(r, (size_t)reduce_blocks(r->sm_count) * 64 + 64);
    if (rc) {
        qd_destroy(r);
        return rc;
    }
    e = init_basis(r->psi, r->prec, (uint64_t)N, (uint64_t)idx, r->sm_count, r->stream);
    if (e != cudaSuccess) {
        qd_destroy(r);
        return cuda_fail(e, "init");
    }
    *out = r;
    return QD_OK;
}

int qd_destroy(qd_reg *r) {
    if (!r) return QD_OK;
    if (r->stream) cudaStreamSynchronize(r->stream);
    else cudaDeviceSynchronize();
    if (r->owns && r->psi) cudaFree(r->psi);
    if (r->red) cudaFree(r->red);
    if (r->cdf) cudaFree(r->cdf);
    if (r->cdf_chunks) cudaFree(r->cdf_chunks);
    if (r->dev_err) cudaFree(r->dev_err);
    delete r;
    return QD_OK;
}

int qd_reset(qd_reg *r, const int32_t *init_levels) {
    if (int rc = reg_ok(r)) return rc;
    int64_t idx = 0;
    for (int q = 0; q < r->n; ++q) {
        const int l = init_levels ? init_levels[q] : 0;
        if (l < 0 || l >= r->dims[q]) return fail(QD_ERR_ARG, "init level out of range");
        idx += (int64_t)l * r->s[q];
    }
    QD_CUDA(init_basis(r->psi, r->prec, (uint64_t)r->N, (uint64_t)idx, r->sm_count, r->stream));
    r->measured = false;
    return QD_OK;
}

int qd_measure_all(qd_reg *r) {
    if (int rc = reg_ok(r)) return rc;
    r->measured = true;
    return QD_OK;
}

int qd_is_measured(const qd_reg *r, int32_t *measured) {
    if (int rc = reg_ok(r)) return rc;
    if (!measured) return fail(QD_ERR_ARG, "null output");
    *measured = r->measured ? 1 : 0;
    return QD_OK;
}

int qd_info(const qd_reg *r, int64_t *N, int32_t *n, void **state, int32_t *precision) {
    if (int rc = reg_ok(r)) return rc;
    if (N) *N = r->N;
    if (n) *n = r->n;
    if (state) *state = r->psi;
    if (precision) *precision = r->prec;
    return QD_OK;
}

int qd_set_stream(qd_reg *r, void *stream) {
    if (int rc = reg_ok(r)) return rc;
    r->stream = static_cast<cudaStream_t>(stream);
    return QD_OK;
}

int qd_set_tuning(qd_reg *r, int32_t key, int64_t value) {
    if (int rc = reg_ok(r)) return rc;
    switch (key) {
        case QD_TUNE_TILE_STRIDE:
            if (value < 0) return fail(QD_ERR_ARG, "tile stride must be >= 0");
            r->tile_stride = value;
            return QD_OK;
        case QD_TUNE_FUSE_KMAX:
            if (value < 1 || value > QD_MAX_TARGETS) return fail(QD_ERR_ARG, "fusion qudit limit must be in [1, 6]");
            r->fuse_kmax = (int32_t)value;
            return QD_OK;
        case QD_TUNE_FUSE_DMAX: {
            const int64_t cap = r->prec == QD_C64 ? kTcMaxD : QD_MAX_D;
            if (value < 2 || value > cap) return fail(QD_ERR_ARG, "fusion dimension limit must be in [2, 64] (c64) or [2, 32] (c128)");
            r->fuse_dmax = (int32_t)value;
            return QD_OK;
        }
        case QD_TUNE_TC_MIN_D:
            if (value != 0 && (value < kTcMinD || value > kTcMaxD + 1))
                return fail(QD_ERR_ARG, "tensor-core block threshold must be 0 (cost model) or in [9, 65]");
            r->tc_min_d = (int32_t)value;
            return QD_OK;
        case QD_TUNE_INDEX64:
            if (value != 0 && value != 1) return fail(QD_ERR_ARG, "index width flag must be 0 or 1");
            r->index64 = (int32_t)value;
            return QD_OK;
        default:
            return fail(QD_ERR_ARG, "unknown tuning key");
    }
}

int qd_apply(qd_reg *r, const double *matrix, const int32_t *targets, int32_t k, const int32_t *controls,
             const int32_t *ctrl_levels, int32_t nc) {
    if (int rc = reg_ok(r)) return rc;
    if (!targets || k < 1 || k > QD_MAX_TARGETS) return fail(QD_ERR_ARG, "need 1..QD_MAX_TARGETS targets");
    qd_gate g = make_record(QD_GATE_U, targets, k, controls, ctrl_levels, nc, 0, matrix);
    return apply_record(r, &g);
}

int qd_apply_diag(qd_reg *r, const double *diag, const int32_t *targets, int32_t k, const int32_t *controls,
                  const int32_t *ctrl_levels, int32_t nc) {
    if (int rc = reg_ok(r)) return rc;
    if (!targets || k < 1 || k > QD_MAX_TARGETS) return fail(QD_ERR_ARG, "need 1..QD_MAX_TARGETS targets");
    qd_gate g = make_record(QD_GATE_DIAG, targets, k, controls, ctrl_levels, nc, 0, diag);
    return apply_record(r, &g);
}

int qd_apply_x(qd_reg *r, int32_t t, int32_t shift) {
    if (int rc = reg_ok(r)) return rc;
    qd_gate g = make_record(QD_GATE_X, &t, 1, nullptr, nullptr, 0, shift, nullptr);
    return apply_record(r, &g);
}

int qd_apply_z(qd_reg *r, int32_t t, int32_t power) {
    if (int rc = reg_ok(r)) return rc;
    qd_gate g = make_record(QD_GATE_Z, &t, 1, nullptr, nullptr, 0, power, nullptr);
    return apply_record(r, &g);
}

int qd_apply_h(qd_reg *r, int32_t t) {
    if (int rc = reg_ok(r)) return rc;
    qd_gate g = make_record(QD_GATE_H, &t, 1, nullptr, nullptr, 0, 0, nullptr);
    return apply_record(r, &g);
}

int qd_apply_cx(qd_reg *r, int32_t c, int32_t t, int32_t shift, int32_t ctrl_level) {
    if (int rc = reg_ok(r)) return rc;
    qd_gate g = make_record(QD_GATE_X, &t, 1, &c, &ctrl_level, 1, shift, nullptr);
    return apply_record(r, &g);
}

int qd_apply_mct(qd_reg *r, const int32_t *controls, const int32_t *ctrl_levels, int32_t nc, int32_t t,
                 int32_t shift) {
    if (int rc = reg_ok(r)) return rc;
    if (nc < 0 || nc > QD_MAX_CONTROLS || (nc > 0 && !controls)) return fail(QD_ERR_ARG, "bad control list");
    qd_gate g = make_record(QD_GATE_X, &t, 1, controls, ctrl_levels, nc, shift, nullptr);
    return apply_record(r, &g);
}

int qd_apply_gate(qd_reg *r, const qd_gate *gate) {
    if (int rc = reg_ok(r)) return rc;
    return apply_record(r, gate);
}

}  // extern "C"

namespace {

RegisterShape shape_of(const qd_reg *r) {
    const int dmax = r->fuse_dmax > 0 ? r->fuse_dmax : (r->prec == QD_C64 ? kTcMaxD : QD_MAX_D);
    return RegisterShape{r->n, r->dims, r->s, r->N, r->prec, r->tc_min_d, dmax};
}

bool has_measure(const qd_gate *gates, int32_t ngates) {
    for (int i = 0; i < ngates; ++i)
        if (gates[i].kind == QD_GATE_MEASURE) return true;
    return false;
}

// Validate every gate, drop identities, and collect both the fusion view
// (matrix over controls + targets) and the original records.
int collect_gates(const qd_reg *r, const qd_gate *gates, int32_t ngates, std::vector<FuseGate> &fg,
                  std::vector<const qd_gate *> &orig) {
    for (int i = 0; i < ngates; ++i) {
        const qd_gate *gt = &gates[i];
        if (gt->kind == QD_GATE_MEASURE) break;  // gates after the measurement flag are ignored (Sec. 3.4)
        Acting a;
        int rc = validate(r, gt->targets, gt->k, gt->controls, gt->ctrl_levels, gt->nc, a);
        if (rc == QD_OK) {
            std::vector<double> M;
            bool diag = false;
            rc = gate_matrix(r, gt, a, M, &diag);
            GatePlan g;
            bool noop = false;
            if (rc == QD_OK) rc = plan_gate(r, M.data(), a, diag, g, &noop);
            if (rc == QD_OK && !noop) {
                if (diag) {  // expand the diagonal to a full matrix
                    std::vector<double> F((size_t)2 * a.D * a.D, 0.0);
                    for (int j = 0; j < a.D; ++j) {
                        F[2 * (j * a.D + j)] = M[2 * j];
                        F[2 * (j * a.D + j) + 1] = M[2 * j + 1];
                    }
                    M.swap(F);
                }
                std::vector<int> c(a.c, a.c + a.nc), lv(a.lv, a.lv + a.nc), t(a.t, a.t + a.k);
                fg.push_back(make_fuse_gate(c, lv, t, M, r->dims, g.kind == Kind::Mono));
                bool ident = g.kind == Kind::Mono;  // a permutation with phases whose permutation is the identity
                for (int j = 0; ident && j < a.D; ++j) ident = g.src[j] == j;
                fg.back().diag = ident;
                orig.push_back(gt);
            }
        }
        if (rc) {
            g_last_error = "gate " + std::to_string(i) + ": " + g_last_error;
            return rc;
        }
    }
    return QD_OK;
}

CostFn cost_for(const qd_reg *r, int plan_kind) {
    const RegisterShape sh = shape_of(r);
    (void)plan_kind;
    return [sh](const LaunchFeatures &f) { return analytic_cost(sh, f); };
}

int segments_for(const qd_reg *r, const std::vector<FuseGate> &fg, int plan_kind,
                 std::vector<std::pair<int, int>> &segs, std::vector<int> &kinds, double *model_cost) {
    const RegisterShape sh = shape_of(r);
    const int kmax = r->fuse_kmax;
    const int dmax = r->fuse_dmax > 0 ? r->fuse_dmax : (r->prec == QD_C64 ? kTcMaxD : QD_MAX_D);
    CostFn cost = cost_for(r, plan_kind);
    // learned costs of every candidate segment; declared here because the
    // final cost function, used after the switch, refers to it
    std::map<std::array<float, kFeatures>, double> table;
    switch (plan_kind) {
        case QD_PLAN_NONE:
            segs.clear();
            for (int i = 0; i < (int)fg.size(); ++i) segs.push_back({i, i});
            break;
        case QD_PLAN_GREEDY:
            segs = segment_greedy(fg, sh, cost, kmax, dmax);
            break;
        case QD_PLAN_EXHAUSTIVE:
            segs = segment_exhaustive(fg, sh, cost, kmax, dmax, nullptr);
            break;
        case QD_PLAN_LEARNED: {
            if (!r->model) return fail(QD_ERR_UNSUPPORTED, "QD_PLAN_LEARNED needs a cost model (qd_set_cost_model)");
            // every feasible candidate segment, predicted in one batched inference
            std::vector<std::array<float, kFeatures>> feats;
            CostFn collect = [&](const LaunchFeatures &f) {
                std::array<float, kFeatures> k;
                std::copy(f.f, f.f + kFeatures, k.begin());
                if (table.emplace(k, 0.0).second) feats.push_back(k);
                return 0.0;
            };
            segment_exhaustive(fg, sh, collect, kmax, dmax, nullptr);
            std::vector<float> X, y(feats.size());
            for (auto &k : feats) X.insert(X.end(), k.begin(), k.end());
            if (int rc = qd_model_predict(r->model, X.data(), (int32_t)feats.size(), y.data())) return rc;
            for (size_t i = 0; i < feats.size(); ++i) table[feats[i]] = std::exp((double)y[i]) * 1e-6;
            CostFn learned = [&table, sh](const LaunchFeatures &f) {
                std::array<float, kFeatures> k;
                std::copy(f.f, f.f + kFeatures, k.begin());
                auto it = table.find(k);
                return it != table.end() ? it->second : analytic_cost(sh, f);
            };
            segs = segment_exhaustive(fg, sh, learned, kmax, dmax, nullptr);
            cost = learned;
            break;
        }
        default:
            return fail(QD_ERR_ARG, "unknown plan kind");
    }
    // the kernel of every segment, as the final cost function priced it
    double c = 0.0;
    kinds.assign(segs.size(), 0);
    for (size_t i = 0; i < segs.size(); ++i)
        c += segment_cost(fg, segs[i].first, segs[i].second, sh, cost, kmax, &kinds[i]);
    if (model_cost) *model_cost = c;
    return QD_OK;
}

// Tensor-core plan of one fused block (complex64): direct group geometry over
// the block's qudits, no controls; the BF16 terms are packed into `terms`.
int plan_block_tc(const qd_reg *r, const FuseBlock &b, GatePlan &g, std::vector<uint16_t> &terms) {
    g = GatePlan{};
    g.mode = Mode::Tensor;
    g.kind = Kind::Dense;
    g.D = b.D;
    g.Dp = tc_padded_dim(b.D);
    g.N = (uint64_t)r->N;
    g.wide = r->index64 != 0;
    g.pow2 = all_pow2(r);
    g.R = (uint64_t)(r->N / b.D);
    std::vector<int> asc(b.qudits.rbegin(), b.qudits.rend());
    std::vector<std::pair<int64_t, int64_t>> ins;
    for (int q : asc) ins.push_back({r->s[q], r->dims[q]});
    set_expand64(g.ex, ins);
    for (int j = 0; j < b.D; ++j) {
        int rem = j;
        int64_t o = 0;
        for (int m = (int)b.qudits.size() - 1; m >= 0; --m) {
            const int q = b.qudits[m];
            o += (int64_t)(rem % r->dims[q]) * r->s[q];
            rem /= r->dims[q];
        }
        g.off[j] = o;
    }
    g.alg_bytes = 2.0 * (double)r->N * (double)r->esize;
    terms.resize(tc_terms_bytes(g.Dp) / 2);
    tc_pack_terms(b.M.data(), b.D, g.Dp, terms.data());
    return QD_OK;
}

// A diagonal run awaiting its table: covered range, gates and their diagonals.
struct DiagRunSpec {
    int plan_index = 0;  // position of its GatePlan in the plan
    DiagRange range{};
    std::vector<DiagGateDesc> gates;
    std::vector<double> pool;  // interleaved complex diagonal entries of every gate
};

// Plan of a diagonal run gates[first..last] (every gate diagonal): the
// covered qudit range [qa, qb], each gate's acting qudits as range positions
// and its full diagonal (controls included) from its matrix over them.
int plan_diag_run(const qd_reg *r, const std::vector<FuseGate> &fg, int first, int last, GatePlan &g,
                  DiagRunSpec &spec) {
    static_assert(kDiagRunMaxTable == kDiagTableMax, "diagonal table limits of the planner and kernel differ");
    int qa = r->n, qb = -1;
    for (int i = first; i <= last; ++i)
        for (int q : fg[i].acting) {
            qa = std::min(qa, q);
            qb = std::max(qb, q);
        }
    if (qb - qa + 1 > kDiagMaxRange) return fail(QD_ERR_DIM, "diagonal run spans too many qudits");
    g = GatePlan{};
    g.mode = Mode::Table;
    g.kind = Kind::Mono;
    g.N = (uint64_t)r->N;
    g.wide = r->index64 != 0;
    g.pow2 = all_pow2(r);
    g.tab_div = (uint64_t)r->s[qa];
    uint64_t TS = 1;
    spec.range.nr = qb - qa + 1;
    for (int q = qa; q <= qb; ++q) {
        spec.range.d[q - qa] = r->dims[q];
        TS *= (uint64_t)r->dims[q];
    }
    if (TS > kDiagTableMax) return fail(QD_ERR_DIM, "diagonal run table too large");
    g.tab_size = TS;
    g.D = spec.range.nr;  // reported as the kernel class's D: qudits of the covered range
    g.alg_bytes = 2.0 * (double)r->N * (double)r->esize;
    for (int i = first; i <= last; ++i) {
        const FuseGate &x = fg[i];
        if ((int)x.acting.size() > kDiagMaxActing) return fail(QD_ERR_DIM, "diagonal gate acts on too many qudits");
        DiagGateDesc d{};
        d.nq = (int32_t)x.acting.size();
        for (int m = 0; m < d.nq; ++m) d.q[m] = x.acting[m] - qa;
        d.off = (int64_t)(spec.pool.size() / 2);
        for (int j = 0; j < x.Dact; ++j) {
            spec.pool.push_back(x.M[2 * ((size_t)j * x.Dact + j)]);
            spec.pool.push_back(x.M[2 * ((size_t)j * x.Dact + j) + 1]);
        }
        spec.gates.push_back(d);
    }
    return QD_OK;
}

// Launch plan of a dense part followed by a diagonal run: the dense kernel
// (direct geometry) on the part's qudits with the run's table as epilogue;
// the table itself is built once the plan's table buffer exists.
int plan_dense_table(const qd_reg *r, const std::vector<FuseGate> &fg, int first, int last, int kmax, GatePlan &g,
                     DiagRunSpec &spec) {
    const DenseTableSplit dt = dense_table_split(fg, first, last, shape_of(r), kmax);
    if (!dt.ok) return fail(QD_ERR_DIM, "segment is not a dense part followed by a diagonal run");
    const FuseBlock b = build_block(fg, first, dt.split, r->dims);
    Acting a;
    a.k = (int)b.qudits.size();
    a.nc = 0;
    a.D = b.D;
    for (int m = 0; m < a.k; ++m) a.t[m] = b.qudits[m];
    GatePlan run;
    if (int rc = plan_diag_run(r, fg, dt.split + 1, last, run, spec)) return rc;
    bool noop = false;
    if (int rc = plan_gate(r, b.M.data(), a, false, g, &noop, true)) return rc;
    g.mode = Mode::Direct;
    g.tab_div = run.tab_div;
    g.tab_size = run.tab_size;
    return QD_OK;
}

// Launch plan of one fused block: a dense gate on the block's qudits.
int plan_block(const qd_reg *r, const FuseBlock &b, GatePlan &g) {
    Acting a;
    a.k = (int)b.qudits.size();
    a.nc = 0;
    a.D = b.D;
    if (a.k > QD_MAX_TARGETS || b.D > QD_MAX_D) return fail(QD_ERR_DIM, "fused block too large");
    for (int m = 0; m < a.k; ++m) a.t[m] = b.qudits[m];
    bool noop = false;
    int rc = plan_gate(r, b.M.data(), a, false, g, &noop);
    if (rc == QD_OK && noop) g = GatePlan{};  // identity block: no launch (D stays 0)
    return rc;
}

}  // namespace

extern "C" {

}  // extern "C"

namespace {
// Plan from a segmentation of the collected gates.  enforce_limits: fused
// blocks must respect the register's QD_TUNE_FUSE_* limits (planner output
// does by construction; explicit segmentations only need the hard limits).
int build_plan(qd_reg *r, const std::vector<FuseGate> &fg, const std::vector<const qd_gate *> &orig,
               const std::vector<std::pair<int, int>> &segs, const std::vector<int> &kinds, int kmax,
               qd_plan **out) {
    qd_plan *p = new qd_plan();
    p->reg = r;
    p->gates.reserve(segs.size());
    std::vector<std::vector<uint16_t>> tc_terms;
    std::vector<int> tc_index;
    std::vector<DiagRunSpec> runs;
    const RegisterShape sh = shape_of(r);
    int rc = QD_OK;
    for (size_t si = 0; si < segs.size(); ++si) {
        const auto &sg = segs[si];
        GatePlan g;
        if (sg.first == sg.second) {
            bool noop = false;
            rc = prepare_gate(r, orig[sg.first], g, &noop);
            if (rc == QD_OK && noop) continue;
        } else {
            bool all_mono = true, all_diag = true;  // the product is then a permutation with phases / a diagonal
            std::vector<int> uq;
            for (int i = sg.first; i <= sg.second; ++i) {
                all_mono = all_mono && fg[i].mono;
                all_diag = all_diag && fg[i].diag;
                for (int q : fg[i].acting)
                    if (std::find(uq.begin(), uq.end(), q) == uq.end()) uq.push_back(q);
            }
            (void)sh;
            if (kinds[si] == kKernelDenseTable) {
                runs.emplace_back();
                runs.back().plan_index = (int)p->gates.size();
                rc = plan_dense_table(r, fg, sg.first, sg.second, kmax, g, runs.back());
                if (rc == QD_OK) {
                    ++p->blocks;
                    p->gates.push_back(g);
                    continue;
                }
                delete p;
                return rc;
            }
            if (kinds[si] == kKernelDiagTable) {
                runs.emplace_back();
                runs.back().plan_index = (int)p->gates.size();
                rc = plan_diag_run(r, fg, sg.first, sg.second, g, runs.back());
                if (rc == QD_OK) {
                    ++p->blocks;
                    p->gates.push_back(g);
                    continue;
                }
                delete p;
                return rc;
            }
            FuseBlock b = build_block(fg, sg.first, sg.second, r->dims);
            if ((int)b.qudits.size() > QD_MAX_TARGETS) {
                rc = fail(QD_ERR_DIM, "fused block spans more than 6 qudits");
            } else if (b.D <= kTcMaxD && kinds[si] == kKernelBlockTc) {
                tc_terms.emplace_back();
                rc = plan_block_tc(r, b, g, tc_terms.back());
                tc_index.push_back((int)p->gates.size());
            } else {
                rc = plan_block(r, b, g);
                if (rc == QD_OK && g.D == 0) continue;
            }
            if (rc == QD_OK) ++p->blocks;
        }
        if (rc) {
            delete p;
            return rc;
        }
        p->gates.push_back(g);
    }
    if (!tc_terms.empty()) {  // one device buffer for every tensor-core block's terms
        size_t total = 0;
        for (auto &t : tc_terms) total += (t.size() * 2 + 255) / 256 * 256;
        if (cudaMalloc(&p->tc_buf, total) != cudaSuccess) {
            cudaGetLastError();
            p->tc_buf = nullptr;
            delete p;
            return fail(QD_ERR_OOM, "tensor-core block terms allocation failed");
        }
        size_t off = 0;
        for (size_t i = 0; i < tc_terms.size(); ++i) {
            char *dst = static_cast<char *>(p->tc_buf) + off;
            cudaError_t e = cudaMemcpy(dst, tc_terms[i].data(), tc_terms[i].size() * 2, cudaMemcpyHostToDevice);
            if (e != cudaSuccess) {
                delete p;
                return cuda_fail(e, "tensor-core block terms upload");
            }
            p->gates[tc_index[i]].tc_terms = dst;
            off += (tc_terms[i].size() * 2 + 255) / 256 * 256;
        }
    }
    if (!runs.empty()) {  // one device buffer for every diagonal run's table, built on the device
        const size_t esz = 16;  // float4 (hi, lo) or double2
        size_t total = 0;
        for (auto &ru : runs) total += (p->gates[ru.plan_index].tab_size * esz + 255) / 256 * 256;
        if (cudaMalloc(&p->tab_buf, total) != cudaSuccess) {
            cudaGetLastError();
            p->tab_buf = nullptr;
            delete p;
            return fail(QD_ERR_OOM, "diagonal run table allocation failed");
        }
        size_t off = 0;
        for (auto &ru : runs) {
            GatePlan &gp = p->gates[ru.plan_index];
            char *dst = static_cast<char *>(p->tab_buf) + off;
            DiagGateDesc *dg = nullptr;
            double2 *pool = nullptr;
            cudaError_t e = cudaMalloc(&dg, sizeof(DiagGateDesc) * ru.gates.size());
            if (e == cudaSuccess) e = cudaMalloc(&pool, sizeof(double) * ru.pool.size());
            if (e == cudaSuccess)
                e = cudaMemcpy(dg, ru.gates.data(), sizeof(DiagGateDesc) * ru.gates.size(), cudaMemcpyHostToDevice);
            if (e == cudaSuccess) e = cudaMemcpy(pool, ru.pool.data(), sizeof(double) * ru.pool.size(), cudaMemcpyHostToDevice);
            if (e == cudaSuccess)
                e = diag_table_build(dst, r->prec, gp.tab_size, ru.range, dg, (int32_t)ru.gates.size(), pool,
                                     r->sm_count, r->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(r->stream);
            if (dg) cudaFree(dg);
            if (pool) cudaFree(pool);
            if (e != cudaSuccess) {
                delete p;
                return cuda_fail(e, "diagonal run table");
            }
            gp.tab = dst;
            off += (gp.tab_size * esz + 255) / 256 * 256;
        }
    }
    *out = p;
    return QD_OK;
}
}  // namespace

extern "C" {

int qd_plan_create(qd_reg *r, const qd_gate *gates, int32_t ngates, int32_t plan_kind, qd_plan **out) {
    if (!out) return fail(QD_ERR_ARG, "null output handle");
    *out = nullptr;
    if (int rc = reg_ok(r)) return rc;
    if (ngates < 0 || (ngates > 0 && !gates)) return fail(QD_ERR_ARG, "bad gate list");
    if (plan_kind < QD_PLAN_NONE || plan_kind > QD_PLAN_EXHAUSTIVE) return fail(QD_ERR_ARG, "unknown plan kind");
    std::vector<FuseGate> fg;
    std::vector<const qd_gate *> orig;
    int rc = collect_gates(r, gates, ngates, fg, orig);
    if (rc) return rc;
    std::vector<std::pair<int, int>> segs;
    std::vector<int> kinds;
    if ((rc = segments_for(r, fg, plan_kind, segs, kinds, nullptr))) return rc;
    rc = build_plan(r, fg, orig, segs, kinds, r->fuse_kmax, out);
    if (rc == QD_OK) (*out)->measure_after = has_measure(gates, ngates);
    return rc;
}

static_assert(kKernelMono == QD_FORM_MONO && kKernelDense == QD_FORM_DENSE && kKernelBlock == QD_FORM_BLOCK &&
                  kKernelBlockTc == QD_FORM_BLOCK_TC && kKernelDiagTable == QD_FORM_DIAG_RUN &&
                  kKernelDenseTable == QD_FORM_DENSE_RUN,
              "kernel forms of the planner and the C ABI differ");

namespace {
// The register's shape with the hard block limits of an explicit
// segmentation (not the register's fusion limits).
RegisterShape hard_shape(const qd_reg *r) {
    RegisterShape sh = shape_of(r);
    sh.fuse_dmax = r->prec == QD_C64 ? kTcMaxD : QD_MAX_D;
    return sh;
}
}  // namespace

int qd_plan_create_segmented(qd_reg *r, const qd_gate *gates, int32_t ngates, const int32_t *seg_first,
                             const int32_t *seg_last, int32_t nseg, qd_plan **out) {
    return qd_plan_create_forms(r, gates, ngates, seg_first, seg_last, nullptr, nseg, out);
}

int qd_plan_create_forms(qd_reg *r, const qd_gate *gates, int32_t ngates, const int32_t *seg_first,
                         const int32_t *seg_last, const int32_t *seg_kind, int32_t nseg, qd_plan **out) {
    if (!out) return fail(QD_ERR_ARG, "null output handle");
    *out = nullptr;
    if (int rc = reg_ok(r)) return rc;
    if (ngates < 0 || (ngates > 0 && !gates) || nseg < 0 || (nseg > 0 && (!seg_first || !seg_last)))
        return fail(QD_ERR_ARG, "bad arguments");
    std::vector<FuseGate> fg;
    std::vector<const qd_gate *> orig;
    int rc = collect_gates(r, gates, ngates, fg, orig);
    if (rc) return rc;
    std::vector<std::pair<int, int>> segs;
    int next = 0;
    for (int i = 0; i < nseg; ++i) {
        if (seg_first[i] != next || seg_last[i] < seg_first[i] || seg_last[i] >= (int)fg.size())
            return fail(QD_ERR_ARG, "segments must cover the non-identity gates contiguously and in order");
        segs.push_back({seg_first[i], seg_last[i]});
        next = seg_last[i] + 1;
    }
    if (next != (int)fg.size()) return fail(QD_ERR_ARG, "segments do not cover every gate");
    for (auto &sg : segs) {
        if (sg.first == sg.second) continue;
        std::vector<int> qs;
        int64_t D = 1;
        bool all_diag = true;
        for (int gi = sg.first; gi <= sg.second; ++gi) {
            all_diag = all_diag && fg[gi].diag;
            for (int q : fg[gi].acting)
                if (std::find(qs.begin(), qs.end(), q) == qs.end()) {
                    qs.push_back(q);
                    D = std::min<int64_t>(D * r->dims[q], int64_t(1) << 40);
                }
        }
        // a run of diagonal gates may span any qudits whose range table fits,
        // and so may a dense part of at most 16 states followed by such a run
        if (all_diag && diag_table_size(shape_of(r), qs) <= kDiagRunMaxTable) continue;
        if (dense_table_split(fg, sg.first, sg.second, shape_of(r), QD_MAX_TARGETS).ok) continue;
        const int64_t cap = r->prec == QD_C64 ? kTcMaxD : QD_MAX_D;
        if ((int)qs.size() > QD_MAX_TARGETS || D > cap) return fail(QD_ERR_DIM, "segment block too large");
    }
    // kernels of the given segments as the register's cost model prices them,
    // within the hard block limits rather than the register's fusion limits
    // (or as given: each given form must be one of the segment's feasible ones)
    std::vector<int> kinds(segs.size(), 0);
    {
        const RegisterShape sh = hard_shape(r);
        const CostFn cost = cost_for(r, QD_PLAN_GREEDY);
        for (size_t i = 0; i < segs.size(); ++i) {
            if (!seg_kind || seg_kind[i] < 0) {
                segment_cost(fg, segs[i].first, segs[i].second, sh, cost, QD_MAX_TARGETS, &kinds[i]);
                continue;
            }
            bool ok = false;
            for (const LaunchFeatures &f : segment_forms(fg, segs[i].first, segs[i].second, sh, QD_MAX_TARGETS))
                ok = ok || (int)f.f[10] == seg_kind[i];
            if (!ok) return fail(QD_ERR_ARG, "kernel form not feasible for the segment");
            kinds[i] = seg_kind[i];
        }
    }
    rc = build_plan(r, fg, orig, segs, kinds, QD_MAX_TARGETS, out);
    if (rc == QD_OK) (*out)->measure_after = has_measure(gates, ngates);
    return rc;
}

int qd_set_cost_model(qd_reg *r, qd_model *model) {
    if (int rc = reg_ok(r)) return rc;
    r->model = model;
    return QD_OK;
}

int qd_segment_features(qd_reg *r, const qd_gate *gates, int32_t ngates, int32_t first, int32_t last, float *out) {
    if (int rc = reg_ok(r)) return rc;
    if (!out) return fail(QD_ERR_ARG, "null output");
    std::vector<FuseGate> fg;
    std::vector<const qd_gate *> orig;
    if (int rc = collect_gates(r, gates, ngates, fg, orig)) return rc;
    if (first < 0 || last < first || last >= (int)fg.size()) return fail(QD_ERR_ARG, "bad segment");
    // the form an explicit segmentation of this segment runs
    const RegisterShape sh = hard_shape(r);
    int kind = -1;
    segment_cost(fg, first, last, sh, cost_for(r, QD_PLAN_GREEDY), QD_MAX_TARGETS, &kind);
    for (const LaunchFeatures &f : segment_forms(fg, first, last, sh, QD_MAX_TARGETS))
        if ((int)f.f[10] == kind) {
            std::copy(f.f, f.f + kFeatures, out);
            return QD_OK;
        }
    return fail(QD_ERR_ARG, "segment has no feasible form");
}

int qd_segment_forms(qd_reg *r, const qd_gate *gates, int32_t ngates, int32_t first, int32_t last, int32_t *kinds,
                     float *features, int32_t cap, int32_t *nforms) {
    if (int rc = reg_ok(r)) return rc;
    if (!nforms || cap < 0 || (cap > 0 && (!kinds || !features))) return fail(QD_ERR_ARG, "bad output arrays");
    std::vector<FuseGate> fg;
    std::vector<const qd_gate *> orig;
    if (int rc = collect_gates(r, gates, ngates, fg, orig)) return rc;
    if (first < 0 || last < first || last >= (int)fg.size()) return fail(QD_ERR_ARG, "bad segment");
    const std::vector<LaunchFeatures> forms = segment_forms(fg, first, last, hard_shape(r), QD_MAX_TARGETS);
    *nforms = (int32_t)forms.size();
    for (int i = 0; i < (int)forms.size() && i < cap; ++i) {
        kinds[i] = (int32_t)forms[i].f[10];
        std::copy(forms[i].f, forms[i].f + kFeatures, features + (size_t)i * kFeatures);
    }
    if (cap == 0 && !kinds && !features) return QD_OK;  // a count query
    return (int)forms.size() > cap ? fail(QD_ERR_OOM, "more forms than the arrays hold") : QD_OK;
}

namespace {
// Enqueue every launch of the plan (and, when profiling, an event before each
// launch and after the last) on stream s.
cudaError_t enqueue_plan(qd_plan *p, cudaStream_t s) {
    const bool prof = p->profile && p->events.size() == p->gates.size() + 1;
    qd_reg tmp = *p->reg;
    tmp.stream = s;
    for (size_t i = 0; i < p->gates.size(); ++i) {
        if (prof) {
            cudaError_t e = cudaEventRecord(p->events[i], s);
            if (e != cudaSuccess) return e;
        }
        cudaError_t e = launch_plan(&tmp, p->gates[i]);
        if (e != cudaSuccess) return e;
    }
    if (prof) return cudaEventRecord(p->events[p->gates.size()], s);
    return cudaSuccess;
}
}  // namespace

namespace {
// Host function that holds the stream until the enqueueing thread has
// submitted the whole profiled run (bounded: gives up after ~2 s), so the
// per-launch events measure back-to-back kernels, not host submission.
void CUDART_CB hold_until_open(void *arg) {
    auto *flag = static_cast<std::atomic<int> *>(arg);
    for (int i = 0; i < 200000 && flag->load(std::memory_order_acquire) == 0; ++i)
        std::this_thread::sleep_for(std::chrono::microseconds(10));
}
}  // namespace

int qd_plan_run(qd_plan *p) {
    if (!p) return fail(QD_ERR_ARG, "null plan");
    if (p->reg->measured) return QD_OK;  // gates after the measurement flag are ignored (Sec. 3.4)
    if (p->measure_after) p->reg->measured = true;  // set now: the launches below are still ordered before any later call
    cudaStream_t s = p->reg->stream;
    if (p->profile) {  // events cannot be timed inside a graph: direct launches behind a hold
        QD_CUDA(cudaStreamSynchronize(s));
        p->gate_open.store(0, std::memory_order_release);
        cudaError_t e = cudaLaunchHostFunc(s, hold_until_open, &p->gate_open);
        if (e == cudaSuccess) e = enqueue_plan(p, s);
        p->gate_open.store(1, std::memory_order_release);
        if (e != cudaSuccess) return cuda_fail(e, "profiled launch");
        return QD_OK;
    }
    if (!s || !p->use_graph) {  // the legacy default stream cannot be captured: launch directly
        cudaError_t e = enqueue_plan(p, s);
        if (e != cudaSuccess) return cuda_fail(e, "gate launch");
        return QD_OK;
    }
    if (!p->exec) {
        p->drop_graph();
        QD_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = enqueue_plan(p, s);
        cudaGraph_t graph = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(s, &graph);
        if (e != cudaSuccess || e2 != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            return cuda_fail(e != cudaSuccess ? e : e2, "plan capture");
        }
        e = cudaGraphInstantiate(&p->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            p->exec = nullptr;
            return cuda_fail(e, "graph instantiate");
        }
    }
    QD_CUDA(cudaGraphLaunch(p->exec, s));
    return QD_OK;
}

int qd_plan_profile(qd_plan *p, int32_t enable) {
    if (!p) return fail(QD_ERR_ARG, "null plan");
    p->profile = enable != 0;
    if (p->profile && p->events.size() != p->gates.size() + 1) {
        for (cudaEvent_t e : p->events) cudaEventDestroy(e);
        p->events.clear();
        for (size_t i = 0; i <= p->gates.size(); ++i) {
            cudaEvent_t e;
            QD_CUDA(cudaEventCreate(&e));
            p->events.push_back(e);
        }
    }
    return QD_OK;
}

int qd_plan_timings(qd_plan *p, float *ms, double *alg_bytes, int32_t *kclass) {
    if (!p) return fail(QD_ERR_ARG, "null plan");
    const size_t n = p->gates.size();
    if (ms) {
        if (!p->profile || p->events.size() != n + 1) return fail(QD_ERR_ARG, "profiling is not enabled");
        QD_CUDA(cudaStreamSynchronize(p->reg->stream));
        for (size_t i = 0; i < n; ++i) QD_CUDA(cudaEventElapsedTime(&ms[i], p->events[i], p->events[i + 1]));
    }
    for (size_t i = 0; i < n; ++i) {
        const GatePlan &g = p->gates[i];
        if (alg_bytes) alg_bytes[i] = g.alg_bytes;
        if (kclass) {
            int c = g.kind == Kind::Dense ? (g.mode == Mode::Direct ? QD_KCLASS_DENSE_DIRECT : QD_KCLASS_DENSE_TILE)
                                          : (g.mode == Mode::Direct ? QD_KCLASS_MONO_DIRECT : QD_KCLASS_MONO_TILE);
            if (g.mode == Mode::Tensor) c = QD_KCLASS_TENSOR_BLOCK;
            if (g.mode == Mode::Table) c = QD_KCLASS_DIAG_TABLE;
            if (g.mode == Mode::Direct && g.tab) c = QD_KCLASS_DENSE_TABLE;
            kclass[i] = c | (g.D << 8);
        }
    }
    return QD_OK;
}

int qd_plan_info(const qd_plan *p, int32_t *launches, int32_t *blocks) {
    if (!p) return fail(QD_ERR_ARG, "null plan");
    if (launches) *launches = (int32_t)p->gates.size();
    if (blocks) *blocks = p->blocks;
    return QD_OK;
}

int qd_plan_destroy(qd_plan *p) {
    delete p;
    return QD_OK;
}

int qd_run_circuit(qd_reg *r, const qd_gate *gates, int32_t ngates, int32_t plan_kind) {
    qd_plan *p = nullptr;
    int rc = qd_plan_create(r, gates, ngates, plan_kind, &p);
    if (rc) return rc;
    p->use_graph = false;  // one run: direct launches, no capture cost
    rc = qd_plan_run(p);
    qd_plan_destroy(p);
    return rc;
}

int qd_norm(qd_reg *r, double *out) {
    if (int rc = reg_ok(r)) return rc;
    if (!out) return fail(QD_ERR_ARG, "null output");
    const int nb = reduce_blocks(r->sm_count);
    Expand64 ex{};
    double *res = r->red + nb * 64;
    QD_CUDA(slice_norms(r->psi, r->prec, (uint64_t)r->N, ex, 0, 1, r->red, nb, res, r->stream));
    QD_CUDA(cudaMemcpyAsync(out, res, sizeof(double), cudaMemcpyDeviceToHost, r->stream));
    QD_CUDA(cudaStreamSynchronize(r->stream));
    return QD_OK;
}

int qd_overlap(qd_reg *a, qd_reg *b, double *re, double *im) {
    if (int rc = reg_ok(a)) return rc;
    if (int rc = reg_ok(b)) return rc;
    if (!re || !im) return fail(QD_ERR_ARG, "null output");
    if (a->N != b->N) return fail(QD_ERR_DIM, "registers differ in size");
    const int nb = reduce_blocks(a->sm_count);
    double *res = a->red + (size_t)nb * 64;
    if (b->stream != a->stream) {  // b's pending work must finish before a's stream reads it
        QD_CUDA(cudaStreamSynchronize(b->stream));
    }
    QD_CUDA(overlap(a->psi, a->prec, b->psi, b->prec, (uint64_t)a->N, a->red, nb, res, a->stream));
    double h[2];
    QD_CUDA(cudaMemcpyAsync(h, res, sizeof(h), cudaMemcpyDeviceToHost, a->stream));
    QD_CUDA(cudaStreamSynchronize(a->stream));
    *re = h[0];
    *im = h[1];
    return QD_OK;
}

int qd_marginal(qd_reg *r, int32_t q, double *out) {
    if (int rc = reg_ok(r)) return rc;
    if (!out) return fail(QD_ERR_ARG, "null output");
    if (q < 0 || q >= r->n) return fail(QD_ERR_ARG, "qudit out of range");
    const int nb = reduce_blocks(r->sm_count);
    const int d = r->dims[q];
    Expand64 ex{};
    set_expand64(ex, {{r->s[q], d}});
    double *res = r->red + (size_t)nb * 64;
    QD_CUDA(slice_norms(r->psi, r->prec, (uint64_t)(r->N / d), ex, (uint64_t)r->s[q], d, r->red, nb, res, r->stream));
    QD_CUDA(cudaMemcpyAsync(out, res, sizeof(double) * d, cudaMemcpyDeviceToHost, r->stream));
    QD_CUDA(cudaStreamSynchronize(r->stream));
    return QD_OK;
}

int qd_probabilities(qd_reg *r, double *out, int32_t where) {
    if (int rc = reg_ok(r)) return rc;
    if (!out) return fail(QD_ERR_ARG, "null output");
    if (where == QD_DEVICE) {
        QD_CUDA(probabilities(r->psi, r->prec, (uint64_t)r->N, out, r->sm_count, r->stream));
        return QD_OK;
    }
    if (where != QD_HOST) return fail(QD_ERR_ARG, "where must be QD_HOST or QD_DEVICE");
    int rc = ensure_cdf(r);  // reuse the CDF buffer as staging
    if (rc) return rc;
    QD_CUDA(probabilities(r->psi, r->prec, (uint64_t)r->N, r->cdf, r->sm_count, r->stream));
    QD_CUDA(cudaMemcpyAsync(out, r->cdf, sizeof(double) * r->N, cudaMemcpyDeviceToHost, r->stream));
    QD_CUDA(cudaStreamSynchronize(r->stream));
    return QD_OK;
}

int qd_cdf(qd_reg *r, double *out, int32_t where) {
    if (int rc = reg_ok(r)) return rc;
    if (!out) return fail(QD_ERR_ARG, "null output");
    if (where != QD_HOST && where != QD_DEVICE) return fail(QD_ERR_ARG, "where must be QD_HOST or QD_DEVICE");
    int rc = compute_cdf(r);
    if (rc) return rc;
    QD_CUDA(cudaMemcpyAsync(out, r->cdf, sizeof(double) * r->N,
                            where == QD_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, r->stream));
    if (where == QD_HOST) QD_CUDA(cudaStreamSynchronize(r->stream));
    return QD_OK;
}

static int sample_impl(qd_reg *r, const double *u_host, uint64_t seed, int64_t shots, int64_t *out) {
    if (int rc = reg_ok(r)) return rc;
    if (!out || shots < 0) return fail(QD_ERR_ARG, "bad sample arguments");
    if (shots == 0) return QD_OK;
    int rc = compute_cdf(r);
    if (rc) return rc;
    double *u_dev = nullptr;
    int64_t *o_dev = nullptr;
    if (u_host && cudaMalloc(&u_dev, sizeof(double) * shots) != cudaSuccess) return fail(QD_ERR_OOM, "sample buffer");
    if (cudaMalloc(&o_dev, sizeof(int64_t) * shots) != cudaSuccess) {
        if (u_dev) cudaFree(u_dev);
        return fail(QD_ERR_OOM, "sample buffer");
    }
    cudaError_t e = cudaSuccess;
    if (u_host) e = cudaMemcpyAsync(u_dev, u_host, sizeof(double) * shots, cudaMemcpyHostToDevice, r->stream);
    if (e == cudaSuccess) e = sample(r->cdf, (uint64_t)r->N, u_dev, seed, shots, o_dev, r->sm_count, r->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, o_dev, sizeof(int64_t) * shots, cudaMemcpyDeviceToHost, r->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(r->stream);
    if (u_dev) cudaFree(u_dev);
    cudaFree(o_dev);
    if (e != cudaSuccess) return cuda_fail(e, "sample");
    return QD_OK;
}

int qd_sample(qd_reg *r, uint64_t seed, int64_t shots, int64_t *out) { return sample_impl(r, nullptr, seed, shots, out); }

int qd_sample_u(qd_reg *r, const double *u, int64_t shots, int64_t *out) {
    if (!u) return fail(QD_ERR_ARG, "null uniforms");
    return sample_impl(r, u, 0, shots, out);
}

int qd_get_amplitudes(qd_reg *r, void *out, int32_t where) {
    if (int rc = reg_ok(r)) return rc;
    if (!out) return fail(QD_ERR_ARG, "null output");
    if (where != QD_HOST && where != QD_DEVICE) return fail(QD_ERR_ARG, "where must be QD_HOST or QD_DEVICE");
    QD_CUDA(cudaMemcpyAsync(out, r->psi, r->esize * r->N,
                            where == QD_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, r->stream));
    if (where == QD_HOST) QD_CUDA(cudaStreamSynchronize(r->stream));
    return QD_OK;
}

int qd_set_amplitudes(qd_reg *r, const void *in, int32_t where) {
    if (int rc = reg_ok(r)) return rc;
    if (!in) return fail(QD_ERR_ARG, "null input");
    if (where != QD_HOST && where != QD_DEVICE) return fail(QD_ERR_ARG, "where must be QD_HOST or QD_DEVICE");
    QD_CUDA(cudaMemcpyAsync(r->psi, in, r->esize * r->N,
                            where == QD_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, r->stream));
    r->measured = false;  // a new input state starts a new circuit
    return QD_OK;
}

int qd_ket_list(qd_reg *r, int32_t method, double threshold, int64_t cap, int64_t *indices, double *values,
                int64_t *count) {
    if (int rc = reg_ok(r)) return rc;
    if (method != QD_OUT_AMPLITUDE && method != QD_OUT_PROBABILITY) return fail(QD_ERR_ARG, "unknown output method");
    if (!count || cap < 0 || (cap > 0 && (!indices || !values))) return fail(QD_ERR_ARG, "bad output arguments");
    if (!(threshold >= 0.0)) return fail(QD_ERR_ARG, "threshold must be >= 0");
    const uint64_t nch = ket_chunks((uint64_t)r->N);
    const size_t per = method == QD_OUT_AMPLITUDE ? 2 : 1;
    int64_t *counts = nullptr, *idx_dev = nullptr;
    double *val_dev = nullptr;
    int rc = QD_OK;
    if (cudaMalloc(&counts, sizeof(int64_t) * (2 * nch + 1)) != cudaSuccess) return fail(QD_ERR_OOM, "ket scratch");
    if (cap > 0 && (cudaMalloc(&idx_dev, sizeof(int64_t) * cap) != cudaSuccess ||
                    cudaMalloc(&val_dev, sizeof(double) * per * cap) != cudaSuccess))
        rc = fail(QD_ERR_OOM, "ket output buffers");
    int64_t total = 0;
    if (rc == QD_OK) {
        int64_t *offsets = counts + nch;
        cudaError_t e = ket_select(r->psi, r->prec, (uint64_t)r->N, threshold, method == QD_OUT_AMPLITUDE ? 0 : 1,
                                   cap, counts, offsets, idx_dev, val_dev, r->sm_count, r->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(&total, offsets + nch, sizeof(int64_t), cudaMemcpyDeviceToHost, r->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(r->stream);
        const int64_t n = total < cap ? total : cap;
        if (e == cudaSuccess && n > 0)
            e = cudaMemcpy(indices, idx_dev, sizeof(int64_t) * n, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && n > 0) e = cudaMemcpy(values, val_dev, sizeof(double) * per * n, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) rc = cuda_fail(e, "ket readout");
    }
    if (counts) cudaFree(counts);
    if (idx_dev) cudaFree(idx_dev);
    if (val_dev) cudaFree(val_dev);
    if (rc == QD_OK) *count = total;
    return rc;
}

int qd_run_moments(qd_reg *r, const qd_gate *gates, int32_t ngates, int32_t *n_moments) {
    if (int rc = reg_ok(r)) return rc;
    if (ngates < 0 || (ngates > 0 && !gates)) return fail(QD_ERR_ARG, "bad gate list");
    if (r->N > kKronMaxN || r->n > kKronMaxQudits)
        return fail(QD_ERR_DIM, "the moment path keeps N x N operators: registers of at most 4096 amplitudes");
    if (r->measured) {
        if (n_moments) *n_moments = 0;
        return QD_OK;
    }
    std::vector<FuseGate> fg;
    std::vector<const qd_gate *> orig;
    if (int rc = collect_gates(r, gates, ngates, fg, orig)) return rc;
    int nm = 0;
    cudaError_t e = run_moments(r->psi, r->prec, r->N, r->n, r->dims, fg, &nm, r->stream);
    if (e != cudaSuccess) return cuda_fail(e, "moment path");
    if (has_measure(gates, ngates)) r->measured = true;
    if (n_moments) *n_moments = nm;
    return QD_OK;
}

int qd_apply_toffoli(qd_reg *r, int32_t c1, int32_t carrier, int32_t t, int32_t shift) {
    if (int rc = reg_ok(r)) return rc;
    qd_gate g[3];
    if (int rc = qd_toffoli_gates(r->dims, r->n, c1, carrier, t, shift, g)) return rc;
    for (const qd_gate &x : g)
        if (int rc = apply_record(r, &x)) return rc;
    return QD_OK;
}

int qd_apply_mct_tree(qd_reg *r, const int32_t *controls, const int32_t *ctrl_levels, int32_t nc, int32_t t,
                      int32_t shift) {
    if (int rc = reg_ok(r)) return rc;
    int32_t count = 0;
    if (int rc = qd_mct_tree_gates(r->dims, r->n, controls, ctrl_levels, nc, t, shift, nullptr, 0, &count, nullptr))
        return rc;
    std::vector<qd_gate> g((size_t)count);
    if (int rc = qd_mct_tree_gates(r->dims, r->n, controls, ctrl_levels, nc, t, shift, g.data(), count, &count,
                                   nullptr))
        return rc;
    for (const qd_gate &x : g)
        if (int rc = apply_record(r, &x)) return rc;
    return QD_OK;
}

int qd_sync(qd_reg *r, int32_t *device_error) {
    if (int rc = reg_ok(r)) return rc;
    int32_t err = 0;
    QD_CUDA(cudaMemcpyAsync(&err, r->dev_err, sizeof(int32_t), cudaMemcpyDeviceToHost, r->stream));
    QD_CUDA(cudaStreamSynchronize(r->stream));
    if (device_error) *device_error = err;
    if (err == 1) return fail(QD_ERR_TIMEOUT, "a bounded device wait of the tensor-core kernel expired");
    if (err) return fail(QD_ERR_DEVICE, "device error word set: " + std::to_string(err));
    return QD_OK;
}

int qd_debug_gate_members(const int32_t *dims, int32_t n, const qd_gate *gate, int64_t *out, int64_t cap,
                          int64_t *info) {
    return qd_debug_gate_members_tuned(dims, n, gate, -1, out, cap, info);
}

int qd_debug_gate_members_tuned(const int32_t *dims, int32_t n, const qd_gate *gate, int64_t tile_stride,
                                int64_t *out, int64_t cap, int64_t *info) {
    if (!dims || n < 1 || n > QD_MAX_QUDITS || !info) return fail(QD_ERR_ARG, "bad arguments");
    qd_reg r;
    r.n = n;
    int64_t s = 1;
    for (int q = 0; q < n; ++q) {
        if (dims[q] < 2 || dims[q] > 64) return fail(QD_ERR_DIM, "qudit dimension must be in [2, 64]");
        r.dims[q] = dims[q];
        r.s[q] = s;
        s *= dims[q];
    }
    r.s[n] = s;
    r.N = s;
    r.esize = 8;
    r.tile_stride = tile_stride;
    GatePlan g;
    bool noop = false;
    int rc = prepare_gate(&r, gate, g, &noop);
    if (rc) return rc;
    for (int i = 0; i < 7; ++i) info[i] = 0;
    info[6] = noop ? 1 : 0;
    if (noop) return QD_OK;
    const int D = g.D;
    info[0] = g.mode == Mode::Tile ? 1 : 0;
    info[1] = D;
    info[3] = g.kind == Kind::Mono ? 1 : 0;
    info[4] = g.active;
    info[5] = g.B;
    int64_t w = 0;
    auto put = [&](int64_t v) {
        if (out && w < cap) out[w] = v;
        ++w;
    };
    if (g.mode == Mode::Direct) {
        info[2] = (int64_t)g.R;
        for (uint64_t gi = 0; gi < g.R; ++gi) {
            const uint64_t base = expand(gi, g.ex) + g.base_off;
            for (int j = 0; j < D; ++j) put((int64_t)(base + g.off[j]));
        }
        return QD_OK;
    }
    info[2] = (int64_t)(g.R_tiles * g.G_in);
    std::vector<uint64_t> cb(g.DH);
    for (uint64_t t = 0; t < g.R_tiles; ++t) {
        for (uint32_t h = 0; h < g.DH; ++h) cb[h] = expand(t, g.ex_hi) * g.B + g.base_off_hi + g.offH[h];
        for (uint32_t gl = 0; gl < g.G_in; ++gl) {
            const uint32_t eb = expand(gl, g.ex_lo) + g.lo_off;
            for (int j = 0; j < D; ++j) {
                const uint32_t p = eb + (uint32_t)g.smoff[j];
                const uint32_t c = fdiv(p, g.divB);
                put((int64_t)(cb[c] + (p - c * g.B)));
            }
        }
    }
    return QD_OK;
}

namespace {
int host_register(const int32_t *dims, int32_t n, int32_t precision, qd_reg &r) {
    if (!dims || n < 1 || n > QD_MAX_QUDITS) return fail(QD_ERR_ARG, "bad dims");
    r.n = n;
    int64_t s = 1;
    for (int q = 0; q < n; ++q) {
        if (dims[q] < 2 || dims[q] > 64) return fail(QD_ERR_DIM, "qudit dimension must be in [2, 64]");
        r.dims[q] = dims[q];
        r.s[q] = s;
        s *= dims[q];
    }
    r.s[n] = s;
    r.N = s;
    r.prec = precision == QD_C128 ? QD_C128 : QD_C64;
    r.esize = r.prec == QD_C64 ? 8 : 16;
    return QD_OK;
}
}  // namespace

int qd_moment_packing(const int32_t *dims, int32_t n, const qd_gate *gates, int32_t ngates, int32_t *moment_of_gate,
                      int32_t *n_moments) {
    qd_reg r;
    if (int rc = host_register(dims, n, QD_C128, r)) return rc;
    if (ngates < 0 || (ngates > 0 && !gates)) return fail(QD_ERR_ARG, "bad gate list");
    std::vector<FuseGate> fg;
    std::vector<const qd_gate *> orig;
    if (int rc = collect_gates(&r, gates, ngates, fg, orig)) return rc;
    int nm = 0;
    const std::vector<int> m = pack_moments(n, fg, &nm);
    // identity gates were dropped: report -1 for them, the moment otherwise
    if (moment_of_gate) {
        for (int i = 0; i < ngates; ++i) moment_of_gate[i] = -1;
        for (size_t k = 0; k < orig.size(); ++k) moment_of_gate[orig[k] - gates] = m[k];
    }
    if (n_moments) *n_moments = nm;
    return QD_OK;
}


int qd_debug_fuse_plan(const int32_t *dims, int32_t n, int32_t precision, const qd_gate *gates, int32_t ngates,
                       int32_t plan_kind, int32_t kmax, int32_t dmax, int32_t *seg_first, int32_t *seg_last,
                       int32_t cap, int32_t *nseg, double *model_cost) {
    qd_reg r;
    if (int rc = host_register(dims, n, precision, r)) return rc;
    r.fuse_kmax = kmax;
    r.fuse_dmax = dmax;
    std::vector<FuseGate> fg;
    std::vector<const qd_gate *> orig;
    if (int rc = collect_gates(&r, gates, ngates, fg, orig)) return rc;
    std::vector<std::pair<int, int>> segs;
    std::vector<int> kinds;
    if (int rc = segments_for(&r, fg, plan_kind, segs, kinds, model_cost)) return rc;
    for (size_t i = 0; i < segs.size() && (int32_t)i < cap; ++i) {
        if (seg_first) seg_first[i] = segs[i].first;
        if (seg_last) seg_last[i] = segs[i].second;
    }
    if (nseg) *nseg = (int32_t)segs.size();
    return QD_OK;
}

int qd_debug_segment_cost(const int32_t *dims, int32_t n, int32_t precision, const qd_gate *gates, int32_t ngates,
                          int32_t first, int32_t last, double *cost) {
    qd_reg r;
    if (int rc = host_register(dims, n, precision, r)) return rc;
    std::vector<FuseGate> fg;
    std::vector<const qd_gate *> orig;
    if (int rc = collect_gates(&r, gates, ngates, fg, orig)) return rc;
    if (first < 0 || last < first || last >= (int)fg.size() || !cost) return fail(QD_ERR_ARG, "bad segment");
    *cost = segment_cost(fg, first, last, shape_of(&r), cost_for(&r, QD_PLAN_GREEDY), r.fuse_kmax);
    return QD_OK;
}

int qd_debug_segment_forms(const int32_t *dims, int32_t n, int32_t precision, const qd_gate *gates, int32_t ngates,
                           int32_t first, int32_t last, int32_t *kinds, float *features, int32_t cap,
                           int32_t *nforms) {
    qd_reg r;
    if (int rc = host_register(dims, n, precision, r)) return rc;
    if (!nforms || cap < 0 || (cap > 0 && (!kinds || !features))) return fail(QD_ERR_ARG, "bad output arrays");
    std::vector<FuseGate> fg;
    std::vector<const qd_gate *> orig;
    if (int rc = collect_gates(&r, gates, ngates, fg, orig)) return rc;
    if (first < 0 || last < first || last >= (int)fg.size()) return fail(QD_ERR_ARG, "bad segment");
    const std::vector<LaunchFeatures> forms = segment_forms(fg, first, last, hard_shape(&r), QD_MAX_TARGETS);
    *nforms = (int32_t)forms.size();
    for (int i = 0; i < (int)forms.size() && i < cap; ++i) {
        kinds[i] = (int32_t)forms[i].f[10];
        std::copy(forms[i].f, forms[i].f + kFeatures, features + (size_t)i * kFeatures);
    }
    return (int)forms.size() > cap ? fail(QD_ERR_OOM, "more forms than the arrays hold") : QD_OK;
}

int qd_debug_fuse_block(const int32_t *dims, int32_t n, const qd_gate *gates, int32_t ngates, int32_t first,
                        int32_t last, int32_t *qudits, int32_t *k, int32_t *D, double *matrix, int64_t cap) {
    qd_reg r;
    if (int rc = host_register(dims, n, QD_C128, r)) return rc;
    std::vector<FuseGate> fg;
    std::vector<const qd_gate *> orig;
    if (int rc = collect_gates(&r, gates, ngates, fg, orig)) return rc;
    if (first < 0 || last < first || last >= (int)fg.size()) return fail(QD_ERR_ARG, "bad segment");
    FuseBlock b = build_block(fg, first, last, r.dims);
    if ((int)b.qudits.size() > 6 || (int64_t)b.M.size() > cap) return fail(QD_ERR_DIM, "block too large for output");
    for (size_t i = 0; i < b.qudits.size(); ++i) qudits[i] = b.qudits[i];
    *k = (int32_t)b.qudits.size();
    *D = b.D;
    std::copy(b.M.begin(), b.M.end(), matrix);
    return QD_OK;
}

// ---------------------------------------------------------------- batches

}  // extern "C"

struct qd_batch {
    // One validated gate of a circuit: acting qudits and its matrix over the
    // targets (as in the per-gate path), kept until the batch is prepared.
    struct Stored {
        Acting a;
        std::vector<double> M;
        bool diag = false;
        uint64_t mask = 0;  // acting qudits (targets and controls)
    };
    int32_t ncirc = 0;
    std::vector<std::vector<int32_t>> dims;
    std::vector<uint64_t> N, offs, basis;
    std::vector<std::vector<Stored>> circ;
    uint64_t total = 0;       // amplitudes of all registers
    uint64_t arena_amps = 0;  // arena size: every register padded to an even count
    uint32_t tile_amps = 4096;
    int32_t ctas_per_sm = 0;
    uint32_t small_amps = 2048;
    uint64_t group_amps = uint64_t(1) << 25;
    uint32_t tiles_per_item = 1;
    uint32_t poll_limit = kBatchPollLimit;
    uint32_t tile_cap = 0;
    uint32_t desc_bytes = kBatchDescBytes;
    double alg_bytes = 0;
    int64_t nsegs = 0;
    bool profile = false;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    cudaStream_t stream = nullptr;
    int sm_count = 0;
    int32_t nitems = 0;
    bool dirty = true;
    // device
    float2 *arena = nullptr;
    double *probs = nullptr;
    BSeg *dsegs = nullptr;
    BChunk *dchunks = nullptr;
    BGate *dgates = nullptr;
    float2 *dcoef = nullptr;
    uint32_t *dhoff = nullptr;
    BItem *ditems = nullptr;
    uint64_t *doffs = nullptr, *dbasis = nullptr;
    uint32_t *dcounters = nullptr;
    int32_t *derr = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool host_only = false;  // host-side replay object: owns no device memory
    void free_tables() {
        if (host_only) return;
        cudaFree(dsegs);
        cudaFree(dchunks);
        cudaFree(dgates);
        cudaFree(dcoef);
        cudaFree(dhoff);
        cudaFree(ditems);
        dsegs = nullptr;
        dchunks = nullptr;
        dgates = nullptr;
        dcoef = nullptr;
        dhoff = nullptr;
        ditems = nullptr;
        if (exec) cudaGraphExecDestroy(exec);
        exec = nullptr;
    }
    ~qd_batch() {
        if (host_only) return;
        if (stream) cudaStreamSynchronize(stream);
        else cudaDeviceSynchronize();
        free_tables();
        cudaFree(arena);
        cudaFree(probs);
        cudaFree(doffs);
        cudaFree(dbasis);
        cudaFree(dcounters);
        cudaFree(derr);
        if (ev0) cudaEventDestroy(ev0);
        if (ev1) cudaEventDestroy(ev1);
    }
};

namespace {

uint64_t mask_product(const std::vector<int32_t> &dims, uint64_t m) {
    uint64_t p = 1;
    for (size_t q = 0; q < dims.size(); ++q)
        if ((m >> q) & 1u) p *= (uint64_t)dims[q];
    return p;
}

// Greedy segmentation of circuit c: a segment starts with one gate's acting
// qudits S and takes the following gates while the union stays within tmax
// amplitudes; S is then widened with the lowest remaining qudits that still
// fit (longer contiguous runs, fewer tiles), and the following gates acting
// inside the widened S join the segment.
std::vector<std::pair<int, uint64_t>> batch_segments(const qd_batch *b, int c, uint64_t tmax) {
    const auto &gs = b->circ[c];
    const auto &d = b->dims[c];
    std::vector<std::pair<int, uint64_t>> segs;  // (first gate, S)
    size_t i = 0;
    while (i < gs.size()) {
        uint64_t S = gs[i].mask;
        size_t j = i + 1;
        while (j < gs.size() && mask_product(d, S | gs[j].mask) <= tmax) S |= gs[j++].mask;
        uint64_t P = mask_product(d, S);
        for (size_t q = 0; q < d.size(); ++q)
            if (!((S >> q) & 1u) && P * (uint64_t)d[q] <= tmax) {
                S |= uint64_t(1) << q;
                P *= (uint64_t)d[q];
            }
        while (j < gs.size() && (gs[j].mask & ~S) == 0) ++j;
        segs.push_back({(int)i, S});
        i = j;
    }
    return segs;
}

// FP32 hi + lo parts of a gate's coefficients (dense: D x D, else D phases),
// appended to coef: ncoef hi entries, then ncoef lo entries.
void split_coef(const GatePlan &g, BGate &bg, std::vector<float2> &coef) {
    const int n = bg.kind == 0 ? g.D * g.D : g.D;
    const double *src = bg.kind == 0 ? g.U : g.lam;
    bg.ncoef = (uint32_t)n;
    std::vector<float2> hi(n), lo(n);
    for (int k = 0; k < n; ++k) {
        const double re = src[2 * k], im = src[2 * k + 1];
        hi[k] = make_float2((float)re, (float)im);
        lo[k] = make_float2((float)(re - (double)hi[k].x), (float)(im - (double)hi[k].y));
    }
    coef.insert(coef.end(), hi.begin(), hi.end());
    coef.insert(coef.end(), lo.begin(), lo.end());
}

// Expansion with adjacent insertions merged into runs (at most kBExMax).
bool merge_expand(const Expand64 &e, BEx &out) {
    out = BEx{};
    uint64_t dv[kMaxIns], sp[kMaxIns];
    int n = 0;
    for (int k = 0; k < e.n; ++k) {
        if (n > 0 && e.div[k].d == sp[n - 1]) {
            sp[n - 1] = e.span[k];
        } else {
            dv[n] = e.div[k].d;
            sp[n] = e.span[k];
            ++n;
        }
    }
    if (n > kBExMax) return false;
    out.n = n;
    for (int k = 0; k < n; ++k) {
        out.div[k] = make_fastdiv32((uint32_t)dv[k]);
        out.span[k] = (uint32_t)sp[k];
    }
    return true;
}

struct BatchTables {
    std::vector<BSeg> segs;
    std::vector<BChunk> chunks;
    std::vector<BGate> gates;
    std::vector<float2> coef;
    std::vector<uint32_t> hoff;
    std::vector<BItem> items;
    uint32_t cap = 1;
    uint32_t desc_bytes = kBatchDescBytes;  // largest chunk, at least the target size
    double bytes = 0;
};

// Segment and encode every circuit; build the work queue (host only).
int batch_tables(const qd_batch *b, BatchTables &tb) {
    std::vector<BSeg> &segs = tb.segs;
    std::vector<BChunk> &chunks = tb.chunks;
    std::vector<BGate> &gates = tb.gates;
    std::vector<float2> &coef = tb.coef;
    std::vector<uint32_t> &hoff = tb.hoff;
    std::vector<std::vector<int>> cseg(b->ncirc);  // segment indices per circuit
    uint32_t cap = 0;
    double bytes = 0;
    for (int c = 0; c < b->ncirc; ++c) {
        const auto &d = b->dims[c];
        const int n = (int)d.size();
        const uint64_t N = b->N[c];
        const uint64_t tmax = N <= b->small_amps ? N : std::min<uint64_t>(N, b->tile_amps);
        const auto parts = batch_segments(b, c, tmax);
        for (size_t p = 0; p < parts.size(); ++p) {
            const int first = parts[p].first;
            const int last = p + 1 < parts.size() ? parts[p + 1].first : (int)b->circ[c].size();
            const uint64_t S = parts[p].second;
            const uint64_t T = mask_product(d, S);
            if (T > kBatchMaxTile)
                return fail(QD_ERR_UNSUPPORTED, "a batched gate acts on more than 24576 amplitudes of its register");
            cap = std::max<uint32_t>(cap, (uint32_t)T);
            // local register over S (ascending qudits) and the position map
            std::vector<int32_t> ldims;
            int pos[QD_MAX_QUDITS];
            for (int q = 0; q < n; ++q)
                if ((S >> q) & 1u) {
                    pos[q] = (int)ldims.size();
                    ldims.push_back(d[q]);
                }
            qd_reg lr;
            if (int rc = host_register(ldims.data(), (int32_t)ldims.size(), QD_C64, lr)) return rc;
            lr.tile_stride = 0;  // direct geometry
            BSeg sg{};
            sg.chunk0 = (int32_t)chunks.size();
            const size_t gate_begin = gates.size();
            BChunk ch{(int32_t)gates.size(), 0, (uint32_t)coef.size(), 0};
            for (int gi = first; gi < last; ++gi) {
                const auto &st = b->circ[c][gi];
                Acting la = st.a;
                for (int m = 0; m < la.k; ++m) la.t[m] = pos[la.t[m]];
                for (int m = 0; m < la.nc; ++m) la.c[m] = pos[la.c[m]];
                GatePlan g;
                bool noop = false;
                if (int rc = plan_gate(&lr, st.M.data(), la, st.diag, g, &noop)) return rc;
                if (noop) continue;
                BGate bg{};
                bg.kind = g.kind == Kind::Dense ? 0 : 1;
                bg.D = g.D;
                bg.R = (uint32_t)g.R;
                bg.base = (uint32_t)g.base_off;
                if (!merge_expand(g.ex, bg.ex)) return fail(QD_ERR_UNSUPPORTED, "gate geometry exceeds the batch descriptor");
                for (int j = 0; j < g.D; ++j) {
                    bg.off[j] = (uint16_t)g.off[j];
                    bg.src[j] = (int8_t)g.src[j];
                }
                bg.active = g.active;
                bg.unit = g.unit;
                std::vector<float2> gc;
                split_coef(g, bg, gc);
                // close the chunk when this gate's descriptor and coefficients would overflow it
                const size_t need = (size_t)(ch.ngates + 1) * sizeof(BGate) + (ch.ncoef + gc.size()) * sizeof(float2);
                if (ch.ngates > 0 && need > kBatchDescBytes) {
                    chunks.push_back(ch);
                    ch = BChunk{(int32_t)gates.size(), 0, (uint32_t)coef.size(), 0};
                }
                bg.coef = ch.ncoef;
                ch.ncoef += (uint32_t)gc.size();
                ch.ngates += 1;
                coef.insert(coef.end(), gc.begin(), gc.end());
                gates.push_back(bg);
            }
            if (ch.ngates > 0) chunks.push_back(ch);
            sg.nchunks = (int32_t)chunks.size() - sg.chunk0;
            if (gates.size() == gate_begin) continue;
            // tile geometry: contiguous low block, run table over the rest of S
            int m = 0;
            uint64_t B = 1;
            while (m < n && ((S >> m) & 1u)) B *= (uint64_t)d[m++];
            sg.T = (uint32_t)T;
            sg.B = (uint32_t)B;
            sg.divB = make_fastdiv32((uint32_t)B);
            sg.pair = (B % 2 == 0) ? 1u : 0u;
            sg.hoff = (uint32_t)hoff.size();
            const uint64_t H = T / B;
            {
                // strides of the register
                std::vector<uint64_t> s(n + 1, 1);
                for (int q = 0; q < n; ++q) s[q + 1] = s[q] * (uint64_t)d[q];
                for (uint64_t h = 0; h < H; ++h) {
                    uint64_t rem = h, o = 0;
                    for (int q = m; q < n; ++q)
                        if ((S >> q) & 1u) {
                            o += (rem % (uint64_t)d[q]) * s[q];
                            rem /= (uint64_t)d[q];
                        }
                    hoff.push_back((uint32_t)o);
                }
                // tile index -> flat base: insert a zero digit run at every run of S
                std::vector<std::pair<int64_t, int64_t>> runs;
                for (int q = 0; q < n;) {
                    if (!((S >> q) & 1u)) {
                        ++q;
                        continue;
                    }
                    int e = q;
                    int64_t dp = 1;
                    while (e < n && ((S >> e) & 1u)) dp *= d[e++];
                    runs.push_back({(int64_t)s[q], dp});
                    q = e;
                }
                Expand64 ex64;
                set_expand64(ex64, runs);
                sg.ex = narrow(ex64);
            }
            sg.ntiles = (uint32_t)(N / T);
            cseg[c].push_back((int)segs.size());
            segs.push_back(sg);
            bytes += 16.0 * (double)N;
        }
    }
    // Work queue.  Circuits in groups of about group_amps amplitudes (a
    // circuit no larger than small_amps is one item); within a group items
    // go segment level by segment level, so that a group's states stay in L2.
    std::vector<BItem> &items = tb.items;
    std::vector<int> grp;
    uint64_t in_group = 0;
    auto flush_group = [&]() {
        size_t maxs = 0;
        for (int c : grp) maxs = std::max(maxs, cseg[c].size());
        std::vector<uint32_t> cum(grp.size(), 0);
        for (size_t L = 0; L < maxs; ++L)
            for (size_t k = 0; k < grp.size(); ++k) {
                const int c = grp[k];
                if (L >= cseg[c].size()) continue;
                const BSeg &sg = segs[cseg[c][L]];
                for (uint32_t t = 0; t < sg.ntiles; t += b->tiles_per_item) {
                    const uint32_t cnt = std::min(b->tiles_per_item, sg.ntiles - t);
                    items.push_back(BItem{c, cseg[c][L], t, cnt, cum[k], 0});
                }
                cum[k] += sg.ntiles;
            }
        grp.clear();
        in_group = 0;
    };
    for (int c = 0; c < b->ncirc; ++c) {
        if (cseg[c].empty()) continue;
        if (!grp.empty() && in_group + b->N[c] > b->group_amps) flush_group();
        grp.push_back(c);
        in_group += b->N[c];
    }
    if (!grp.empty()) flush_group();
    tb.cap = std::max<uint32_t>(cap, 1);
    tb.bytes = bytes;
    tb.desc_bytes = kBatchDescBytes;
    for (const BChunk &ch : chunks) {
        const size_t need = (size_t)ch.ngates * sizeof(BGate) + (size_t)ch.ncoef * sizeof(float2);
        tb.desc_bytes = std::max<uint32_t>(tb.desc_bytes, (uint32_t)((need + 15) / 16 * 16));
    }
    return QD_OK;
}

// Segment, encode and upload every circuit; build the work queue.
int batch_prepare(qd_batch *b) {
    b->free_tables();
    BatchTables tb;
    if (int rc = batch_tables(b, tb)) return rc;
    const auto &segs = tb.segs;
    const auto &gates = tb.gates;
    const auto &coef = tb.coef;
    const auto &hoff = tb.hoff;
    const auto &items = tb.items;
    b->nitems = (int32_t)items.size();
    b->nsegs = (int64_t)segs.size();
    b->alg_bytes = tb.bytes;
    b->tile_cap = tb.cap;
    b->desc_bytes = tb.desc_bytes;
    auto up = [&](void **dst, const void *src, size_t bytes_) -> int {
        if (bytes_ == 0) bytes_ = 16;
        if (cudaMalloc(dst, bytes_) != cudaSuccess) {
            cudaGetLastError();
            return fail(QD_ERR_OOM, "batch table allocation failed");
        }
        if (src && cudaMemcpy(*dst, src, bytes_, cudaMemcpyHostToDevice) != cudaSuccess)
            return fail(QD_ERR_CUDA, "batch table upload failed");
        return QD_OK;
    };
    if (int rc = up((void **)&b->dsegs, segs.data(), segs.size() * sizeof(BSeg))) return rc;
    if (int rc = up((void **)&b->dchunks, tb.chunks.data(), tb.chunks.size() * sizeof(BChunk))) return rc;
    if (int rc = up((void **)&b->dgates, gates.data(), gates.size() * sizeof(BGate))) return rc;
    if (int rc = up((void **)&b->dcoef, coef.data(), coef.size() * sizeof(float2))) return rc;
    if (int rc = up((void **)&b->dhoff, hoff.data(), hoff.size() * sizeof(uint32_t))) return rc;
    if (int rc = up((void **)&b->ditems, items.data(), items.size() * sizeof(BItem))) return rc;
    b->dirty = false;
    return QD_OK;
}

// Validate and keep circuit c's gates (host only).
int batch_store(qd_batch *b, int32_t c, const qd_gate *gates, int32_t ngates) {
    qd_reg r;
    if (int rc = host_register(b->dims[c].data(), (int32_t)b->dims[c].size(), QD_C64, r)) return rc;
    r.tile_stride = 0;
    std::vector<qd_batch::Stored> out;
    for (int i = 0; i < ngates; ++i) {
        qd_batch::Stored st;
        const qd_gate *gt = &gates[i];
        if (gt->kind == QD_GATE_MEASURE) break;  // gates after the measurement flag are ignored (Sec. 3.4)
        int rc = validate(&r, gt->targets, gt->k, gt->controls, gt->ctrl_levels, gt->nc, st.a);
        if (!rc) rc = gate_matrix(&r, gt, st.a, st.M, &st.diag);
        GatePlan g;
        bool noop = false;
        if (!rc) rc = plan_gate(&r, st.M.data(), st.a, st.diag, g, &noop);
        if (rc) {
            g_last_error = "circuit " + std::to_string(c) + " gate " + std::to_string(i) + ": " + g_last_error;
            return rc;
        }
        if (noop) continue;
        if (st.a.D > kBatchMaxD) return fail(QD_ERR_DIM, "batched gates need a target dimension <= 25");
        for (int m = 0; m < st.a.k; ++m) st.mask |= uint64_t(1) << st.a.t[m];
        for (int m = 0; m < st.a.nc; ++m) st.mask |= uint64_t(1) << st.a.c[m];
        if (mask_product(b->dims[c], st.mask) > kBatchMaxTile)
            return fail(QD_ERR_UNSUPPORTED, "a batched gate acts on more than 24576 amplitudes of its register");
        out.push_back(std::move(st));
    }
    b->circ[c].swap(out);
    b->dirty = true;
    return QD_OK;
}

// Registers of the batch: dims, sizes and arena offsets (host only).
int batch_shape(qd_batch *b, int32_t ncirc, const int32_t *nqudits, const int32_t *dims_concat) {
    b->ncirc = ncirc;
    int k = 0;
    for (int c = 0; c < ncirc; ++c) {
        if (nqudits[c] < 1 || nqudits[c] > QD_MAX_QUDITS) return fail(QD_ERR_ARG, "bad qudit count");
        std::vector<int32_t> d(dims_concat + k, dims_concat + k + nqudits[c]);
        k += nqudits[c];
        uint64_t N = 1;
        for (int32_t x : d) {
            if (x < 2 || x > 64) return fail(QD_ERR_DIM, "qudit dimension must be in [2, 64]");
            N *= (uint64_t)x;
            if (N >= (uint64_t(1) << 31))
                return fail(QD_ERR_DIM, "a batched register must hold fewer than 2^31 amplitudes");
        }
        b->dims.push_back(d);
        b->N.push_back(N);
        b->offs.push_back(b->arena_amps);
        b->basis.push_back(0);
        b->total += N;
        b->arena_amps += (N + 1) & ~uint64_t(1);
    }
    b->circ.assign(ncirc, {});
    return QD_OK;
}

BatchLaunch batch_desc(const qd_batch *b) {
    BatchLaunch L;
    L.arena = b->arena;
    L.total = b->arena_amps;
    L.offs = b->doffs;
    L.basis = b->dbasis;
    L.segs = b->dsegs;
    L.chunks = b->dchunks;
    L.gates = b->dgates;
    L.coef = b->dcoef;
    L.hoff = b->dhoff;
    L.items = b->ditems;
    L.nitems = b->nitems;
    L.ncirc = b->ncirc;
    L.counters = b->dcounters;
    L.err = b->derr;
    L.probs = b->probs;
    L.sm_count = b->sm_count;
    L.ctas_per_sm = b->ctas_per_sm;
    L.tile_cap = b->tile_cap;
    L.desc_bytes = b->desc_bytes;
    L.poll_limit = b->poll_limit;
    return L;
}

}  // namespace

extern "C" {

int qd_batch_create(int32_t ncirc, const int32_t *nqudits, const int32_t *dims_concat, void *stream, qd_batch **out) {
    if (!out) return fail(QD_ERR_ARG, "null output handle");
    *out = nullptr;
    if (ncirc < 1 || !nqudits || !dims_concat) return fail(QD_ERR_ARG, "bad batch description");
    qd_batch *b = new qd_batch();
    b->stream = static_cast<cudaStream_t>(stream);
    if (int rc = batch_shape(b, ncirc, nqudits, dims_concat)) {
        delete b;
        return rc;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
        delete b;
        return cuda_fail(e, "device query");
    }
    if (cudaMalloc(&b->arena, b->arena_amps * sizeof(float2)) != cudaSuccess ||
        cudaMalloc(&b->probs, b->arena_amps * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&b->doffs, ncirc * sizeof(uint64_t)) != cudaSuccess ||
        cudaMalloc(&b->dbasis, ncirc * sizeof(uint64_t)) != cudaSuccess ||
        cudaMalloc(&b->dcounters, (ncirc + 1) * sizeof(uint32_t)) != cudaSuccess ||
        cudaMalloc(&b->derr, sizeof(int32_t)) != cudaSuccess) {
        cudaGetLastError();
        delete b;
        return fail(QD_ERR_OOM, "batch allocation failed");
    }
    if (cudaMemcpy(b->doffs, b->offs.data(), ncirc * sizeof(uint64_t), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->dbasis, b->basis.data(), ncirc * sizeof(uint64_t), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(b->derr, 0, sizeof(int32_t)) != cudaSuccess) {
        delete b;
        return fail(QD_ERR_CUDA, "batch table upload failed");
    }
    *out = b;
    return QD_OK;
}

int qd_batch_set_circuit(qd_batch *b, int32_t c, const qd_gate *gates, int32_t ngates) {
    if (!b || c < 0 || c >= b->ncirc || ngates < 0 || (ngates > 0 && !gates)) return fail(QD_ERR_ARG, "bad arguments");
    return batch_store(b, c, gates, ngates);
}

int qd_batch_tune(qd_batch *b, int32_t key, int64_t value) {
    if (!b) return fail(QD_ERR_ARG, "null batch");
    switch (key) {
        case QD_BATCH_TILE_AMPS:
            if (value < 1 || value > (int64_t)kBatchMaxTile) return fail(QD_ERR_ARG, "tile size out of range");
            b->tile_amps = (uint32_t)value;
            break;
        case QD_BATCH_CTAS_PER_SM:
            if (value < 0 || value > 8) return fail(QD_ERR_ARG, "CTAs per SM out of range");
            b->ctas_per_sm = (int32_t)value;
            break;
        case QD_BATCH_SMALL_AMPS:
            if (value < 0 || value > (int64_t)kBatchMaxTile) return fail(QD_ERR_ARG, "shared-memory register size out of range");
            b->small_amps = (uint32_t)value;
            break;
        case QD_BATCH_GROUP_AMPS:
            if (value < 1) return fail(QD_ERR_ARG, "group size out of range");
            b->group_amps = (uint64_t)value;
            break;
        case QD_BATCH_TILES_PER_ITEM:
            if (value < 1 || value > 4096) return fail(QD_ERR_ARG, "tiles per item out of range");
            b->tiles_per_item = (uint32_t)value;
            break;
        case QD_BATCH_POLL_LIMIT:
            if (value < 0 || value > (int64_t(1) << 30)) return fail(QD_ERR_ARG, "poll limit out of range");
            b->poll_limit = (uint32_t)value;
            if (b->exec) {  // a new kernel argument: capture the graph again
                cudaGraphExecDestroy(b->exec);
                b->exec = nullptr;
            }
            return QD_OK;
        default:
            return fail(QD_ERR_ARG, "unknown batch tuning key");
    }
    b->dirty = true;
    return QD_OK;
}

int qd_batch_run(qd_batch *b) {
    if (!b) return fail(QD_ERR_ARG, "null batch");
    if (b->dirty) {
        if (b->stream) cudaStreamSynchronize(b->stream);
        if (int rc = batch_prepare(b)) return rc;
    }
    const BatchLaunch desc = batch_desc(b);
    if (b->profile) {
        if (!b->ev0) {
            QD_CUDA(cudaEventCreate(&b->ev0));
            QD_CUDA(cudaEventCreate(&b->ev1));
        }
        QD_CUDA(batch_launch(desc, b->stream, b->ev0, b->ev1));
        return QD_OK;
    }
    if (!b->stream) {
        QD_CUDA(batch_launch(desc, b->stream));
        return QD_OK;
    }
    if (!b->exec) {
        batch_occupancy(b->tile_cap, b->desc_bytes);  // sets the kernel's shared-memory attribute outside the capture
        QD_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = batch_launch(desc, b->stream);
        cudaGraph_t graph = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(b->stream, &graph);
        if (e != cudaSuccess || e2 != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            return cuda_fail(e != cudaSuccess ? e : e2, "batch capture");
        }
        e = cudaGraphInstantiate(&b->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            b->exec = nullptr;
            return cuda_fail(e, "batch graph instantiate");
        }
    }
    QD_CUDA(cudaGraphLaunch(b->exec, b->stream));
    return QD_OK;
}

int qd_batch_probabilities(qd_batch *b, int32_t c, double *out) {
    if (!b || !out || c < 0 || c >= b->ncirc) return fail(QD_ERR_ARG, "bad arguments");
    QD_CUDA(cudaMemcpyAsync(out, b->probs + b->offs[c], b->N[c] * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
    QD_CUDA(cudaStreamSynchronize(b->stream));
    return QD_OK;
}

int qd_batch_get_amplitudes(qd_batch *b, int32_t c, void *out) {
    if (!b || !out || c < 0 || c >= b->ncirc) return fail(QD_ERR_ARG, "bad arguments");
    QD_CUDA(cudaMemcpyAsync(out, b->arena + b->offs[c], b->N[c] * sizeof(float2), cudaMemcpyDeviceToHost, b->stream));
    QD_CUDA(cudaStreamSynchronize(b->stream));
    return QD_OK;
}

int qd_batch_info(qd_batch *b, int64_t *total, int32_t *items, int32_t *launches, int32_t *device_error) {
    if (!b) return fail(QD_ERR_ARG, "null batch");
    if (b->dirty) {
        if (b->stream) cudaStreamSynchronize(b->stream);
        if (int rc = batch_prepare(b)) return rc;
    }
    if (total) *total = (int64_t)b->total;
    if (items) *items = b->nitems;
    if (launches) *launches = b->nitems > 0 ? 4 : 3;  // zero fill, basis ones, persistent kernel, probabilities
    if (device_error) {
        int32_t e = 0;
        QD_CUDA(cudaMemcpyAsync(&e, b->derr, sizeof(int32_t), cudaMemcpyDeviceToHost, b->stream));
        QD_CUDA(cudaStreamSynchronize(b->stream));
        *device_error = e;
    }
    return QD_OK;
}

int qd_batch_sync(qd_batch *b, int32_t *device_error) {
    if (!b) return fail(QD_ERR_ARG, "null batch");
    int32_t e = 0;
    if (b->derr) {
        QD_CUDA(cudaMemcpyAsync(&e, b->derr, sizeof(int32_t), cudaMemcpyDeviceToHost, b->stream));
        QD_CUDA(cudaStreamSynchronize(b->stream));
    }
    if (device_error) *device_error = e;
    if (e == 2) return fail(QD_ERR_TIMEOUT, "a work item's bounded wait on its circuit counter expired");
    if (e) return fail(QD_ERR_DEVICE, "batch device error word set: " + std::to_string(e));
    return QD_OK;
}

int qd_batch_profile(qd_batch *b, int32_t enable) {
    if (!b) return fail(QD_ERR_ARG, "null batch");
    b->profile = enable != 0;
    return QD_OK;
}

int qd_batch_timings(qd_batch *b, float *kernel_ms, double *alg_bytes) {
    if (!b) return fail(QD_ERR_ARG, "null batch");
    if (alg_bytes) {
        if (b->dirty) {
            if (b->stream) cudaStreamSynchronize(b->stream);
            if (int rc = batch_prepare(b)) return rc;
        }
        *alg_bytes = b->alg_bytes;
    }
    if (kernel_ms) {
        if (!b->profile || !b->ev1) return fail(QD_ERR_ARG, "no profiled run");
        QD_CUDA(cudaEventSynchronize(b->ev1));
        QD_CUDA(cudaEventElapsedTime(kernel_ms, b->ev0, b->ev1));
    }
    return QD_OK;
}

int qd_batch_autotune(qd_batch *b, int32_t reps, int64_t *chosen, float *best_ms) {
    if (!b || reps < 1) return fail(QD_ERR_ARG, "bad arguments");
    struct Shape {
        uint32_t tile, small;
        int32_t ctas;
        uint32_t tpi;
    };
    const Shape cand[] = {{4096, 2048, 0, 1}, {2048, 2048, 0, 1}, {8192, 2048, 0, 1}, {4096, 1024, 0, 1},
                          {4096, 6144, 0, 1}, {4096, 2048, 4, 1}, {4096, 2048, 0, 2}, {6144, 2048, 0, 1}};
    const bool was_profile = b->profile;
    b->profile = true;
    float best = 0.f;
    int bi = -1;
    for (int i = 0; i < (int)(sizeof(cand) / sizeof(cand[0])); ++i) {
        b->tile_amps = cand[i].tile;
        b->small_amps = cand[i].small;
        b->ctas_per_sm = cand[i].ctas;
        b->tiles_per_item = cand[i].tpi;
        b->dirty = true;
        float t = 0.f;
        for (int k = 0; k <= reps; ++k) {  // the first run prepares and warms up
            if (int rc = qd_batch_run(b)) {
                b->profile = was_profile;
                return rc;
            }
            float ms = 0.f;
            if (int rc = qd_batch_timings(b, &ms, nullptr)) {
                b->profile = was_profile;
                return rc;
            }
            if (k > 0) t = (k == 1) ? ms : std::min(t, ms);
        }
        if (bi < 0 || t < best) {
            best = t;
            bi = i;
        }
    }
    b->profile = was_profile;
    b->tile_amps = cand[bi].tile;
    b->small_amps = cand[bi].small;
    b->ctas_per_sm = cand[bi].ctas;
    b->tiles_per_item = cand[bi].tpi;
    b->dirty = true;
    if (chosen) {
        chosen[0] = cand[bi].tile;
        chosen[1] = cand[bi].small;
        chosen[2] = cand[bi].ctas;
        chosen[3] = cand[bi].tpi;
    }
    if (best_ms) *best_ms = best;
    return QD_OK;
}

int qd_batch_destroy(qd_batch *b) {
    delete b;
    return QD_OK;
}

// Host replay of the batched kernel over the encoded tables (debug).
int qd_debug_batch_emulate(int32_t ncirc, const int32_t *nqudits, const int32_t *dims_concat, const qd_gate *gates,
                           const int32_t *ngates, const int64_t *tune, double *amps, int64_t *info) {
    if (ncirc < 1 || !nqudits || !dims_concat || !ngates || !amps || !info) return fail(QD_ERR_ARG, "bad arguments");
    qd_batch b;
    b.host_only = true;
    if (int rc = batch_shape(&b, ncirc, nqudits, dims_concat)) return rc;
    if (tune) {
        const int32_t keys[4] = {QD_BATCH_TILE_AMPS, QD_BATCH_SMALL_AMPS, QD_BATCH_GROUP_AMPS, QD_BATCH_TILES_PER_ITEM};
        for (int i = 0; i < 4; ++i)
            if (tune[i] >= 0)
                if (int rc = qd_batch_tune(&b, keys[i], tune[i])) return rc;
    }
    int g0 = 0;
    for (int c = 0; c < ncirc; ++c) {
        if (ngates[c] < 0) return fail(QD_ERR_ARG, "bad gate count");
        if (int rc = batch_store(&b, c, gates ? gates + g0 : nullptr, ngates[c])) return rc;
        g0 += ngates[c];
    }
    BatchTables tb;
    if (int rc = batch_tables(&b, tb)) return rc;
    std::vector<std::complex<double>> psi(b.arena_amps);
    for (int c = 0; c < ncirc; ++c) psi[b.offs[c] + b.basis[c]] = 1.0;
    std::vector<uint32_t> done(ncirc, 0);
    std::vector<int> cur_seg(ncirc, -1);
    std::vector<std::vector<uint32_t>> visits(ncirc);
    int64_t errors = 0;
    auto close_segment = [&](int c) {
        for (uint32_t v : visits[c])
            if (v != 1) errors |= 4;  // a segment's tiles must cover the register exactly once
        std::fill(visits[c].begin(), visits[c].end(), 0u);
    };
    std::vector<std::complex<double>> st, v;
    for (const BItem &it : tb.items) {
        const int c = it.circuit;
        const uint64_t N = b.N[c];
        if (done[c] < it.wait_target) errors |= 1;  // would wait on a later item
        if (visits[c].empty()) visits[c].assign(N, 0u);
        if (cur_seg[c] != it.seg) {
            if (cur_seg[c] >= 0) close_segment(c);
            cur_seg[c] = it.seg;
        }
        const BSeg &S = tb.segs[it.seg];
        st.assign(S.T, 0.0);
        for (uint32_t t = it.first; t < it.first + it.count; ++t) {
            if (t >= S.ntiles) {
                errors |= 2;
                continue;
            }
            const uint32_t base_t = expand(t, S.ex);
            std::vector<uint64_t> idx(S.T);
            for (uint32_t l = 0; l < S.T; ++l) {
                const uint32_t h = fdiv(l, S.divB);
                idx[l] = (uint64_t)base_t + (l - h * S.B) + tb.hoff[S.hoff + h];
                // paired segments: every even l starts a 16-byte aligned amplitude pair
                if (S.pair && (l % 2 == 0) && (((b.offs[c] + idx[l]) & 1u) || l + 1 >= S.T)) errors |= 32;
                if (idx[l] >= N) {
                    errors |= 2;
                    idx[l] = 0;
                }
                ++visits[c][idx[l]];
                st[l] = psi[b.offs[c] + idx[l]];
            }
            for (int g = -1, ci = S.chunk0, gi = 0; ci < S.chunk0 + S.nchunks;) {
                const BChunk &ch = tb.chunks[ci];
                if (gi >= ch.ngates) {
                    ++ci;
                    gi = 0;
                    continue;
                }
                if ((size_t)ch.ngates * sizeof(BGate) + (size_t)ch.ncoef * sizeof(float2) > tb.desc_bytes ||
                    (ch.coef0 & 1u) || (tb.desc_bytes & 15u))
                    errors |= 16;  // a chunk must fit its shared-memory area, 16-byte aligned
                g = ch.gate0 + gi++;
                const BGate &G = tb.gates[g];
                if (G.coef + 2 * G.ncoef > ch.ncoef || (G.coef & 1u)) errors |= 16;
                auto cf = [&](int k, int n) {
                    const float2 hi = tb.coef[ch.coef0 + G.coef + k], lo = tb.coef[ch.coef0 + G.coef + n + k];
                    return std::complex<double>((double)hi.x + (double)lo.x, (double)hi.y + (double)lo.y);
                };
                v.assign(G.D, 0.0);
                for (uint32_t r = 0; r < G.R; ++r) {
                    const uint32_t base = expand(r, G.ex) + G.base;
                    bool ok = true;
                    for (int j = 0; j < G.D; ++j)
                        if ((uint64_t)base + G.off[j] >= S.T) ok = false;
                    if (!ok) {
                        errors |= 8;
                        continue;
                    }
                    for (int j = 0; j < G.D; ++j) v[j] = st[base + G.off[j]];
                    for (int i = 0; i < G.D; ++i) {
                        if (G.kind == 0) {
                            std::complex<double> acc = 0.0;
                            for (int j = 0; j < G.D; ++j) acc += cf(i * G.D + j, G.D * G.D) * v[j];
                            st[base + G.off[i]] = acc;
                        } else if ((G.active >> i) & 1u) {
                            const std::complex<double> in = v[G.src[i]];
                            st[base + G.off[i]] = ((G.unit >> i) & 1u) ? in : cf(i, G.D) * in;
                        }
                    }
                }
            }
            for (uint32_t l = 0; l < S.T; ++l) psi[b.offs[c] + idx[l]] = st[l];
        }
        done[c] += it.count;
    }
    for (int c = 0; c < ncirc; ++c)
        if (cur_seg[c] >= 0) close_segment(c);
    uint64_t o = 0;
    for (int c = 0; c < ncirc; ++c)
        for (uint64_t i = 0; i < b.N[c]; ++i, ++o) {
            amps[2 * o] = psi[b.offs[c] + i].real();
            amps[2 * o + 1] = psi[b.offs[c] + i].imag();
        }
    info[0] = (int64_t)tb.segs.size();
    info[1] = (int64_t)tb.items.size();
    info[2] = (int64_t)tb.cap;
    info[3] = (int64_t)tb.bytes;
    info[4] = errors;
    return QD_OK;
}

}  // extern "C"
