// Gate-fusion planner (host code): block construction, cost models,
// greedy and exhaustive segmentations.  See qd_fuse.h.
#include <algorithm>
#include <cmath>
#include <limits>
#include <map>

#include "qd_fuse.h"

namespace qd {

namespace {

// digits of local index j over the listed qudits (first most significant)
void local_digits(int j, const std::vector<int> &qs, const int32_t *dims, int *out) {
    for (int m = (int)qs.size() - 1; m >= 0; --m) {
        out[m] = j % dims[qs[m]];
        j /= dims[qs[m]];
    }
}

int local_index(const int *digs, const std::vector<int> &qs, const int32_t *dims) {
    int j = 0;
    for (size_t m = 0; m < qs.size(); ++m) j = j * dims[qs[m]] + digs[m];
    return j;
}

// C = A * B for D x D interleaved complex matrices
void cmatmul(const std::vector<double> &A, const std::vector<double> &B, std::vector<double> &C, int D) {
    C.assign((size_t)2 * D * D, 0.0);
    for (int i = 0; i < D; ++i)
        for (int k = 0; k < D; ++k) {
            const double ar = A[2 * (i * D + k)], ai = A[2 * (i * D + k) + 1];
            if (ar == 0.0 && ai == 0.0) continue;
            for (int j = 0; j < D; ++j) {
                const double br = B[2 * (k * D + j)], bi = B[2 * (k * D + j) + 1];
                C[2 * (i * D + j)] += ar * br - ai * bi;
                C[2 * (i * D + j) + 1] += ar * bi + ai * br;
            }
        }
}

std::vector<int> union_qudits(const std::vector<FuseGate> &gates, int first, int last) {
    std::vector<int> s;
    for (int g = first; g <= last; ++g)
        for (int q : gates[g].acting)
            if (std::find(s.begin(), s.end(), q) == s.end()) s.push_back(q);
    std::sort(s.begin(), s.end(), std::greater<int>());
    return s;
}

int64_t dim_of(const std::vector<int> &qs, const int32_t *dims) {
    int64_t D = 1;
    for (int q : qs) D *= dims[q];
    return D;
}

}  // namespace

FuseGate make_fuse_gate(const std::vector<int> &controls, const std::vector<int> &levels,
                        const std::vector<int> &targets, const std::vector<double> &Mt, const int32_t *dims,
                        bool mono) {
    FuseGate g;
    g.acting = controls;
    g.acting.insert(g.acting.end(), targets.begin(), targets.end());
    g.nc = (int)controls.size();
    g.mono = mono;
    const int Dt = (int)dim_of(targets, dims);
    const int C = (int)dim_of(controls, dims);
    g.Dact = C * Dt;
    g.M.assign((size_t)2 * g.Dact * g.Dact, 0.0);
    // identity everywhere except the block at the control combination `levels`
    int csel = 0;
    for (size_t m = 0; m < controls.size(); ++m) csel = csel * dims[controls[m]] + levels[m];
    for (int c = 0; c < C; ++c)
        for (int i = 0; i < Dt; ++i) {
            if (c != csel) {
                g.M[2 * ((c * Dt + i) * g.Dact + c * Dt + i)] = 1.0;
                continue;
            }
            for (int j = 0; j < Dt; ++j) {
                g.M[2 * ((c * Dt + i) * g.Dact + c * Dt + j)] = Mt[2 * (i * Dt + j)];
                g.M[2 * ((c * Dt + i) * g.Dact + c * Dt + j) + 1] = Mt[2 * (i * Dt + j) + 1];
            }
        }
    return g;
}

FuseBlock build_block(const std::vector<FuseGate> &gates, int first, int last, const int32_t *dims) {
    FuseBlock b;
    b.first = first;
    b.last = last;
    b.qudits = union_qudits(gates, first, last);
    const int D = (int)dim_of(b.qudits, dims);
    b.D = D;
    b.M.assign((size_t)2 * D * D, 0.0);
    for (int i = 0; i < D; ++i) b.M[2 * (i * D + i)] = 1.0;
    std::vector<double> E, T;
    int xs[16], ys[16], ga[16];
    for (int gi = first; gi <= last; ++gi) {
        const FuseGate &g = gates[gi];
        // position of each acting qudit in the block list
        int pos[16];
        for (size_t a = 0; a < g.acting.size(); ++a)
            pos[a] = (int)(std::find(b.qudits.begin(), b.qudits.end(), g.acting[a]) - b.qudits.begin());
        E.assign((size_t)2 * D * D, 0.0);
        for (int x = 0; x < D; ++x) {
            local_digits(x, b.qudits, dims, xs);
            for (size_t a = 0; a < g.acting.size(); ++a) ga[a] = xs[pos[a]];
            const int col = local_index(ga, g.acting, dims);
            for (int row = 0; row < g.Dact; ++row) {
                const double re = g.M[2 * (row * g.Dact + col)], im = g.M[2 * (row * g.Dact + col) + 1];
                if (re == 0.0 && im == 0.0) continue;
                local_digits(row, g.acting, dims, ga);
                std::copy(xs, xs + b.qudits.size(), ys);
                for (size_t a = 0; a < g.acting.size(); ++a) ys[pos[a]] = ga[a];
                const int y = local_index(ys, b.qudits, dims);
                E[2 * (y * D + x)] = re;
                E[2 * (y * D + x) + 1] = im;
            }
        }
        cmatmul(E, b.M, T, D);
        b.M.swap(T);
    }
    return b;
}

LaunchFeatures launch_features(const RegisterShape &reg, const std::vector<int> &qudits, int D, int kernel,
                               double slice_fraction) {
    LaunchFeatures lf;
    for (float &v : lf.f) v = 0.f;
    std::vector<int> qs = qudits;
    std::sort(qs.begin(), qs.end());  // ascending stride
    lf.f[0] = (float)std::log2((double)D);
    lf.f[1] = (float)qs.size();
    for (int i = 0; i < 3; ++i) {
        if (i < (int)qs.size()) {
            lf.f[2 + i] = (float)std::log2((double)reg.strides[qs[i]]);
            lf.f[5 + i] = (float)((qs[i] + 0.5) / reg.n);
        } else {
            lf.f[2 + i] = -1.f;
            lf.f[5 + i] = -1.f;
        }
    }
    lf.f[8] = (float)std::log2((double)reg.N);
    lf.f[9] = reg.precision == 2 ? 1.f : 0.f;
    lf.f[10] = (float)kernel;
    lf.f[11] = (float)std::log2(slice_fraction);
    return lf;
}

int block_kernels(const RegisterShape &reg, int64_t D, int nq, int kmax, bool all_mono, bool all_diag, int *kinds) {
    if (all_diag && (nq > kmax || D > kMonoBlockMaxD)) {
        kinds[0] = kKernelDiagTable;
        return 1;
    }
    if (all_mono && D <= kMonoBlockMaxD) {
        kinds[0] = kKernelMono;
        return 1;
    }
    if (reg.precision != 1) {
        kinds[0] = kKernelBlock;
        return 1;
    }
    if (D > kDenseBlockMaxD) {
        kinds[0] = kKernelBlockTc;
        return 1;
    }
    if (reg.tc_min_d == 0 && D >= kTcMinBlockD) {
        kinds[0] = kKernelBlock;
        kinds[1] = kKernelBlockTc;
        return 2;
    }
    kinds[0] = (reg.tc_min_d > 0 && D >= reg.tc_min_d) ? kKernelBlockTc : kKernelBlock;
    return 1;
}

uint64_t diag_table_size(const RegisterShape &reg, const std::vector<int> &qudits) {
    int lo = reg.n, hi = -1;
    for (int q : qudits) {
        lo = std::min(lo, q);
        hi = std::max(hi, q);
    }
    uint64_t T = 1;
    for (int q = lo; q <= hi; ++q) {
        T *= (uint64_t)reg.dims[q];
        if (T > kDiagRunMaxTable) return kDiagRunMaxTable + 1;
    }
    return T;
}

DenseTableSplit dense_table_split(const std::vector<FuseGate> &gates, int first, int last, const RegisterShape &reg,
                                  int kmax) {
    DenseTableSplit d;
    int k = last;
    while (k >= first && gates[k].diag) --k;
    d.split = k;
    if (k < first || k == last) return d;  // all diagonal, or no diagonal suffix
    d.dense_q = union_qudits(gates, first, k);
    d.run_q = union_qudits(gates, k + 1, last);
    d.dense_D = dim_of(d.dense_q, reg.dims);
    d.table = diag_table_size(reg, d.run_q);
    d.ok = (int)d.dense_q.size() <= kmax && d.dense_D <= kDenseTableMaxD && d.table <= kDiagRunMaxTable;
    return d;
}

double analytic_cost(const RegisterShape &reg, const LaunchFeatures &lf) {
    const double D = std::exp2((double)lf.f[0]);
    const bool c128 = lf.f[9] > 0.5f;
    const bool dense = lf.f[10] > 0.5f;
    const bool block = lf.f[10] > 2.5f && lf.f[10] < 3.5f;  // fused block on the tensor cores
    const bool table = lf.f[10] > 3.5f && lf.f[10] < 4.5f; // diagonal run through a table
    const bool dense_table = lf.f[10] > 4.5f;              // dense part + diagonal table
    // feature 11: log2 of the control-slice fraction, or (dense + table) of the table entries
    const double touched = dense_table ? (double)reg.N : (double)reg.N * std::exp2((double)lf.f[11]);
    const double b = c128 ? 16.0 : 8.0;
    double t_mem = 2.0 * touched * b / 5.0e12;
    if (table) t_mem += std::exp2((double)lf.f[0]) * 16.0 / 5.0e12;
    if (dense_table) t_mem += std::exp2((double)lf.f[11]) * 16.0 / 5.0e12;
    double t_cmp = table ? touched * 40.0 / 2.0e13 : 0.0;  // index arithmetic per amplitude
    if (dense_table) t_cmp = c128 ? touched * 4.0 * D / 0.5e12 : touched * (8.0 * D + 64.0) / 2.0e13;
    if (dense && !table && !dense_table) {
        if (!c128 && block) {
            // fused block on the tensor cores: 6 exact BF16 slice products of
            // (2 Dp) x (2 Dp) per group; measured on GB300 the kernel moves
            // about 3.5 TB/s at D = Dp, less in proportion to the padding
            const double Dp = D <= 32 ? std::ceil(D / 8.0) * 8.0 : std::ceil(D / 16.0) * 16.0;
            t_cmp = 2.0 * touched * b / (3.5e12 * D / Dp);
        } else {
            // complex64 with hi+lo coefficients: 8 D FFMA per amplitude plus
            // index work; complex128: 4 D DFMA per amplitude
            t_cmp = c128 ? touched * 4.0 * D / 0.5e12 : touched * (8.0 * D + 24.0) / 2.0e13;
        }
    }
    return std::max(t_mem, t_cmp) + 4.0e-6;
}

double segment_cost(const std::vector<FuseGate> &gates, int first, int last, const RegisterShape &reg,
                    const CostFn &cost, int kmax, int *kind_out) {
    if (first == last) {
        const FuseGate &g = gates[first];
        double frac = 1.0;
        int Dt = g.Dact;
        for (int m = 0; m < g.nc; ++m) {
            frac /= reg.dims[g.acting[m]];
            Dt /= reg.dims[g.acting[m]];
        }
        if (kind_out) *kind_out = g.mono ? kKernelMono : kKernelDense;
        return cost(launch_features(reg, g.acting, Dt, g.mono ? kKernelMono : kKernelDense, frac));
    }
    const std::vector<int> s = union_qudits(gates, first, last);
    const int64_t D = dim_of(s, reg.dims);
    // a product of permutations with phases is one: it runs on the mono
    // kernel (up to its 32 local states), not as a dense block
    bool all_mono = true, all_diag = true;
    for (int i = first; i <= last; ++i) {
        all_mono = all_mono && gates[i].mono;
        all_diag = all_diag && gates[i].diag;
    }
    // the segment's feasible forms: a block (or a diagonal run), and a dense
    // part followed by a diagonal run
    int kinds[2];
    int nk = 0;
    if (((int)s.size() <= kmax && D <= reg.fuse_dmax) ||
        (all_diag && diag_table_size(reg, s) <= kDiagRunMaxTable))
        nk = block_kernels(reg, D, (int)s.size(), kmax, all_mono, all_diag, kinds);
    double best = std::numeric_limits<double>::infinity();
    for (int k = 0; k < nk; ++k) {
        const int kind = kinds[k];
        const double c = kind == kKernelDiagTable
                             ? cost(launch_features(reg, s, (int)diag_table_size(reg, s), kind, 1.0))
                             : cost(launch_features(reg, s, (int)D, kind, 1.0));
        if (c < best) {
            best = c;
            if (kind_out) *kind_out = kind;
        }
    }
    const DenseTableSplit dt = dense_table_split(gates, first, last, reg, kmax);
    if (dt.ok) {
        const double c =
            cost(launch_features(reg, dt.dense_q, (int)dt.dense_D, kKernelDenseTable, (double)dt.table));
        if (c < best) {
            best = c;
            if (kind_out) *kind_out = kKernelDenseTable;
        }
    }
    return best;
}

std::vector<LaunchFeatures> segment_forms(const std::vector<FuseGate> &gates, int first, int last,
                                          const RegisterShape &reg, int kmax) {
    std::vector<LaunchFeatures> out;
    const CostFn grab = [&out](const LaunchFeatures &f) {
        out.push_back(f);
        return 0.0;
    };
    segment_cost(gates, first, last, reg, grab, kmax);
    return out;
}

namespace {
// A multi-gate segment is feasible as a block within the qudit and dimension
// limits, and as a diagonal run (every gate diagonal) on any number of qudits
// whose covering range gives a table of at most kDiagRunMaxTable entries.
bool feasible(const std::vector<FuseGate> &gates, int first, int last, const RegisterShape &reg, int kmax,
              int Dmax) {
    if (first == last) return true;
    const std::vector<int> s = union_qudits(gates, first, last);
    bool all_diag = true;
    for (int i = first; i <= last && all_diag; ++i) all_diag = gates[i].diag;
    if (all_diag && diag_table_size(reg, s) <= kDiagRunMaxTable) return true;
    if ((int)s.size() <= kmax && dim_of(s, reg.dims) <= Dmax) return true;
    return dense_table_split(gates, first, last, reg, kmax).ok;
}
}  // namespace

std::vector<std::pair<int, int>> segment_greedy(const std::vector<FuseGate> &gates, const RegisterShape &reg,
                                                const CostFn &cost, int kmax, int Dmax) {
    std::vector<std::pair<int, int>> segs;
    const int n = (int)gates.size();
    int start = 0;
    for (int i = 1; i <= n; ++i) {
        if (i < n && feasible(gates, start, i, reg, kmax, Dmax)) {
            const double merged = segment_cost(gates, start, i, reg, cost, kmax);
            const double split =
                segment_cost(gates, start, i - 1, reg, cost, kmax) + segment_cost(gates, i, i, reg, cost, kmax);
            if (merged <= split) continue;
        }
        segs.push_back({start, i - 1});
        start = i;
    }
    return segs;
}

std::vector<std::pair<int, int>> segment_exhaustive(const std::vector<FuseGate> &gates, const RegisterShape &reg,
                                                    const CostFn &cost, int kmax, int Dmax, double *best_cost) {
    const int n = (int)gates.size();
    std::vector<double> best(n + 1, std::numeric_limits<double>::infinity());
    std::vector<int> from(n + 1, -1);
    best[0] = 0.0;
    for (int i = 1; i <= n; ++i) {
        for (int j = i - 1; j >= 0; --j) {
            if (!feasible(gates, j, i - 1, reg, kmax, Dmax)) break;  // unions only grow as j decreases
            const double c = best[j] + segment_cost(gates, j, i - 1, reg, cost, kmax);
            if (c < best[i]) {
                best[i] = c;
                from[i] = j;
            }
        }
    }
    std::vector<std::pair<int, int>> segs;
    for (int i = n; i > 0; i = from[i]) segs.push_back({from[i], i - 1});
    std::reverse(segs.begin(), segs.end());
    if (best_cost) *best_cost = best[n];
    return segs;
}

}  // namespace qd
