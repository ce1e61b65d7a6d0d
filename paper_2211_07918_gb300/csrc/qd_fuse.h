// Gate-fusion planner (host): groups runs of consecutive gates into blocks
// whose product matrix is applied in one pass over the state.
//
// A segmentation splits the gate list into contiguous segments; a segment of
// one gate runs that gate's own kernel, a longer segment runs one dense
// kernel with the product of its gates embedded in the union of their acting
// qudits (controls included, expanded to dense).  The greedy planner extends
// the current segment while the cost model says the merged block is cheaper
// than closing it; the exhaustive planner is an exact dynamic program over
// all contiguous segmentations (the reference the other two are measured against).
#pragma once
#include <cstdint>
#include <functional>
#include <vector>

namespace qd {

// One validated gate: its matrix over the acting qudits (controls first,
// then targets; first listed = most significant), with controls expanded.
struct FuseGate {
    std::vector<int> acting;
    std::vector<double> M;  // Dact x Dact, interleaved complex, row-major
    int Dact = 1;
    bool mono = false;      // the original gate is a permutation with phases
    bool diag = false;      // ... and its permutation is the identity (a diagonal gate)
    int nc = 0;             // number of controls in `acting`
};

struct FuseBlock {
    std::vector<int> qudits;  // descending qudit index: first = most significant local digit
    int D = 1;
    std::vector<double> M;    // D x D product, interleaved complex
    int first = 0, last = 0;  // gate range [first, last]
};

// Features of one candidate launch for the cost models.
constexpr int kFeatures = 12;
struct LaunchFeatures {
    float f[kFeatures];
};

struct RegisterShape {
    int n;
    const int32_t *dims;
    const int64_t *strides;
    int64_t N;
    int precision;  // 1 = complex64, 2 = complex128
    int tc_min_d;   // complex64 fused blocks with D >= tc_min_d (or D > 32) run on the tensor cores;
                    // 0: the cost model chooses per block between the CUDA cores and the tensor cores
    int fuse_dmax;  // largest dimension of a fused block
};

// Kernel kind of a launch (feature 10).
constexpr int kKernelMono = 0;   // per-gate permutation with phases
constexpr int kKernelDense = 1;  // per-gate dense (CUDA cores)
constexpr int kKernelBlock = 2;    // fused block on the CUDA-core dense kernels (D <= 32)
constexpr int kKernelBlockTc = 3;  // fused block on the tensor cores (complex64)
constexpr int kKernelDiagTable = 4;  // run of diagonal gates applied through one table (any qudit count)
constexpr int kKernelDenseTable = 5; // dense gate or block followed by a diagonal run, one launch
constexpr int kDenseTableMaxD = 16;  // largest dense part of such a launch
constexpr uint64_t kDiagRunMaxTable = uint64_t(1) << 24;  // entries of a diagonal run's table
constexpr int kMonoBlockMaxD = 32;  // a fused block of permutations with phases up to this D runs as mono
constexpr int kDenseBlockMaxD = 32;  // largest fused block the CUDA-core dense kernels take

// Candidate kernels of a fused (multi-gate) segment over nq qudits of
// dimension D (written to kinds[], count returned): a diagonal table when
// every gate is diagonal and the segment is beyond the block limits (more
// than kmax qudits or D > kMonoBlockMaxD); mono when every gate is a
// permutation with phases and D <= kMonoBlockMaxD; else dense on the CUDA
// cores, or on the tensor cores for complex64 when D >= tc_min_d or D > 32.
// With tc_min_d = 0 a complex64 dense block of kTcMinBlockD <= D <= 32 has
// both dense kernels as candidates and the cost model picks the cheaper.
constexpr int kTcMinBlockD = 9;
int block_kernels(const RegisterShape &reg, int64_t D, int nq, int kmax, bool all_mono, bool all_diag, int *kinds);

// Entries of the table of a diagonal run over `qudits`: the product of the
// dimensions of the contiguous range [min, max] of those qudits.
uint64_t diag_table_size(const RegisterShape &reg, const std::vector<int> &qudits);

// A multi-gate segment as a dense part followed by a diagonal run: split is
// the last gate of the dense part (the segment's maximal all-diagonal suffix
// starts after it; -1 when the whole segment is diagonal); ok when the dense
// part spans at most kmax qudits and kDenseTableMaxD states and the run's
// table fits kDiagRunMaxTable.  dense_q: the dense part's qudits; run_q: the
// run's; table: the run's table entries.
struct DenseTableSplit {
    bool ok = false;
    int split = -1;
    std::vector<int> dense_q, run_q;
    int64_t dense_D = 1;
    uint64_t table = 0;
};
DenseTableSplit dense_table_split(const std::vector<FuseGate> &gates, int first, int last, const RegisterShape &reg,
                                  int kmax);

// Feature vector of a launch acting on `qudits` with target dimension D:
// log2 D, qudit count, log2 of the (up to three) smallest strides, relative
// positions, log2 N, precision, kernel kind, log2 of the control-slice
// fraction.
LaunchFeatures launch_features(const RegisterShape &reg, const std::vector<int> &qudits, int D, int kernel,
                               double slice_fraction);

// Analytic cost (seconds): max(HBM time, arithmetic time) + launch overhead,
// with GB300 rates measured for the per-gate kernels.
double analytic_cost(const RegisterShape &reg, const LaunchFeatures &f);

using CostFn = std::function<double(const LaunchFeatures &)>;

// Expand a gate over (controls, targets) into its full matrix over `acting`.
FuseGate make_fuse_gate(const std::vector<int> &controls, const std::vector<int> &levels,
                        const std::vector<int> &targets, const std::vector<double> &Mt, const int32_t *dims, bool mono);

// Product of gates[first..last] embedded in the union of their qudits.
FuseBlock build_block(const std::vector<FuseGate> &gates, int first, int last, const int32_t *dims);

// Segmentations: list of [first, last] gate ranges covering the gate list.
std::vector<std::pair<int, int>> segment_greedy(const std::vector<FuseGate> &gates, const RegisterShape &reg,
                                                const CostFn &cost, int kmax, int Dmax);
std::vector<std::pair<int, int>> segment_exhaustive(const std::vector<FuseGate> &gates, const RegisterShape &reg,
                                                    const CostFn &cost, int kmax, int Dmax, double *best_cost);

// Cost the model assigns to one segment (single gate: its own kernel; a
// block: its cheapest candidate kernel, returned in *kind if not NULL); kmax
// is the block limit that decides between a mono block and a diagonal table.
double segment_cost(const std::vector<FuseGate> &gates, int first, int last, const RegisterShape &reg,
                    const CostFn &cost, int kmax, int *kind = nullptr);

// Launch features of every feasible form of one segment (the candidates
// segment_cost weighs; the kernel class is feature 10).
std::vector<LaunchFeatures> segment_forms(const std::vector<FuseGate> &gates, int first, int last,
                                          const RegisterShape &reg, int kmax);

}  // namespace qd
