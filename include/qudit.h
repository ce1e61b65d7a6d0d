/*
 * qudit.h - C ABI of libqudit, a GB300 (sm_103a) engine that applies
 * generalized qudit gates in place to a mixed-radix state vector.
 *
 * The calls follow the problem statement of QuDiet (arXiv 2211.07918):
 *   - a register is a heterogeneous list of qudit dimensions whose state has
 *     N = prod d_q entries (Sec. 2.2); the first qudit is the least
 *     significant digit (Sec. 3.2, qregs), so amplitude i is the basis state
 *     with digits x_q = (i / s_q) mod d_q, s_q = prod_{p<q} d_p;
 *   - each qudit starts in a chosen computational basis level, |0> by default
 *     (Sec. 3.2, init_states);
 *   - gates (Sec. 2.1.2 and Sec. 3.4): generalized NOT X^d_{+a}, phase shift
 *     Z_d, generalized Hadamard F_d, generalized CNOT / multi-controlled
 *     Toffoli that fire on a control level (d_c - 1 in the paper; any chosen
 *     level here, after Fig. 1), and user-defined k-qudit matrices;
 *   - the result is read as amplitudes or probabilities of the basis states
 *     (Sec. 3.8, OutputMethod).
 *
 * Conventions for every call
 *   - Return value: QD_OK (0) or a negative QD_ERR_* code.  No call aborts the
 *     process or traps the GPU.  qd_last_error() gives a message for the
 *     calling thread's most recent failure.
 *   - Ownership: the caller owns every pointer it passes (dims, matrices,
 *     target lists, output buffers); the library copies what it keeps.  A
 *     device buffer given to qd_create stays owned by the caller (for example
 *     torch storage) and must outlive the register.
 *   - Streams: a stream argument is a cudaStream_t passed as void* (NULL is
 *     the legacy default stream).  All device work of a register is ordered
 *     on its stream; calls that return host values synchronise that stream.
 *   - Gate matrices are host arrays of complex128 values stored as
 *     interleaved (re, im) doubles, row-major D x D, D = prod of the target
 *     dimensions.  The local index of a multi-qudit gate takes the
 *     first-listed target as its most significant digit.  Matrices are
 *     rounded to the register precision on the host.
 *   - Amplitude buffers are complex64 (interleaved float) or complex128
 *     (interleaved double) in the flat index order above.
 */
#ifndef QUDIT_H
#define QUDIT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ------------------------------------------------------ */
#define QD_OK 0
#define QD_ERR_ARG (-1)         /* null pointer, bad count, bad enum, bad shift or level */
#define QD_ERR_DIM (-2)         /* dimension outside [2, 64], N above the limit, D too large */
#define QD_ERR_OVERLAP (-3)     /* repeated target, or a control that is also a target */
#define QD_ERR_OOM (-4)         /* device allocation failed or caller buffer too small */
#define QD_ERR_CUDA (-5)        /* a CUDA runtime call failed */
#define QD_ERR_TIMEOUT (-6)     /* a bounded device wait expired */
#define QD_ERR_DEVICE (-7)      /* a kernel reported an error through the device error word */
#define QD_ERR_UNSUPPORTED (-8) /* valid request this build does not implement */

/* ---- enums ------------------------------------------------------------ */
#define QD_C64 1  /* complex64 state: FP32 arithmetic */
#define QD_C128 2 /* complex128 state: FP64 arithmetic */

#define QD_HOST 0   /* output/input pointer is host memory */
#define QD_DEVICE 1 /* output/input pointer is device memory */

#define QD_GATE_X 1    /* X^d_{+a}: |x> -> |(x+a) mod d>, a = param in [1, d-1] (Sec. 2.1.2) */
#define QD_GATE_Z 2    /* Z_d^p = diag(w^{p j}), w = exp(2 pi i/d), p = param (Sec. 2.1.2) */
#define QD_GATE_H 3    /* F_d[j][k] = w^{jk}/sqrt(d) (Sec. 2.1.2) */
#define QD_GATE_U 4    /* dense user matrix, D x D (Sec. 3.4 User Defined Gate) */
#define QD_GATE_DIAG 5 /* diagonal user matrix, D entries */
#define QD_GATE_MEASURE 6 /* measurement flag on all qudits (Sec. 3.4 Measurement Gate, Sec. 3.6 measure_all):
                             no unitary; every gate after it is ignored.  targets, controls, param ignored */

#define QD_PLAN_NONE 0       /* one kernel per gate, no fusion */
#define QD_PLAN_GREEDY 1     /* greedy gate fusion into blocks */
#define QD_PLAN_LEARNED 2    /* exact segmentation under the learned cost model (qd_set_cost_model) */
#define QD_PLAN_EXHAUSTIVE 3 /* exact optimum over contiguous segmentations (small circuits) */

#define QD_MAX_QUDITS 48
#define QD_MAX_TARGETS 6
#define QD_MAX_CONTROLS 8
#define QD_MAX_D 32          /* largest target-space dimension of one per-gate kernel */
#define QD_MAX_AMPLITUDES (((int64_t)1) << 40)

/* One gate of a circuit.  Controls fire when every control qudit holds its
 * level; a level of -1 means d_c - 1 (the paper's C_{X,d} and C^n_{X,d}). */
typedef struct qd_gate {
    int32_t kind;                          /* QD_GATE_* */
    int32_t k;                             /* number of targets, 1..QD_MAX_TARGETS */
    int32_t targets[QD_MAX_TARGETS];       /* first listed = most significant local digit */
    int32_t nc;                            /* number of controls, 0..QD_MAX_CONTROLS */
    int32_t controls[QD_MAX_CONTROLS];
    int32_t ctrl_levels[QD_MAX_CONTROLS];  /* level in [0, d_c) or -1 */
    int32_t param;                         /* X: shift a; Z: power p; otherwise ignored */
    int32_t reserved;
    const double *matrix;                  /* U: 2*D*D doubles; DIAG: 2*D doubles; else NULL */
} qd_gate;

typedef struct qd_reg qd_reg;   /* opaque register handle */
typedef struct qd_plan qd_plan; /* opaque prepared circuit */

/* ---- register (Sec. 2.2, Sec. 3.2, Sec. 3.3) --------------------------- */

/* Create a register of n qudits with dims[q] in [2, 64] and
 * N = prod dims[q] <= QD_MAX_AMPLITUDES, initialised to the basis state
 * |init_levels[0] ... init_levels[n-1]> (NULL: all 0).
 * precision: QD_C64 or QD_C128.  dev_buf: NULL to let the library allocate
 * the N amplitudes, or a caller-owned device buffer of dev_buf_bytes >= N *
 * element size, aligned to 16 bytes.  stream: cudaStream_t as void*.
 * Errors: QD_ERR_ARG, QD_ERR_DIM, QD_ERR_OOM, QD_ERR_CUDA. */
int qd_create(const int32_t *dims, int32_t n, const int32_t *init_levels, int32_t precision,
              void *dev_buf, size_t dev_buf_bytes, void *stream, qd_reg **out);

/* Release the register and everything the library allocated for it. */
int qd_destroy(qd_reg *reg);

/* Re-initialise to a basis state (NULL: all 0): one memset-class pass. */
int qd_reset(qd_reg *reg, const int32_t *init_levels);

/* Register facts: amplitude count, qudit count, device pointer of the state,
 * precision.  Any output pointer may be NULL. */
int qd_info(const qd_reg *reg, int64_t *num_amplitudes, int32_t *n, void **state, int32_t *precision);

/* Move subsequent work of the register to another stream. */
int qd_set_stream(qd_reg *reg, void *stream);

/* Launch-shape tuning of later gate plans on this register.
 * QD_TUNE_TILE_STRIDE: gates whose lowest target or control stride (in
 * amplitudes) is below value are staged through shared memory ("tile"
 * kernels); 0 never tiles.  Default: environment QD_TILE_STRIDE, else 0.
 * Errors: QD_ERR_ARG for an unknown key or a negative value. */
#define QD_TUNE_TILE_STRIDE 1
/* QD_TUNE_FUSE_KMAX: most qudits a fused block may span (1..6, default 3).
 * QD_TUNE_FUSE_DMAX: largest dimension of a fused block: complex64 2..64
 * (default 64), complex128 2..QD_MAX_D (default 32).
 * QD_TUNE_TC_MIN_D: which kernel runs a complex64 fused dense block of
 * dimension D <= 32: 0 (default) lets the plan's cost model (analytic, or the
 * learned model for QD_PLAN_LEARNED) price both and take the cheaper, for D
 * >= 9; a value in 9..65 sends blocks of D >= value to the tensor cores
 * (exact BF16 slice products with FP32 accumulation) and smaller ones to the
 * CUDA-core dense kernels.  Blocks above 32 always run on the tensor cores. */
#define QD_TUNE_FUSE_KMAX 2
#define QD_TUNE_FUSE_DMAX 3
#define QD_TUNE_TC_MIN_D 4
/* QD_TUNE_INDEX64: 1 runs the 64-bit index kernels on this register
 * whatever its size (by default they run on registers of 2^31 amplitudes
 * or more, except registers of up to 2^32 whose dimensions are all powers
 * of two, which keep 32-bit indices), for plans created afterwards and for
 * one-shot gate calls; 0 (default) lets the size decide. */
#define QD_TUNE_INDEX64 5
int qd_set_tuning(qd_reg *reg, int32_t key, int64_t value);

/* ---- gate application, in place (Sec. 2.1.2, Sec. 3.4) ---------------- */

/* Apply a dense D x D matrix to targets[0..k) under controls[0..nc) at
 * ctrl_levels (NULL or -1 entries: d_c - 1).  The matrix is classified on
 * the host: a diagonal or a permutation-with-phases matrix runs the
 * data-movement kernels, anything else the dense kernels.  No check of
 * unitarity.  Errors: QD_ERR_ARG, QD_ERR_DIM (D > QD_MAX_D), QD_ERR_OVERLAP. */
int qd_apply(qd_reg *reg, const double *matrix, const int32_t *targets, int32_t k,
             const int32_t *controls, const int32_t *ctrl_levels, int32_t nc);

/* Apply a diagonal matrix given by its D complex entries. */
int qd_apply_diag(qd_reg *reg, const double *diag, const int32_t *targets, int32_t k,
                  const int32_t *controls, const int32_t *ctrl_levels, int32_t nc);

/* X^d_{+shift} on t, shift in [1, d_t - 1] (Sec. 2.1.2 generalized NOT). */
int qd_apply_x(qd_reg *reg, int32_t t, int32_t shift);
/* Z_d^power on t (Sec. 2.1.2 phase shift; power is reduced mod d). */
int qd_apply_z(qd_reg *reg, int32_t t, int32_t power);
/* F_d on t (Sec. 2.1.2 generalized Hadamard). */
int qd_apply_h(qd_reg *reg, int32_t t);
/* C_{X,d}: X^{d_t}_{+shift} on t when control c holds ctrl_level
 * (-1: d_c - 1) (Sec. 2.1.2 generalized CNOT; Sec. 3.4 cx((c,t), plus)). */
int qd_apply_cx(qd_reg *reg, int32_t c, int32_t t, int32_t shift, int32_t ctrl_level);
/* C^n_{X,d}: X_{+shift} on t when every control holds its level (NULL or -1:
 * d_c - 1) (Sec. 2.1.2 multi-controlled Toffoli). */
int qd_apply_mct(qd_reg *reg, const int32_t *controls, const int32_t *ctrl_levels, int32_t nc,
                 int32_t t, int32_t shift);
/* Apply one gate record.  A QD_GATE_MEASURE record sets the register's
 * measurement flag (qd_measure_all). */
int qd_apply_gate(qd_reg *reg, const qd_gate *gate);

/* Measurement flag (Sec. 3.4: the Measurement Gate only marks the end of the
 * circuit; any gate after it is ignored; Sec. 3.6 measure_all).  After
 * qd_measure_all every later gate call, qd_plan_run, qd_run_circuit and
 * qd_run_moments on the register returns QD_OK without touching the state,
 * until qd_reset or qd_set_amplitudes starts a new circuit.  Readouts are
 * unaffected.  qd_is_measured reports the flag (0 or 1). */
int qd_measure_all(qd_reg *reg);
int qd_is_measured(const qd_reg *reg, int32_t *measured);

/* Toffoli through an elevated carrier level (Sec. 3.4: cx((0,1), plus=1),
 * cx((1,2), plus=1), cx((0,1), plus=2)): X^{d_t}_{+shift} on t when c1 holds
 * d_c1 - 1 and the carrier holds d_carrier - 2, its top logical level.  The
 * three generalized CNOTs, each firing on its control's top level d - 1, are
 * CX_{+1}(c1 -> carrier), CX_{+shift}(carrier -> t), CX_{+(d_carrier-1)}(c1 ->
 * carrier); the carrier's level d_carrier - 1 is the elevated "|d>" level,
 * so the carrier needs dimension >= 3 and returns to its input.
 * qd_toffoli_gates writes the three records (host only, no register needed);
 * qd_apply_toffoli applies them.  Errors: QD_ERR_ARG (index, shift),
 * QD_ERR_OVERLAP (repeated qudit), QD_ERR_DIM (carrier dimension < 3). */
int qd_toffoli_gates(const int32_t *dims, int32_t n, int32_t c1, int32_t carrier, int32_t t, int32_t shift,
                     qd_gate *out3);
int qd_apply_toffoli(qd_reg *reg, int32_t c1, int32_t carrier, int32_t t, int32_t shift);

/* Logarithmic-depth multi-controlled Toffoli through |d>-level controls
 * (Sec. 2.1.2, Fig. 1: controls firing on |d-1> and on |d>): X^{d_t}_{+shift}
 * on t when every control q holds its active level l_q (ctrl_levels[i], NULL
 * or -1: d_q - 2).  The controls form a balanced binary tree in heap order
 * (control i has children 2i+1 and 2i+2); deepest level first, each inner
 * control is shifted +1 under its children (a leaf child firing on l_u, an
 * inner child on its elevated level l_u + 1), which raises it to l_v + 1 iff
 * every control of its subtree is active; then the target fires under the
 * root; then the raises are undone in reverse order.  Every inner control
 * needs l_q + 1 < d_q, and the state's values of each control must not exceed
 * its active level.  Gates: 2 floor(nc / 2) + 1 records with at most two
 * controls each; depth 2 floor(log2 nc) + 1 (gates of one tree level act on
 * disjoint qudits).  qd_mct_tree_gates writes *count records to out (NULL
 * out: count only) and the depth; qd_apply_mct_tree applies them.
 * Errors: QD_ERR_ARG, QD_ERR_OVERLAP, QD_ERR_DIM (no free level on an inner
 * control), QD_ERR_OOM (cap < *count). */
int qd_mct_tree_gates(const int32_t *dims, int32_t n, const int32_t *controls, const int32_t *ctrl_levels, int32_t nc,
                      int32_t t, int32_t shift, qd_gate *out, int32_t cap, int32_t *count, int32_t *depth);
int qd_apply_mct_tree(qd_reg *reg, const int32_t *controls, const int32_t *ctrl_levels, int32_t nc, int32_t t,
                      int32_t shift);

/* ---- circuits ---------------------------------------------------------- */

/* Validate and prepare a gate list for repeated runs on this register:
 * kernel choice, launch parameters and (plan_kind != QD_PLAN_NONE) gate
 * fusion.  Fusion splits the gate list into contiguous segments; a segment of
 * several gates becomes one dense block (the FP64 product of its gates,
 * controls expanded, over the union of their qudits, at most
 * QD_TUNE_FUSE_KMAX qudits and QD_TUNE_FUSE_DMAX states) applied in one pass.
 * QD_PLAN_GREEDY extends a segment while the cost model prefers the merged
 * block; QD_PLAN_EXHAUSTIVE takes the exact minimum-cost segmentation.
 * Identity gates are dropped.  The gates array and its matrices may be freed
 * after the call.  Errors: those of the gates (prefixed with the gate index),
 * QD_ERR_UNSUPPORTED for a plan kind without its cost model. */
int qd_plan_create(qd_reg *reg, const qd_gate *gates, int32_t ngates, int32_t plan_kind, qd_plan **out);
/* Enqueue the prepared circuit on the register's stream.  On a non-default
 * stream the first run captures the launches into a CUDA graph and later runs
 * replay it (one launch call per run); on the legacy default stream every run
 * launches the kernels directly. */
int qd_plan_run(qd_plan *plan);
/* Number of kernel launches one run enqueues, and of fused blocks. */
int qd_plan_info(const qd_plan *plan, int32_t *launches, int32_t *blocks);
int qd_plan_destroy(qd_plan *plan);
/* Per-launch timing: with enable != 0 every qd_plan_run launches directly
 * (no graph), holds the stream with a host function until all launches are
 * enqueued, and records a CUDA event before each launch and after the last.
 * qd_plan_timings then synchronises the stream and writes, for launch i of
 * the latest run, its device time in ms (events), its algorithmic HBM bytes
 * (2 x bytes of the amplitudes it reads and writes) and its kernel class
 * (QD_KCLASS_* | D << 8).  Any output pointer may be NULL. */
#define QD_KCLASS_DENSE_DIRECT 0
#define QD_KCLASS_DENSE_TILE 1
#define QD_KCLASS_MONO_DIRECT 2
#define QD_KCLASS_MONO_TILE 3
#define QD_KCLASS_TENSOR_BLOCK 4 /* fused block on tcgen05 (exact BF16 slices, FP32 accumulate) */
#define QD_KCLASS_DIAG_TABLE 5   /* run of diagonal gates through one table (D = qudits the table covers) */
#define QD_KCLASS_DENSE_TABLE 6  /* dense part followed by a diagonal run's table, one pass (D = dense part) */
int qd_plan_profile(qd_plan *plan, int32_t enable);
int qd_plan_timings(qd_plan *plan, float *ms, double *alg_bytes, int32_t *kclass);
/* Plan, run once with direct launches (no graph capture) and release. */
int qd_run_circuit(qd_reg *reg, const qd_gate *gates, int32_t ngates, int32_t plan_kind);

/* ---- readout (Sec. 3.8), FP64 on the device ---------------------------- */

/* sum_i |psi_i|^2 (FP64) into *out (host).  Synchronises. */
int qd_norm(qd_reg *reg, double *out);
/* p_i = |psi_i|^2 (FP64) for all N entries into out (QD_HOST or QD_DEVICE
 * buffer of N doubles). */
int qd_probabilities(qd_reg *reg, double *out, int32_t where);
/* <a|b> = sum_i conj(a_i) b_i in FP64 over two registers of equal size (the
 * precisions may differ), into *re, *im (host).  Fidelity |<a|b>|^2 between
 * a complex64 result and a complex128 reference stays on the device.
 * Synchronises both streams.  Errors: QD_ERR_ARG, QD_ERR_DIM. */
int qd_overlap(qd_reg *a, qd_reg *b, double *re, double *im);
/* P(x_q = v), v < d_q, into the host array out[d_q].  Synchronises. */
int qd_marginal(qd_reg *reg, int32_t q, double *out);
/* Inclusive prefix sum of p_i (FP64, left to right) into N doubles. */
int qd_cdf(qd_reg *reg, double *out, int32_t where);
/* Measurement sampling: shot s returns the smallest i with
 * CDF_i > u_s * CDF_{N-1}, u_s = 2^-53 * (word 0 of Philox4x64-10 at
 * counter (s,0,0,0), key (seed,0)) >> 11).  out: host array of shots int64. */
int qd_sample(qd_reg *reg, uint64_t seed, int64_t shots, int64_t *out);
/* The same with caller-supplied uniforms u[0..shots) in [0,1) (host). */
int qd_sample_u(qd_reg *reg, const double *u, int64_t shots, int64_t *out);

/* Prefix sums without any device allocation.  The paper has no counterpart
 * to this call; it exists for callers that may not allocate device memory,
 * such as code running under an application allocator that owns all of the
 * device heap, or a latency-critical loop where an allocation (which can
 * synchronise the device) is not allowed.
 * It writes the same inclusive FP64 prefix sums of |state_i|^2 as qd_cdf to
 * the caller's device buffer cdf_out[0..n_amplitudes), reading the caller's
 * device state (QD_C64 or QD_C128 amplitudes), on stream (cudaStream_t as
 * void*, NULL = legacy default stream); it returns once the work is enqueued.
 * Its scratch is a fixed array of 65536 FP64 chunk sums inside the library's
 * device image (512 KiB, held on every GPU that loads the library until the
 * process exits), so n_amplitudes may not exceed 2^28 (QD_ERR_DIM beyond).
 * The first call on each device looks up the array's device address with
 * that device current; make that first call before any stream capture.  Only
 * a successful lookup is kept: after a failed one the next call tries again.
 * All calls share the one array: calls whose work overlaps on the GPU (for
 * example on two streams at once) race on it and must be ordered by the
 * caller.  Values an earlier call left in the array are never read.
 * Errors: QD_ERR_ARG (null pointer, bad precision), QD_ERR_DIM, QD_ERR_CUDA. */
int qd_cdf_noalloc(const void *state, int64_t n_amplitudes, int32_t precision, double *cdf_out, void *stream);

/* Ket readout (Sec. 3.8 OutputType / OutputMethod; Sec. 3.9 prints the
 * basis states of nonzero probability with their amplitudes): the basis
 * indices i with |psi_i|^2 > threshold (FP64), in ascending order, found on
 * the device.  The first min(cap, total) go to indices[] (host) and values[]
 * (host: method QD_OUT_AMPLITUDE writes re, im per entry, 2 doubles;
 * QD_OUT_PROBABILITY writes |psi_i|^2, 1 double); *count receives the total
 * (may exceed cap).  Synchronises.  Errors: QD_ERR_ARG, QD_ERR_OOM. */
#define QD_OUT_AMPLITUDE 0
#define QD_OUT_PROBABILITY 1
int qd_ket_list(qd_reg *reg, int32_t method, double threshold, int64_t cap, int64_t *indices, double *values,
                int64_t *count);
/* Ket label of basis index (OutputType.print): "|x_0 x_1 ... x_{n-1}>",
 * qudit 0 first (the paper prints |120> for x_0 = 1, x_1 = 2, x_2 = 0),
 * digits in decimal, comma-separated when some dimension exceeds 10.
 * Host only.  Errors: QD_ERR_ARG, QD_ERR_DIM, QD_ERR_OOM (cap too small). */
int qd_ket_label(const int32_t *dims, int32_t n, int64_t index, char *buf, int32_t cap);

/* Copy the N amplitudes out of / into the register (register precision). */
int qd_get_amplitudes(qd_reg *reg, void *out, int32_t where);
int qd_set_amplitudes(qd_reg *reg, const void *in, int32_t where);

/* Wait for the register's stream; report a device-side error word (0 if
 * none) in *device_error (may be NULL).  Returns QD_ERR_TIMEOUT when a
 * bounded wait expired (word 1), QD_ERR_DEVICE for any other nonzero word. */
int qd_sync(qd_reg *reg, int32_t *device_error);

/* ---- batched persistent execution -------------------------------------- */
/* Many independent circuits, each on its own register (dims of uneven count
 * and value), complex64 states in one device arena, run by one persistent
 * kernel launch (QuDiet Sec. 2.2 registers, Sec. 2.1.2 / 3.4 gates).  Each
 * circuit is cut into segments of consecutive gates whose acting qudits fit a
 * shared-memory tile; a work item loads tiles of a segment, applies all its
 * gates in shared memory and writes them back (a register of at most
 * QD_BATCH_SMALL_AMPS amplitudes is one segment and one tile).  Items of a
 * circuit's later segments wait on per-circuit completion counters (bounded
 * waits).  Each run resets every register to |0...0>, applies all circuits
 * and writes the FP64 probabilities of every amplitude; on a non-default
 * stream the sequence is captured into a CUDA graph on the first run and
 * replayed afterwards.  Gates: target dimension <= 25, acting qudits (targets
 * and controls) spanning <= 24576 amplitudes; every register holds fewer than
 * 2^31 amplitudes.  The batch owns its device memory; the caller owns every
 * host buffer passed in. */
typedef struct qd_batch qd_batch;
#define QD_BATCH_TILE_AMPS 1   /* largest shared-memory tile of a large circuit's segment (default 4096) */
#define QD_BATCH_CTAS_PER_SM 2 /* persistent CTAs per SM (0: as many as fit; default 0) */
#define QD_BATCH_SMALL_AMPS 3  /* largest register simulated whole in shared memory (default 2048) */
#define QD_BATCH_GROUP_AMPS 4  /* large circuits are queued in groups of about this many amplitudes,
                                  level by level within a group, so that a group's states stay in L2
                                  (default 2^25) */
#define QD_BATCH_TILES_PER_ITEM 5 /* tiles one work item processes (default 1) */
#define QD_BATCH_POLL_LIMIT 6     /* polls of a work item's wait on its circuit's counter before it gives
                                     up, skips its tiles and sets the error word to 2 (0..2^30; default
                                     2^22, over 0.5 s); a small limit makes waits expire on purpose */
/* ncirc registers; register c has nqudits[c] qudits whose dims follow in
 * dims_concat (concatenated in circuit order).  stream: cudaStream_t as void*. */
int qd_batch_create(int32_t ncirc, const int32_t *nqudits, const int32_t *dims_concat, void *stream, qd_batch **out);
/* Set (replace) the gate list of circuit c (copied; identity gates dropped).
 * Errors as for qd_plan_create, plus QD_ERR_DIM for a target dimension above
 * 25 and QD_ERR_UNSUPPORTED for acting qudits spanning more than 24576
 * amplitudes. */
int qd_batch_set_circuit(qd_batch *b, int32_t c, const qd_gate *gates, int32_t ngates);
/* Launch-shape tuning (QD_BATCH_*), used by the autotuner; takes effect at the next run. */
int qd_batch_tune(qd_batch *b, int32_t key, int64_t value);
/* Run every circuit once (asynchronous on the batch's stream).  The first
 * run after a change segments and uploads every circuit. */
int qd_batch_run(qd_batch *b);
/* FP64 probabilities / amplitudes of circuit c after the last run (host
 * buffers of N_c entries; synchronise the stream). */
int qd_batch_probabilities(qd_batch *b, int32_t c, double *out);
int qd_batch_get_amplitudes(qd_batch *b, int32_t c, void *out);
/* Total amplitudes, work items of a run, launches per run, and the device
 * error word (synchronises; nonzero: a bounded wait expired). */
int qd_batch_info(qd_batch *b, int64_t *total_amplitudes, int32_t *items, int32_t *launches, int32_t *device_error);
/* Wait for the batch's stream and report the last run's device error word:
 * QD_ERR_TIMEOUT when a work item's bounded wait expired (word 2; the run's
 * results are not valid), QD_ERR_DEVICE for any other nonzero word (3: a
 * gate descriptor failed its bounds check).  Each run clears the word. */
int qd_batch_sync(qd_batch *b, int32_t *device_error);
/* Profiling mode: runs launch directly (no graph) with CUDA events around the
 * persistent kernel.  qd_batch_timings (synchronises) returns that kernel's
 * time in the last run and its algorithmic bytes (every segment reads and
 * writes its register once: 16 bytes per complex64 amplitude per segment). */
int qd_batch_profile(qd_batch *b, int32_t enable);
int qd_batch_timings(qd_batch *b, float *kernel_ms, double *alg_bytes);
/* Autotuner: runs the batch (reps timed runs after one warm-up run each) in
 * a fixed set of launch shapes - tile amplitudes, shared-memory register
 * limit, CTAs per SM, tiles per item - and keeps the one whose persistent
 * kernel was fastest.  chosen (4 int64, may be NULL): tile amplitudes, small
 * register limit, CTAs per SM, tiles per item; best_ms (may be NULL): its
 * kernel time.  Synchronises; the registers hold the last run's result. */
int qd_batch_autotune(qd_batch *b, int32_t reps, int64_t *chosen, float *best_ms);
int qd_batch_destroy(qd_batch *b);

/* ---- learned cost model ------------------------------------------------ */
/* The fusion planner's learned cost model: an MLP 12 -> 64 -> 64 -> 64 -> 1
 * (ReLU) predicting log(launch time in microseconds) from the 12 launch
 * features of a candidate segment (qd_segment_features).  Trained on the GPU
 * by the library's own forward, backward and Adam kernels; inference uses
 * FP16 weights with FP32 accumulation.  The paper has no such component; it
 * steers the fusion of the paper's gates (QD_PLAN_LEARNED).  Parameters are
 * QD_MODEL_PARAMS floats: W1 (12x64, row = input), b1, W2 (64x64), b2, W3,
 * b3, W4 (64), b4. */
#define QD_MODEL_FEATURES 12
#define QD_MODEL_PARAMS 9217
typedef struct qd_model qd_model;
int qd_model_create(qd_model **out);
int qd_model_destroy(qd_model *model);
/* Set parameters and the feature / target normalisation (NULL mean or std:
 * 0 and 1). */
int qd_model_set(qd_model *model, const float *params, const float *feat_mean, const float *feat_std, float y_mean,
                 float y_std);
int qd_model_get(const qd_model *model, float *params, float *feat_mean, float *feat_std, float *y_mean, float *y_std);
/* Fit to n samples (features X[n][12] host, targets y[n] = log time) with Adam:
 * epochs over shuffled mini-batches, learning rate lr, seeded initialisation;
 * *final_loss = mean squared error over the set in normalised units. */
int qd_model_train(qd_model *model, const float *X, const float *y, int32_t n, int32_t epochs, int32_t batch,
                   float lr, uint64_t seed, double *final_loss);
/* Predicted targets for n feature rows (host arrays), FP16 weights. */
int qd_model_predict(qd_model *model, const float *X, int32_t n, float *y);
/* Network on already-normalised rows (fp16 = 0: FP32 weights). */
int qd_model_forward_raw(qd_model *model, const float *Xn, int32_t n, float *y, int32_t fp16);
/* Mean-squared-error loss and its gradient (QD_MODEL_PARAMS floats) for
 * already-normalised rows and targets, by the forward and backward kernels. */
int qd_model_grad_raw(qd_model *model, const float *Xn, const float *t, int32_t n, double *loss, float *grad);
/* Attach a model to a register for QD_PLAN_LEARNED (NULL detaches; the
 * model must outlive the plans made with it). */
int qd_set_cost_model(qd_reg *reg, qd_model *model);
/* Kernel forms of one launch (launch feature 10). */
#define QD_FORM_MONO 0       /* one permutation / diagonal gate */
#define QD_FORM_DENSE 1      /* one dense gate */
#define QD_FORM_BLOCK 2      /* fused block, CUDA-core dense kernel (D <= 32) */
#define QD_FORM_BLOCK_TC 3   /* fused block, tensor-core kernel (complex64, 9 <= D <= 64) */
#define QD_FORM_DIAG_RUN 4   /* run of diagonal gates through one table */
#define QD_FORM_DENSE_RUN 5  /* dense part (<= 16 states) followed by a diagonal run */
/* The 12 launch features of gates[first..last] (indices of the non-identity
 * gates) as one launch on this register, in the form that
 * qd_plan_create_segmented gives that segment: log2 D (of the table, for a
 * diagonal run), qudit count, log2 of the three smallest strides, relative
 * positions, log2 N, precision, kernel form (QD_FORM_*), log2 of the
 * control-slice fraction (of the table size, for a dense part + run).  Errors: QD_ERR_ARG (bad segment). */
int qd_segment_features(qd_reg *reg, const qd_gate *gates, int32_t ngates, int32_t first, int32_t last, float *out);
/* Every feasible kernel form of gates[first..last] under the hard limits of
 * qd_plan_create_segmented (the candidates a planner weighs): *nforms of
 * them (at most 3), kinds[i] the kernel form (QD_FORM_*) and features[i*12..] its 12
 * launch features, for i < cap.  QD_ERR_OOM when *nforms > cap (the first
 * cap are written), except for a count query (cap 0, both arrays NULL). */
int qd_segment_forms(qd_reg *reg, const qd_gate *gates, int32_t ngates, int32_t first, int32_t last, int32_t *kinds,
                     float *features, int32_t cap, int32_t *nforms);
/* A plan from an explicit segmentation: segment i covers the non-identity
 * gates [seg_first[i], seg_last[i]] (contiguous, in order, covering all);
 * multi-gate segments become fused blocks regardless of the size limits of
 * QD_TUNE_FUSE_*, up to 6 qudits and D <= 64 (complex64) or 32 (complex128),
 * or, when every gate of the segment is diagonal, one diagonal-run launch
 * over any qudits whose covering range has at most 2^24 states, or, when the
 * segment is a dense part of at most 16 states followed by such a run, one
 * dense launch that applies the run's table to its outputs. */
int qd_plan_create_segmented(qd_reg *reg, const qd_gate *gates, int32_t ngates, const int32_t *seg_first,
                             const int32_t *seg_last, int32_t nseg, qd_plan **out);
/* qd_plan_create_segmented with the kernel form of every segment given:
 * seg_kind[i] a kernel form from qd_segment_forms for that segment, or -1
 * for the cost model's choice (seg_kind NULL: all -1).  Errors: QD_ERR_ARG
 * when a given form is not feasible for its segment. */
int qd_plan_create_forms(qd_reg *reg, const qd_gate *gates, int32_t ngates, const int32_t *seg_first,
                         const int32_t *seg_last, const int32_t *seg_kind, int32_t nseg, qd_plan **out);

/* ---- QuDiet QASM front end (Sec. 4) ----------------------------------- */
/* Parse a QuDiet QASM program: ".qudit n"; n declarations "qudit NAME (d)" in
 * qudit order (the first declared is qudit 0); ".begin"; gate lines "X q [a]"
 * (X^d_{+a}, a = 1 if absent), "Z q [p]" (Z_d^p, p = 1 if absent), "H q"
 * (F_d), "CX c t [a]" (X^{d_t}_{+a} on t when c holds d_c - 1); ".end".
 * Names are case-insensitive; '#' or "//" starts a comment.  Writes the dims
 * (dims_cap entries) and gate records (gates_cap entries; named gates carry
 * no matrix), *n and *ngates the counts (written also when an array is too
 * small, which returns QD_ERR_OOM; NULL arrays query the counts).  On a
 * syntax error *error_line is the 1-based line.  Errors: QD_ERR_ARG
 * (syntax, unknown name or gate, shift out of [1, d-1]), QD_ERR_DIM
 * (dimension outside [2, 64]), QD_ERR_OVERLAP (CX on one qudit). */
int qd_qasm_parse(const char *text, int32_t *dims, int32_t dims_cap, int32_t *n, qd_gate *gates, int32_t gates_cap,
                  int32_t *ngates, int32_t *error_line);

/* ---- the paper's execution model, for comparison (Sec. 3.5-3.6) -------- */
/* Apply the gate list to the register's current state the way the paper's
 * backends do: gates are packed into moments (each gate in the first moment
 * after the last one holding a gate on any of its qudits), every moment
 * becomes its full N x N Kronecker-product operator with identities on the
 * untouched qudits, the operators are multiplied from the last moment down
 * to the first (GEMM chain) and the product is applied to the state (GEMV),
 * all in complex128 on the device.  Registers of at most 4096 amplitudes
 * (QD_ERR_DIM beyond); allocates three N x N operators per call;
 * synchronises.  *n_moments (may be NULL) receives the moment count. */
int qd_run_moments(qd_reg *reg, const qd_gate *gates, int32_t ngates, int32_t *n_moments);
/* Host only: the moment of every gate (-1 for gates dropped as identities or
 * after a measurement flag) and the moment count. */
int qd_moment_packing(const int32_t *dims, int32_t n, const qd_gate *gates, int32_t ngates, int32_t *moment_of_gate,
                      int32_t *n_moments);

/* Static message for an error code; thread-local message of the last failure. */
const char *qd_strerror(int code);
const char *qd_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* QUDIT_H */
