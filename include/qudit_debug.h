/*
 * qudit_debug.h - host-only inspection entry point of libqudit, for tests.
 *
 * qd_debug_gate_members runs the library's gate planner for a register of
 * dims[0..n) (no device, no allocation) and replays on the host the index
 * arithmetic the chosen kernel performs: for every group it writes the flat
 * amplitude indices of the group's D members, in local-index order, to
 * out[group * D + j] (up to cap entries).  info (7 int64) receives: mode
 * (0 direct, 1 tile), D, number of groups, kind (0 dense, 1 diagonal or
 * permutation with phases), active-member mask, tile block length B, and
 * the noop flag (1 if the gate is the identity and launches nothing).
 *
 * The groups of a gate are the sets of amplitudes it mixes: with targets T
 * and controls C at levels l_c, one group per assignment of the qudits
 * outside T and C, restricted to x_c = l_c (QuDiet Sec. 2.1.2, the block
 * structure of C_{X,d} and C^n_{X,d}).
 * Returns QD_OK or the planner's error code.
 */
#ifndef QUDIT_DEBUG_H
#define QUDIT_DEBUG_H
#include "qudit.h"
#ifdef __cplusplus
extern "C" {
#endif
int qd_debug_gate_members(const int32_t *dims, int32_t n, const qd_gate *gate, int64_t *out, int64_t cap,
                          int64_t *info);
/* The same with an explicit tile-stride threshold (see QD_TUNE_TILE_STRIDE). */
int qd_debug_gate_members_tuned(const int32_t *dims, int32_t n, const qd_gate *gate, int64_t tile_stride,
                                int64_t *out, int64_t cap, int64_t *info);

/* Fusion planner replay (host only, no device).  For a register of dims[0..n)
 * at `precision`, plan gates[0..ngates) with plan_kind and the fusion limits
 * kmax, dmax (as QD_TUNE_FUSE_KMAX / QD_TUNE_FUSE_DMAX): writes the chosen
 * contiguous segments as [seg_first[i], seg_last[i]] gate ranges (indices of
 * the non-identity gates, in order; up to cap), their count in *nseg, and the
 * cost model's total in *model_cost. */
int qd_debug_fuse_plan(const int32_t *dims, int32_t n, int32_t precision, const qd_gate *gates, int32_t ngates,
                       int32_t plan_kind, int32_t kmax, int32_t dmax, int32_t *seg_first, int32_t *seg_last,
                       int32_t cap, int32_t *nseg, double *model_cost);
/* Cost the model assigns to the segment [first, last] of the non-identity
 * gates (one gate: its own kernel; several: one dense block). */
int qd_debug_segment_cost(const int32_t *dims, int32_t n, int32_t precision, const qd_gate *gates, int32_t ngates,
                          int32_t first, int32_t last, double *cost);
/* The feasible kernel forms of the segment [first, last] (as
 * qd_segment_forms, for a register of dims[0..n) at `precision`, no device):
 * *nforms of them, kinds[i] (QD_FORM_*) and features[i*12..] for i < cap. */
int qd_debug_segment_forms(const int32_t *dims, int32_t n, int32_t precision, const qd_gate *gates, int32_t ngates,
                           int32_t first, int32_t last, int32_t *kinds, float *features, int32_t cap,
                           int32_t *nforms);
/* The fused block of gates [first, last]: its qudits (first = most
 * significant local digit, at most 6) and its D x D FP64 matrix (interleaved
 * complex, row-major; cap doubles available). */
int qd_debug_fuse_block(const int32_t *dims, int32_t n, const qd_gate *gates, int32_t ngates, int32_t first,
                        int32_t last, int32_t *qudits, int32_t *k, int32_t *D, double *matrix, int64_t cap);
/* Batched execution replay (host only, no device).  Builds the batch of
 * ncirc registers (as qd_batch_create; circuit c's ngates[c] gates follow one
 * another in `gates`), applies the tuning tune[0..4) = tile amplitudes, small
 * register limit, group amplitudes, tiles per item (a negative entry keeps
 * the default; tune may be NULL), encodes the segments, tiles, local gate
 * geometry and work queue exactly as a run does, and replays the queue in
 * order on the host in FP64 with the kernel's index arithmetic, from every
 * register at |0...0>.  amps (2 * total doubles) receives the final states
 * (interleaved complex, circuit after circuit); info (5 int64): segments, work items,
 * largest tile, algorithmic bytes, and an error mask: 1 an item waits on a
 * later one, 2 a tile index leaves its register, 4 a segment's tiles do not
 * cover the register exactly once, 8 a gate index leaves its tile, 16 a
 * chunk of gate descriptors overflows its shared-memory area or is
 * misaligned, 32 a tile gathered as amplitude pairs has a pair that is not
 * 16-byte aligned in the arena. */
int qd_debug_batch_emulate(int32_t ncirc, const int32_t *nqudits, const int32_t *dims_concat, const qd_gate *gates,
                           const int32_t *ngates, const int64_t *tune, double *amps, int64_t *info);
#ifdef __cplusplus
}
#endif
#endif
