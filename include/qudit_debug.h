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
#ifdef __cplusplus
}
#endif
#endif
