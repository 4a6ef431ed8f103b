// Candidate schedules of the forward / inverse transform, per N.
//
// A schedule fixes how the log2 N butterfly stages of Sec. II-D are split
// into kernels and fused register passes (the stage-fusion and switch-point
// design space of Sec. V-A/B/D, re-expressed for sm_103a):
//
//   S1(LOGN, LOGT, LOGRP, TPC, PIPE)
//       one kernel, one row per tile: 2^LOGT threads per row, R = N/2^LOGT
//       coefficients per thread, passes of up to LOGRP fused stages,
//       TPC rows per CTA.
//   S2(LOGN, SPLIT, LOGP, LOGTA, LOGRPA, TPCA, LOGTB, LOGRPB, TPCB, PIPE)
//       two kernels: a column kernel runs stages [0, SPLIT) on tiles of
//       2^SPLIT x 2^LOGP (2^LOGP adjacent columns for 128-byte coalescing),
//       then a row kernel runs [SPLIT, LOGN) on contiguous blocks of
//       2^(LOGN - SPLIT).  The inverse runs them in the opposite order.
//   PIPE is the kernel form: 1 the persistent, double-buffered form fed by
//       bulk asynchronous copies; 0 the direct form; 2 the direct form
//       reading twiddles through the read-only cache instead of staging them
//       in shared memory.  An S2 entry may give its row kernel another form:
//       PIPE = A | B << 2 with B != 0 runs the column kernel in form A and
//       the row kernel in form B (8 = column direct, rows read-only); below
//       4 both kernels use PIPE.
//
// The lists are split by N so that the kernel translation units can be
// compiled in parallel; NTT_SCHEDULES_ALL keeps the table order (which is
// the schedule id order within each N).
#pragma once

#define NTT_SCHEDULES_SMALL(S1, S2)                                                   \
    S1(1, 0, 1, 128, 0)                                                           \
    S1(2, 0, 2, 128, 0)                                                           \
    S1(3, 0, 3, 128, 0)                                                           \
    S1(4, 0, 4, 64, 0) S1(4, 1, 3, 64, 0)                                         \
    S1(5, 0, 5, 32, 0) S1(5, 1, 4, 32, 0) S1(5, 2, 3, 32, 0)                      \
    S1(6, 1, 5, 32, 0) S1(6, 2, 4, 16, 0) S1(6, 3, 3, 16, 0)                      \
    S1(7, 2, 5, 16, 0) S1(7, 3, 4, 8, 0) S1(7, 4, 3, 8, 0)                        \
    S1(8, 3, 5, 8, 0) S1(8, 4, 4, 8, 0) S1(8, 5, 3, 4, 0) S1(8, 5, 3, 4, 1)       \
    S1(9, 4, 5, 4, 0) S1(9, 5, 4, 4, 0) S1(9, 6, 3, 2, 0) S1(9, 6, 3, 2, 1)

#define NTT_SCHEDULES_MID(S1, S2)                                                     \
    S1(10, 7, 3, 1, 0) S1(10, 7, 3, 1, 1) S1(10, 6, 4, 2, 0) S1(10, 6, 4, 2, 1)   \
    S1(10, 5, 5, 4, 0) S1(10, 8, 2, 1, 1) S1(10, 8, 2, 1, 0) S1(10, 7, 3, 1, 2)   \
    S1(11, 8, 3, 1, 0) S1(11, 8, 3, 1, 1) S1(11, 7, 4, 1, 0) S1(11, 7, 4, 1, 1)   \
    S1(11, 6, 5, 2, 0) S1(11, 8, 3, 1, 2)                                         \
    S1(12, 9, 3, 1, 0) S1(12, 9, 3, 1, 1) S1(12, 8, 4, 1, 0) S1(12, 8, 4, 1, 1)   \
    S1(12, 7, 5, 1, 0) S1(12, 9, 3, 1, 2)

#define NTT_SCHEDULES_LARGE(S1, S2)                                                   \
    S1(13, 9, 4, 1, 0) S1(13, 8, 5, 1, 0) S1(13, 10, 3, 1, 0)                     \
    S2(13, 6, 4, 6, 4, 1, 5, 3, 4, 0) S2(13, 6, 4, 6, 4, 1, 5, 3, 4, 2)           \
    S2(13, 6, 4, 6, 4, 1, 5, 3, 4, 8)                                             \
    S1(14, 10, 4, 1, 0) S1(14, 9, 5, 1, 0)                                        \
    S2(14, 7, 4, 7, 4, 1, 4, 4, 8, 1) S2(14, 7, 4, 7, 4, 1, 4, 3, 8, 0)           \
    S2(14, 7, 4, 7, 4, 1, 5, 2, 4, 0) S2(14, 7, 4, 7, 4, 1, 4, 3, 8, 2)           \
    S2(14, 7, 4, 7, 4, 1, 4, 3, 8, 8)                                             \
    S2(15, 7, 4, 7, 4, 1, 4, 4, 8, 1) S2(15, 7, 4, 6, 5, 1, 3, 5, 16, 0)          \
    S2(15, 5, 4, 4, 5, 4, 5, 5, 4, 0) S2(15, 7, 4, 8, 3, 1, 5, 3, 8, 0)           \
    S2(15, 7, 4, 7, 4, 1, 5, 3, 4, 0) S2(15, 7, 4, 7, 4, 1, 5, 3, 4, 2)           \
    S2(15, 7, 4, 7, 4, 1, 5, 3, 4, 8)

#define NTT_SCHEDULES_HUGE(S1, S2)                                                    \
    S2(16, 8, 4, 8, 4, 1, 5, 3, 4, 0) S2(16, 7, 4, 7, 4, 1, 6, 3, 2, 2)           \
    S2(16, 8, 4, 8, 4, 1, 5, 3, 8, 0) S2(16, 8, 4, 8, 4, 1, 5, 3, 2, 0)           \
    S2(16, 8, 4, 8, 4, 1, 6, 2, 2, 0) S2(16, 7, 4, 7, 4, 1, 6, 3, 2, 8)           \
    S2(16, 7, 4, 7, 4, 1, 6, 3, 2, 0) S2(16, 8, 4, 8, 4, 1, 5, 3, 4, 2)           \
    S2(16, 7, 4, 7, 4, 1, 5, 3, 4, 8) S2(16, 7, 4, 7, 4, 1, 5, 4, 4, 8)           \
    S2(16, 7, 4, 7, 4, 1, 5, 3, 2, 8)

#define NTT_SCHEDULES_ALL(S1, S2)                                           \
    NTT_SCHEDULES_SMALL(S1, S2) NTT_SCHEDULES_MID(S1, S2) NTT_SCHEDULES_LARGE(S1, S2) \
    NTT_SCHEDULES_HUGE(S1, S2)

// On-the-fly-twiddle transforms (NTT_FLAG_OTF_TWIDDLES): one configuration
// per N >= 2^10, the measured default geometry with every kernel in form 3
// (twiddles generated from two small per-limb tables, see ntt_tile.cuh).
#define NTT_OTF_CONFIGS(S1, S2)                                                       \
    S1(10, 7, 3, 1, 3) S1(11, 8, 3, 1, 3) S1(12, 9, 3, 1, 3)                      \
    S2(13, 6, 4, 6, 4, 1, 5, 3, 4, 3) S2(14, 7, 4, 7, 4, 1, 4, 3, 8, 3)           \
    S2(15, 7, 4, 7, 4, 1, 5, 3, 4, 3) S2(16, 7, 4, 7, 4, 1, 6, 3, 2, 3)
