// Tile configurations of the mixed-batch persistent kernel: one per N in
// [2^10, 2^16], all with 128-thread CTAs (so a single kernel can run any of
// them) and at most 18 KiB of shared memory (a 2^11-word tile and its staged
// twiddles).  For N >= 2^14 they are the geometries of the standalone
// schedules measured fastest on GB300 (column tiles of 2^7 x 16 with 16
// coefficients per thread in passes of 4 stages, row tiles of 8 coefficients
// per thread in passes of 3 stages), so a row in the persistent kernel runs
// the same tile code as in a plain launch.
//   SINGLE(LOGN, LOGT, LOGRP, TPC, MODE)   one tile kernel's phases (whole rows)
//   SPLIT(LOGN, SPLIT, LOGP, LOGTA, LOGRPA, TPCA, LOGTB, LOGRPB, TPCB, MODE)
//                                    column phase then row phase per row
// MODE as in the schedule list: 0 stages twiddles in shared memory, 2 reads
// them through the read-only cache, 8 = column phase 0 and row phase 2 (the
// forms measured fastest on GB300).
// The host emulation checks the same list against the oracle.
#pragma once

#define NTT_BATCH_CONFIGS(SINGLE, SPLIT)                                   \
    SINGLE(10, 7, 3, 1, 2)                                                 \
    SINGLE(11, 7, 4, 1, 2)                                                 \
    SPLIT(12, 6, 4, 6, 4, 2, 3, 3, 16, 8)                                  \
    SPLIT(13, 6, 4, 6, 4, 2, 4, 3, 8, 8)                                   \
    SPLIT(14, 7, 4, 7, 4, 1, 4, 3, 8, 8)                                   \
    SPLIT(15, 7, 4, 7, 4, 1, 5, 3, 4, 8)                                   \
    SPLIT(16, 7, 4, 7, 4, 1, 6, 3, 2, 8)
