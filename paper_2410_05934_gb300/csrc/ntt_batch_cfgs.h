// Tile configurations of the mixed-batch persistent kernel: one per N in
// [2^10, 2^16], all with 256-thread CTAs (so a single kernel can run any of
// them), at most 8 coefficients per thread (the kernel's register budget is
// set by its largest path) and at most 18 KiB of shared memory (a 2^11-word
// tile and its staged twiddles), so three CTAs fit on an SM by registers and
// the rest of the SM's 256 KiB of L1/shared memory caches the twiddle tables.
//   SINGLE(LOGN, LOGT, LOGRP, TPC, MODE)   one tile kernel's phases (whole rows)
//   SPLIT(LOGN, SPLIT, LOGP, LOGTA, LOGRPA, TPCA, LOGTB, LOGRPB, TPCB, MODE)
//                                    column phase then row phase per row
// MODE as in the schedule list: 0 stages twiddles in shared memory, 2 reads
// them through the read-only cache, 8 = column phase 0 and row phase 2 (the
// forms measured fastest on GB300).
// The host emulation checks the same list against the oracle.
#pragma once

#define NTT_BATCH_CONFIGS(SINGLE, SPLIT)                                   \
    SINGLE(10, 7, 3, 2, 2)                                                 \
    SINGLE(11, 8, 3, 1, 2)                                                 \
    SPLIT(12, 6, 4, 8, 2, 1, 3, 3, 32, 8)                                  \
    SPLIT(13, 6, 4, 8, 2, 1, 4, 3, 16, 8)                                  \
    SPLIT(14, 7, 4, 8, 3, 1, 4, 3, 16, 8)                                  \
    SPLIT(15, 7, 4, 8, 3, 1, 5, 3, 8, 8)                                   \
    SPLIT(16, 7, 4, 8, 3, 1, 6, 3, 4, 8)
