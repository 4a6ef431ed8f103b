// Tile configurations of the mixed-batch persistent kernel: one per N in
// [2^10, 2^16], all with 256-thread CTAs (so a single kernel can run any of
// them), at most 8 coefficients per thread (the kernel's register budget is
// set by its largest path) and at most 48 KiB of shared memory, so three
// CTAs fit on an SM.
//   SINGLE(LOGN, LOGT, LOGRP, TPC)   one tile kernel's phases (whole rows)
//   SPLIT(LOGN, SPLIT, LOGP, LOGTA, LOGRPA, TPCA, LOGTB, LOGRPB, TPCB)
//                                    column phase then row phase per row
// The host emulation checks the same list against the oracle.
#pragma once

#define NTT_BATCH_CONFIGS(SINGLE, SPLIT)                                   \
    SINGLE(10, 7, 3, 2)                                                    \
    SINGLE(11, 8, 3, 1)                                                    \
    SPLIT(12, 6, 4, 8, 2, 1, 3, 3, 32)                                     \
    SPLIT(13, 6, 4, 8, 2, 1, 4, 3, 16)                                     \
    SPLIT(14, 7, 4, 8, 3, 1, 4, 3, 16)                                     \
    SPLIT(15, 7, 4, 8, 3, 1, 5, 3, 8)                                      \
    SPLIT(16, 7, 4, 8, 3, 1, 6, 3, 4)
