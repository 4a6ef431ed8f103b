// Launcher interface between the C ABI and the kernel translation units.
#pragma once
#include <stdint.h>

#include "ntt_tile.cuh"

namespace nttgb {

// Device-side view of a plan (host pointers when used by the emulation).
struct PlanDev {
    const TwPair* fwd;
    const TwPair* inv;
    const LimbConst* lc;
    int* status;
    uint32_t n_moduli;
    uint32_t check;
    uint32_t mc;        // modulus class: 1 when every modulus is below 2^57, 2 below 2^50
    uint32_t src_mode;  // 1: the inverse's first kernel computes the CKKS tensor product;
                        // 2: the forward transform is the Rescale by aux_q (TileArgs);
                        // 3: the inverse's first kernel multiplies two rows pointwise
    const uint64_t* in_b;
    uint64_t aux_q;
    uint32_t nat;       // natural-order forward output / inverse input (full-row kernels)
    uint32_t has_map;        // source mode 3: polynomial maps of the two factors
    uint8_t a_map[NTT_MUL_MAX_MAPPED], b_map[NTT_MUL_MAX_MAPPED];
    const TwPair* otf_fwd = nullptr;   // on-the-fly twiddle tables (form 3 kernels)
    const TwPair* otf_inv = nullptr;
    uint32_t in_skip = 0;              // TileArgs.in_skip of the first kernel
};

// Transforms rows [row_begin, row_begin + n_rows) of the layout that starts
// at in/out.  Returns NTT_OK or NTT_ERR_CUDA; adds its launch count.
typedef int (*LaunchFn)(const PlanDev& p, const uint64_t* in, uint64_t* out, uint64_t row_begin,
                        uint64_t n_rows, void* stream, uint32_t* launches);

template <int LOGN, int LOGT, int LOGRP, int TPC, int PIPE, bool INV>
int launch_s1(const PlanDev& p, const uint64_t* in, uint64_t* out, uint64_t row_begin,
              uint64_t n_rows, void* stream, uint32_t* launches);

template <int LOGN, int SPLIT, int LOGP, int LOGTA, int LOGRPA, int TPCA, int LOGTB, int LOGRPB,
          int TPCB, int PIPE, bool INV>
int launch_s2(const PlanDev& p, const uint64_t* in, uint64_t* out, uint64_t row_begin,
              uint64_t n_rows, void* stream, uint32_t* launches);

// c = a (.) b over n_rows rows of 2^log2n, row r using modulus (row_begin + r) mod n_moduli
int launch_pointwise(const PlanDev& p, uint32_t log2n, const uint64_t* a, const uint64_t* b,
                     uint64_t* c, uint64_t row_begin, uint64_t n_rows, void* stream,
                     uint32_t* launches);

// 32-bit-word plans (NTT_FLAG_WORD32)
struct Tw32;
struct LimbConst32;
struct Plan32Dev {
    const Tw32* fwd;
    const Tw32* inv;
    const LimbConst32* lc;
    int* status;
    uint32_t n_moduli;
    uint32_t check;
};
int launch_ntt32(const Plan32Dev& p, bool inverse, const uint32_t* in, uint32_t* out, uint64_t row_begin,
                 uint64_t n_rows, uint32_t log2n, void* stream, uint32_t* launches);
// the forward rows of pf and the inverse rows of pi (independent buffers):
// one grid at N = 1024, else the two transforms in stream order
int launch_ntt32_fwd_inv(const Plan32Dev& pf, const uint32_t* fin, uint32_t* fout, uint64_t f_rows,
                         const Plan32Dev& pi, const uint32_t* iin, uint32_t* iout, uint64_t i_rows, uint32_t log2n,
                         void* stream, uint32_t* launches);
// the 32-bit butterfly probe with compare-and-select conditional subtractions (kind 8)
int launch_bench_bfly32_cmp(uint64_t q, uint32_t blocks, uint32_t threads, uint32_t iters, uint64_t* sink,
                            void* stream);
int launch_pointwise32(const Plan32Dev& p, uint32_t log2n, const uint32_t* a, const uint32_t* b, uint32_t* c,
                       uint64_t n_rows, void* stream, uint32_t* launches);

// bit-reversal permutation of rows (in == out: in place)
int launch_bitrev_rows(const uint64_t* in, uint64_t* out, uint64_t row_begin, uint64_t n_rows, uint32_t log2n,
                       void* stream, uint32_t* launches);

// ---- grouped launches (batch.cu / grouped.cu) ----
// One request's segment of a grouped grid for one kernel phase.
struct GroupSeg {
    const uint64_t* in;
    uint64_t* out;
    const TwPair* tw;          // the request's forward or inverse tables
    const LimbConst* lc;
    uint64_t n_tiles;          // tiles of this phase's configuration over the request's rows
    uint64_t group_begin;      // first CTA of the segment in the grid
    uint64_t mod_magic;        // fdiv_magic(n_moduli)
    uint32_t n_moduli, inverse, fast32, pad;
};
// kernel phases of N's grouped configuration (0: N not covered)
int grouped_phases(uint32_t log2n);
// log2 tiles per row and tiles per CTA of one phase and direction
int grouped_geometry(uint32_t log2n, int phase, bool inverse, uint32_t* log_tiles_per_row, uint32_t* tpc);
int launch_grouped(uint32_t log2n, uint32_t mc, int phase, const GroupSeg* d_segs, uint32_t n_segs, uint64_t grid,
                   int* status, uint32_t check, void* stream);
// phase `phase` of one forward and one inverse segment of N in one grid, the
// segments passed by value (the inverse's CTAs first: sf.group_begin is
// their count); status / check: {forward plan's, inverse plan's}
int launch_pair(uint32_t log2n, uint32_t mc, int phase, const GroupSeg& sf, const GroupSeg& si, uint64_t grid,
                int* const* status, const uint32_t* check, void* stream);

int launch_bench_bfly(uint64_t q, uint32_t kind, uint32_t blocks, uint32_t threads, uint32_t iters,
                      uint64_t* sink, void* stream);

// one CTA waiting, bounded, on an mbarrier that only a 16-byte copy from src
// completes (issued when deliver != 0); records NTT_STATUS_TIMEOUT when the
// wait runs out
int launch_debug_bounded_wait(const void* src, uint32_t deliver, uint32_t limit, int* status, uint64_t* out,
                              void* stream);

struct SchedEntry {
    uint32_t log2n;
    uint32_t kernels;
    const char* name;
    LaunchFn fwd, inv;
};

// the table of NTT_SCHEDULES_ALL, in order
const SchedEntry* sched_table(int* count);

}  // namespace nttgb
