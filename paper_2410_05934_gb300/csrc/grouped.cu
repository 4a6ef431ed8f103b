// Grouped launches of independent transform requests (C ABI: ntt_batch_* with
// NTT_BATCH_GROUPED).
//
// The paper batches the independent operations of one iteration into one
// launch (Sec. IV-A).  Here every request of one N becomes a segment of one
// grid: the tile groups of all segments are numbered consecutively and CTA b
// finds its segment by a binary search over the segments' first group, so a
// batch of R requests of one N costs one launch per kernel phase instead of
// R launch sequences, and no request leaves its own partly filled last wave.
// Forward and inverse requests share a grid (both configurations have the
// same CTA shape).  Each N has one configuration: the measured large-batch
// schedule of that N, re-shaped where needed so that its phases use the same
// thread count.
#include <cuda_runtime.h>

#include "ntt_gb300.h"
#include "ntt_kernels.cuh"
#include "ntt_launch.h"

namespace nttgb {

// SINGLE(LOGN, LOGT, LOGRP, TPC, MODE) / SPLIT(LOGN, SPLIT, LOGP, LOGTA, LOGRPA,
// TPCA, LOGTB, LOGRPB, TPCB, MODE) as in the schedule list.
#define NTT_GROUP_CONFIGS(SINGLE, SPLIT)                  \
    SINGLE(10, 7, 3, 1, 2)                                \
    SINGLE(11, 8, 3, 1, 2)                                \
    SINGLE(12, 9, 3, 1, 2)                                \
    SPLIT(13, 6, 4, 6, 4, 2, 5, 3, 4, 8)                  \
    SPLIT(14, 7, 4, 7, 4, 1, 4, 3, 8, 8)                  \
    SPLIT(15, 7, 4, 7, 4, 1, 5, 3, 4, 8)                  \
    SPLIT(16, 7, 4, 7, 4, 1, 6, 3, 2, 8)

// CTA b of a grouped grid: the last segment whose first group is <= b
NTT_HD uint32_t group_segment(const GroupSeg* segs, uint32_t n_segs, uint64_t b) {
    uint32_t lo = 0, hi = n_segs;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (segs[mid].group_begin <= b) lo = mid; else hi = mid;
    }
    return lo;
}

// One phase of a grouped grid: CF runs the forward segments, CI the inverse ones.
template <class CF, class CI>
__global__ void __launch_bounds__(CF::THREADS) k_ntt_grouped(const GroupSeg* __restrict__ segs, uint32_t n_segs,
                                                              int* status, uint32_t check) {
    static_assert(CF::THREADS == CI::THREADS, "forward and inverse segments share the CTA shape");
    extern __shared__ __align__(16) uint64_t smem[];
    pdl_begin();
    const uint64_t b = blockIdx.x;
    const GroupSeg sg = segs[group_segment(segs, n_segs, b)];
    TileArgs a;
    a.in = sg.in;
    a.out = sg.out;
    a.tw = sg.tw;
    a.lc = sg.lc;
    a.status = status;
    a.row_begin = 0;
    a.n_tiles = sg.n_tiles;
    a.n_moduli = sg.n_moduli;
    a.check = check;
    a.fast32 = sg.fast32;
    a.mod_magic = sg.mod_magic;
    a.src_mode = 0;
    a.in_b = nullptr;
    a.aux_q = 0;
    a.nat = 0;
    a.has_map = 0;
    a.otf = nullptr;
    a.in_skip = 0;
    if (sg.inverse)
        tile_group<CI>(a, b - sg.group_begin, smem);
    else
        tile_group<CF>(a, b - sg.group_begin, smem);
}

// Two segments passed by value (ntt_forward_inverse): CTAs [0, si.group_begin
// + groups of si) would be the inverse segment; here the inverse segment
// starts at CTA 0 and the forward one at sf.group_begin.
template <class CF, class CI>
__global__ void __launch_bounds__(CF::THREADS) k_ntt_pair(GroupSeg sf, GroupSeg si, int* status_f, int* status_i,
                                                           uint32_t check_f, uint32_t check_i) {
    static_assert(CF::THREADS == CI::THREADS, "forward and inverse segments share the CTA shape");
    extern __shared__ __align__(16) uint64_t smem[];
    pdl_begin();
    const uint64_t b = blockIdx.x;
    const bool inv = b < sf.group_begin;
    const GroupSeg& sg = inv ? si : sf;
    TileArgs a;
    a.in = sg.in;
    a.out = sg.out;
    a.tw = sg.tw;
    a.lc = sg.lc;
    a.status = inv ? status_i : status_f;
    a.row_begin = 0;
    a.n_tiles = sg.n_tiles;
    a.n_moduli = sg.n_moduli;
    a.check = inv ? check_i : check_f;
    a.fast32 = sg.fast32;
    a.mod_magic = sg.mod_magic;
    a.src_mode = 0;
    a.in_b = nullptr;
    a.aux_q = 0;
    a.nat = 0;
    a.has_map = 0;
    a.otf = nullptr;
    a.in_skip = 0;
    if (inv)
        tile_group<CI>(a, b, smem);
    else
        tile_group<CF>(a, b - sf.group_begin, smem);
}

template <class CF, class CI>
static int launch_pair_cfg(const GroupSeg& sf, const GroupSeg& si, uint64_t grid, int* const* status,
                           const uint32_t* check, cudaStream_t st) {
    constexpr size_t smem = CF::SMEM_BYTES > CI::SMEM_BYTES ? CF::SMEM_BYTES : CI::SMEM_BYTES;
    if (grid == 0) return NTT_OK;
    if (grid > 0x7fffffffull) return NTT_ERR_ARG;
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(k_ntt_pair<CF, CI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
        return NTT_ERR_CUDA;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(CF::THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cudaLaunchKernelEx(&cfg, k_ntt_pair<CF, CI>, sf, si, status[0], status[1], check[0], check[1]) != cudaSuccess)
        return NTT_ERR_CUDA;
    return cudaPeekAtLastError() == cudaSuccess ? NTT_OK : NTT_ERR_CUDA;
}

template <class CF, class CI>
static int launch_grouped_cfg(const GroupSeg* d_segs, uint32_t n_segs, uint64_t grid, int* status, uint32_t check,
                              cudaStream_t st) {
    constexpr size_t smem = CF::SMEM_BYTES > CI::SMEM_BYTES ? CF::SMEM_BYTES : CI::SMEM_BYTES;
    if (grid == 0) return NTT_OK;
    if (grid > 0x7fffffffull) return NTT_ERR_ARG;
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(k_ntt_grouped<CF, CI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
        return NTT_ERR_CUDA;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(CF::THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (cudaLaunchKernelEx(&cfg, k_ntt_grouped<CF, CI>, d_segs, n_segs, status, check) != cudaSuccess)
        return NTT_ERR_CUDA;
    return cudaPeekAtLastError() == cudaSuccess ? NTT_OK : NTT_ERR_CUDA;
}

int grouped_phases(uint32_t log2n) {
#define NTT_GP_S(LOGN, LOGT, LOGRP, TPC, MODE) \
    case LOGN: return 1;
#define NTT_GP_2(LOGN, SPLIT, LOGP, LOGTA, LOGRPA, TPCA, LOGTB, LOGRPB, TPCB, MODE) \
    case LOGN: return 2;
    switch (log2n) {
        NTT_GROUP_CONFIGS(NTT_GP_S, NTT_GP_2)
        default: return 0;
    }
#undef NTT_GP_S
#undef NTT_GP_2
}

// tiles per row and rows per CTA of phase `phase` (0 first) for direction `inverse`
int grouped_geometry(uint32_t log2n, int phase, bool inverse, uint32_t* log_tiles_per_row, uint32_t* tpc) {
#define NTT_GG_S(LOGN, LOGT, LOGRP, TPC, MODE)        \
    case LOGN:                                        \
        *log_tiles_per_row = 0;                       \
        *tpc = TPC;                                   \
        return NTT_OK;
#define NTT_GG_2(LOGN, SPLIT, LOGP, LOGTA, LOGRPA, TPCA, LOGTB, LOGRPB, TPCB, MODE)                 \
    case LOGN: {                                                                                   \
        const bool col = (phase == 0) != inverse;      /* forward: column first; inverse: row first */ \
        *log_tiles_per_row = col ? (LOGN - SPLIT - LOGP) : SPLIT;                                  \
        *tpc = col ? TPCA : TPCB;                                                                  \
        return NTT_OK;                                                                             \
    }
    switch (log2n) {
        NTT_GROUP_CONFIGS(NTT_GG_S, NTT_GG_2)
        default: return NTT_ERR_UNSUPPORTED;
    }
#undef NTT_GG_S
#undef NTT_GG_2
}

// one-kernel configurations; MCF / MCI are the forward / inverse modulus classes
template <int LOGN, int LOGT, int LOGRP, int TPC, int MODE, int MCF, int MCI>
static int launch_grouped_single(int phase, const GroupSeg* d_segs, uint32_t n_segs, uint64_t grid, int* status,
                                 uint32_t check, cudaStream_t st) {
    using F = TileCfg<LOGN, 0, LOGN, 0, LOGT, LOGRP, TPC, false, MCF, MODE>;
    using I = TileCfg<LOGN, 0, LOGN, 0, LOGT, LOGRP, TPC, true, MCI, MODE>;
    if (phase != 0) return NTT_ERR_ARG;
    return launch_grouped_cfg<F, I>(d_segs, n_segs, grid, status, check, st);
}

// two-kernel configurations: phase 0 = forward column kernel || inverse row
// kernel, phase 1 = forward row kernel || inverse column kernel
template <int LOGN, int SPLIT, int LOGP, int LOGTA, int LOGRPA, int TPCA, int LOGTB, int LOGRPB, int TPCB, int MODE,
          int MCF, int MCI>
static int launch_grouped_split(int phase, const GroupSeg* d_segs, uint32_t n_segs, uint64_t grid, int* status,
                                uint32_t check, cudaStream_t st) {
    using F0 = TileCfg<LOGN, 0, SPLIT, LOGP, LOGTA, LOGRPA, TPCA, false, MCF, form_col(MODE)>;
    using I0 = TileCfg<LOGN, SPLIT, LOGN, 0, LOGTB, LOGRPB, TPCB, true, MCI, form_row(MODE)>;
    using F1 = TileCfg<LOGN, SPLIT, LOGN, 0, LOGTB, LOGRPB, TPCB, false, MCF, form_row(MODE)>;
    using I1 = TileCfg<LOGN, 0, SPLIT, LOGP, LOGTA, LOGRPA, TPCA, true, MCI, form_col(MODE)>;
    if (phase == 0) return launch_grouped_cfg<F0, I0>(d_segs, n_segs, grid, status, check, st);
    if (phase == 1) return launch_grouped_cfg<F1, I1>(d_segs, n_segs, grid, status, check, st);
    return NTT_ERR_ARG;
}

template <int LOGN, int LOGT, int LOGRP, int TPC, int MODE, int MCF, int MCI>
static int launch_pair_single(int phase, const GroupSeg& sf, const GroupSeg& si, uint64_t grid, int* const* status,
                              const uint32_t* check, cudaStream_t st) {
    using F = TileCfg<LOGN, 0, LOGN, 0, LOGT, LOGRP, TPC, false, MCF, MODE>;
    using I = TileCfg<LOGN, 0, LOGN, 0, LOGT, LOGRP, TPC, true, MCI, MODE>;
    if (phase != 0) return NTT_ERR_ARG;
    return launch_pair_cfg<F, I>(sf, si, grid, status, check, st);
}

template <int LOGN, int SPLIT, int LOGP, int LOGTA, int LOGRPA, int TPCA, int LOGTB, int LOGRPB, int TPCB, int MODE,
          int MCF, int MCI>
static int launch_pair_split(int phase, const GroupSeg& sf, const GroupSeg& si, uint64_t grid, int* const* status,
                             const uint32_t* check, cudaStream_t st) {
    using F0 = TileCfg<LOGN, 0, SPLIT, LOGP, LOGTA, LOGRPA, TPCA, false, MCF, form_col(MODE)>;
    using I0 = TileCfg<LOGN, SPLIT, LOGN, 0, LOGTB, LOGRPB, TPCB, true, MCI, form_row(MODE)>;
    using F1 = TileCfg<LOGN, SPLIT, LOGN, 0, LOGTB, LOGRPB, TPCB, false, MCF, form_row(MODE)>;
    using I1 = TileCfg<LOGN, 0, SPLIT, LOGP, LOGTA, LOGRPA, TPCA, true, MCI, form_col(MODE)>;
    if (phase == 0) return launch_pair_cfg<F0, I0>(sf, si, grid, status, check, st);
    if (phase == 1) return launch_pair_cfg<F1, I1>(sf, si, grid, status, check, st);
    return NTT_ERR_ARG;
}

// Phase `phase` of a forward segment sf and an inverse segment si of one N in
// one grid (si's CTAs first, sf.group_begin = si's CTA count).
int launch_pair(uint32_t log2n, uint32_t mc, int phase, const GroupSeg& sf, const GroupSeg& si, uint64_t grid,
                int* const* status, const uint32_t* check, void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
#define NTT_LP_S(LOGN, LOGT, LOGRP, TPC, MODE)                                                                  \
    case LOGN:                                                                                                 \
        return mc == 0 ? launch_pair_single<LOGN, LOGT, LOGRP, TPC, MODE, 0, 0>(phase, sf, si, grid, status, check, st) \
             : mc == 1 ? launch_pair_single<LOGN, LOGT, LOGRP, TPC, MODE, 1, 1>(phase, sf, si, grid, status, check, st) \
                       : launch_pair_single<LOGN, LOGT, LOGRP, TPC, MODE, 1, 2>(phase, sf, si, grid, status, check, st);
#define NTT_LP_2(LOGN, SPLIT, LOGP, LOGTA, LOGRPA, TPCA, LOGTB, LOGRPB, TPCB, MODE)                               \
    case LOGN:                                                                                                 \
        return mc == 0 ? launch_pair_split<LOGN, SPLIT, LOGP, LOGTA, LOGRPA, TPCA, LOGTB, LOGRPB, TPCB, MODE, 0, 0>( \
                             phase, sf, si, grid, status, check, st)                                             \
             : mc == 1 ? launch_pair_split<LOGN, SPLIT, LOGP, LOGTA, LOGRPA, TPCA, LOGTB, LOGRPB, TPCB, MODE, 1, 1>( \
                             phase, sf, si, grid, status, check, st)                                             \
                       : launch_pair_split<LOGN, SPLIT, LOGP, LOGTA, LOGRPA, TPCA, LOGTB, LOGRPB, TPCB, MODE, 1, 2>( \
                             phase, sf, si, grid, status, check, st);
    switch (log2n) {
        NTT_GROUP_CONFIGS(NTT_LP_S, NTT_LP_2)
        default: return NTT_ERR_UNSUPPORTED;
    }
#undef NTT_LP_S
#undef NTT_LP_2
}

// Launches phase `phase` of the grouped grid of one N (mc: the N's modulus
// class; the forward of class 2 runs the class-1 kernels, as plain launches do).
int launch_grouped(uint32_t log2n, uint32_t mc, int phase, const GroupSeg* d_segs, uint32_t n_segs, uint64_t grid,
                   int* status, uint32_t check, void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
#define NTT_GL_S(LOGN, LOGT, LOGRP, TPC, MODE)                                                                \
    case LOGN:                                                                                               \
        return mc == 0 ? launch_grouped_single<LOGN, LOGT, LOGRP, TPC, MODE, 0, 0>(phase, d_segs, n_segs, grid, \
                                                                                   status, check, st)         \
             : mc == 1 ? launch_grouped_single<LOGN, LOGT, LOGRP, TPC, MODE, 1, 1>(phase, d_segs, n_segs, grid, \
                                                                                   status, check, st)         \
                       : launch_grouped_single<LOGN, LOGT, LOGRP, TPC, MODE, 1, 2>(phase, d_segs, n_segs, grid, \
                                                                                   status, check, st);
#define NTT_GL_2(LOGN, SPLIT, LOGP, LOGTA, LOGRPA, TPCA, LOGTB, LOGRPB, TPCB, MODE)                             \
    case LOGN:                                                                                                 \
        return mc == 0 ? launch_grouped_split<LOGN, SPLIT, LOGP, LOGTA, LOGRPA, TPCA, LOGTB, LOGRPB, TPCB, MODE, 0, 0>( \
                             phase, d_segs, n_segs, grid, status, check, st)                                   \
             : mc == 1 ? launch_grouped_split<LOGN, SPLIT, LOGP, LOGTA, LOGRPA, TPCA, LOGTB, LOGRPB, TPCB, MODE, 1, 1>( \
                             phase, d_segs, n_segs, grid, status, check, st)                                   \
                       : launch_grouped_split<LOGN, SPLIT, LOGP, LOGTA, LOGRPA, TPCA, LOGTB, LOGRPB, TPCB, MODE, 1, 2>( \
                             phase, d_segs, n_segs, grid, status, check, st);
    switch (log2n) {
        NTT_GROUP_CONFIGS(NTT_GL_S, NTT_GL_2)
        default: return NTT_ERR_UNSUPPORTED;
    }
#undef NTT_GL_S
#undef NTT_GL_2
}

}  // namespace nttgb
