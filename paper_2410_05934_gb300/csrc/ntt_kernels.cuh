// Kernel and launcher templates of the tile NTT (see ntt_tile.cuh for the
// tile geometry).  Included by the kernel translation units, each of which
// explicitly instantiates one slice of the schedule list.
#pragma once
#include <cuda_runtime.h>

#include "ntt_gb300.h"
#include "ntt_launch.h"
#include "ntt_tile.cuh"

namespace nttgb {

template <class C, int I>
__device__ __forceinline__ void run_passes(const TileArgs& a, const TileLoc& L, int t, uint64_t* sm) {
    if constexpr (I < C::NPASS) {
        constexpr int P = C::INV ? (C::NPASS - 1 - I) : I;
        phase_pass<C, P>(a, L, t, sm);
        __syncthreads();
        run_passes<C, I + 1>(a, L, t, sm);
    }
}

// One CTA = TPC tiles; each tile is staged through shared memory, runs the
// kernel's fused passes, and is written back with 16-byte stores.
template <class C>
__global__ void __launch_bounds__(C::THREADS) k_ntt_tile(TileArgs a) {
    extern __shared__ __align__(16) uint64_t smem[];
    const int tid = threadIdx.x;
    const int tin = tid >> C::LOGT;
    const int t = tid & (C::T - 1);
    const uint64_t tile = (uint64_t)blockIdx.x * C::TPC + tin;
    const TileLoc L = locate<C>(a, tile);
    uint64_t* sm = smem + (size_t)tin * C::E;
    phase_load<C>(a, L, t, sm);
    __syncthreads();
    run_passes<C, 0>(a, L, t, sm);
    phase_store<C>(a, L, t, sm);
}

template <class C>
int launch_tile_kernel(const PlanDev& p, const uint64_t* in, uint64_t* out, uint64_t row_begin,
                       uint64_t n_rows, cudaStream_t st) {
    TileArgs a;
    a.in = in;
    a.out = out;
    a.tw = C::INV ? p.inv : p.fwd;
    a.lc = p.lc;
    a.status = p.status;
    a.row_begin = row_begin;
    a.n_tiles = n_rows << C::LOGTPR;
    a.n_moduli = p.n_moduli;
    a.check = p.check;
    const uint64_t ctas = (a.n_tiles + C::TPC - 1) / C::TPC;
    if (ctas == 0) return NTT_OK;
    if (ctas > 0x7fffffffull) return NTT_ERR_ARG;
    if (C::SMEM_BYTES > 48 * 1024) {
        // per-function attribute; cheap to repeat, needed once per device
        cudaError_t e = cudaFuncSetAttribute(k_ntt_tile<C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)C::SMEM_BYTES);
        if (e != cudaSuccess) return NTT_ERR_CUDA;
    }
    k_ntt_tile<C><<<(unsigned)ctas, C::THREADS, C::SMEM_BYTES, st>>>(a);
    return cudaPeekAtLastError() == cudaSuccess ? NTT_OK : NTT_ERR_CUDA;
}

template <int LOGN, int LOGT, int LOGRP, int TPC, bool INV>
int launch_s1(const PlanDev& p, const uint64_t* in, uint64_t* out, uint64_t row_begin,
              uint64_t n_rows, void* stream, uint32_t* launches) {
    using C = TileCfg<LOGN, 0, LOGN, 0, LOGT, LOGRP, TPC, INV>;
    int rc = launch_tile_kernel<C>(p, in, out, row_begin, n_rows, (cudaStream_t)stream);
    if (rc == NTT_OK && launches) *launches += 1;
    return rc;
}

template <int LOGN, int SPLIT, int LOGP, int LOGTA, int LOGRPA, int TPCA, int LOGTB, int LOGRPB,
          int TPCB, bool INV>
int launch_s2(const PlanDev& p, const uint64_t* in, uint64_t* out, uint64_t row_begin,
              uint64_t n_rows, void* stream, uint32_t* launches) {
    using CA = TileCfg<LOGN, 0, SPLIT, LOGP, LOGTA, LOGRPA, TPCA, INV>;
    using CB = TileCfg<LOGN, SPLIT, LOGN, 0, LOGTB, LOGRPB, TPCB, INV>;
    cudaStream_t st = (cudaStream_t)stream;
    int rc;
    if (!INV) {
        rc = launch_tile_kernel<CA>(p, in, out, row_begin, n_rows, st);
        if (rc == NTT_OK) rc = launch_tile_kernel<CB>(p, in, out, row_begin, n_rows, st);
    } else {
        rc = launch_tile_kernel<CB>(p, in, out, row_begin, n_rows, st);
        if (rc == NTT_OK) rc = launch_tile_kernel<CA>(p, in, out, row_begin, n_rows, st);
    }
    if (rc == NTT_OK && launches) *launches += 2;
    return rc;
}

#define NTT_INST_S1(LOGN, LOGT, LOGRP, TPC)                                                     \
    template int launch_s1<LOGN, LOGT, LOGRP, TPC, false>(const PlanDev&, const uint64_t*,      \
                                                          uint64_t*, uint64_t, uint64_t, void*, \
                                                          uint32_t*);                           \
    template int launch_s1<LOGN, LOGT, LOGRP, TPC, true>(const PlanDev&, const uint64_t*,       \
                                                         uint64_t*, uint64_t, uint64_t, void*,  \
                                                         uint32_t*);
#define NTT_INST_S2(LOGN, SPLIT, LOGP, LOGTA, LOGRPA, TPCA, LOGTB, LOGRPB, TPCB)                \
    template int launch_s2<LOGN, SPLIT, LOGP, LOGTA, LOGRPA, TPCA, LOGTB, LOGRPB, TPCB, false>( \
        const PlanDev&, const uint64_t*, uint64_t*, uint64_t, uint64_t, void*, uint32_t*);      \
    template int launch_s2<LOGN, SPLIT, LOGP, LOGTA, LOGRPA, TPCA, LOGTB, LOGRPB, TPCB, true>(  \
        const PlanDev&, const uint64_t*, uint64_t*, uint64_t, uint64_t, void*, uint32_t*);

}  // namespace nttgb
