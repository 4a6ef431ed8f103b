// Kernel and launcher templates of the tile NTT (see ntt_tile.cuh for the
// tile geometry and the two kernel forms).  Included by the kernel
// translation units, each of which explicitly instantiates one slice of the
// schedule list.
#pragma once
#include <cuda_runtime.h>

#include "ntt_gb300.h"
#include "ntt_launch.h"
#include "ntt_tile.cuh"

namespace nttgb {

// ---- PTX helpers: mbarrier and bulk asynchronous copies (sm_90+) ----
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Bounded wait: each try_wait suspends for a hardware-chosen interval, so
// the iteration limit bounds the total time; false means it ran out.
#define NTT_MBAR_SPIN_LIMIT (1u << 22)
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  uint32_t limit = NTT_MBAR_SPIN_LIMIT) {
    for (uint32_t i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// global -> shared bulk copy completing on `bar` (addresses 16-byte aligned,
// size a multiple of 16)
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

template <int ID, int COUNT>
__device__ __forceinline__ void named_barrier() {
    asm volatile("bar.sync %0, %1;" ::"n"(ID), "n"(COUNT) : "memory");
}

// barrier 1 + tin for tile slots 0 .. TILES - 1 (literal ids, so a CTA
// reserves only the barriers it uses)
template <int COUNT, int TILES, int K = 0>
__device__ __forceinline__ void tile_barrier(int tin) {
    if constexpr (K + 1 < TILES) {
        if (tin == K) {
            named_barrier<1 + K, COUNT>();
            return;
        }
        tile_barrier<COUNT, TILES, K + 1>(tin);
    } else {
        named_barrier<1 + K, COUNT>();
    }
}

// Orders one tile's shared-memory words between passes.  The passes of a
// tile read and write only that tile's words (staged twiddles are written
// before the CTA-wide barrier that precedes the first pass and are read-only
// afterwards), so only the tile's own threads synchronise: a tile of at most
// one warp with __syncwarp, a wider tile on a named barrier of its own
// (ids 1..TILES; id 0 is __syncthreads).  TILES is the number of tiles side
// by side in the CTA: C::TPC, or 2 in the CMux kernel, whose two slots each
// run a one-tile config.
template <class C, int TILES = C::TPC>
__device__ __forceinline__ void tile_sync() {
    if constexpr (TILES == 1 || TILES > 8) {
        __syncthreads();
    } else if constexpr (C::T <= 32) {
        __syncwarp();
    } else {
        tile_barrier<C::T, TILES>((int)threadIdx.x >> C::LOGT);
    }
}

template <class C, int I, int TILES = C::TPC>
__device__ __forceinline__ void run_passes(TileRegs<C>& st, const TileArgs& a, const TileLoc& L, int t,
                                           uint64_t* sm) {
    if constexpr (I < C::NPASS) {
        constexpr int P = C::INV ? (C::NPASS - 1 - I) : I;
        pass_read<C, P>(st, L, t, sm);
        pass_compute<C, P>(st, a, L, t, sm);
        pass_write<C, P>(st, L, t, sm);
        tile_sync<C, TILES>();
        run_passes<C, I + 1, TILES>(st, a, L, t, sm);
    }
}

// Programmatic dependent launch: the direct-form kernels are launched with
// programmatic stream serialization, so the next kernel on the stream may be
// scheduled once every CTA of this one has started (its CTAs then fill the
// SMs this grid's last wave leaves idle); griddepcontrol.wait holds a kernel
// until the previous grid has completed and its writes are visible, before
// it touches global data.  Without the launch attribute both are no-ops.
__device__ __forceinline__ void pdl_begin() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// ---- direct form: one CTA = TPC tiles, loaded with 16-byte loads ----
// tile group g of config C (the CTA's whole work in the direct form)
template <class C>
__device__ __forceinline__ void tile_group(const TileArgs& a, uint64_t g, uint64_t* smem) {
    const int tid = threadIdx.x;
    const int tin = tid >> C::LOGT;
    const int t = tid & (C::T - 1);
    const TileLoc L = locate_in_group<C>(a, g, tin);
    uint64_t* sm = smem + (size_t)tin * C::TILE_WORDS;
    TileRegs<C> st;
    load_direct<C>(st, a, L, t, sm);
    write_input_tile<C>(st, a, L, t, sm);
    async_wait_all();
    __syncthreads();
    run_passes<C, 0>(st, a, L, t, sm);
    store_tile<C>(a, L, t, sm);
}

#ifndef NTT_TILE_MIN_CTAS
#define NTT_TILE_MIN_CTAS 1
#endif
#ifndef NTT_ROW_MIN_CTAS
#define NTT_ROW_MIN_CTAS 8     // measured: the N = 2^16 row kernels fit 64 registers, 8 CTAs per SM, 2.6 % faster forward
#endif
// resident 128-thread-equivalent CTAs per SM the register budget must allow
template <class C>
constexpr int tile_min_ctas() {
    // row kernels of two-kernel schedules with at most 8 coefficients per thread
    constexpr int m = (C::S0 > 0 && C::S1 == C::LOGN && C::LOGP == 0 && C::R <= 8 && C::MODE != 3)
                          ? NTT_ROW_MIN_CTAS
                          : NTT_TILE_MIN_CTAS;
    return m * 128 / C::THREADS > 0 ? m * 128 / C::THREADS : 1;
}
template <class C>
__global__ void __launch_bounds__(C::THREADS) k_ntt_tile(TileArgs a) {
    extern __shared__ __align__(16) uint64_t smem[];
    pdl_begin();
    tile_group<C>(a, blockIdx.x, smem);
}

// The same kernel with a register bound for tile_min_ctas resident CTAs.
// Kept apart: an explicit minimum of one CTA changes the code ptxas emits
// for the other configurations (N <= 2^12 measured up to 34 % slower with
// the same register count), so only the bounded kernels carry one.
template <class C>
__global__ void __launch_bounds__(C::THREADS, tile_min_ctas<C>()) k_ntt_tile_bounded(TileArgs a) {
    extern __shared__ __align__(16) uint64_t smem[];
    pdl_begin();
    tile_group<C>(a, blockIdx.x, smem);
}

// the direct-form kernel of config C (only the one it uses is instantiated)
template <class C>
constexpr auto tile_kernel() {
    if constexpr (tile_min_ctas<C>() > 1)
        return k_ntt_tile_bounded<C>;
    else
        return k_ntt_tile<C>;
}

// Issues the bulk copies of tile group g into buffer `buf` (all threads take
// part; thread 0 arms the barrier with the byte count).
template <class C>
__device__ __forceinline__ void issue_group(const TileArgs& a, uint64_t g, int buf, uint64_t* bars,
                                           uint64_t* smem, uint64_t g_prev, bool have_prev) {
    const int tid = threadIdx.x;
    fence_proxy_async_smem();
    if (tid == 0) {
        uint32_t bytes = 0;
        for (int tin = 0; tin < C::TPC; ++tin) {
            const TileLoc L = locate<C>(a, g * C::TPC + tin);
            if (!L.valid) continue;
            bytes += (uint32_t)C::DATA_BYTES;
            if (twiddles_needed<C>(a, g, g_prev, have_prev, tin))
                bytes += (uint32_t)(C::TILE_TX_BYTES - C::DATA_BYTES);
        }
        mbar_arrive_expect_tx(&bars[buf], bytes);
    }
    for (int c = tid; c < C::TPC * C::COPIES; c += C::THREADS) {
        const int tin = c / C::COPIES, cc = c % C::COPIES;
        const TileLoc L = locate<C>(a, g * C::TPC + tin);
        if (!L.valid) continue;
        if (cc >= C::RUNS && !twiddles_needed<C>(a, g, g_prev, have_prev, tin)) continue;
        const CopyDesc d = tile_copy<C>(a, L, cc);
        uint64_t* dst = smem + (size_t)buf * C::BUF_WORDS + (size_t)tin * C::TILE_WORDS + d.dst_word;
        bulk_load(dst, d.src, d.bytes, &bars[buf]);
    }
}

// ---- pipelined form: persistent CTAs, two buffers, bulk copies ----
template <class C>
__global__ void __launch_bounds__(C::THREADS) k_ntt_tile_pipe(TileArgs a, uint64_t groups) {
    extern __shared__ __align__(16) uint64_t smem[];
    uint64_t* bars = smem + C::BAR_OFFSET / sizeof(uint64_t);
    const int tid = threadIdx.x;
    const int tin = tid >> C::LOGT;
    const int t = tid & (C::T - 1);
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        mbar_fence_init();
    }
    __syncthreads();
    const uint64_t step = gridDim.x;
    uint64_t g = blockIdx.x;
    if (g < groups) issue_group<C>(a, g, 0, bars, smem, 0, false);
    uint32_t parity = 0;   // bit b: phase parity expected next on buffer b
    for (uint32_t it = 0; g < groups; ++it, g += step) {
        const int b = it & 1;
        const uint64_t gn = g + step;
        if (gn < groups) issue_group<C>(a, gn, b ^ 1, bars, smem, g - step, it >= 1);
        const bool ok = mbar_wait_bounded(&bars[b], (parity >> b) & 1u);
        parity ^= 1u << b;
        if (__syncthreads_or(!ok)) {
            // A copy of buffer b did not complete within the bound.  Report it,
            // then wait once more (bounded) on BOTH buffers before leaving: on
            // b, whose late copy may still be writing, and on b ^ 1, whose
            // copies for the next group were issued above.  A CTA must not
            // exit while a bulk copy may still write its shared memory (the
            // next CTA on the SM could own those bytes by then); a copy that
            // is still pending after a second full bound is taken as lost,
            // i.e. one that never writes.
            if (tid == 0) record_status(a.status, NTT_STATUS_TIMEOUT);
            (void)mbar_wait_bounded(&bars[b], ((parity >> b) & 1u) ^ 1u);   // the phase waited on above
            if (gn < groups) (void)mbar_wait_bounded(&bars[b ^ 1], (parity >> (b ^ 1)) & 1u);
            return;
        }
        const TileLoc L = locate_in_group<C>(a, g, tin);
        uint64_t* sm = smem + (size_t)b * C::BUF_WORDS + (size_t)tin * C::TILE_WORDS;
        TileRegs<C> st;
        relayout_read<C>(st, a, L, t, sm);
        __syncthreads();
        write_input_tile<C>(st, a, L, t, sm);
        __syncthreads();
        run_passes<C, 0>(st, a, L, t, sm);
        store_tile<C>(a, L, t, sm);
        __syncthreads();   // buffer b is refilled by the next iteration's issue
    }
}

template <class C>
int resident_ctas_per_sm() {
    static int cached[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (!cached[dev]) {
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_ntt_tile_pipe<C>, C::THREADS, C::SMEM_BYTES) !=
                cudaSuccess ||
            n < 1)
            n = 1;
        int sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cached[dev] = n * (sms > 0 ? sms : 1);
    }
    return cached[dev];
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
    a.fast32 = (row_begin + n_rows < (1ull << 32) && a.n_tiles < (1ull << 32)) ? 1u : 0u;
    a.mod_magic = fdiv_magic(a.n_moduli);
    a.src_mode = p.src_mode;
    a.in_b = p.in_b;
    a.aux_q = p.aux_q;
    a.nat = p.nat;
    a.has_map = p.has_map;
    for (int i = 0; i < NTT_MUL_MAX_MAPPED; ++i) {
        a.a_map[i] = p.a_map[i];
        a.b_map[i] = p.b_map[i];
    }
    a.otf = C::INV ? p.otf_inv : p.otf_fwd;
    a.in_skip = p.in_skip;
    if (C::MODE == 3 && !a.otf) return NTT_ERR_ARG;
    if (C::PIPE && C::FIRST && p.src_mode) return NTT_ERR_UNSUPPORTED;  // direct form only
    const uint64_t groups = (a.n_tiles + C::TPC - 1) / C::TPC;
    if (groups == 0) return NTT_OK;
    if (groups > 0x7fffffffull) return NTT_ERR_ARG;
    // only the kernel of the config's form is instantiated
    if constexpr (C::PIPE) {
        if (C::SMEM_BYTES > 48 * 1024 &&
            cudaFuncSetAttribute(k_ntt_tile_pipe<C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)C::SMEM_BYTES) != cudaSuccess)
            return NTT_ERR_CUDA;
        uint64_t grid = (uint64_t)resident_ctas_per_sm<C>();
        if (grid > groups) grid = groups;
        k_ntt_tile_pipe<C><<<(unsigned)grid, C::THREADS, C::SMEM_BYTES, st>>>(a, groups);
    } else {
        constexpr auto kernel = tile_kernel<C>();
        if (C::SMEM_BYTES > 48 * 1024 &&
            cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM_BYTES) !=
                cudaSuccess)
            return NTT_ERR_CUDA;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)groups);
        cfg.blockDim = dim3(C::THREADS);
        cfg.dynamicSmemBytes = C::SMEM_BYTES;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        if (cudaLaunchKernelEx(&cfg, kernel, a) != cudaSuccess) return NTT_ERR_CUDA;
    }
    return cudaPeekAtLastError() == cudaSuccess ? NTT_OK : NTT_ERR_CUDA;
}

template <int LOGN, int LOGT, int LOGRP, int TPC, int PIPE, bool INV>
int launch_s1(const PlanDev& p, const uint64_t* in, uint64_t* out, uint64_t row_begin,
              uint64_t n_rows, void* stream, uint32_t* launches) {
    int rc;
    // class 2 differs from class 1 only in the inverse: the forward runs the class-1 kernels
    if (INV && p.mc == 2)
        rc = launch_tile_kernel<TileCfg<LOGN, 0, LOGN, 0, LOGT, LOGRP, TPC, INV, INV ? 2 : 1, PIPE>>(
            p, in, out, row_begin, n_rows, (cudaStream_t)stream);
    else if (p.mc >= 1)
        rc = launch_tile_kernel<TileCfg<LOGN, 0, LOGN, 0, LOGT, LOGRP, TPC, INV, 1, PIPE>>(
            p, in, out, row_begin, n_rows, (cudaStream_t)stream);
    else
        rc = launch_tile_kernel<TileCfg<LOGN, 0, LOGN, 0, LOGT, LOGRP, TPC, INV, 0, PIPE>>(
            p, in, out, row_begin, n_rows, (cudaStream_t)stream);
    if (rc == NTT_OK && launches) *launches += 1;
    return rc;
}

template <int LOGN, int SPLIT, int LOGP, int LOGTA, int LOGRPA, int TPCA, int LOGTB, int LOGRPB,
          int TPCB, int PIPE, bool INV, int MC>
int launch_s2_mc(const PlanDev& p, const uint64_t* in, uint64_t* out, uint64_t row_begin,
                 uint64_t n_rows, cudaStream_t st) {
    using CA = TileCfg<LOGN, 0, SPLIT, LOGP, LOGTA, LOGRPA, TPCA, INV, MC, form_col(PIPE)>;
    using CB = TileCfg<LOGN, SPLIT, LOGN, 0, LOGTB, LOGRPB, TPCB, INV, MC, form_row(PIPE)>;
    int rc;
    if (!INV) {
        rc = launch_tile_kernel<CA>(p, in, out, row_begin, n_rows, st);
        if (rc == NTT_OK) rc = launch_tile_kernel<CB>(p, in, out, row_begin, n_rows, st);
    } else {
        rc = launch_tile_kernel<CB>(p, in, out, row_begin, n_rows, st);
        if (rc == NTT_OK) rc = launch_tile_kernel<CA>(p, in, out, row_begin, n_rows, st);
    }
    return rc;
}

template <int LOGN, int SPLIT, int LOGP, int LOGTA, int LOGRPA, int TPCA, int LOGTB, int LOGRPB,
          int TPCB, int PIPE, bool INV>
int launch_s2(const PlanDev& p, const uint64_t* in, uint64_t* out, uint64_t row_begin,
              uint64_t n_rows, void* stream, uint32_t* launches) {
    cudaStream_t st = (cudaStream_t)stream;
    // class 2 differs from class 1 only in the inverse: the forward runs the class-1 kernels
    int rc = (INV && p.mc == 2)
        ? launch_s2_mc<LOGN, SPLIT, LOGP, LOGTA, LOGRPA, TPCA, LOGTB, LOGRPB, TPCB, PIPE, INV, INV ? 2 : 1>(p, in, out, row_begin, n_rows, st)
        : p.mc >= 1
        ? launch_s2_mc<LOGN, SPLIT, LOGP, LOGTA, LOGRPA, TPCA, LOGTB, LOGRPB, TPCB, PIPE, INV, 1>(p, in, out, row_begin, n_rows, st)
        : launch_s2_mc<LOGN, SPLIT, LOGP, LOGTA, LOGRPA, TPCA, LOGTB, LOGRPB, TPCB, PIPE, INV, 0>(p, in, out, row_begin, n_rows, st);
    if (rc == NTT_OK && launches) *launches += 2;
    return rc;
}

#define NTT_INST_S1(LOGN, LOGT, LOGRP, TPC, PIPE)                                                  \
    template int launch_s1<LOGN, LOGT, LOGRP, TPC, PIPE, false>(const PlanDev&, const uint64_t*,  \
                                                                uint64_t*, uint64_t, uint64_t,    \
                                                                void*, uint32_t*);                \
    template int launch_s1<LOGN, LOGT, LOGRP, TPC, PIPE, true>(const PlanDev&, const uint64_t*,   \
                                                               uint64_t*, uint64_t, uint64_t,     \
                                                               void*, uint32_t*);
#define NTT_INST_S2(LOGN, SPLIT, LOGP, LOGTA, LOGRPA, TPCA, LOGTB, LOGRPB, TPCB, PIPE)              \
    template int launch_s2<LOGN, SPLIT, LOGP, LOGTA, LOGRPA, TPCA, LOGTB, LOGRPB, TPCB, PIPE,      \
                           false>(const PlanDev&, const uint64_t*, uint64_t*, uint64_t, uint64_t, \
                                  void*, uint32_t*);                                              \
    template int launch_s2<LOGN, SPLIT, LOGP, LOGTA, LOGRPA, TPCA, LOGTB, LOGRPB, TPCB, PIPE,      \
                           true>(const PlanDev&, const uint64_t*, uint64_t*, uint64_t, uint64_t,  \
                                 void*, uint32_t*);

}  // namespace nttgb
