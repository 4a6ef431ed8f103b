// Uneven mixed batches in one persistent launch (C ABI: ntt_batch_*).
//
// The paper batches the independent CMux operations of all slots into one
// launch instead of one launch per ciphertext (Sec. IV-A); here the same
// idea is applied to whole transform requests: requests of different N,
// limb counts, polynomial counts and directions become (request, row range)
// work items, sorted largest first, and one persistent kernel with a fixed
// 256-thread CTA pulls them from an atomic queue.  Every N in [2^10, 2^16]
// has a 256-thread tile configuration: one tile kernel's phases for
// N <= 2^13, and for N >= 2^14 the column phase then the row phase of a
// row inside the same CTA (the intermediate goes through the output buffer;
// __syncthreads orders the CTA's global writes before its reads).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "ntt_gb300.h"
#include "ntt_internal.h"
#include "ntt_batch_cfgs.h"
#include "ntt_kernels.cuh"
#include "ntt_launch.h"

namespace nttgb {

struct BatchReq {
    const uint64_t* in;
    uint64_t* out;
    const TwPair* tw_fwd;     // pool tables of this N, offset to the request's first modulus
    const TwPair* tw_inv;
    const LimbConst* lc;
    uint32_t log2n, n_moduli, inverse, pad;
};

struct BatchItem {
    uint32_t req;
    uint32_t n_rows;
    uint64_t row_begin;
};

#define NTT_BATCH_THREADS 256

// One phase (stage range) of a config over rows [a.row_begin, +n_rows).
template <class C>
__device__ __forceinline__ void batch_phase(TileArgs a, uint64_t n_rows, uint64_t* smem) {
    static_assert(C::THREADS == NTT_BATCH_THREADS, "batch configs use 256-thread CTAs");
    a.n_tiles = n_rows << C::LOGTPR;
    const int tin = threadIdx.x >> C::LOGT, t = threadIdx.x & (C::T - 1);
    uint64_t* sm = smem + (size_t)tin * C::TILE_WORDS;
    for (uint64_t g = 0; g * C::TPC < a.n_tiles; ++g) {
        const TileLoc L = locate<C>(a, g * C::TPC + tin);
        TileRegs<C> st;
        load_direct<C>(st, a, L, t, sm);
        write_pairs_swizzled<C>(st, L, t, sm);
        __syncthreads();
        run_passes<C, 0>(st, a, L, t, sm);
        store_tile<C>(a, L, t, sm);
        __syncthreads();
    }
}

template <int LOGN, int LOGT, int LOGRP, int TPC, bool INV, int MC>
__device__ __forceinline__ void batch_single(const TileArgs& a, const BatchReq& rq, uint64_t n_rows,
                                             uint64_t* smem) {
    TileArgs b = a;
    b.tw = INV ? rq.tw_inv : rq.tw_fwd;
    batch_phase<TileCfg<LOGN, 0, LOGN, 0, LOGT, LOGRP, TPC, INV, MC>>(b, n_rows, smem);
}

template <int LOGN, int SPLIT, int LOGP, int LOGTA, int LOGRPA, int TPCA, int LOGTB, int LOGRPB, int TPCB,
          bool INV, int MC>
__device__ __forceinline__ void batch_split(const TileArgs& a, const BatchReq& rq, uint64_t n_rows,
                                            uint64_t* smem) {
    using CA = TileCfg<LOGN, 0, SPLIT, LOGP, LOGTA, LOGRPA, TPCA, INV, MC>;
    using CB = TileCfg<LOGN, SPLIT, LOGN, 0, LOGTB, LOGRPB, TPCB, INV, MC>;
    TileArgs b = a;
    b.tw = INV ? rq.tw_inv : rq.tw_fwd;
    // one row at a time so the row phase reads what this CTA's column phase wrote
    for (uint64_t r = 0; r < n_rows; ++r) {
        b.row_begin = a.row_begin + r;
        if (!INV) {
            batch_phase<CA>(b, 1, smem);
            batch_phase<CB>(b, 1, smem);
        } else {
            batch_phase<CB>(b, 1, smem);
            batch_phase<CA>(b, 1, smem);
        }
    }
}

#define NTT_BATCH_CASE_SINGLE(LOGN, LOGT, LOGRP, TPC) \
    case LOGN: batch_single<LOGN, LOGT, LOGRP, TPC, INV, MC>(a, rq, n_rows, smem); break;
#define NTT_BATCH_CASE_SPLIT(LOGN, SPLIT, LOGP, LOGTA, LOGRPA, TPCA, LOGTB, LOGRPB, TPCB)                 \
    case LOGN:                                                                                         \
        batch_split<LOGN, SPLIT, LOGP, LOGTA, LOGRPA, TPCA, LOGTB, LOGRPB, TPCB, INV, MC>(a, rq, n_rows, \
                                                                                         smem);         \
        break;

template <bool INV, int MC>
__device__ __forceinline__ void batch_dispatch(const TileArgs& a, const BatchReq& rq, uint64_t n_rows,
                                               uint64_t* smem) {
    switch (rq.log2n) {
        NTT_BATCH_CONFIGS(NTT_BATCH_CASE_SINGLE, NTT_BATCH_CASE_SPLIT)
        default: break;
    }
}

// Largest shared-memory footprint among the batch configurations (N = 2^12
// single tile and N = 2^16 row phase: 96 KiB).
static constexpr size_t kBatchSmem = 96 * 1024;

template <int MC>
__global__ void __launch_bounds__(NTT_BATCH_THREADS, 2)
    k_ntt_batch(const BatchReq* __restrict__ reqs, const BatchItem* __restrict__ items, uint32_t n_items,
                uint32_t* counter, int* status, uint32_t check) {
    extern __shared__ __align__(16) uint64_t smem[];
    __shared__ uint32_t s_item;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(counter, 1u);
        __syncthreads();
        const uint32_t item = s_item;
        __syncthreads();
        if (item >= n_items) break;
        const BatchItem it = items[item];
        const BatchReq rq = reqs[it.req];
        TileArgs a;
        a.in = rq.in;
        a.out = rq.out;
        a.tw = nullptr;
        a.lc = rq.lc;
        a.status = status;
        a.row_begin = it.row_begin;
        a.n_tiles = 0;
        a.n_moduli = rq.n_moduli;
        a.check = check;
        if (rq.inverse)
            batch_dispatch<true, MC>(a, rq, it.n_rows, smem);
        else
            batch_dispatch<false, MC>(a, rq, it.n_rows, smem);
    }
}

// rows per work item: about one 2^13-coefficient chunk, whole rows above
static uint32_t rows_per_item(uint32_t log2n) { return log2n >= 13 ? 1u : (1u << (13 - log2n)); }

struct NTableSet {
    PlanHost host;              // pool prefix tables of one N
    TwPair* d_fwd = nullptr;
    TwPair* d_inv = nullptr;
    LimbConst* d_lc = nullptr;
};

}  // namespace nttgb

struct ntt_batch_s {
    std::vector<ntt_request_t> reqs;
    std::vector<nttgb::BatchReq> hreqs;
    std::vector<nttgb::BatchItem> hitems;
    nttgb::NTableSet tables[NTT_MAX_LOG2N + 1];
    nttgb::BatchReq* d_reqs = nullptr;
    nttgb::BatchItem* d_items = nullptr;
    uint32_t* d_counter = nullptr;
    int* d_status = nullptr;
    uint32_t flags = 0, mc = 0, check = 0;
    int device = -1;
    int grid = 0;
    uint64_t coefficients = 0;
    uint32_t last_launches = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    cudaStream_t graph_stream = nullptr;
};

namespace nttgb {

static void batch_free(ntt_batch_s* b) {
    if (b->graph_exec) cudaGraphExecDestroy(b->graph_exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (auto& t : b->tables) {
        if (t.d_fwd) cudaFree(t.d_fwd);
        if (t.d_inv) cudaFree(t.d_inv);
        if (t.d_lc) cudaFree(t.d_lc);
    }
    if (b->d_reqs) cudaFree(b->d_reqs);
    if (b->d_items) cudaFree(b->d_items);
    if (b->d_counter) cudaFree(b->d_counter);
    if (b->d_status) cudaFree(b->d_status);
    delete b;
}

static bool aligned16p(const void* p) { return ((uintptr_t)p & 15u) == 0; }

static int validate_reqs(const ntt_request_t* reqs, uint32_t n, uint32_t pool_len) {
    if (!reqs || n == 0) return NTT_ERR_ARG;
    for (uint32_t i = 0; i < n; ++i) {
        const ntt_request_t& r = reqs[i];
        if (r.log2n > NTT_MAX_LOG2N || r.n_moduli == 0 || r.n_polys == 0 || r.inverse > 1)
            return NTT_ERR_ARG;
        if (r.log2n < NTT_BATCH_MIN_LOG2N) return NTT_ERR_UNSUPPORTED;
        if ((uint64_t)r.moduli_offset + r.n_moduli > pool_len) return NTT_ERR_ARG;
        if (!r.in || !r.out) return NTT_ERR_ARG;
        if (!aligned16p(r.in) || !aligned16p(r.out)) return NTT_ERR_ALIGN;
        if (((unsigned __int128)r.n_polys * r.n_moduli << r.log2n) >= ((unsigned __int128)1 << 40))
            return NTT_ERR_ARG;
    }
    return NTT_OK;
}

}  // namespace nttgb

using namespace nttgb;

extern "C" {

int ntt_batch_plan(ntt_batch_t* out, const ntt_request_t* reqs, uint32_t n_reqs,
                   const uint64_t* moduli_pool, uint32_t pool_len, uint32_t flags) {
    if (!out) return NTT_ERR_ARG;
    *out = nullptr;
    if (!moduli_pool || pool_len == 0) return NTT_ERR_ARG;
    if (flags & ~(NTT_BATCH_GRAPH | NTT_FLAG_CHECK)) return NTT_ERR_ARG;
    int rc = validate_reqs(reqs, n_reqs, pool_len);
    if (rc) return rc;
    ntt_batch_s* b = new (std::nothrow) ntt_batch_s();
    if (!b) return NTT_ERR_NOMEM;
    b->flags = flags;
    b->check = (flags & NTT_FLAG_CHECK) ? 1u : 0u;
    try {
        b->reqs.assign(reqs, reqs + n_reqs);
        // pool prefix needed per N
        uint32_t need[NTT_MAX_LOG2N + 1] = {0};
        for (const auto& r : b->reqs) need[r.log2n] = std::max(need[r.log2n], r.moduli_offset + r.n_moduli);
        b->mc = 1;
        for (uint32_t ln = 0; ln <= NTT_MAX_LOG2N; ++ln) {
            if (!need[ln]) continue;
            rc = build_plan_host(b->tables[ln].host, ln, moduli_pool, need[ln], 1, NTT_FLAG_HOST_ONLY);
            if (rc) {
                batch_free(b);
                return rc;
            }
            if (!b->tables[ln].host.mc) b->mc = 0;
        }
        // work items, largest transforms first (longest-processing-time order)
        for (uint32_t i = 0; i < n_reqs; ++i) {
            const auto& r = b->reqs[i];
            const uint64_t rows = (uint64_t)r.n_polys * r.n_moduli;
            const uint32_t per = rows_per_item(r.log2n);
            for (uint64_t r0 = 0; r0 < rows; r0 += per)
                b->hitems.push_back({i, (uint32_t)std::min<uint64_t>(per, rows - r0), r0});
            b->coefficients += rows << r.log2n;
        }
        std::stable_sort(b->hitems.begin(), b->hitems.end(), [&](const BatchItem& x, const BatchItem& y) {
            return b->reqs[x.req].log2n > b->reqs[y.req].log2n;
        });
        if (b->hitems.size() >= 0xffffffffull) {
            batch_free(b);
            return NTT_ERR_ARG;
        }
    } catch (const std::bad_alloc&) {
        batch_free(b);
        return NTT_ERR_NOMEM;
    }
    // device side
    bool ok = cudaGetDevice(&b->device) == cudaSuccess;
    for (uint32_t ln = 0; ok && ln <= NTT_MAX_LOG2N; ++ln) {
        NTableSet& t = b->tables[ln];
        if (t.host.fwd.empty()) continue;
        const size_t twb = t.host.fwd.size() * sizeof(TwPair), lcb = t.host.consts.size() * sizeof(LimbConst);
        ok = cudaMalloc(&t.d_fwd, twb) == cudaSuccess && cudaMalloc(&t.d_inv, twb) == cudaSuccess &&
             cudaMalloc(&t.d_lc, lcb) == cudaSuccess &&
             cudaMemcpy(t.d_fwd, t.host.fwd.data(), twb, cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemcpy(t.d_inv, t.host.inv.data(), twb, cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemcpy(t.d_lc, t.host.consts.data(), lcb, cudaMemcpyHostToDevice) == cudaSuccess;
        std::vector<TwPair>().swap(t.host.fwd);
        std::vector<TwPair>().swap(t.host.inv);
    }
    if (ok) {
        b->hreqs.resize(n_reqs);
        for (uint32_t i = 0; i < n_reqs; ++i) {
            const auto& r = b->reqs[i];
            const NTableSet& t = b->tables[r.log2n];
            BatchReq& d = b->hreqs[i];
            d.in = r.in;
            d.out = r.out;
            d.tw_fwd = t.d_fwd + ((size_t)r.moduli_offset << r.log2n);
            d.tw_inv = t.d_inv + ((size_t)r.moduli_offset << r.log2n);
            d.lc = t.d_lc + r.moduli_offset;
            d.log2n = r.log2n;
            d.n_moduli = r.n_moduli;
            d.inverse = r.inverse;
            d.pad = 0;
        }
        ok = cudaMalloc(&b->d_reqs, sizeof(BatchReq) * n_reqs) == cudaSuccess &&
             cudaMalloc(&b->d_items, sizeof(BatchItem) * b->hitems.size()) == cudaSuccess &&
             cudaMalloc(&b->d_counter, sizeof(uint32_t)) == cudaSuccess &&
             cudaMalloc(&b->d_status, sizeof(int)) == cudaSuccess &&
             cudaMemcpy(b->d_reqs, b->hreqs.data(), sizeof(BatchReq) * n_reqs, cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemcpy(b->d_items, b->hitems.data(), sizeof(BatchItem) * b->hitems.size(),
                        cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemset(b->d_status, 0, sizeof(int)) == cudaSuccess;
    }
    if (ok) {
        cudaError_t e = b->mc ? cudaFuncSetAttribute(k_ntt_batch<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBatchSmem)
                              : cudaFuncSetAttribute(k_ntt_batch<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBatchSmem);
        int per_sm = 0, sms = 0;
        ok = e == cudaSuccess &&
             (b->mc ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ntt_batch<1>, NTT_BATCH_THREADS, kBatchSmem)
                    : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ntt_batch<0>, NTT_BATCH_THREADS, kBatchSmem)) == cudaSuccess &&
             cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device) == cudaSuccess;
        b->grid = std::max(1, per_sm) * std::max(1, sms);
        if ((uint64_t)b->grid > b->hitems.size()) b->grid = (int)b->hitems.size();
    }
    if (!ok) {
        cudaGetLastError();
        batch_free(b);
        return NTT_ERR_CUDA;
    }
    *out = b;
    return NTT_OK;
}

int ntt_batch_update(ntt_batch_t b, const ntt_request_t* reqs, uint32_t n_reqs, void* cuda_stream) {
    if (!b || !reqs || n_reqs != b->reqs.size()) return NTT_ERR_ARG;
    for (uint32_t i = 0; i < n_reqs; ++i) {
        const ntt_request_t& r = reqs[i];
        const ntt_request_t& o = b->reqs[i];
        if (r.log2n != o.log2n || r.n_moduli != o.n_moduli || r.n_polys != o.n_polys ||
            r.moduli_offset != o.moduli_offset || r.inverse != o.inverse || !r.in || !r.out)
            return NTT_ERR_ARG;
        if (!aligned16p(r.in) || !aligned16p(r.out)) return NTT_ERR_ALIGN;
    }
    for (uint32_t i = 0; i < n_reqs; ++i) {
        b->reqs[i].in = reqs[i].in;
        b->reqs[i].out = reqs[i].out;
        b->hreqs[i].in = reqs[i].in;
        b->hreqs[i].out = reqs[i].out;
    }
    // pageable source: the runtime stages it before returning, so hreqs may change afterwards
    return cudaMemcpyAsync(b->d_reqs, b->hreqs.data(), sizeof(BatchReq) * n_reqs, cudaMemcpyHostToDevice,
                           (cudaStream_t)cuda_stream) == cudaSuccess ? NTT_OK : NTT_ERR_CUDA;
}

static int batch_enqueue(ntt_batch_t b, cudaStream_t st) {
    if (cudaMemsetAsync(b->d_counter, 0, sizeof(uint32_t), st) != cudaSuccess) return NTT_ERR_CUDA;
    if (b->mc)
        k_ntt_batch<1><<<b->grid, NTT_BATCH_THREADS, kBatchSmem, st>>>(b->d_reqs, b->d_items, (uint32_t)b->hitems.size(),
                                                                      b->d_counter, b->d_status, b->check);
    else
        k_ntt_batch<0><<<b->grid, NTT_BATCH_THREADS, kBatchSmem, st>>>(b->d_reqs, b->d_items, (uint32_t)b->hitems.size(),
                                                                      b->d_counter, b->d_status, b->check);
    return cudaPeekAtLastError() == cudaSuccess ? NTT_OK : NTT_ERR_CUDA;
}

int ntt_batch_execute(ntt_batch_t b, void* cuda_stream) {
    if (!b) return NTT_ERR_ARG;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != b->device) return NTT_ERR_ARG;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    b->last_launches = 0;
    if (!(b->flags & NTT_BATCH_GRAPH)) {
        int rc = batch_enqueue(b, st);
        if (rc == NTT_OK) b->last_launches = 1;
        return rc;
    }
    if (!b->graph_exec) {
        // capture on a private stream (the legacy default stream cannot be captured)
        cudaStream_t cap;
        if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) return NTT_ERR_CUDA;
        int rc = NTT_OK;
        if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) rc = NTT_ERR_CUDA;
        if (rc == NTT_OK) rc = batch_enqueue(b, cap);
        cudaGraph_t g = nullptr;
        if (cudaStreamEndCapture(cap, &g) != cudaSuccess) rc = NTT_ERR_CUDA;
        cudaStreamDestroy(cap);
        if (rc == NTT_OK && cudaGraphInstantiate(&b->graph_exec, g, 0) != cudaSuccess) rc = NTT_ERR_CUDA;
        if (rc != NTT_OK) {
            if (g) cudaGraphDestroy(g);
            b->graph_exec = nullptr;
            cudaGetLastError();
            return rc;
        }
        b->graph = g;
    }
    if (cudaGraphLaunch(b->graph_exec, st) != cudaSuccess) return NTT_ERR_CUDA;
    b->last_launches = 1;
    return NTT_OK;
}

int ntt_batch_execute_plain(ntt_batch_t b, const uint32_t* schedules, void* cuda_stream) {
    if (!b) return NTT_ERR_ARG;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != b->device) return NTT_ERR_ARG;
    int count = 0;
    const SchedEntry* table = sched_table(&count);
    b->last_launches = 0;
    for (size_t i = 0; i < b->reqs.size(); ++i) {
        const ntt_request_t& r = b->reqs[i];
        const uint64_t rows = (uint64_t)r.n_polys * r.n_moduli;
        uint32_t sid = schedules ? schedules[i] : default_schedule(r.log2n, rows);
        int idx = -1;
        for (int k = 0, seen = 0; k < count; ++k) {
            if (table[k].log2n != r.log2n) continue;
            if ((uint32_t)seen++ == sid) {
                idx = k;
                break;
            }
        }
        if (idx < 0) return NTT_ERR_ARG;
        PlanDev d;
        d.fwd = b->hreqs[i].tw_fwd;
        d.inv = b->hreqs[i].tw_inv;
        d.lc = b->hreqs[i].lc;
        d.status = b->d_status;
        d.n_moduli = r.n_moduli;
        d.check = b->check;
        d.mc = b->tables[r.log2n].host.mc;
        const LaunchFn fn = r.inverse ? table[idx].inv : table[idx].fwd;
        int rc = fn(d, r.in, r.out, 0, rows, cuda_stream, &b->last_launches);
        if (rc) return rc;
    }
    return NTT_OK;
}

int ntt_batch_destroy(ntt_batch_t b) {
    if (!b) return NTT_ERR_ARG;
    batch_free(b);
    return NTT_OK;
}

int ntt_batch_status(ntt_batch_t b, void* cuda_stream) {
    if (!b) return NTT_ERR_ARG;
    int host = 0;
    if (cudaStreamSynchronize((cudaStream_t)cuda_stream) != cudaSuccess) return NTT_ERR_CUDA;
    if (cudaMemcpy(&host, b->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return NTT_ERR_CUDA;
    if (host && cudaMemset(b->d_status, 0, sizeof(int)) != cudaSuccess) return NTT_ERR_CUDA;
    return host;
}

int ntt_batch_info(ntt_batch_t b, uint64_t* items, uint32_t* last_launches, uint64_t* coefficients) {
    if (!b) return NTT_ERR_ARG;
    if (items) *items = b->hitems.size();
    if (last_launches) *last_launches = b->last_launches;
    if (coefficients) *coefficients = b->coefficients;
    return NTT_OK;
}

}  // extern "C"
