// Uneven mixed batches in one persistent launch (C ABI: ntt_batch_*).
//
// The paper batches the independent CMux operations of all slots into one
// launch instead of one launch per ciphertext (Sec. IV-A); here the same
// idea is applied to whole transform requests: requests of different N,
// limb counts, polynomial counts and directions become (request, row range)
// work items, sorted largest first, and one persistent kernel with a fixed
// 128-thread CTA pulls them from an atomic queue.  Every N in [2^10, 2^16]
// has a 128-thread tile configuration: one tile kernel's phases for
// N <= 2^11, and for N >= 2^12 the column phase then the row phase of a
// row inside the same CTA (the intermediate goes through the output buffer;
// __syncthreads orders the CTA's global writes before its reads).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
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

#define NTT_BATCH_THREADS 128
#define NTT_BATCH_BRANCHES 4     // concurrent graph branches for the scheduled requests
static constexpr size_t kBatchSmemBound = 18 * 1024;

// One phase (stage range) of a config over rows [a.row_begin, +n_rows).
template <class C>
__device__ __forceinline__ void batch_phase(TileArgs a, uint64_t n_rows, uint64_t* smem) {
    static_assert(C::THREADS == NTT_BATCH_THREADS, "batch configs use 128-thread CTAs");
    static_assert(C::SMEM_BYTES <= kBatchSmemBound, "batch configs fit the kernel's shared memory");
    a.n_tiles = n_rows << C::LOGTPR;
    const int tin = threadIdx.x >> C::LOGT, t = threadIdx.x & (C::T - 1);
    uint64_t* sm = smem + (size_t)tin * C::TILE_WORDS;
    for (uint64_t g = 0; g * C::TPC < a.n_tiles; ++g) {
        const TileLoc L = locate_in_group<C>(a, g, tin);
        TileRegs<C> st;
        load_direct<C>(st, a, L, t, sm);
        write_pairs_swizzled<C>(st, L, t, sm);
        async_wait_all();
        __syncthreads();
        run_passes<C, 0>(st, a, L, t, sm);
        store_tile<C>(a, L, t, sm);
        __syncthreads();
    }
}

template <int LOGN, int LOGT, int LOGRP, int TPC, int MODE, bool INV, int MC>
__device__ __forceinline__ void batch_single(const TileArgs& a, const BatchReq& rq, uint64_t n_rows,
                                             uint64_t* smem) {
    TileArgs b = a;
    b.tw = INV ? rq.tw_inv : rq.tw_fwd;
    batch_phase<TileCfg<LOGN, 0, LOGN, 0, LOGT, LOGRP, TPC, INV, MC, MODE>>(b, n_rows, smem);
}

template <int LOGN, int SPLIT, int LOGP, int LOGTA, int LOGRPA, int TPCA, int LOGTB, int LOGRPB, int TPCB,
          int MODE, bool INV, int MC>
__device__ __forceinline__ void batch_split(const TileArgs& a, const BatchReq& rq, uint64_t n_rows,
                                            uint64_t* smem) {
    using CA = TileCfg<LOGN, 0, SPLIT, LOGP, LOGTA, LOGRPA, TPCA, INV, MC, form_col(MODE)>;
    using CB = TileCfg<LOGN, SPLIT, LOGN, 0, LOGTB, LOGRPB, TPCB, INV, MC, form_row(MODE)>;
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

// Only the paths with N <= 2^NMAX are compiled into a kernel variant: a
// batch of short polynomials runs a variant whose register budget is not
// set by the long-polynomial paths.
#define NTT_BATCH_CASE_SINGLE(LOGN, LOGT, LOGRP, TPC, MODE)                             \
    case LOGN:                                                                         \
        if constexpr (LOGN <= NMAX) batch_single<LOGN, LOGT, LOGRP, TPC, MODE, INV, MC>(a, rq, n_rows, smem); \
        break;
#define NTT_BATCH_CASE_SPLIT(LOGN, SPLIT, LOGP, LOGTA, LOGRPA, TPCA, LOGTB, LOGRPB, TPCB, MODE)           \
    case LOGN:                                                                                         \
        if constexpr (LOGN <= NMAX)                                                                    \
            batch_split<LOGN, SPLIT, LOGP, LOGTA, LOGRPA, TPCA, LOGTB, LOGRPB, TPCB, MODE, INV, MC>(   \
                a, rq, n_rows, smem);                                                                  \
        break;

template <bool INV, int MC, int NMAX>
__device__ __forceinline__ void batch_dispatch(const TileArgs& a, const BatchReq& rq, uint64_t n_rows,
                                               uint64_t* smem) {
    switch (rq.log2n) {
        NTT_BATCH_CONFIGS(NTT_BATCH_CASE_SINGLE, NTT_BATCH_CASE_SPLIT)
        default: break;
    }
}

// Largest shared-memory footprint among the batch configurations (18 KiB).
static constexpr size_t kBatchSmem = kBatchSmemBound;
// kernel variants: all N (NMAX 16), or short polynomials only (NMAX 11)
#define NTT_BATCH_SHORT_NMAX 11
// CTAs per SM the register budget is set for (the standalone column kernels'
// 72 registers): the exact-quotient class (q >= 2^57) needs more registers
// per butterfly than the small-modulus class
template <int MC, int NMAX>
struct BatchOcc {
    static constexpr int ctas = MC ? 6 : 5;
};

template <int MC, int NMAX>
__global__ void __launch_bounds__(NTT_BATCH_THREADS, BatchOcc<MC, NMAX>::ctas)
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
        a.fast32 = 0;
        a.mod_magic = 0;
        a.src_mode = 0;
        a.in_b = nullptr;
        a.aux_q = 0;
        a.nat = 0;
        a.has_map = 0;
        a.in_skip = 0;
        if (rq.inverse)
            batch_dispatch<true, MC, NMAX>(a, rq, it.n_rows, smem);
        else
            batch_dispatch<false, MC, NMAX>(a, rq, it.n_rows, smem);
    }
}

static const void* batch_kernel(uint32_t mc, uint32_t short_only) {
    if (mc) return short_only ? (const void*)k_ntt_batch<1, NTT_BATCH_SHORT_NMAX> : (const void*)k_ntt_batch<1, 16>;
    return short_only ? (const void*)k_ntt_batch<0, NTT_BATCH_SHORT_NMAX> : (const void*)k_ntt_batch<0, 16>;
}

// rows per work item: one tile group of the batch configuration (two rows at
// N = 2^10, one row above), so that the queue's last wave is short
static uint32_t rows_per_item(uint32_t log2n) { return log2n <= 10 ? 2u : 1u; }

struct NTableSet {
    PlanHost host;              // pool prefix tables of one N
    TwPair* d_fwd = nullptr;
    TwPair* d_inv = nullptr;
    LimbConst* d_lc = nullptr;
};


// ---- allocation-free variant: scratch in a file-scope device array ----
//
// Layout of g_ntt_static_scratch: the work-queue counter in the first 256
// bytes, then up to NTT_STATIC_MAX_REQUESTS descriptors.  Work items are not
// stored: item k belongs to the request whose [item_begin, next item_begin)
// range holds k (binary search), rows in chunks of rows_per_item(N).
struct StaticReq {
    const uint64_t* in;
    uint64_t* out;
    const TwPair* tw_fwd;
    const TwPair* tw_inv;
    const LimbConst* lc;
    int* status;
    uint32_t log2n, n_moduli, inverse, item_begin;
    uint32_t rows, check, per_item, pad;
};
static_assert(sizeof(StaticReq) == 80, "descriptor size");
static_assert(256 + sizeof(StaticReq) * NTT_STATIC_MAX_REQUESTS <= NTT_STATIC_SCRATCH_BYTES,
              "descriptors fit the static scratch array");

static __device__ __align__(256) unsigned char g_ntt_static_scratch[NTT_STATIC_SCRATCH_BYTES];

template <int MC>
__global__ void __launch_bounds__(NTT_BATCH_THREADS, BatchOcc<MC, 16>::ctas)
    k_ntt_batch_static(const StaticReq* __restrict__ reqs, uint32_t n_reqs, uint32_t n_items,
                       uint32_t* counter) {
    extern __shared__ __align__(16) uint64_t smem[];
    __shared__ uint32_t s_item;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(counter, 1u);
        __syncthreads();
        const uint32_t item = s_item;
        __syncthreads();
        if (item >= n_items) break;
        uint32_t lo = 0, hi = n_reqs;    // last request with item_begin <= item
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (reqs[mid].item_begin <= item) lo = mid; else hi = mid;
        }
        const StaticReq sr = reqs[lo];
        const uint64_t row_begin = (uint64_t)(item - sr.item_begin) * sr.per_item;
        const uint64_t n_rows = min((uint64_t)sr.per_item, (uint64_t)sr.rows - row_begin);
        BatchReq rq;
        rq.in = sr.in;
        rq.out = sr.out;
        rq.tw_fwd = sr.tw_fwd;
        rq.tw_inv = sr.tw_inv;
        rq.lc = sr.lc;
        rq.log2n = sr.log2n;
        rq.n_moduli = sr.n_moduli;
        rq.inverse = sr.inverse;
        TileArgs a;
        a.in = sr.in;
        a.out = sr.out;
        a.tw = nullptr;
        a.lc = sr.lc;
        a.status = sr.status;
        a.row_begin = row_begin;
        a.n_tiles = 0;
        a.n_moduli = sr.n_moduli;
        a.check = sr.check;
        a.fast32 = 0;
        a.mod_magic = 0;
        a.src_mode = 0;
        a.in_b = nullptr;
        a.aux_q = 0;
        a.nat = 0;
        a.has_map = 0;
        a.in_skip = 0;
        if (sr.inverse)
            batch_dispatch<true, MC, 16>(a, rq, n_rows, smem);
        else
            batch_dispatch<false, MC, 16>(a, rq, n_rows, smem);
    }
}

struct StaticDevice {
    bool ready = false;
    unsigned char* scratch = nullptr;   // device address of g_ntt_static_scratch
    int grid[2] = {0, 0};
};
static StaticDevice g_static_dev[64];
static std::mutex g_static_mu;

// Once per device, with that device current: the array's device address
// (its name is only a host-side stand-in) and the kernel's launch shape.
static int static_setup(int dev, StaticDevice** out) {
    if (dev < 0 || dev >= 64) return NTT_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_static_mu);
    StaticDevice& d = g_static_dev[dev];
    if (!d.ready) {
        void* ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_ntt_static_scratch) != cudaSuccess || !ptr) return NTT_ERR_CUDA;
        int sms = 0, n0 = 0, n1 = 0;
        if (cudaFuncSetAttribute(k_ntt_batch_static<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBatchSmem) != cudaSuccess ||
            cudaFuncSetAttribute(k_ntt_batch_static<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBatchSmem) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n0, k_ntt_batch_static<0>, NTT_BATCH_THREADS, kBatchSmem) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n1, k_ntt_batch_static<1>, NTT_BATCH_THREADS, kBatchSmem) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return NTT_ERR_CUDA;
        d.scratch = static_cast<unsigned char*>(ptr);
        d.grid[0] = std::max(1, n0) * std::max(1, sms);
        d.grid[1] = std::max(1, n1) * std::max(1, sms);
        d.ready = true;
    }
    *out = &d;
    return NTT_OK;
}

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
    uint32_t short_only = 0;    // every request has N <= 2^NTT_BATCH_SHORT_NMAX
    std::vector<uint32_t> scheduled;   // requests that run as their own launches
    // their branches (request k on branch k mod n_branches), forked from and
    // joined to the caller's stream
    uint32_t n_branches = 0;
    cudaStream_t side[NTT_BATCH_BRANCHES] = {};
    cudaEvent_t ev_fork = nullptr;
    cudaEvent_t ev_join[NTT_BATCH_BRANCHES] = {};
    int device = -1;
    int grid = 0;
    uint64_t coefficients = 0;
    uint32_t last_launches = 0;
    uint32_t graph_kernels = 0;        // kernels one replay of the graph runs
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    cudaStream_t graph_stream = nullptr;
    // NTT_BATCH_GROUPED: one group per N of the unscheduled requests
    struct Group {
        uint32_t log2n = 0, mc = 0, phases = 0, n_segs = 0;
        std::vector<uint32_t> reqs;                 // request indices, in order
        std::vector<nttgb::GroupSeg> hsegs[2];      // per phase
        nttgb::GroupSeg* d_segs[2] = {nullptr, nullptr};
        uint64_t grid[2] = {0, 0};
    };
    std::vector<Group> groups;
};

namespace nttgb {

static void batch_drop_graph(ntt_batch_s* b) {
    if (b->graph_exec) cudaGraphExecDestroy(b->graph_exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->graph_exec = nullptr;
    b->graph = nullptr;
}

static void batch_free(ntt_batch_s* b) {
    batch_drop_graph(b);
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    for (int k = 0; k < NTT_BATCH_BRANCHES; ++k) {
        if (b->ev_join[k]) cudaEventDestroy(b->ev_join[k]);
        if (b->side[k]) cudaStreamDestroy(b->side[k]);
    }
    for (auto& t : b->tables) {
        if (t.d_fwd) cudaFree(t.d_fwd);
        if (t.d_inv) cudaFree(t.d_inv);
        if (t.d_lc) cudaFree(t.d_lc);
    }
    for (auto& g : b->groups)
        for (auto* d : g.d_segs)
            if (d) cudaFree(d);
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
        if (r.schedule > (uint32_t)schedule_count(r.log2n)) return NTT_ERR_ARG;
        if ((uint64_t)r.moduli_offset + r.n_moduli > pool_len) return NTT_ERR_ARG;
        if (!r.in || !r.out) return NTT_ERR_ARG;
        if (!aligned16p(r.in) || !aligned16p(r.out)) return NTT_ERR_ALIGN;
        if (((unsigned __int128)r.n_polys * r.n_moduli << r.log2n) >= ((unsigned __int128)1 << 40))
            return NTT_ERR_ARG;
    }
    return NTT_OK;
}

// The segments of group g's requests for every phase of its configuration:
// tile counts of that phase's config over each request's rows, consecutive
// ranges of CTAs.
static void batch_fill_segments(ntt_batch_s* b, ntt_batch_s::Group& g) {
    for (uint32_t p = 0; p < g.phases; ++p) {
        g.hsegs[p].resize(g.reqs.size());
        uint64_t begin = 0;
        for (size_t k = 0; k < g.reqs.size(); ++k) {
            const uint32_t i = g.reqs[k];
            const ntt_request_t& r = b->reqs[i];
            const BatchReq& d = b->hreqs[i];
            uint32_t ltpr = 0, tpc = 1;
            grouped_geometry(r.log2n, (int)p, r.inverse != 0, &ltpr, &tpc);
            const uint64_t rows = (uint64_t)r.n_polys * r.n_moduli;
            GroupSeg& sg = g.hsegs[p][k];
            sg.in = r.in;
            sg.out = r.out;
            sg.tw = r.inverse ? d.tw_inv : d.tw_fwd;
            sg.lc = d.lc;
            sg.n_tiles = rows << ltpr;
            sg.group_begin = begin;
            sg.mod_magic = fdiv_magic(r.n_moduli);
            sg.n_moduli = r.n_moduli;
            sg.inverse = r.inverse;
            sg.fast32 = (rows < (1ull << 32) && sg.n_tiles < (1ull << 32)) ? 1u : 0u;
            sg.pad = 0;
            begin += (sg.n_tiles + tpc - 1) / tpc;
        }
        g.grid[p] = begin;
    }
}

}  // namespace nttgb

using namespace nttgb;

extern "C" {

int ntt_batch_plan(ntt_batch_t* out, const ntt_request_t* reqs, uint32_t n_reqs,
                   const uint64_t* moduli_pool, uint32_t pool_len, uint32_t flags) {
    if (!out) return NTT_ERR_ARG;
    *out = nullptr;
    if (!moduli_pool || pool_len == 0) return NTT_ERR_ARG;
    if (flags & ~(NTT_BATCH_GRAPH | NTT_FLAG_CHECK | NTT_BATCH_GROUPED)) return NTT_ERR_ARG;
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
            b->coefficients += rows << r.log2n;
            if (r.schedule) {
                b->scheduled.push_back(i);
                continue;
            }
            if (flags & NTT_BATCH_GROUPED) {
                auto it = std::find_if(b->groups.begin(), b->groups.end(),
                                       [&](const ntt_batch_s::Group& g) { return g.log2n == r.log2n; });
                if (it == b->groups.end()) {
                    b->groups.emplace_back();
                    it = b->groups.end() - 1;
                    it->log2n = r.log2n;
                    it->phases = (uint32_t)grouped_phases(r.log2n);
                }
                it->reqs.push_back(i);
                continue;
            }
            const uint32_t per = rows_per_item(r.log2n);
            for (uint64_t r0 = 0; r0 < rows; r0 += per)
                b->hitems.push_back({i, (uint32_t)std::min<uint64_t>(per, rows - r0), r0});
        }
        b->short_only = 1;
        for (const auto& r : b->reqs)
            if (!r.schedule && r.log2n > NTT_BATCH_SHORT_NMAX) b->short_only = 0;
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
        const size_t n_items = std::max<size_t>(1, b->hitems.size());
        ok = cudaMalloc(&b->d_reqs, sizeof(BatchReq) * n_reqs) == cudaSuccess &&
             cudaMalloc(&b->d_items, sizeof(BatchItem) * n_items) == cudaSuccess &&
             cudaMalloc(&b->d_counter, sizeof(uint32_t)) == cudaSuccess &&
             cudaMalloc(&b->d_status, sizeof(int)) == cudaSuccess &&
             cudaMemcpy(b->d_reqs, b->hreqs.data(), sizeof(BatchReq) * n_reqs, cudaMemcpyHostToDevice) == cudaSuccess &&
             (b->hitems.empty() ||
              cudaMemcpy(b->d_items, b->hitems.data(), sizeof(BatchItem) * b->hitems.size(),
                         cudaMemcpyHostToDevice) == cudaSuccess) &&
             cudaMemset(b->d_status, 0, sizeof(int)) == cudaSuccess;
    }
    if (ok && !b->groups.empty()) {
        // largest N first; segments of every phase, uploaded once
        std::sort(b->groups.begin(), b->groups.end(),
                  [](const ntt_batch_s::Group& x, const ntt_batch_s::Group& y) { return x.log2n > y.log2n; });
        for (auto& g : b->groups) {
            g.mc = b->tables[g.log2n].host.mc;
            g.n_segs = (uint32_t)g.reqs.size();
            batch_fill_segments(b, g);
            for (uint32_t p = 0; ok && p < g.phases; ++p)
                ok = cudaMalloc(&g.d_segs[p], sizeof(GroupSeg) * g.n_segs) == cudaSuccess &&
                     cudaMemcpy(g.d_segs[p], g.hsegs[p].data(), sizeof(GroupSeg) * g.n_segs,
                                cudaMemcpyHostToDevice) == cudaSuccess;
        }
    }
    const size_t branch_users = b->scheduled.size() + (b->groups.size() > 1 ? b->groups.size() : 0);
    if (ok && branch_users) {
        b->n_branches = (uint32_t)std::min<size_t>(NTT_BATCH_BRANCHES, branch_users);
        ok = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) == cudaSuccess;
        for (uint32_t k = 0; ok && k < b->n_branches; ++k)
            ok = cudaStreamCreateWithFlags(&b->side[k], cudaStreamNonBlocking) == cudaSuccess &&
                 cudaEventCreateWithFlags(&b->ev_join[k], cudaEventDisableTiming) == cudaSuccess;
    }
    if (ok) {
        const void* fn = batch_kernel(b->mc, b->short_only);
        int per_sm = 0, sms = 0;
        ok = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBatchSmem) == cudaSuccess &&
             cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, NTT_BATCH_THREADS, kBatchSmem) == cudaSuccess &&
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
    // the scheduled requests' pointers are kernel arguments of the captured graph
    if (!b->scheduled.empty()) batch_drop_graph(b);
    // grouped segments hold the pointers in device memory: refresh them in stream order
    for (auto& g : b->groups) {
        batch_fill_segments(b, g);
        for (uint32_t p = 0; p < g.phases; ++p)
            if (cudaMemcpyAsync(g.d_segs[p], g.hsegs[p].data(), sizeof(GroupSeg) * g.n_segs, cudaMemcpyHostToDevice,
                                (cudaStream_t)cuda_stream) != cudaSuccess)
                return NTT_ERR_CUDA;
    }
    // pageable source: the runtime stages it before returning, so hreqs may change afterwards
    return cudaMemcpyAsync(b->d_reqs, b->hreqs.data(), sizeof(BatchReq) * n_reqs, cudaMemcpyHostToDevice,
                           (cudaStream_t)cuda_stream) == cudaSuccess ? NTT_OK : NTT_ERR_CUDA;
}

// One launch sequence of request i with schedule `sid` of its N on the batch's tables.
static int batch_launch_request(ntt_batch_t b, size_t i, uint32_t sid, cudaStream_t st, uint32_t* launches) {
    int count = 0;
    const SchedEntry* table = sched_table(&count);
    const ntt_request_t& r = b->reqs[i];
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
    d.src_mode = 0;
    d.in_b = nullptr;
    d.aux_q = 0;
    d.nat = 0;
    d.has_map = 0;
    const LaunchFn fn = r.inverse ? table[idx].inv : table[idx].fwd;
    return fn(d, r.in, r.out, 0, (uint64_t)r.n_polys * r.n_moduli, st, launches);
}

// [fork -> scheduled requests on up to NTT_BATCH_BRANCHES branches] ||
// [reset counter, persistent kernel] -> join
static int batch_enqueue(ntt_batch_t b, cudaStream_t st, uint32_t* launches) {
    *launches = 0;
    if (!b->scheduled.empty()) {
        if (cudaEventRecord(b->ev_fork, st) != cudaSuccess) return NTT_ERR_CUDA;
        for (uint32_t k = 0; k < b->n_branches; ++k)
            if (cudaStreamWaitEvent(b->side[k], b->ev_fork, 0) != cudaSuccess) return NTT_ERR_CUDA;
        for (size_t k = 0; k < b->scheduled.size(); ++k) {
            const uint32_t i = b->scheduled[k];
            int rc = batch_launch_request(b, i, b->reqs[i].schedule - 1, b->side[k % b->n_branches], launches);
            if (rc) return rc;
        }
    }
    // grouped grids: one N per branch after the scheduled requests (or on the
    // caller's stream when there is a single N)
    const bool group_branches = b->groups.size() > 1;
    if (group_branches && b->scheduled.empty()) {
        if (cudaEventRecord(b->ev_fork, st) != cudaSuccess) return NTT_ERR_CUDA;
        for (uint32_t k = 0; k < b->n_branches; ++k)
            if (cudaStreamWaitEvent(b->side[k], b->ev_fork, 0) != cudaSuccess) return NTT_ERR_CUDA;
    }
    for (size_t j = 0; j < b->groups.size(); ++j) {
        const auto& g = b->groups[j];
        cudaStream_t gs = group_branches ? b->side[(b->scheduled.size() + j) % b->n_branches] : st;
        for (uint32_t p = 0; p < g.phases; ++p) {
            int rc = launch_grouped(g.log2n, g.mc, (int)p, g.d_segs[p], g.n_segs, g.grid[p], b->d_status, b->check,
                                    gs);
            if (rc) return rc;
            ++*launches;
        }
    }
    if (!b->scheduled.empty() || group_branches) {
        for (uint32_t k = 0; k < b->n_branches; ++k)
            if (cudaEventRecord(b->ev_join[k], b->side[k]) != cudaSuccess) return NTT_ERR_CUDA;
    }
    const uint32_t n = (uint32_t)b->hitems.size();
    if (n) {
        if (cudaMemsetAsync(b->d_counter, 0, sizeof(uint32_t), st) != cudaSuccess) return NTT_ERR_CUDA;
#define NTT_BATCH_LAUNCH(MC, NMAX) \
    k_ntt_batch<MC, NMAX><<<b->grid, NTT_BATCH_THREADS, kBatchSmem, st>>>(b->d_reqs, b->d_items, n, b->d_counter, \
                                                                       b->d_status, b->check)
        if (b->mc) {
            if (b->short_only) NTT_BATCH_LAUNCH(1, NTT_BATCH_SHORT_NMAX); else NTT_BATCH_LAUNCH(1, 16);
        } else {
            if (b->short_only) NTT_BATCH_LAUNCH(0, NTT_BATCH_SHORT_NMAX); else NTT_BATCH_LAUNCH(0, 16);
        }
#undef NTT_BATCH_LAUNCH
        if (cudaPeekAtLastError() != cudaSuccess) return NTT_ERR_CUDA;
        ++*launches;
    }
    if (!b->scheduled.empty() || group_branches)
        for (uint32_t k = 0; k < b->n_branches; ++k)
            if (cudaStreamWaitEvent(st, b->ev_join[k], 0) != cudaSuccess) return NTT_ERR_CUDA;
    return NTT_OK;
}

int ntt_batch_execute(ntt_batch_t b, void* cuda_stream) {
    if (!b) return NTT_ERR_ARG;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != b->device) return NTT_ERR_ARG;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    b->last_launches = 0;
    if (!(b->flags & NTT_BATCH_GRAPH)) {
        uint32_t launches = 0;
        int rc = batch_enqueue(b, st, &launches);
        if (rc == NTT_OK) b->last_launches = launches;
        return rc;
    }
    if (!b->graph_exec) {
        // capture on a private stream (the legacy default stream cannot be captured)
        cudaStream_t cap;
        if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) return NTT_ERR_CUDA;
        int rc = NTT_OK;
        if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) rc = NTT_ERR_CUDA;
        if (rc == NTT_OK) rc = batch_enqueue(b, cap, &b->graph_kernels);
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
    b->last_launches = b->graph_kernels;
    return NTT_OK;
}

int ntt_batch_execute_plain(ntt_batch_t b, const uint32_t* schedules, void* cuda_stream) {
    if (!b) return NTT_ERR_ARG;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != b->device) return NTT_ERR_ARG;
    b->last_launches = 0;
    for (size_t i = 0; i < b->reqs.size(); ++i) {
        const ntt_request_t& r = b->reqs[i];
        const uint32_t sid = schedules ? schedules[i] : default_schedule(r.log2n, (uint64_t)r.n_polys * r.n_moduli);
        int rc = batch_launch_request(b, i, sid, (cudaStream_t)cuda_stream, &b->last_launches);
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

int ntt_batch_execute_static(const ntt_plan_request_t* reqs, uint32_t n_reqs, void* cuda_stream) {
    if (!reqs || n_reqs == 0 || n_reqs > NTT_STATIC_MAX_REQUESTS) return NTT_ERR_ARG;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return NTT_ERR_CUDA;
    // host-side staging of the descriptors (host memory only)
    std::vector<StaticReq> desc(n_reqs), sorted(n_reqs);
    std::vector<uint32_t> order(n_reqs);
    uint32_t mc = 1;
    for (uint32_t i = 0; i < n_reqs; ++i) {
        const ntt_plan_request_t& r = reqs[i];
        const ntt_plan_s* p = r.plan;
        if (!p || (p->h.flags & NTT_FLAG_HOST_ONLY) || p->device != dev || r.inverse > 1 || !r.in || !r.out)
            return NTT_ERR_ARG;
        if (p->h.log2n < NTT_BATCH_MIN_LOG2N || (p->h.flags & (NTT_FLAG_NATURAL_ORDER | NTT_FLAG_WORD32))) return NTT_ERR_UNSUPPORTED;
        const uint32_t polys = r.n_polys ? r.n_polys : p->h.batch;
        if (polys > p->h.batch) return NTT_ERR_ARG;
        if (!aligned16p(r.in) || !aligned16p(r.out)) return NTT_ERR_ALIGN;
        StaticReq& d = desc[i];
        d.in = r.in;
        d.out = r.out;
        d.tw_fwd = p->d_fwd;
        d.tw_inv = p->d_inv;
        d.lc = p->d_consts;
        d.status = p->d_status;
        d.log2n = p->h.log2n;
        d.n_moduli = p->h.n_moduli;
        d.inverse = r.inverse;
        d.rows = polys * p->h.n_moduli;
        d.check = (p->h.flags & NTT_FLAG_CHECK) ? 1u : 0u;
        d.per_item = rows_per_item(d.log2n);
        d.pad = 0;
        if (!p->h.mc) mc = 0;
        order[i] = i;
    }
    // largest transforms first, then item ranges in that order
    std::stable_sort(order.begin(), order.end(),
                     [&](uint32_t x, uint32_t y) { return desc[x].log2n > desc[y].log2n; });
    uint64_t items = 0;
    for (uint32_t k = 0; k < n_reqs; ++k) {
        sorted[k] = desc[order[k]];
        sorted[k].item_begin = (uint32_t)items;
        items += (sorted[k].rows + sorted[k].per_item - 1) / sorted[k].per_item;
    }
    if (items >= 0xffffffffull) return NTT_ERR_ARG;
    StaticDevice* sd = nullptr;
    int rc = static_setup(dev, &sd);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    uint32_t* counter = reinterpret_cast<uint32_t*>(sd->scratch);
    StaticReq* d_reqs = reinterpret_cast<StaticReq*>(sd->scratch + 256);
    // pageable source: staged by the runtime before the call returns
    if (cudaMemcpyAsync(d_reqs, sorted.data(), sizeof(StaticReq) * n_reqs, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemsetAsync(counter, 0, sizeof(uint32_t), st) != cudaSuccess)
        return NTT_ERR_CUDA;
    const int grid = (int)std::min<uint64_t>((uint64_t)sd->grid[mc], items);
    if (mc)
        k_ntt_batch_static<1><<<grid, NTT_BATCH_THREADS, kBatchSmem, st>>>(d_reqs, n_reqs, (uint32_t)items, counter);
    else
        k_ntt_batch_static<0><<<grid, NTT_BATCH_THREADS, kBatchSmem, st>>>(d_reqs, n_reqs, (uint32_t)items, counter);
    return cudaPeekAtLastError() == cudaSuccess ? NTT_OK : NTT_ERR_CUDA;
}

}  // extern "C"
