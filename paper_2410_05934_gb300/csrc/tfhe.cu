// C ABI of the batched TFHE external product / CMux step (declared in
// include/ntt_gb300.h) and its kernel; the per-thread steps live in
// tfhe_cmux.cuh so that the host emulation runs the same code.
#include <cuda_runtime.h>

#include <algorithm>

#include "ntt_gb300.h"
#include "ntt_internal.h"
#include "ntt_kernels.cuh"
#include "tfhe_cmux.cuh"

namespace nttgb {

template <int LOGN, int MC>
__global__ void __launch_bounds__(CmuxCfg<LOGN, MC>::THREADS, CmuxCfg<LOGN, MC>::MIN_CTAS) k_tfhe_cmux(CmuxArgs c, TileArgs af, TileArgs ai) {
    using K = CmuxCfg<LOGN, MC>;
    using F = typename K::F;
    using I = typename K::I;
    extern __shared__ __align__(16) uint64_t smem[];
    pdl_begin();     // consecutive CMux steps: launched early, reading only after the previous step
    const int s = threadIdx.x >> K::LOGT;
    const int t = threadIdx.x & (K::T - 1);
    uint64_t* sm = smem + (size_t)s * K::N;
    TileLoc L;
    L.row = 0;
    L.rowq = 0;
    L.limb = 0;
    L.hi = 0;
    L.gbase = 0;
    L.tw_off = 0;
    L.valid = true;
    const LimbConst lc = af.lc[0];
    for (uint64_t ct = blockIdx.x; ct < c.n_ct; ct += gridDim.x) {
        CmuxRegs<K> cr;
        cmux_load<K>(cr, c, ct, s, t, smem);
        // the two slots touch only their own row and partial sums until the
        // exchange, so they synchronise separately (a named barrier each)
        for (uint32_t j = 0; j < c.levels; ++j) {
            TileRegs<F> st;
            cmux_digits<K>(st, cr, j, c);
            write_pairs_swizzled<F>(st, L, t, sm);
            tile_sync<F, 2>();
            run_passes<F, 0, 2>(st, af, L, t, sm);
            cmux_mac<K>(c, lc, (uint32_t)s * c.levels + j, s, t, smem);
        }
        __syncthreads();    // exchange: each slot reads both slots' partial sums
        TileRegs<I> si;
        cmux_inverse_input<K>(si, lc, s, t, smem);
        write_pairs_swizzled<I>(si, L, t, sm);
        tile_sync<I, 2>();
        run_passes<I, 0, 2>(si, ai, L, t, sm);
        cmux_store<K>(c, lc, ct, s, t, sm);
        __syncthreads();    // partial sums read by the other slot before they are cleared
    }
}

template <int LOGN, int MC>
static int launch_cmux(const CmuxArgs& c, const TileArgs& af, const TileArgs& ai, cudaStream_t st) {
    using K = CmuxCfg<LOGN, MC>;
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaFuncSetAttribute(k_tfhe_cmux<LOGN, MC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)K::SMEM_BYTES) != cudaSuccess ||
        cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tfhe_cmux<LOGN, MC>, K::THREADS,
                                                      K::SMEM_BYTES) != cudaSuccess)
        return NTT_ERR_CUDA;
    // enough CTAs for several waves; each walks ciphertexts ct, ct + grid, ...
    const uint64_t cap = (uint64_t)std::max(1, sms) * (uint64_t)std::max(1, per_sm) * 16u;
    const unsigned grid = (unsigned)std::min<uint64_t>(c.n_ct, cap);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(K::THREADS);
    cfg.dynamicSmemBytes = K::SMEM_BYTES;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_tfhe_cmux<LOGN, MC>, c, af, ai) == cudaSuccess ? NTT_OK : NTT_ERR_CUDA;
}

// Shared argument checks of both entry points; fills c (not in/rot/out) and
// the two tile argument blocks.
static int cmux_setup(ntt_plan_t plan, const uint64_t* d_key, uint32_t levels, uint32_t log2_base, uint64_t n_ct,
                      CmuxArgs& c, TileArgs& af, TileArgs& ai) {
    // d_key: [2 levels][2][N] pairs {w, floor(w 2^64 / q)} (tfhe_key_prepare)
    if (!plan || !d_key) return NTT_ERR_ARG;
    if (plan->h.flags & NTT_FLAG_HOST_ONLY) return NTT_ERR_ARG;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != plan->device) return NTT_ERR_ARG;
    if (plan->h.n_moduli != 1) return NTT_ERR_ARG;
    if (plan->h.flags & (NTT_FLAG_NATURAL_ORDER | NTT_FLAG_WORD32)) return NTT_ERR_UNSUPPORTED;
    if (plan->h.log2n < NTT_TFHE_MIN_LOG2N || plan->h.log2n > NTT_TFHE_MAX_LOG2N) return NTT_ERR_UNSUPPORTED;
    if (((uintptr_t)d_key & 15u) != 0) return NTT_ERR_ALIGN;
    const uint64_t q = plan->h.moduli[0];
    const uint32_t sigma = 63u - (uint32_t)__builtin_clzll(q);
    if (levels < 1 || levels > NTT_TFHE_MAX_LEVELS || log2_base < 1 || levels * log2_base > 32 ||
        levels * log2_base > sigma)
        return NTT_ERR_ARG;
    if (n_ct > (1ull << 40)) return NTT_ERR_ARG;
    c.key = reinterpret_cast<const TwPair*>(d_key);
    c.status = plan->d_status;
    c.q = q;
    c.half_q = q >> 1;
    c.m = (uint64_t)(((unsigned __int128)1 << (64 + sigma)) / q);
    c.n_ct = n_ct;
    c.sigma = sigma;
    c.levels = levels;
    c.log2_base = log2_base;
    c.check = (plan->h.flags & NTT_FLAG_CHECK) ? 1u : 0u;
    TileArgs a{};
    a.lc = plan->d_consts;
    a.status = plan->d_status;
    a.n_moduli = 1;
    af = a;
    ai = a;
    af.tw = plan->d_fwd;
    ai.tw = plan->d_inv;
    return NTT_OK;
}

static int cmux_dispatch(ntt_plan_t plan, const CmuxArgs& c, const TileArgs& af, const TileArgs& ai, void* stream) {
    plan->last_launches = 0;
    if (c.n_ct == 0) return NTT_OK;
    cudaStream_t st = (cudaStream_t)stream;
    int rc;
    const bool small = plan->h.mc != 0;
    switch (plan->h.log2n) {
        case 10: rc = small ? launch_cmux<10, 1>(c, af, ai, st) : launch_cmux<10, 0>(c, af, ai, st); break;
        case 11: rc = small ? launch_cmux<11, 1>(c, af, ai, st) : launch_cmux<11, 0>(c, af, ai, st); break;
        default: return NTT_ERR_UNSUPPORTED;
    }
    if (rc == NTT_OK) plan->last_launches = 1;
    return rc;
}

// key rows -> {w, floor(w 2^64 / q)} pairs; range check under NTT_FLAG_CHECK
__global__ void k_tfhe_key_prepare(const uint64_t* __restrict__ key, TwPair* __restrict__ out, uint64_t count,
                                   uint64_t q, int* status, uint32_t check) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t w = key[i];
        if (check && w >= q) record_status(status, NTT_STATUS_RANGE);
        out[i] = TwPair{w, (uint64_t)(((unsigned __int128)w << 64) / q)};
    }
}

}  // namespace nttgb

using namespace nttgb;

extern "C" {

int tfhe_key_prepare(ntt_plan_t plan, const uint64_t* d_key, uint32_t levels, uint64_t* d_key_shoup,
                     void* cuda_stream) {
    if (!plan || !d_key || !d_key_shoup) return NTT_ERR_ARG;
    if (plan->h.flags & NTT_FLAG_HOST_ONLY) return NTT_ERR_ARG;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != plan->device) return NTT_ERR_ARG;
    if (plan->h.n_moduli != 1 || levels < 1 || levels > NTT_TFHE_MAX_LEVELS) return NTT_ERR_ARG;
    if (plan->h.flags & NTT_FLAG_WORD32) return NTT_ERR_UNSUPPORTED;
    if (((uintptr_t)d_key & 7u) || ((uintptr_t)d_key_shoup & 15u)) return NTT_ERR_ALIGN;
    const uint64_t count = (uint64_t)4 * levels << plan->h.log2n;
    const unsigned grid = (unsigned)std::min<uint64_t>((count + 255) / 256, 4096);
    k_tfhe_key_prepare<<<grid, 256, 0, (cudaStream_t)cuda_stream>>>(
        d_key, reinterpret_cast<TwPair*>(d_key_shoup), count, plan->h.moduli[0], plan->d_status,
        (plan->h.flags & NTT_FLAG_CHECK) ? 1u : 0u);
    plan->last_launches = 1;
    return cudaPeekAtLastError() == cudaSuccess ? NTT_OK : NTT_ERR_CUDA;
}

int tfhe_external_product(ntt_plan_t plan, const uint64_t* d_in, const uint64_t* d_key, uint32_t levels,
                          uint32_t log2_base, uint64_t* d_out, uint64_t n_ct, void* cuda_stream) {
    CmuxArgs c;
    TileArgs af, ai;
    int rc = cmux_setup(plan, d_key, levels, log2_base, n_ct, c, af, ai);
    if (rc) return rc;
    if (n_ct == 0) return cmux_dispatch(plan, c, af, ai, cuda_stream);    // nothing to read or write
    if (!d_in || !d_out) return NTT_ERR_ARG;
    if (((uintptr_t)d_in & 15u) || ((uintptr_t)d_out & 15u)) return NTT_ERR_ALIGN;
    c.in = d_in;
    c.rot = nullptr;
    c.out = d_out;
    return cmux_dispatch(plan, c, af, ai, cuda_stream);
}

int tfhe_cmux_rotate(ntt_plan_t plan, const uint64_t* d_acc, const uint32_t* d_rot, const uint64_t* d_key,
                     uint32_t levels, uint32_t log2_base, uint64_t* d_out, uint64_t n_ct, void* cuda_stream) {
    CmuxArgs c;
    TileArgs af, ai;
    int rc = cmux_setup(plan, d_key, levels, log2_base, n_ct, c, af, ai);
    if (rc) return rc;
    if (n_ct == 0) return cmux_dispatch(plan, c, af, ai, cuda_stream);    // nothing to read or write
    if (!d_acc || !d_rot || !d_out) return NTT_ERR_ARG;
    if (((uintptr_t)d_acc & 15u) || ((uintptr_t)d_out & 15u) || ((uintptr_t)d_rot & 3u)) return NTT_ERR_ALIGN;
    c.in = d_acc;
    c.rot = d_rot;
    c.out = d_out;
    return cmux_dispatch(plan, c, af, ai, cuda_stream);
}

}  // extern "C"
