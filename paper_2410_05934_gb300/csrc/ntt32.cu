// 32-bit-word transforms and pointwise product (plans with NTT_FLAG_WORD32):
// kernels, launchers and the 32-bit tables built from the plan's host tables.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "ntt_gb300.h"
#include "ntt_internal.h"
#include "ntt32.cuh"
#include "ntt_kernels.cuh"

namespace nttgb {

template <class C, int I>
__device__ __forceinline__ void run_passes32(Regs32<C>& st, const Args32& a, const Loc32& L, int t, uint32_t* sm) {
    if constexpr (I < C::NPASS) {
        constexpr int P = C::INV ? (C::NPASS - 1 - I) : I;
        pass32<C, P>(st, a, L, t, sm);
        tile_sync<C>();     // a row's passes touch only that row's words
        run_passes32<C, I + 1>(st, a, L, t, sm);
    }
}

template <class C>
__global__ void __launch_bounds__(C::THREADS) k_ntt32(Args32 a) {
    extern __shared__ __align__(16) uint32_t smem32[];
    pdl_begin();
    const int tin = threadIdx.x >> C::LOGT;
    const int t = threadIdx.x & (C::T - 1);
    const Loc32 L = locate32<C>(a, blockIdx.x, tin);
    uint32_t* sm = smem32 + (size_t)tin * C::E;
    Regs32<C> st;
    load32<C>(st, a, L, t, sm);
    __syncthreads();
    run_passes32<C, 0>(st, a, L, t, sm);
    store32<C>(a, L, t, sm);
}

// N = 1024: persistent CTAs of NTT_W1024_WARPS warps, each warp walking its
// list of rows with the next rows' loads in flight (see ntt32.cuh); inverse
// rows of ai (quads [0, quads_i)) and forward rows of af in one grid.  Every
// four warps of a CTA take one quad of rows per step (a CTA of 4 m warps
// counts as m consecutive quad walkers).  Shared memory per warp: two
// landing buffers and the work buffer (12 KiB); with a single modulus (SMTW)
// the CTA also holds both twiddle tables (2 x 8 KiB), copied once, so the
// butterflies read them from shared memory.
#ifndef NTT_W1024_WARPS
#define NTT_W1024_WARPS 4           // warps per CTA, a multiple of 4
#endif
#ifndef NTT_W1024_CTAS_PER_SM
#define NTT_W1024_CTAS_PER_SM 3     // resident CTAs per SM the grid is sized for
#endif
static_assert(NTT_W1024_WARPS % 4 == 0 && NTT_W1024_WARPS <= 16, "quads of warps");
#define NTT_W1024_SMEM (NTT_W1024_WARPS * 3 * 1024 * sizeof(uint32_t))
#define NTT_W1024_TW_SMEM (2 * 1024 * sizeof(Tw32))
template <bool SMTW>
__global__ void __launch_bounds__(32 * NTT_W1024_WARPS, NTT_W1024_CTAS_PER_SM)
    k_ntt32_w1024(Args32 af, Args32 ai, uint32_t quads_i, uint32_t quads) {
    extern __shared__ __align__(16) uint32_t sm_w1024[];
    pdl_begin();
    constexpr uint32_t SUB = NTT_W1024_WARPS / 4;      // quad walkers per CTA
    const int wc = threadIdx.x >> 5, t = threadIdx.x & 31;
    const int w = wc & 3;
    uint32_t* const land0 = sm_w1024 + wc * 3072;      // landing buffers at +0 and +1024
    uint32_t* work = sm_w1024 + wc * 3072 + 2048;
    Tw32* tws_f = reinterpret_cast<Tw32*>(sm_w1024 + NTT_W1024_WARPS * 3072);
    Tw32* tws_i = tws_f + 1024;
    const uint32_t grid = gridDim.x * SUB, cta = blockIdx.x * SUB + (uint32_t)(wc >> 2);
    if (SMTW) {     // both tables of the single modulus, 16 bytes per copy
        for (uint32_t i = threadIdx.x; i < 512; i += 32 * NTT_W1024_WARPS) {
            async_copy16(tws_f + 2 * i, af.tw + 2 * i);
            async_copy16(tws_i + 2 * i, ai.tw + 2 * i);
        }
        async_commit();
    }
    W1024Pick cur = w1024_pick(af, ai, quads_i, quads, cta, grid, 0, w);
    W1024Pick nxt = w1024_pick(af, ai, quads_i, quads, cta, grid, 1, w);
    w1024_prefetch(cur.inv ? ai : af, cur.L, t, land0);
    async_commit();
    w1024_prefetch(nxt.inv ? ai : af, nxt.L, t, land0 + 1024);
    async_commit();
    if (SMTW) {     // the tables' group (the two row groups may stay in flight)
        asm volatile("cp.async.wait_group 2;" ::: "memory");
        __syncthreads();
    }
    Row1024 r;
    for (uint32_t k = 0; cur.live; ++k) {
        uint32_t* ld = land0 + ((k & 1u) << 10);
        async_wait_prev();          // row k has landed (row k + 1 may be in flight)
        __syncwarp();
        const W1024Pick after = w1024_pick(af, ai, quads_i, quads, cta, grid, k + 2, w);
        if (!cur.inv) {
            w1024_fwd_a_land<SMTW>(r, af, cur.L, t, ld, tws_f);
            __syncwarp();           // every lane has read the landing buffer: refill it
            w1024_prefetch(after.inv ? ai : af, after.L, t, ld);
            async_commit();
            w1024_write_a(r, cur.L, t, work);
            __syncwarp();
            w1024_fwd_b<SMTW>(r, af, cur.L, t, work, tws_f);
            __syncwarp();
            w1024_store(af, cur.L, t, work);
        } else {
            w1024_inv_a_land(ai, cur.L, t, ld, work);
            __syncwarp();
            w1024_prefetch(after.inv ? ai : af, after.L, t, ld);
            async_commit();
            w1024_inv_b<SMTW>(r, ai, cur.L, t, work, tws_i);
            __syncwarp();
            w1024_inv_c<SMTW>(r, ai, cur.L, t, work, tws_i);
        }
        __syncwarp();               // the work buffer is free for the next row
        cur = nxt;
        nxt = after;
    }
    async_wait_all();
}

static int launch32_w1024_rows(const Args32& af, const Args32& ai, uint64_t f_rows, uint64_t i_rows, cudaStream_t st) {
    const uint64_t quads_i = (i_rows + 3) / 4, quads = quads_i + (f_rows + 3) / 4;
    if (quads == 0) return NTT_OK;
    if (quads > 0x7fffffffull) return NTT_ERR_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return NTT_ERR_CUDA;
    uint64_t ctas = (uint64_t)(sms > 0 ? sms : 1) * NTT_W1024_CTAS_PER_SM;
    const uint64_t need = (quads + NTT_W1024_WARPS / 4 - 1) / (NTT_W1024_WARPS / 4);
    if (ctas > need) ctas = need;
    const bool smtw = af.n_moduli == 1 && ai.n_moduli == 1;
    const auto kernel = smtw ? k_ntt32_w1024<true> : k_ntt32_w1024<false>;
    const size_t smem = NTT_W1024_SMEM + (smtw ? NTT_W1024_TW_SMEM : 0);
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return NTT_ERR_CUDA;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)ctas);
    cfg.blockDim = dim3(32 * NTT_W1024_WARPS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, af, ai, (uint32_t)quads_i, (uint32_t)quads) == cudaSuccess ? NTT_OK
                                                                                                   : NTT_ERR_CUDA;
}

template <bool INV>
static int launch32_w1024(const Args32& a, cudaStream_t st) {
    return INV ? launch32_w1024_rows(a, a, 0, a.n_rows, st) : launch32_w1024_rows(a, a, a.n_rows, 0, st);
}

template <int LOGN, bool INV>
static int launch32_n(const Args32& a, cudaStream_t st) {
    using C = typename Cfg32Sel<LOGN, INV>::C;
    const uint64_t ctas = ((uint64_t)a.n_rows + C::TPC - 1) / C::TPC;
    if (ctas == 0) return NTT_OK;
    if (ctas > 0x7fffffffull) return NTT_ERR_ARG;
    cudaLaunchConfig_t cfg = {};       // programmatic dependent launch, as the 64-bit tile kernels
    cfg.gridDim = dim3((unsigned)ctas);
    cfg.blockDim = dim3(C::THREADS);
    cfg.dynamicSmemBytes = sizeof(uint32_t) * C::E * C::TPC;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_ntt32<C>, a) == cudaSuccess ? NTT_OK : NTT_ERR_CUDA;
}

#define NTT32_CASE(LOGN) \
    case LOGN: return inverse ? launch32_n<LOGN, true>(a, st) : launch32_n<LOGN, false>(a, st);

int launch_ntt32(const Plan32Dev& p, bool inverse, const uint32_t* in, uint32_t* out, uint64_t row_begin,
                 uint64_t n_rows, uint32_t log2n, void* stream, uint32_t* launches) {
    if (n_rows == 0) return NTT_OK;
    if (row_begin + n_rows > 0xffffffffull) return NTT_ERR_ARG;
    Args32 a;
    a.in = in;
    a.out = out;
    a.tw = inverse ? p.inv : p.fwd;
    a.lc = p.lc;
    a.status = p.status;
    a.row_begin = (uint32_t)row_begin;
    a.n_rows = (uint32_t)n_rows;
    a.n_moduli = p.n_moduli;
    a.check = p.check;
    a.mod_magic = fdiv_magic(p.n_moduli);
    cudaStream_t st = (cudaStream_t)stream;
    if (launches) ++*launches;
    switch (log2n) {
        NTT32_CASE(1) NTT32_CASE(2) NTT32_CASE(3) NTT32_CASE(4) NTT32_CASE(5) NTT32_CASE(6)
        NTT32_CASE(7) NTT32_CASE(8) NTT32_CASE(9) NTT32_CASE(11) NTT32_CASE(12)
        case 10: return inverse ? launch32_w1024<true>(a, st) : launch32_w1024<false>(a, st);
        default: return NTT_ERR_UNSUPPORTED;
    }
}

static Args32 args32(const Plan32Dev& p, bool inverse, const uint32_t* in, uint32_t* out, uint64_t n_rows) {
    Args32 a;
    a.in = in;
    a.out = out;
    a.tw = inverse ? p.inv : p.fwd;
    a.lc = p.lc;
    a.status = p.status;
    a.row_begin = 0;
    a.n_rows = (uint32_t)n_rows;
    a.n_moduli = p.n_moduli;
    a.check = p.check;
    a.mod_magic = fdiv_magic(p.n_moduli);
    return a;
}

int launch_ntt32_fwd_inv(const Plan32Dev& pf, const uint32_t* fin, uint32_t* fout, uint64_t f_rows,
                         const Plan32Dev& pi, const uint32_t* iin, uint32_t* iout, uint64_t i_rows, uint32_t log2n,
                         void* stream, uint32_t* launches) {
    if (f_rows > 0xffffffffull || i_rows > 0xffffffffull) return NTT_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    if (log2n != 10 || f_rows == 0 || i_rows == 0) {     // the two transforms in stream order
        int rc = launch_ntt32(pf, false, fin, fout, 0, f_rows, log2n, stream, launches);
        return rc ? rc : launch_ntt32(pi, true, iin, iout, 0, i_rows, log2n, stream, launches);
    }
    const Args32 af = args32(pf, false, fin, fout, f_rows), ai = args32(pi, true, iin, iout, i_rows);
    const int rc = launch32_w1024_rows(af, ai, f_rows, i_rows, st);
    if (rc == NTT_OK && launches) ++*launches;
    return rc;
}

// Probe kind 8: 32-bit Harvey CT butterflies as in k_bench_bfly32 (kind 5),
// with the conditional subtraction written as compare and select
__global__ void __launch_bounds__(256) k_bench_bfly32_cmp(uint32_t q, uint32_t w, uint32_t wp, uint32_t iters,
                                                          uint64_t* sink) {
    constexpr int P = 8;
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t X[P], Y[P];
#pragma unroll
    for (int i = 0; i < P; ++i) {
        X[i] = (uint32_t)((tid * 7919u + (uint64_t)i * 104729u) % q);
        Y[i] = (uint32_t)((tid * 31u + (uint64_t)i * 17u) % q);
    }
    const uint32_t two_q = 2 * q;
    for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < P; ++i) {
            const uint32_t x = X[i] >= two_q ? X[i] - two_q : X[i];
            const uint32_t t = shoup32(Y[i], w, wp, q);
            X[i] = x + t;
            Y[i] = x - t + two_q;
        }
    }
    uint32_t acc = 0;
#pragma unroll
    for (int i = 0; i < P; ++i) acc ^= X[i] ^ Y[i];
    if (acc == 0x5eed5eedu) sink[tid] = acc;   // practically never taken
}

int launch_bench_bfly32_cmp(uint64_t q, uint32_t blocks, uint32_t threads, uint32_t iters, uint64_t* sink,
                            void* stream) {
    const uint32_t w = (uint32_t)(q / 3);
    const uint32_t wp = (uint32_t)(((uint64_t)w << 32) / q);
    k_bench_bfly32_cmp<<<blocks, threads, 0, (cudaStream_t)stream>>>((uint32_t)q, w, wp, iters, sink);
    return cudaPeekAtLastError() == cudaSuccess ? NTT_OK : NTT_ERR_CUDA;
}

__global__ void k_pointwise32(const uint32_t* __restrict__ a, const uint32_t* __restrict__ b, uint32_t* c,
                              const LimbConst32* __restrict__ lc, uint32_t n_moduli, uint32_t log2n, uint64_t total) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (uint64_t)gridDim.x * blockDim.x) {
        const LimbConst32 m = lc[(i >> log2n) % n_moduli];
        c[i] = mulmod32(a[i], b[i], m);
    }
}

int launch_pointwise32(const Plan32Dev& p, uint32_t log2n, const uint32_t* a, const uint32_t* b, uint32_t* c,
                       uint64_t n_rows, void* stream, uint32_t* launches) {
    const uint64_t total = n_rows << log2n;
    if (total == 0) return NTT_OK;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return NTT_ERR_CUDA;
    const unsigned grid = (unsigned)std::min<uint64_t>((total + 255) / 256, (uint64_t)std::max(1, sms) * 32u);
    k_pointwise32<<<grid, 256, 0, (cudaStream_t)stream>>>(a, b, c, p.lc, p.n_moduli, log2n, total);
    if (launches) ++*launches;
    return cudaPeekAtLastError() == cudaSuccess ? NTT_OK : NTT_ERR_CUDA;
}

}  // namespace nttgb
