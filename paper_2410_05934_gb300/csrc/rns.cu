// C ABI of the RNS basis conversion (declared in include/ntt_gb300.h): the
// plan precomputes the CRT constants on the host, the kernel splits each
// coefficient's conversion over the warps of a CTA (rns.cuh holds the
// arithmetic).
#include <cuda_runtime.h>

#include <algorithm>
#include <new>
#include <vector>

#include "ntt_gb300.h"
#include "ntt_internal.h"
#include "rns.cuh"

struct ntt_bconv_s {
    uint32_t L = 0, K = 0, chunk = 0;
    int device = -1;
    std::vector<uint64_t> host;     // the constant block (rns.cuh order)
    uint64_t* d_const = nullptr;
};

namespace nttgb {

// A CTA step converts 64 adjacent coefficients (32 lanes x NTT_BCONV_NC,
// 16-byte loads and stores) with 4 warps: warp w first computes the a_i of
// its quarter of the input limbs i into shared memory, then, after a barrier,
// the outputs j of its quarter of the output limbs from all a_i.  Every a_i is
// computed once, and the shared footprint (a_i of 64 coefficients plus the
// L x K constants c_ij, read at one address by the whole warp) stays small
// enough for ~7 CTAs per SM.
#define NTT_BCONV_WARPS 4
#define NTT_BCONV_THREADS (32 * NTT_BCONV_WARPS)
#define NTT_BCONV_NC 2
#define NTT_BCONV_CPS (32 * NTT_BCONV_NC)      // coefficients per CTA step

static size_t bconv_smem_bytes(uint32_t L, uint32_t K) {
    return sizeof(uint64_t) * ((size_t)L * NTT_BCONV_CPS + (size_t)L * K);
}

// outputs j0 .. j0 + NJ - 1 of one lane's NC coefficients
template <int NJ, class GetA, class GetC>
__device__ __forceinline__ void bconv_store(const BconvView& v, uint32_t j0, GetA a, GetC cij, uint64_t* dst,
                                            uint32_t log2n) {
    uint64_t y[NTT_BCONV_NC][NJ];
    bconv_y<NJ, NTT_BCONV_NC>(v, j0, a, cij, y);
#pragma unroll
    for (int u = 0; u < NJ; ++u)
        *reinterpret_cast<ulonglong2*>(dst + ((uint64_t)(j0 + u) << log2n)) = make_ulonglong2(y[0][u], y[1][u]);
}

__global__ void __launch_bounds__(NTT_BCONV_THREADS) k_bconv(const uint64_t* __restrict__ in, uint64_t* __restrict__ out,
                                                            const uint64_t* __restrict__ cst, uint32_t L, uint32_t K,
                                                            uint32_t chunk, uint32_t log2n, uint64_t total) {
    extern __shared__ __align__(16) uint64_t sa[];   // [L][NC][32] a_i, then [L][K] c_ij
    uint64_t* sc = sa + (size_t)L * NTT_BCONV_CPS;
    const BconvView v = bconv_view(cst, L, K, chunk);
    for (uint32_t e = threadIdx.x; e < L * K; e += NTT_BCONV_THREADS) sc[e] = bconv_ld(v.c + e);
    const uint32_t lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
    const uint32_t i_lo = L * w / NTT_BCONV_WARPS, i_hi = L * (w + 1) / NTT_BCONV_WARPS;
    const uint32_t j_lo = K * w / NTT_BCONV_WARPS, j_hi = K * (w + 1) / NTT_BCONV_WARPS;
    const uint64_t mask = (1ull << log2n) - 1;
    const uint64_t steps = (total + NTT_BCONV_CPS - 1) / NTT_BCONV_CPS;
    auto a = [&](int c, uint32_t i) { return sa[((size_t)i * NTT_BCONV_NC + c) * 32 + lane]; };
    auto cij = [&](uint32_t i, uint32_t j) { return sc[(size_t)i * K + j]; };
    for (uint64_t s = blockIdx.x; s < steps; s += gridDim.x) {
        // a pair never straddles two polynomials (N even), and total is even
        const uint64_t idx = s * NTT_BCONV_CPS + 2u * lane;
        const bool valid = idx < total;
        const uint64_t poly = idx >> log2n, k = idx & mask;
        __syncthreads();    // constants staged / the previous step's a_i consumed
        if (valid) {
            const uint64_t* src = in + ((poly * L) << log2n) + k;
            for (uint32_t i = i_lo; i < i_hi; ++i) {
                const ulonglong2 x = *reinterpret_cast<const ulonglong2*>(src + ((uint64_t)i << log2n));
                sa[((size_t)i * NTT_BCONV_NC + 0) * 32 + lane] = bconv_a(v, i, x.x);
                sa[((size_t)i * NTT_BCONV_NC + 1) * 32 + lane] = bconv_a(v, i, x.y);
            }
        }
        __syncthreads();
        if (valid) {
            uint64_t* dst = out + ((poly * K) << log2n) + k;
            uint32_t j = j_lo;
            for (; j + 4 <= j_hi; j += 4) bconv_store<4>(v, j, a, cij, dst, log2n);
            for (; j + 2 <= j_hi; j += 2) bconv_store<2>(v, j, a, cij, dst, log2n);
            for (; j < j_hi; ++j) bconv_store<1>(v, j, a, cij, dst, log2n);
        }
    }
}

}  // namespace nttgb

using namespace nttgb;

extern "C" {

int ntt_bconv_plan(ntt_bconv_t* out, const uint64_t* q_from, uint32_t L, const uint64_t* p_to, uint32_t K) {
    if (!out) return NTT_ERR_ARG;
    *out = nullptr;
    ntt_bconv_s* b = new (std::nothrow) ntt_bconv_s();
    if (!b) return NTT_ERR_NOMEM;
    int rc;
    try {
        rc = bconv_constants(q_from, L, p_to, K, b->host, b->chunk);
    } catch (const std::bad_alloc&) {
        rc = NTT_ERR_NOMEM;
    }
    if (rc) {
        delete b;
        return rc;
    }
    b->L = L;
    b->K = K;
    const size_t bytes = b->host.size() * sizeof(uint64_t);
    // the kernel's attribute covers the largest bases, so plans never lower it for each other
    const size_t smem_max = bconv_smem_bytes(NTT_BCONV_MAX_MODULI, NTT_BCONV_MAX_MODULI);
    if (cudaGetDevice(&b->device) != cudaSuccess || cudaMalloc(&b->d_const, bytes) != cudaSuccess ||
        cudaMemcpy(b->d_const, b->host.data(), bytes, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaFuncSetAttribute(k_bconv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max) != cudaSuccess) {
        if (b->d_const) cudaFree(b->d_const);
        cudaGetLastError();
        delete b;
        return NTT_ERR_CUDA;
    }
    *out = b;
    return NTT_OK;
}

int ntt_bconv_destroy(ntt_bconv_t b) {
    if (!b) return NTT_ERR_ARG;
    if (b->d_const) cudaFree(b->d_const);
    delete b;
    return NTT_OK;
}


int ntt_bconv(ntt_bconv_t b, const uint64_t* d_in, uint64_t* d_out, uint32_t log2n, uint64_t n_polys,
              void* cuda_stream) {
    if (!b || !d_in || !d_out || log2n < 1 || log2n > NTT_MAX_LOG2N) return NTT_ERR_ARG;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != b->device) return NTT_ERR_ARG;
    if (((uintptr_t)d_in & 15u) || ((uintptr_t)d_out & 15u)) return NTT_ERR_ALIGN;
    if (n_polys > (1ull << 32)) return NTT_ERR_ARG;
    const uint64_t total = n_polys << log2n;
    if (total == 0) return NTT_OK;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return NTT_ERR_CUDA;
    const size_t smem = bconv_smem_bytes(b->L, b->K);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bconv, NTT_BCONV_THREADS, smem) != cudaSuccess)
        return NTT_ERR_CUDA;
    // one wave of persistent CTAs, each walking steps blockIdx.x, + grid, ...
    const uint64_t steps = (total + NTT_BCONV_CPS - 1) / NTT_BCONV_CPS;
    const uint64_t wave = (uint64_t)std::max(1, sms) * (uint64_t)std::max(1, per_sm);
    const unsigned grid = (unsigned)std::min<uint64_t>(steps, wave);
    k_bconv<<<grid, NTT_BCONV_THREADS, smem, (cudaStream_t)cuda_stream>>>(d_in, d_out, b->d_const, b->L, b->K,
                                                                         b->chunk, log2n, total);
    return cudaPeekAtLastError() == cudaSuccess ? NTT_OK : NTT_ERR_CUDA;
}

}  // extern "C"
