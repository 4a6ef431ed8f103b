// C ABI of the RNS basis conversion (declared in include/ntt_gb300.h): the
// plan precomputes the CRT constants on the host, the kernel converts one
// coefficient per thread (rns.cuh).
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

// Each thread converts NTT_BCONV_NC adjacent coefficients (16-byte loads and
// stores); its a_i live in shared memory, the L x K constants c_ij too (read
// by the whole warp at one address: a broadcast).
#define NTT_BCONV_THREADS 128
#define NTT_BCONV_NC 2

static size_t bconv_smem_bytes(uint32_t L, uint32_t K) {
    return sizeof(uint64_t) * ((size_t)L * NTT_BCONV_NC * NTT_BCONV_THREADS + (size_t)L * K);
}

__global__ void __launch_bounds__(NTT_BCONV_THREADS) k_bconv(const uint64_t* __restrict__ in, uint64_t* __restrict__ out,
                                                            const uint64_t* __restrict__ cst, uint32_t L, uint32_t K,
                                                            uint32_t chunk, uint32_t log2n, uint64_t total) {
    extern __shared__ __align__(16) uint64_t sa[];   // [L][NC][THREADS] a_i, then [L][K] c_ij
    uint64_t* sc = sa + (size_t)L * NTT_BCONV_NC * NTT_BCONV_THREADS;
    const BconvView v = bconv_view(cst, L, K, chunk);
    for (uint32_t e = threadIdx.x; e < L * K; e += NTT_BCONV_THREADS) sc[e] = bconv_ld(v.c + e);
    __syncthreads();
    const uint64_t mask = (1ull << log2n) - 1;
    const uint64_t groups = total / NTT_BCONV_NC;        // coefficient pairs (N >= 2)
    for (uint64_t g = (uint64_t)blockIdx.x * NTT_BCONV_THREADS + threadIdx.x; g < groups;
         g += (uint64_t)gridDim.x * NTT_BCONV_THREADS) {
        const uint64_t idx = g * NTT_BCONV_NC;
        const uint64_t poly = idx >> log2n, k = idx & mask;
        const uint64_t* src = in + ((poly * L) << log2n) + k;
        for (uint32_t i = 0; i < L; ++i) {
            const ulonglong2 x = *reinterpret_cast<const ulonglong2*>(src + ((uint64_t)i << log2n));
            sa[((size_t)i * NTT_BCONV_NC + 0) * NTT_BCONV_THREADS + threadIdx.x] = bconv_a(v, i, x.x);
            sa[((size_t)i * NTT_BCONV_NC + 1) * NTT_BCONV_THREADS + threadIdx.x] = bconv_a(v, i, x.y);
        }
        uint64_t* dst = out + ((poly * K) << log2n) + k;
        auto a = [&](int c, uint32_t i) { return sa[((size_t)i * NTT_BCONV_NC + c) * NTT_BCONV_THREADS + threadIdx.x]; };
        auto cij = [&](uint32_t i, uint32_t j) { return sc[(size_t)i * K + j]; };
        uint32_t j = 0;
        for (; j + 4 <= K; j += 4) {
            uint64_t y[NTT_BCONV_NC][4];
            bconv_y<4, NTT_BCONV_NC>(v, j, a, cij, y);
#pragma unroll
            for (int u = 0; u < 4; ++u)
                *reinterpret_cast<ulonglong2*>(dst + ((uint64_t)(j + u) << log2n)) = make_ulonglong2(y[0][u], y[1][u]);
        }
        for (; j < K; ++j) {
            uint64_t y[NTT_BCONV_NC][1];
            bconv_y<1, NTT_BCONV_NC>(v, j, a, cij, y);
            *reinterpret_cast<ulonglong2*>(dst + ((uint64_t)j << log2n)) = make_ulonglong2(y[0][0], y[1][0]);
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
    const uint64_t blocks = (total / NTT_BCONV_NC + NTT_BCONV_THREADS - 1) / NTT_BCONV_THREADS;
    const unsigned grid = (unsigned)std::min<uint64_t>(blocks, (uint64_t)std::max(1, sms) * 64u);
    k_bconv<<<grid, NTT_BCONV_THREADS, smem, (cudaStream_t)cuda_stream>>>(d_in, d_out, b->d_const, b->L, b->K,
                                                                         b->chunk, log2n, total);
    return cudaPeekAtLastError() == cudaSuccess ? NTT_OK : NTT_ERR_CUDA;
}

}  // extern "C"
