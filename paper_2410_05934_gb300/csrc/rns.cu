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

#define NTT_BCONV_THREADS 256

__global__ void __launch_bounds__(NTT_BCONV_THREADS) k_bconv(const uint64_t* __restrict__ in, uint64_t* __restrict__ out,
                                                            const uint64_t* __restrict__ cst, uint32_t L, uint32_t K,
                                                            uint32_t chunk, uint32_t log2n, uint64_t total) {
    extern __shared__ uint64_t sa[];     // [L][NTT_BCONV_THREADS]: this thread's a_i in column threadIdx.x
    const BconvView v = bconv_view(cst, L, K, chunk);
    const uint64_t mask = (1ull << log2n) - 1;
    for (uint64_t idx = (uint64_t)blockIdx.x * NTT_BCONV_THREADS + threadIdx.x; idx < total;
         idx += (uint64_t)gridDim.x * NTT_BCONV_THREADS) {
        const uint64_t poly = idx >> log2n, k = idx & mask;
        const uint64_t* src = in + ((poly * L) << log2n) + k;
        for (uint32_t i = 0; i < L; ++i)
            sa[(size_t)i * NTT_BCONV_THREADS + threadIdx.x] = bconv_a(v, i, src[(uint64_t)i << log2n]);
        uint64_t* dst = out + ((poly * K) << log2n) + k;
        auto a = [&](uint32_t i) { return sa[(size_t)i * NTT_BCONV_THREADS + threadIdx.x]; };
        uint32_t j = 0;
        for (; j + 4 <= K; j += 4) {
            uint64_t y[4];
            bconv_y<4>(v, j, a, y);
#pragma unroll
            for (int u = 0; u < 4; ++u) dst[(uint64_t)(j + u) << log2n] = y[u];
        }
        for (; j < K; ++j) {
            uint64_t y[1];
            bconv_y<1>(v, j, a, y);
            dst[(uint64_t)j << log2n] = y[0];
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
    // the kernel's attribute covers the largest basis, so plans never lower it for each other
    const size_t smem_max = (size_t)NTT_BCONV_MAX_MODULI * NTT_BCONV_THREADS * sizeof(uint64_t);
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
    if (!b || !d_in || !d_out || log2n > NTT_MAX_LOG2N) return NTT_ERR_ARG;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != b->device) return NTT_ERR_ARG;
    if (((uintptr_t)d_in & 7u) || ((uintptr_t)d_out & 7u)) return NTT_ERR_ALIGN;
    if (n_polys > (1ull << 32)) return NTT_ERR_ARG;
    const uint64_t total = n_polys << log2n;
    if (total == 0) return NTT_OK;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return NTT_ERR_CUDA;
    const size_t smem = (size_t)b->L * NTT_BCONV_THREADS * sizeof(uint64_t);
    const uint64_t blocks = (total + NTT_BCONV_THREADS - 1) / NTT_BCONV_THREADS;
    const unsigned grid = (unsigned)std::min<uint64_t>(blocks, (uint64_t)std::max(1, sms) * 64u);
    k_bconv<<<grid, NTT_BCONV_THREADS, smem, (cudaStream_t)cuda_stream>>>(d_in, d_out, b->d_const, b->L, b->K,
                                                                         b->chunk, log2n, total);
    return cudaPeekAtLastError() == cudaSuccess ? NTT_OK : NTT_ERR_CUDA;
}

}  // extern "C"
