// Pointwise product kernel: the (.) of Eq. 1 (arxiv 2410.05934, Sec. II-D),
// c[r][j] = a[r][j] b[r][j] mod q_l(r), exact (Barrett, see ntt_arith.cuh).
// HBM-bound: 24 bytes move per coefficient for one 64x64-bit product.
#include <cuda_runtime.h>

#include "ntt_gb300.h"
#include "ntt_launch.h"

namespace nttgb {

// One thread per coefficient pair; each CTA walks a contiguous slice of one
// row so the modulus lookup is per CTA-iteration, not per element.
__global__ void __launch_bounds__(256) k_pointwise(const uint64_t* __restrict__ a,
                                                   const uint64_t* __restrict__ b,
                                                   uint64_t* c, const LimbConst* lc,
                                                   uint32_t n_moduli, uint32_t log2n,
                                                   uint64_t row_begin, uint64_t n_pairs) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_pairs; i += stride) {
        const uint64_t e = 2 * i;
        const uint64_t row = row_begin + (e >> log2n);
        const LimbConst m = lc[row % n_moduli];
        ulonglong2 x = *reinterpret_cast<const ulonglong2*>(a + e);
        ulonglong2 y = *reinterpret_cast<const ulonglong2*>(b + e);
        ulonglong2 z;
        z.x = barrett_mulmod(x.x, y.x, m.q, m.mu, m.bits);
        z.y = barrett_mulmod(x.y, y.y, m.q, m.mu, m.bits);
        *reinterpret_cast<ulonglong2*>(c + e) = z;
    }
}

int launch_pointwise(const PlanDev& p, uint32_t log2n, const uint64_t* a, const uint64_t* b,
                     uint64_t* c, uint64_t row_begin, uint64_t n_rows, void* stream,
                     uint32_t* launches) {
    const uint64_t n_pairs = (n_rows << log2n) / 2;
    if (n_pairs == 0) return NTT_OK;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    uint64_t blocks = (n_pairs + 255) / 256;
    const uint64_t cap = (uint64_t)(sms > 0 ? sms : 152) * 8;
    if (blocks > cap) blocks = cap;
    k_pointwise<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(
        a + (row_begin << log2n), b + (row_begin << log2n), c + (row_begin << log2n), p.lc,
        p.n_moduli, log2n, row_begin, n_pairs);
    if (cudaPeekAtLastError() != cudaSuccess) return NTT_ERR_CUDA;
    if (launches) *launches += 1;
    return NTT_OK;
}

}  // namespace nttgb
