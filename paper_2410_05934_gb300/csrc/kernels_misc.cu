// Pointwise product kernel: the (.) of Eq. 1 (arxiv 2410.05934, Sec. II-D),
// c[r][j] = a[r][j] b[r][j] mod q_l(r), exact (Barrett, see ntt_arith.cuh).
// HBM-bound: 24 bytes move per coefficient for one 64x64-bit product.
#include <cuda_runtime.h>

#include <algorithm>

#include "ntt_gb300.h"
#include "ntt_kernels.cuh"
#include "ntt_launch.h"
#include "ntt32.cuh"

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

// Throughput probe: independent butterflies per thread, same arithmetic as
// the transform kernels, so butterflies/s measures the integer-pipe ceiling
// of the NTT itself.
template <int KIND>
__global__ void __launch_bounds__(256) k_bench_bfly(uint64_t q, uint64_t w0, uint64_t wp0,
                                                    uint32_t iters, uint64_t* sink) {
    constexpr int P = 8;
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t two_q = 2 * q;
    uint64_t X[P], Y[P];
#pragma unroll
    for (int i = 0; i < P; ++i) {
        X[i] = (tid * 7919u + (uint64_t)i * 104729u) % q;
        Y[i] = (tid * 31u + (uint64_t)i * 17u) % q;
    }
    const uint64_t w = w0, wp = wp0;
    for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < P; ++i) {
            if (KIND == 0) ct_butterfly(X[i], Y[i], w, wp, q, two_q);
            else if (KIND == 1) gs_butterfly(X[i], Y[i], w, wp, q, two_q);
            else if (KIND == 2) ct_butterfly_small(X[i], Y[i], w, wp, q, 2 * two_q);
            else if (KIND == 3) gs_butterfly_small(X[i], Y[i], w, wp, q, 2 * two_q);
            else if (KIND == 6) X[i] = mont_mul(X[i], Y[i], q, wp);   // wp carries -q^-1 mod 2^64
            else if (KIND == 7) gs_butterfly_lazy(X[i], Y[i], w, wp, q, 8 * two_q);
            else {   // 64 x 64 -> 128-bit multiply-accumulate (the inner step of the basis conversion)
                const uint64_t lo = X[i] * w;
                Y[i] += lo;
                X[i] += mulhi64(X[i], w) + (Y[i] < lo ? 1u : 0u);
            }
        }
    }
    uint64_t acc = 0;
#pragma unroll
    for (int i = 0; i < P; ++i) acc ^= X[i] ^ Y[i];
    if (acc == 0x5eed5eed5eedull) sink[tid] = acc;   // practically never taken
}

// Bit-reversal permutation of rows [row_begin, row_begin + n_rows): unit
// u = (row, tile b).  In place, the CTA of the smaller of b and brv(b) swaps
// the pair (both tiles are read before either is written); out of place,
// every tile goes to its image.
__global__ void __launch_bounds__(256) k_bitrev_rows(const uint64_t* in, uint64_t* out, uint64_t row_begin,
                                                     uint64_t n_rows, int log2n, int in_place) {
    __shared__ __align__(16) uint64_t sm[2 * NTT_BRV_PITCH * 32];
    const BrvGeom g = brv_geom(log2n);
    const uint64_t units = n_rows << g.M;
    for (uint64_t u = blockIdx.x; u < units; u += gridDim.x) {
        const uint64_t row = row_begin + (u >> g.M);
        const uint32_t b = (uint32_t)(u & ((1ull << g.M) - 1)), b2 = brv_bits(b, g.M);
        const uint64_t base = row << log2n;
        if (in_place) {
            if (b > b2) continue;           // uniform over the CTA
            brv_tile_load(in + base, g, b, threadIdx.x, blockDim.x, sm);
            if (b2 != b) brv_tile_load(in + base, g, b2, threadIdx.x, blockDim.x, sm + NTT_BRV_PITCH * 32);
            __syncthreads();
            brv_tile_store(out + base, g, b, threadIdx.x, blockDim.x, sm);
            if (b2 != b) brv_tile_store(out + base, g, b2, threadIdx.x, blockDim.x, sm + NTT_BRV_PITCH * 32);
        } else {
            brv_tile_load(in + base, g, b, threadIdx.x, blockDim.x, sm);
            __syncthreads();
            brv_tile_store(out + base, g, b, threadIdx.x, blockDim.x, sm);
        }
        __syncthreads();
    }
}

int launch_bitrev_rows(const uint64_t* in, uint64_t* out, uint64_t row_begin, uint64_t n_rows, uint32_t log2n,
                       void* stream, uint32_t* launches) {
    if (n_rows == 0) return NTT_OK;
    const BrvGeom g = brv_geom((int)log2n);
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return NTT_ERR_CUDA;
    const uint64_t units = n_rows << g.M;
    const unsigned grid = (unsigned)std::min<uint64_t>(units, (uint64_t)std::max(1, sms) * 32u);
    k_bitrev_rows<<<grid, 256, 0, (cudaStream_t)stream>>>(in, out, row_begin, n_rows, (int)log2n, in == out ? 1 : 0);
    if (launches) ++*launches;
    return cudaPeekAtLastError() == cudaSuccess ? NTT_OK : NTT_ERR_CUDA;
}

// 32-bit Harvey CT butterflies (the arithmetic of the NTT_FLAG_WORD32 kernels)
__global__ void __launch_bounds__(256) k_bench_bfly32(uint32_t q, uint32_t w, uint32_t wp, uint32_t iters,
                                                      uint64_t* sink) {
    constexpr int P = 8;
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t X[P], Y[P];
#pragma unroll
    for (int i = 0; i < P; ++i) {
        X[i] = (uint32_t)((tid * 7919u + (uint64_t)i * 104729u) % q);
        Y[i] = (uint32_t)((tid * 31u + (uint64_t)i * 17u) % q);
    }
    const Tw32 tw{w, wp};
    for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int i = 0; i < P; ++i) ct32(X[i], Y[i], tw, q, 2 * q);
    }
    uint32_t acc = 0;
#pragma unroll
    for (int i = 0; i < P; ++i) acc ^= X[i] ^ Y[i];
    if (acc == 0x5eed5eedu) sink[tid] = acc;   // practically never taken
}

int launch_bench_bfly(uint64_t q, uint32_t kind, uint32_t blocks, uint32_t threads, uint32_t iters,
                      uint64_t* sink, void* stream) {
    if (kind == 5) {
        const uint32_t w = (uint32_t)(q / 3);
        const uint32_t wp = (uint32_t)(((uint64_t)w << 32) / q);
        k_bench_bfly32<<<blocks, threads, 0, (cudaStream_t)stream>>>((uint32_t)q, w, wp, iters, sink);
        return cudaPeekAtLastError() == cudaSuccess ? NTT_OK : NTT_ERR_CUDA;
    }
    // a fixed twiddle in Shoup form: w = q/3 rounded, w' = floor(w 2^64 / q)
    const uint64_t w = q / 3;
    const uint64_t wp = (uint64_t)(((unsigned __int128)w << 64) / q);
    cudaStream_t st = (cudaStream_t)stream;
    switch (kind) {
        case 0: k_bench_bfly<0><<<blocks, threads, 0, st>>>(q, w, wp, iters, sink); break;
        case 1: k_bench_bfly<1><<<blocks, threads, 0, st>>>(q, w, wp, iters, sink); break;
        case 2: k_bench_bfly<2><<<blocks, threads, 0, st>>>(q, w, wp, iters, sink); break;
        case 3: k_bench_bfly<3><<<blocks, threads, 0, st>>>(q, w, wp, iters, sink); break;
        case 6: {   // Montgomery products: the second operand stays fixed below q, the first below 2q
            uint64_t inv = q;   // q^-1 mod 2^64 by Newton's iteration (q odd): 3 correct bits, doubled 5 times
            for (int i = 0; i < 5; ++i) inv *= 2 - q * inv;
            k_bench_bfly<6><<<blocks, threads, 0, st>>>(q, w, 0 - inv, iters, sink);
            break;
        }
        case 7: k_bench_bfly<7><<<blocks, threads, 0, st>>>(q, w, wp, iters, sink); break;
        default: k_bench_bfly<4><<<blocks, threads, 0, st>>>(q, w, wp, iters, sink); break;
    }
    return cudaPeekAtLastError() == cudaSuccess ? NTT_OK : NTT_ERR_CUDA;
}

// Test aid for the bounded waits: one CTA arms an mbarrier for 16 bytes and
// waits on it with the transform kernels' bounded wait.  With `deliver` one
// bulk copy of 16 bytes completes it; without, nothing ever arrives, the wait
// runs out after `limit` rounds and the status word records the timeout.
// Nothing is in flight when the CTA leaves: the only copy is issued when
// `deliver` is set, and then the wait ends by its completion (or, if even that
// copy were lost, after the bound, a copy that never writes).
__global__ void __launch_bounds__(32) k_debug_bounded_wait(const uint64_t* src, uint32_t deliver, uint32_t limit,
                                                          int* status, uint64_t* out) {
    __shared__ __align__(16) uint64_t buf[2];
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        buf[0] = buf[1] = 0;
        mbar_init(&bar, 1);
        mbar_fence_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(&bar, 16);
        if (deliver) bulk_load(buf, src, 16, &bar);
    }
    const bool ok = mbar_wait_bounded(&bar, 0, limit);
    if (__syncthreads_or(!ok)) {
        if (threadIdx.x == 0) record_status(status, NTT_STATUS_TIMEOUT);
        return;
    }
    if (threadIdx.x == 0 && out) {
        out[0] = buf[0];
        out[1] = buf[1];
    }
}

int launch_debug_bounded_wait(const void* src, uint32_t deliver, uint32_t limit, int* status, uint64_t* out,
                              void* stream) {
    k_debug_bounded_wait<<<1, 32, 0, (cudaStream_t)stream>>>(static_cast<const uint64_t*>(src), deliver, limit,
                                                            status, out);
    return cudaPeekAtLastError() == cudaSuccess ? NTT_OK : NTT_ERR_CUDA;
}

}  // namespace nttgb
