// RNS basis conversion (BConv) of one coefficient: the CKKS key-switching
// operator beside the NTT (Sec. III, Phase 1):
//   a_i = [x_i Qhat_i^-1]_{q_i}                     (Shoup, exact after one csub)
//   y_j = sum_i a_i [Qhat_i]_{p_j}  mod p_j          (128-bit lazy sum)
// The products a_i c_ij are summed in a 128-bit accumulator that is folded
// back below p_j every `chunk` terms (chunk * max q * max p < 2^128), and the
// final 128-bit value is reduced with two Shoup reductions:
//   hi 2^64 + lo = [hi]_p [2^64]_p + [lo]_p  (mod p).
// Host and device, so the host emulation runs the same arithmetic.
#pragma once
#include "ntt_arith.cuh"

namespace nttgb {

// Device constant block of a conversion, uint64 words in this order:
//   q[L], qhi[L], qhi_p[L]            (Qhat_i^-1 mod q_i and its Shoup form)
//   p[K], p_one[K], r64[K], r64_p[K]  (floor(2^64 / p_j), 2^64 mod p_j, its Shoup form)
//   c[L][K]                           (Qhat_i mod p_j)
struct BconvView {
    const uint64_t *q, *qhi, *qhi_p, *p, *p_one, *r64, *r64_p, *c;
    uint32_t L, K, chunk;
};

NTT_HD BconvView bconv_view(const uint64_t* w, uint32_t L, uint32_t K, uint32_t chunk) {
    BconvView v;
    v.q = w;
    v.qhi = w + L;
    v.qhi_p = w + 2 * L;
    v.p = w + 3 * L;
    v.p_one = v.p + K;
    v.r64 = v.p + 2 * K;
    v.r64_p = v.p + 3 * K;
    v.c = v.p + 4 * K;
    v.L = L;
    v.K = K;
    v.chunk = chunk;
    return v;
}

NTT_HD uint64_t bconv_ld(const uint64_t* p) {
#if defined(__CUDA_ARCH__)
    return __ldg(p);
#else
    return *p;
#endif
}

// (hi 2^64 + lo) mod p
NTT_HD uint64_t reduce128(uint64_t hi, uint64_t lo, uint64_t p, uint64_t p_one, uint64_t r64, uint64_t r64_p) {
    const uint64_t h = csub(shoup_mul(hi, 1, p_one, p), p);
    const uint64_t l = csub(shoup_mul(lo, 1, p_one, p), p);
    const uint64_t t = csub(shoup_mul(h, r64, r64_p, p), p);
    return csub(t + l, p);
}

// a_i of one coefficient, from x_i (any 64-bit value)
NTT_HD uint64_t bconv_a(const BconvView& v, uint32_t i, uint64_t x) {
    const uint64_t q = bconv_ld(v.q + i);
    return csub(shoup_mul(x, bconv_ld(v.qhi + i), bconv_ld(v.qhi_p + i), q), q);
}

// y_j of NC coefficients from their a_i, read through a(c, i), for the NJ
// outputs j0 .. j0 + NJ - 1 at once (independent accumulators: NJ x NC-fold
// ILP; each constant c_ij, read through cij(i, j), serves NC products)
template <int NJ, int NC, class GetA, class GetC>
NTT_HD void bconv_y(const BconvView& v, uint32_t j0, GetA a, GetC cij, uint64_t (&y)[NC][NJ]) {
    uint64_t hi[NC][NJ], lo[NC][NJ];
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
        for (int u = 0; u < NJ; ++u) hi[c][u] = lo[c][u] = 0;
    uint32_t n = 0;
    for (uint32_t i = 0; i < v.L; ++i) {
        uint64_t ai[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) ai[c] = a(c, i);
#pragma unroll
        for (int u = 0; u < NJ; ++u) {
            const uint64_t w = cij(i, j0 + u);
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const uint64_t pl = ai[c] * w;
                lo[c][u] += pl;
                hi[c][u] += mulhi64(ai[c], w) + (lo[c][u] < pl ? 1u : 0u);
            }
        }
        if (++n == v.chunk) {      // uniform: only bases whose products approach 2^128 / L fold
#pragma unroll
            for (int u = 0; u < NJ; ++u) {
                const uint32_t j = j0 + u;
                const uint64_t p = bconv_ld(v.p + j), p_one = bconv_ld(v.p_one + j);
                const uint64_t r64 = bconv_ld(v.r64 + j), r64_p = bconv_ld(v.r64_p + j);
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    lo[c][u] = reduce128(hi[c][u], lo[c][u], p, p_one, r64, r64_p);
                    hi[c][u] = 0;
                }
            }
            n = 1;   // the folded value counts as one more term
        }
    }
#pragma unroll
    for (int u = 0; u < NJ; ++u) {
        const uint32_t j = j0 + u;
        const uint64_t p = bconv_ld(v.p + j), p_one = bconv_ld(v.p_one + j);
        const uint64_t r64 = bconv_ld(v.r64 + j), r64_p = bconv_ld(v.r64_p + j);
#pragma unroll
        for (int c = 0; c < NC; ++c) y[c][u] = reduce128(hi[c][u], lo[c][u], p, p_one, r64, r64_p);
    }
}

}  // namespace nttgb
