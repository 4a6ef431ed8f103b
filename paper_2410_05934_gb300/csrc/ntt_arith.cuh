// Modular arithmetic of the NTT kernels (arxiv 2410.05934, Sec. II-D).
//
// Words are uint64, moduli q < 2^62.  Twiddles are multiplied in Shoup form:
// for a fixed w < q the plan stores w' = floor(w 2^64 / q); then for ANY
// y < 2^64,  Q = floor(y w' / 2^64)  and  r = y w - Q q  satisfy
// r = y w mod q  or  r = y w mod q + q, i.e. r in [0, 2q).  (y w/q - y w'/2^64
// lies in [0, 1), so Q is floor(y w / q) or one less.)  Only the low 64 bits
// of y w and Q q are needed because r < 2q < 2^64.  The kernels estimate Q
// from three of the four 32 x 32-bit partial products (shoup_mul_approx) and
// fix the range with at most one subtraction where a bound needs it.
//
// Butterflies keep values lazily reduced (Harvey's bounds), which q < 2^62
// makes safe in 64-bit words:
//   CT (forward, Eq. 1's NTT^{CT}):  X, Y in [0, 4q) -> X + wY, X - wY in [0, 4q)
//   GS (inverse, Eq. 1's INTT^{GS}): X, Y in [0, 2q) -> X + Y, (X - Y) w in [0, 2q)
//
// Every function here is __host__ __device__ so the kernels' phase functions
// can also run on the CPU (the host emulation used by the CPU test suite).
#pragma once
#include <stdint.h>

#if defined(__CUDACC__)
#define NTT_HD __host__ __device__ __forceinline__
#else
#define NTT_HD inline
#endif

namespace nttgb {

NTT_HD uint64_t mulhi64(uint64_t a, uint64_t b) {
#if defined(__CUDA_ARCH__)
    return __umul64hi(a, b);
#else
    return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

// Shoup product with a three-partial-product quotient: with y = yh 2^32 + yl
// and w' = wh 2^32 + wl,  Q~ = yh wh + floor(yh wl / 2^32) + floor(yl wh / 2^32)
// drops three fractional parts (each < 1) of y w' / 2^64, so
// floor(y w' / 2^64) - Q~ is in {0, 1, 2} and floor(y w / q) - Q~ in {0..3}:
// the result y w - Q~ q is y w mod q plus 0..3 q, i.e. in [0, 4q), for any
// y < 2^64.  The butterflies of moduli below 2^57 use it as it is (4q-wide
// lazy bounds fit); shoup_mul adds one conditional subtraction for the rest.
//
// On the GPU the product is written with 32-bit multiplies of the integer
// multiply pipe, which binds the transforms: two high halves and one
// widening multiply-add for Q~, then y w - Q~ q mod 2^64 as
// y w + Q~ (2^64 - q), each 64 x 64 -> 64-bit low product being one
// widening multiply of the low words plus two low multiplies of the cross
// words added to its high word.  Same value as the host form below (the
// compiler's own lowering of the C form issues ~25 % more multiply-pipe
// cycles per butterfly).
NTT_HD uint64_t shoup_mul_approx(uint64_t y, uint64_t w, uint64_t wp, uint64_t q) {
#if defined(__CUDA_ARCH__)
    const uint64_t nq = 0 - q;
    uint64_t r;
    asm("{\n\t"
        ".reg .u32 yl, yh, wl, wh, pl, ph, nl, nh, a, b, ql, qh, rl, rh;\n\t"
        ".reg .u64 Q, t;\n\t"
        "mov.b64 {yl, yh}, %1;\n\t"
        "mov.b64 {wl, wh}, %2;\n\t"
        "mov.b64 {pl, ph}, %3;\n\t"
        "mov.b64 {nl, nh}, %4;\n\t"
        "mul.hi.u32 a, yh, pl;\n\t"          // floor(yh wl' / 2^32)
        "mul.hi.u32 b, yl, ph;\n\t"          // floor(yl wh' / 2^32)
        "cvt.u64.u32 t, a;\n\t"
        "mad.wide.u32 Q, yh, ph, t;\n\t"     // yh wh' + a
        "mov.b64 {ql, qh}, Q;\n\t"
        "add.cc.u32 ql, ql, b;\n\t"          // Q~ = yh wh' + a + b
        "addc.u32 qh, qh, 0;\n\t"
        "mul.wide.u32 t, yl, wl;\n\t"        // y w mod 2^64
        "mov.b64 {rl, rh}, t;\n\t"
        "mad.lo.u32 rh, yl, wh, rh;\n\t"
        "mad.lo.u32 rh, yh, wl, rh;\n\t"
        "mov.b64 t, {rl, rh};\n\t"
        "mad.wide.u32 t, ql, nl, t;\n\t"     // + Q~ (2^64 - q) mod 2^64
        "mov.b64 {rl, rh}, t;\n\t"
        "mad.lo.u32 rh, ql, nh, rh;\n\t"
        "mad.lo.u32 rh, qh, nl, rh;\n\t"
        "mov.b64 %0, {rl, rh};\n\t"
        "}"
        : "=l"(r)
        : "l"(y), "l"(w), "l"(wp), "l"(nq));
    return r;
#else
    const uint32_t yl = (uint32_t)y, yh = (uint32_t)(y >> 32);
    const uint32_t wl = (uint32_t)wp, wh = (uint32_t)(wp >> 32);
    const uint64_t mid = (((uint64_t)yh * wl) >> 32) + (((uint64_t)yl * wh) >> 32);
    const uint64_t Q = (uint64_t)yh * wh + mid;
    return y * w - Q * q;
#endif
}

// x in [0, 2m) -> [0, m)
NTT_HD uint64_t csub(uint64_t x, uint64_t m) { return x >= m ? x - m : x; }

// y * w mod q lazily: result in [0, 2q) for any y < 2^64 (w < q, wp its
// Shoup form), for every q < 2^62.  The three-partial-product quotient
// leaves y w mod q + {0..3} q, which is below 4q < 2^64, and one conditional
// subtraction of 2q brings it into [0, 2q).  That costs two integer adds
// where the exact quotient floor(y w' / 2^64) costs four more multiplies on
// the integer multiply pipe, which is the one that binds.
NTT_HD uint64_t shoup_mul(uint64_t y, uint64_t w, uint64_t wp, uint64_t q) {
    return csub(shoup_mul_approx(y, w, wp, q), 2 * q);
}

// Cooley-Tukey butterfly, Harvey-lazy.  In/out in [0, 4q).
NTT_HD void ct_butterfly(uint64_t& X, uint64_t& Y, uint64_t w, uint64_t wp, uint64_t q,
                         uint64_t two_q) {
    uint64_t x = csub(X, two_q);
    uint64_t t = shoup_mul(Y, w, wp, q);
    X = x + t;
    Y = x - t + two_q;
}

// Gentleman-Sande butterfly, Harvey-lazy.  In/out in [0, 2q).
NTT_HD void gs_butterfly(uint64_t& X, uint64_t& Y, uint64_t w, uint64_t wp, uint64_t q,
                         uint64_t two_q) {
    uint64_t s = csub(X + Y, two_q);
    uint64_t d = X - Y + two_q;
    Y = shoup_mul(d, w, wp, q);
    X = s;
}

// Modulus class 1 (q < 2^57): quotient-approximate products, 4q-wide bounds.
// Forward CT without any conditional subtraction: X, Y < B q  ->
//   X + wY < (B + 4) q,  X - wY + 4q < (B + 4) q   (wY in [0, 4q)).
// From canonical input the bound after s stages is (1 + 4 s) q <= 65 q < 2^64.
NTT_HD void ct_butterfly_small(uint64_t& X, uint64_t& Y, uint64_t w, uint64_t wp, uint64_t q,
                               uint64_t four_q) {
    uint64_t t = shoup_mul_approx(Y, w, wp, q);
    uint64_t x = X;
    X = x + t;
    Y = x - t + four_q;
}

// GS with 4q-wide bounds: X, Y in [0, 4q) -> X + Y reduced to [0, 4q),
// (X - Y + 4q) w in [0, 4q).  Needs 8q < 2^64.
NTT_HD void gs_butterfly_small(uint64_t& X, uint64_t& Y, uint64_t w, uint64_t wp, uint64_t q,
                               uint64_t four_q) {
    uint64_t s = csub(X + Y, four_q);
    uint64_t d = X - Y + four_q;
    Y = shoup_mul_approx(d, w, wp, q);
    X = s;
}

NTT_HD void gs_butterfly_scaled_small(uint64_t& X, uint64_t& Y, uint64_t ninv, uint64_t ninv_p,
                                      uint64_t wn, uint64_t wn_p, uint64_t q, uint64_t four_q) {
    uint64_t s = X + Y;                 // [0, 8q)
    uint64_t d = X - Y + four_q;        // [0, 8q)
    X = shoup_mul_approx(s, ninv, ninv_p, q);
    Y = shoup_mul_approx(d, wn, wn_p, q);
}

// x in [0, 65q) to [0, q) for q < 2^57 of bit length k (the forward
// transform's output bound in modulus class 1).  With sh = max(k - 25, 0),
// t = floor(x / 2^sh) < 65 * 2^25 < 2^32 and m = floor(2^(32 + sh) / q) < 2^32,
// the estimate Qe = floor(t m / 2^32) of Q = floor(x / q) is short by less
// than t / 2^32 + 2^sh / q + 1 < 0.51 + 2^-24 + 1 < 2, so x - Qe q lies in
// [0, 2q): one conditional subtraction.  Qe <= 65, so Qe q needs only the
// low 64 bits of a 32 x 64 product.
NTT_HD uint64_t reduce_65q(uint64_t x, uint32_t m, uint32_t k, uint64_t q) {
    const uint32_t sh = k > 25 ? k - 25 : 0;
    const uint32_t t = (uint32_t)(x >> sh);
#if defined(__CUDA_ARCH__)
    const uint32_t qe = __umulhi(t, m);
#else
    const uint32_t qe = (uint32_t)(((uint64_t)t * m) >> 32);
#endif
    return csub(x - (uint64_t)qe * q, q);
}

// Modulus class 2 (q < 2^50): the inverse's GS butterflies skip the
// conditional subtraction of the sum.  Before the k-th stage of a kernel
// every value is below B_k = 2^k 4q, so with c = B_k
//   X + Y < B_(k+1),   X - Y + c in (0, 2 B_k),   (X - Y + c) w in [0, 4q)
// and a kernel of at most 11 stages stays below 2^13 q < 2^63.
NTT_HD void gs_butterfly_lazy(uint64_t& X, uint64_t& Y, uint64_t w, uint64_t wp, uint64_t q, uint64_t c) {
    const uint64_t s = X + Y;
    Y = shoup_mul_approx(X - Y + c, w, wp, q);
    X = s;
}

NTT_HD void gs_butterfly_scaled_lazy(uint64_t& X, uint64_t& Y, uint64_t ninv, uint64_t ninv_p, uint64_t wn,
                                     uint64_t wn_p, uint64_t q, uint64_t c) {
    const uint64_t s = X + Y, d = X - Y + c;
    X = shoup_mul_approx(s, ninv, ninv_p, q);
    Y = shoup_mul_approx(d, wn, wn_p, q);
}

// x < 2^(k + 14) (k the bit length of q) to [0, 3q): with sh = max(k - 18, 0),
// t = floor(x / 2^sh) < 2^32 and m = floor(2^(32 + sh) / q), Qe = floor(t m / 2^32)
// is short of floor(x / q) by less than t / 2^32 + 2^sh / q + 1 < 2 + 2^-17.
// Ends a class-2 inverse kernel that is not the last (its values are below
// 2^(A + 2) q for A <= 11 stages), inside the next kernel's input bound 4q.
NTT_HD uint64_t reduce_lazy(uint64_t x, uint32_t m, uint32_t k, uint64_t q) {
    const uint32_t sh = k > 18 ? k - 18 : 0;
    const uint32_t t = (uint32_t)(x >> sh);
#if defined(__CUDA_ARCH__)
    const uint32_t qe = __umulhi(t, m);
#else
    const uint32_t qe = (uint32_t)(((uint64_t)t * m) >> 32);
#endif
    return x - (uint64_t)qe * q;
}

// Last GS stage with the N^-1 scaling folded in:
//   X' = (X + Y) N^-1,  Y' = (X - Y) w N^-1;   in [0, 2q) -> out [0, 2q).
NTT_HD void gs_butterfly_scaled(uint64_t& X, uint64_t& Y, uint64_t ninv, uint64_t ninv_p,
                                uint64_t wn, uint64_t wn_p, uint64_t q, uint64_t two_q) {
    uint64_t s = X + Y;                 // [0, 4q)
    uint64_t d = X - Y + two_q;         // [0, 4q)
    X = shoup_mul(s, ninv, ninv_p, q);
    Y = shoup_mul(d, wn, wn_p, q);
}

// a * b mod q for a, b < q by Barrett reduction with k = bitlen(q) and
// mu = floor(2^(2k) / q) < 2^63:  x = a b < 2^(2k);  q3 = ((x >> (k-1)) mu) >> (k+1)
// underestimates floor(x / q) by at most 2, so r = x - q3 q < 3q (Handbook of
// Applied Cryptography, Alg. 14.42).  The lazy form returns r in [0, 3q); the
// exact form subtracts q up to twice.
// Montgomery product (R = 2^64) of a, b < q < 2^62 with qn = -q^-1 mod 2^64:
// m = (a b mod R) qn mod R makes a b + m q divisible by R, and
// t = (a b + m q) / R < q^2 / R + q < 2q is congruent to a b R^-1 mod q.
// The low words of a b and m q sum to 0 mod R, so their carry is 1 exactly
// when the low word of a b is nonzero.
NTT_HD uint64_t mont_mul(uint64_t a, uint64_t b, uint64_t q, uint64_t qn) {
    const uint64_t lo = a * b, hi = mulhi64(a, b);
    const uint64_t m = lo * qn;
    return hi + mulhi64(m, q) + (lo != 0 ? 1u : 0u);
}

NTT_HD uint64_t barrett_mulmod_lazy(uint64_t a, uint64_t b, uint64_t q, uint64_t mu, uint32_t k) {
    uint64_t lo = a * b;
    uint64_t hi = mulhi64(a, b);
    uint32_t sh = k - 1;
    uint64_t q1 = sh == 0 ? lo : ((lo >> sh) | (hi << (64 - sh)));
    uint64_t plo = q1 * mu;
    uint64_t phi = mulhi64(q1, mu);
    uint32_t sh2 = k + 1;
    uint64_t q3 = (plo >> sh2) | (phi << (64 - sh2));
    return lo - q3 * q;   // [0, 3q)
}

NTT_HD uint64_t barrett_mulmod(uint64_t a, uint64_t b, uint64_t q, uint64_t mu, uint32_t k) {
    return csub(csub(barrett_mulmod_lazy(a, b, q, mu, k), q), q);   // [0, 3q) -> [0, q)
}

}  // namespace nttgb
