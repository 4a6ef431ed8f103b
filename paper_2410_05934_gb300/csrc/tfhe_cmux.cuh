// TFHE external product and CMux step, batched over ciphertexts that share
// one RGSW key (the batched CMux gate of Sec. IV-A; the blind rotation of
// Sec. II-B repeats it once per LWE coefficient).  One CTA takes one RLWE
// ciphertext (B(x), A(x)) at a time, entirely on chip:
//
//   slot s (threads [s T, (s + 1) T)) owns input polynomial s:
//     load    v = x^a d_s - d_s (CMux) or v = d_s (external product) at its
//             coefficients, and t = round(v B^l / q) mod B^l once per value
//     level j = 0..l-1:  signed digit e_j of t (mod q)
//             -> forward NTT in shared memory (the tile phases of the NTT)
//             -> MAC: acc_c += NTT(e_j) * K[s l + j][c] for c = 0, 1
//   output s  the two slots' partial sums of output s, added after a barrier
//             (key rows in Shoup form: products and sums stay in [0, 2q);
//             the sums live in shared memory)
//   output    INTT of acc_s (slot s), plus d_s for the CMux, stored
//
// The digits never leave the SM, the key is read once per ciphertext from
// L2, and HBM sees 16 bytes in and 16 bytes out per coefficient.  Every step
// is a pure function of (thread, shared memory, global memory), so the host
// emulation runs this same code thread by thread with checked indices.
#pragma once
#include "ntt_tile.cuh"

namespace nttgb {

struct CmuxArgs {
    const uint64_t* in;       // [n_ct][2][N]: d (external product) or acc (CMux)
    const uint32_t* rot;      // [n_ct] exponents a (taken mod 2N), or null for the external product
    const TwPair* key;        // [2 levels][2][N] RGSW rows in the NTT domain, {w, floor(w 2^64 / q)}
    uint64_t* out;            // [n_ct][2][N]
    int* status;
    uint64_t q, half_q;       // q and floor(q / 2)
    uint64_t m;               // floor(2^(64 + sigma) / q), sigma = floor(log2 q)
    uint64_t n_ct;
    uint32_t sigma, levels, log2_base, check;
};

// 8 coefficients per thread, passes of up to 3 fused stages, two slots.
// Shared memory (words): [slot 0 row][slot 1 row][partial sums (slot s,
// output c) at (2 + 2 s + c) N]; the MAC sums live in shared memory, not in
// registers, so three CTAs fit on an SM; twiddles come through the
// read-only cache.
template <int LOGN_, int MC_>
struct CmuxCfg {
    static constexpr int LOGN = LOGN_, MC = MC_;
    static constexpr int LOGT = LOGN - 3;
    using F = TileCfg<LOGN, 0, LOGN, 0, LOGT, 3, 1, false, MC, 2>;
    using I = TileCfg<LOGN, 0, LOGN, 0, LOGT, 3, 1, true, MC, 2>;
    static constexpr int N = 1 << LOGN, T = F::T, R = F::R, THREADS = 2 * T;
    static constexpr size_t SMEM_BYTES = sizeof(uint64_t) * (size_t)(6 * N);
    static constexpr int MIN_CTAS = THREADS <= 256 ? 3 : 1;      // register budget: 85 per thread
    static_assert(F::E == N && !F::TWS && !I::TWS, "one whole row per slot, read-only-cache twiddles");
    static constexpr size_t acc_off(int s, int c) { return (size_t)(2 + 2 * s + c) * N; }
};

template <class K>
struct CmuxRegs {
    uint32_t dig[K::R];        // the signed digits of each coefficient, log2_base bits per level
};

// round(v 2^bl / q) mod 2^bl for v < q < 2^62, bl = levels * log2_base <= 32
// and 2^bl < q.  e = floor(v m / 2^64) >> (sigma - bl) is at most 3 below
// Q = floor((v 2^bl + floor(q/2)) / q), so r = v 2^bl + floor(q/2) - e q lies
// in [0, 4q) < 2^64 and wrapping 64-bit arithmetic gives it exactly.
NTT_HD uint32_t cmux_round_top(uint64_t v, const CmuxArgs& c) {
    const uint32_t bl = c.levels * c.log2_base;
    uint64_t e = mulhi64(v, c.m) >> (c.sigma - bl);
    uint64_t r = (v << bl) + c.half_q - e * c.q;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (r >= c.q) {
            r -= c.q;
            ++e;
        }
    }
    return (uint32_t)(e & ((1ull << bl) - 1));
}

// the signed digits e_0..e_(l-1) of t (e_0 most significant), packed as
// log2_base-bit two's-complement fields, level j at bit j * log2_base
NTT_HD uint32_t cmux_pack_digits(uint32_t top, const CmuxArgs& c) {
    const uint64_t base = 1ull << c.log2_base, half = base >> 1, mask = base - 1;
    uint64_t t = top;
    uint64_t packed = 0;
    for (int k = (int)c.levels - 1; k >= 0; --k) {
        const uint64_t d = t & mask;
        t >>= c.log2_base;
        if (d >= half) t += 1;                        // e = d - B, carried into the next level
        packed |= d << (c.log2_base * (uint32_t)k);   // d mod B is e's two's-complement field
    }
    return (uint32_t)packed;
}

// digit j of a packed word, as a residue mod q
NTT_HD uint64_t cmux_digit(uint32_t packed, uint32_t j, const CmuxArgs& c) {
    const uint32_t sh = c.log2_base * j;
    const uint64_t d = ((uint64_t)packed >> sh) & ((1ull << c.log2_base) - 1);
    const uint64_t half = 1ull << (c.log2_base - 1);
    return d < half ? d : c.q - ((1ull << c.log2_base) - d);
}

// coefficient k = 2t + 2iT + h of the slot's row <-> register 2i + h (the
// pair layout of the tile phases, for a tile that is one whole row)
template <class K>
NTT_HD void cmux_load(CmuxRegs<K>& cr, const CmuxArgs& c, uint64_t ct, int s, int t, uint64_t* smem) {
    const uint64_t* row = c.in + ((ct * 2 + (uint64_t)s) << K::LOGN);
    const uint32_t a = c.rot ? (c.rot[ct] & (2u * K::N - 1u)) : 0u;
    bool bad = false;
#pragma unroll
    for (int i = 0; i < K::R / 2; ++i) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const uint32_t k = 2u * (uint32_t)t + 2u * (uint32_t)i * K::T + (uint32_t)h;
            NTT_GMEM_CHECK(k, K::N);
            uint64_t v = row[k];
            bad |= v >= c.q;
            if (c.rot) {
                // (x^a d)[k] = d[e] for e = (k - a) mod 2N < N, else -d[e - N]
                const uint32_t e = (k - a) & (2u * K::N - 1u);
                NTT_GMEM_CHECK(e & (K::N - 1u), K::N);
                const uint64_t w = row[e & (K::N - 1u)];
                bad |= w >= c.q;
                const uint64_t rv = e < (uint32_t)K::N ? w : (w ? c.q - w : 0);
                v = rv >= v ? rv - v : rv + (c.q - v);
            }
            cr.dig[2 * i + h] = cmux_pack_digits(cmux_round_top(v, c), c);
        }
    }
    if (c.check && bad) record_status(c.status, NTT_STATUS_RANGE);
    // this thread's positions of the slot's two partial sums start at zero
    uint64_t* acc0 = smem + K::acc_off(s, 0);
    uint64_t* acc1 = smem + K::acc_off(s, 1);
    const uint32_t b = swz(2u * (uint32_t)t);
#pragma unroll
    for (int i = 0; i < K::R / 2; ++i) {
        const uint32_t cc = swz(2u * (uint32_t)i * K::T);
        NTT_SMEM_CHECK(b ^ cc, K::N);
        acc0[b ^ cc] = acc0[(b ^ cc) ^ 1u] = 0;
        acc1[b ^ cc] = acc1[(b ^ cc) ^ 1u] = 0;
    }
}

template <class K>
NTT_HD void cmux_digits(TileRegs<typename K::F>& st, const CmuxRegs<K>& cr, uint32_t j, const CmuxArgs& c) {
#pragma unroll
    for (int r = 0; r < K::R; ++r) st.x[r] = cmux_digit(cr.dig[r], j, c);
}

// forward result of level j (the slot's row, any lazy range below 2^64)
// times key row p in Shoup form, added to the slot's partial sums (each
// product in [0, 2q), sums kept in [0, 2q) since q < 2^62).  Every thread
// reads and writes only its own positions.
template <class K>
NTT_HD void cmux_mac(const CmuxArgs& c, const LimbConst& lc, uint32_t p, int s, int t, uint64_t* smem) {
    const TwPair* k0 = c.key + ((uint64_t)(2u * p) << K::LOGN);
    const TwPair* k1 = k0 + K::N;
    const uint64_t* sm = smem + (size_t)s * K::N;
    uint64_t* acc0 = smem + K::acc_off(s, 0);
    uint64_t* acc1 = smem + K::acc_off(s, 1);
    const uint32_t b = swz(2u * (uint32_t)t);
#pragma unroll
    for (int i = 0; i < K::R / 2; ++i) {
        const uint32_t cc = swz(2u * (uint32_t)i * K::T);
        const uint32_t e0 = b ^ cc, e1 = e0 ^ 1u;
        NTT_SMEM_CHECK(e0, K::N);
        const uint64_t x = sm[e0], y = sm[e1];
        const uint32_t k = 2u * (uint32_t)t + 2u * (uint32_t)i * K::T;
        NTT_GMEM_CHECK(k + 1, K::N);
        const TwPair a0 = load_tw(k0, k), a1 = load_tw(k0, k + 1);
        const TwPair b0 = load_tw(k1, k), b1 = load_tw(k1, k + 1);
        acc0[e0] = csub(acc0[e0] + shoup_mul(x, a0.w, a0.wp, lc.q), lc.two_q);
        acc0[e1] = csub(acc0[e1] + shoup_mul(y, a1.w, a1.wp, lc.q), lc.two_q);
        acc1[e0] = csub(acc1[e0] + shoup_mul(x, b0.w, b0.wp, lc.q), lc.two_q);
        acc1[e1] = csub(acc1[e1] + shoup_mul(y, b1.w, b1.wp, lc.q), lc.two_q);
    }
}

// after a barrier: output s = partial sum of slot 0 + partial sum of slot 1,
// canonical, into the inverse's registers (pair layout)
template <class K>
NTT_HD void cmux_inverse_input(TileRegs<typename K::I>& st, const LimbConst& lc, int s, int t, const uint64_t* smem) {
    const uint64_t* p0 = smem + K::acc_off(0, s);
    const uint64_t* p1 = smem + K::acc_off(1, s);
    const uint32_t b = swz(2u * (uint32_t)t);
#pragma unroll
    for (int i = 0; i < K::R / 2; ++i) {
        const uint32_t cc = swz(2u * (uint32_t)i * K::T);
        const uint32_t e0 = b ^ cc, e1 = e0 ^ 1u;
        NTT_SMEM_CHECK(e0, K::N);
        st.x[2 * i] = csub(csub(p0[e0], lc.q) + csub(p1[e0], lc.q), lc.q);
        st.x[2 * i + 1] = csub(csub(p0[e1], lc.q) + csub(p1[e1], lc.q), lc.q);
    }
}

// inverse result (shared memory) -> canonical, plus d_s for the CMux -> out
template <class K>
NTT_HD void cmux_store(const CmuxArgs& c, const LimbConst& lc, uint64_t ct, int s, int t, const uint64_t* sm) {
    const uint64_t off = (ct * 2 + (uint64_t)s) << K::LOGN;
    const uint64_t* base = c.in + off;
    uint64_t* dst = c.out + off;
    const uint32_t b = swz(2u * (uint32_t)t);
#pragma unroll
    for (int i = 0; i < K::R / 2; ++i) {
        const uint32_t cc = swz(2u * (uint32_t)i * K::T);
        NTT_SMEM_CHECK(b ^ cc, K::N);
        uint64_t x = sm[b ^ cc], y = sm[(b ^ cc) ^ 1u];
        if (K::MC == 1) {   // [0, 4q) -> [0, q)
            x = csub(csub(x, lc.two_q), lc.q);
            y = csub(csub(y, lc.two_q), lc.q);
        } else {            // [0, 2q) -> [0, q)
            x = csub(x, lc.q);
            y = csub(y, lc.q);
        }
        const uint32_t k = 2u * (uint32_t)t + 2u * (uint32_t)i * K::T;
        NTT_GMEM_CHECK(k + 1, K::N);
        if (c.rot) {
            uint64_t ax, ay;
            load_pair(base + k, ax, ay);
            x = csub(x + ax, lc.q);
            y = csub(y + ay, lc.q);
        }
        store_pair(dst + k, x, y);
    }
}

}  // namespace nttgb
