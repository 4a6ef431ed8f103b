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
//   exchange  slot s hands acc_(1-s) to the other slot, adds the one it gets
//             (key rows in Shoup form: products and sums stay in [0, 2q))
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
// Shared memory (words): [slot 0 row][slot 1 row][forward twiddles][inverse
// twiddles]; the twiddles are staged once per CTA (every ciphertext uses the
// same tables) in the tile phases' slot order (slot i = table entry i + 1
// for a tile that is one whole row), and each slot's TileLoc points its
// pass twiddles there through tw_off.
template <int LOGN_, int MC_>
struct CmuxCfg {
    static constexpr int LOGN = LOGN_, MC = MC_;
    static constexpr int LOGT = LOGN - 3;
    using F = TileCfg<LOGN, 0, LOGN, 0, LOGT, 3, 1, false, MC, 0>;
    using I = TileCfg<LOGN, 0, LOGN, 0, LOGT, 3, 1, true, MC, 0>;
    static constexpr int N = 1 << LOGN, T = F::T, R = F::R, THREADS = 2 * T;
    static constexpr int TW_WORDS = 2 * (N - 1);                 // N - 1 TwPairs
    static constexpr int FWD_TW = 2 * N, INV_TW = 2 * N + TW_WORDS;
    static constexpr size_t SMEM_BYTES = sizeof(uint64_t) * (size_t)(2 * N + 2 * TW_WORDS);
    static constexpr int MIN_CTAS = THREADS <= 256 ? 2 : 1;      // register budget: 128 per thread
    static_assert(F::E == N && F::TWS && I::TWS, "one whole row per slot, twiddles staged in shared memory");
    // tw_off of slot s: from the slot's row + E to the twiddle region
    static constexpr int32_t tw_off(int s, bool inv) { return (1 - s) * N + (inv ? TW_WORDS : 0); }
};

// all threads of the CTA: both tables into their regions
template <class K>
NTT_HD void cmux_stage_twiddles(const TwPair* fwd, const TwPair* inv, int tid, uint64_t* smem) {
    TwPair* f = reinterpret_cast<TwPair*>(smem + K::FWD_TW);
    TwPair* v = reinterpret_cast<TwPair*>(smem + K::INV_TW);
    for (int i = tid; i < K::N - 1; i += K::THREADS) {
        NTT_GMEM_CHECK(i + 1, K::N);
        f[i] = load_tw(fwd, (uint32_t)i + 1u);
        v[i] = load_tw(inv, (uint32_t)i + 1u);
    }
}

template <class K>
struct CmuxRegs {
    uint32_t dig[K::R];        // the signed digits of each coefficient, log2_base bits per level
    uint64_t acc[2][K::R];     // lazy sums of outputs 0 and 1 (pair layout), each < 2 levels q
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
NTT_HD void cmux_load(CmuxRegs<K>& cr, const CmuxArgs& c, uint64_t ct, int s, int t) {
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
#pragma unroll
    for (int r = 0; r < K::R; ++r) cr.acc[0][r] = cr.acc[1][r] = 0;
}

template <class K>
NTT_HD void cmux_digits(TileRegs<typename K::F>& st, const CmuxRegs<K>& cr, uint32_t j, const CmuxArgs& c) {
#pragma unroll
    for (int r = 0; r < K::R; ++r) st.x[r] = cmux_digit(cr.dig[r], j, c);
}

// forward result of level j (shared memory, any lazy range below 2^64) times
// key row p in Shoup form: each product lies in [0, 2q) and the sums are
// kept in [0, 2q) (q < 2^62, so sum + product < 4q < 2^64)
template <class K>
NTT_HD void cmux_mac(CmuxRegs<K>& cr, const CmuxArgs& c, const LimbConst& lc, uint32_t p, int t,
                     const uint64_t* sm) {
    const TwPair* k0 = c.key + ((uint64_t)(2u * p) << K::LOGN);
    const TwPair* k1 = k0 + K::N;
    const uint32_t b = swz(2u * (uint32_t)t);
#pragma unroll
    for (int i = 0; i < K::R / 2; ++i) {
        const uint32_t cc = swz(2u * (uint32_t)i * K::T);
        NTT_SMEM_CHECK(b ^ cc, K::N);
        const uint64_t x = sm[b ^ cc], y = sm[(b ^ cc) ^ 1u];
        const uint32_t k = 2u * (uint32_t)t + 2u * (uint32_t)i * K::T;
        NTT_GMEM_CHECK(k + 1, K::N);
        const TwPair a0 = load_tw(k0, k), a1 = load_tw(k0, k + 1);
        const TwPair b0 = load_tw(k1, k), b1 = load_tw(k1, k + 1);
        cr.acc[0][2 * i] = csub(cr.acc[0][2 * i] + shoup_mul(x, a0.w, a0.wp, lc.q), lc.two_q);
        cr.acc[0][2 * i + 1] = csub(cr.acc[0][2 * i + 1] + shoup_mul(y, a1.w, a1.wp, lc.q), lc.two_q);
        cr.acc[1][2 * i] = csub(cr.acc[1][2 * i] + shoup_mul(x, b0.w, b0.wp, lc.q), lc.two_q);
        cr.acc[1][2 * i + 1] = csub(cr.acc[1][2 * i + 1] + shoup_mul(y, b1.w, b1.wp, lc.q), lc.two_q);
    }
}

// a lazy sum in [0, 2q) to [0, q)
NTT_HD uint64_t cmux_reduce(uint64_t x, const LimbConst& lc) { return csub(x, lc.q); }

// Slot s hands the other output's partial sums over through its own tile
// and adds what the other slot handed it (same thread index, same
// positions).  The accumulator of each slot is picked with a branch, so the
// arrays stay in registers.
template <class K>
NTT_HD void cmux_put_pairs(const uint64_t (&v)[K::R], int t, uint64_t* sm) {
    const uint32_t b = swz(2u * (uint32_t)t);
#pragma unroll
    for (int i = 0; i < K::R / 2; ++i) {
        const uint32_t cc = swz(2u * (uint32_t)i * K::T);
        NTT_SMEM_CHECK(b ^ cc, K::N);
        sm[b ^ cc] = v[2 * i];
        sm[(b ^ cc) ^ 1u] = v[2 * i + 1];
    }
}

template <class K>
NTT_HD void cmux_add_pairs(uint64_t (&v)[K::R], const LimbConst& lc, int t, const uint64_t* sm) {
    const uint32_t b = swz(2u * (uint32_t)t);
#pragma unroll
    for (int i = 0; i < K::R / 2; ++i) {
        const uint32_t cc = swz(2u * (uint32_t)i * K::T);
        NTT_SMEM_CHECK(b ^ cc, K::N);
        v[2 * i] = csub(cmux_reduce(v[2 * i], lc) + cmux_reduce(sm[b ^ cc], lc), lc.q);
        v[2 * i + 1] = csub(cmux_reduce(v[2 * i + 1], lc) + cmux_reduce(sm[(b ^ cc) ^ 1u], lc), lc.q);
    }
}

template <class K>
NTT_HD void cmux_exchange_put(const CmuxRegs<K>& cr, int s, int t, uint64_t* sm) {
    if (s == 0)
        cmux_put_pairs<K>(cr.acc[1], t, sm);
    else
        cmux_put_pairs<K>(cr.acc[0], t, sm);
}

template <class K>
NTT_HD void cmux_exchange_get(CmuxRegs<K>& cr, const LimbConst& lc, int s, int t, const uint64_t* sm_other) {
    if (s == 0)
        cmux_add_pairs<K>(cr.acc[0], lc, t, sm_other);
    else
        cmux_add_pairs<K>(cr.acc[1], lc, t, sm_other);
}

template <class K>
NTT_HD void cmux_inverse_input(TileRegs<typename K::I>& st, const CmuxRegs<K>& cr, int s) {
#pragma unroll
    for (int r = 0; r < K::R; ++r) st.x[r] = s == 0 ? cr.acc[0][r] : cr.acc[1][r];
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
