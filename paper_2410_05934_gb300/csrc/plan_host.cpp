// Host side of ntt_plan: argument validation, the number theory that fixes
// psi (arxiv 2410.05934, Sec. II-D: psi is a primitive 2N-th root of unity
// mod q, which needs q prime and q = 1 mod 2N) and the twiddle tables.
//
// Twiddles follow the merged-psi negacyclic layout of Eq. 1: forward entry
// k = psi^{brv(k)}, inverse entry k = psi^{-brv(k)} (brv over log2 N bits),
// each with its Shoup companion w' = floor(w 2^64 / q).
#include <algorithm>
#include <cstring>

#include "ntt_internal.h"

namespace nttgb {

typedef unsigned __int128 u128;

uint64_t mul_mod(uint64_t a, uint64_t b, uint64_t q) { return (uint64_t)((u128)a * b % q); }

uint64_t pow_mod(uint64_t a, uint64_t e, uint64_t q) {
    uint64_t acc = 1 % q;
    a %= q;
    for (; e; e >>= 1) {
        if (e & 1) acc = mul_mod(acc, a, q);
        a = mul_mod(a, a, q);
    }
    return acc;
}

// Deterministic Miller-Rabin for 64-bit n with the seven bases found by
// J. Sinclair (2, 325, 9375, 28178, 450775, 9780504, 1795265022), which
// admit no strong pseudoprime below 2^64.
bool is_prime_u64(uint64_t n) {
    if (n < 2) return false;
    static const uint64_t small[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    for (uint64_t p : small) {
        if (n == p) return true;
        if (n % p == 0) return false;
    }
    uint64_t d = n - 1;
    unsigned s = __builtin_ctzll(d);
    d >>= s;
    static const uint64_t bases[] = {2, 325, 9375, 28178, 450775, 9780504, 1795265022};
    for (uint64_t b : bases) {
        uint64_t a = b % n;
        if (a == 0) continue;
        uint64_t x = pow_mod(a, d, n);
        if (x == 1 || x == n - 1) continue;
        bool witness = true;
        for (unsigned i = 1; i < s && witness; ++i) {
            x = mul_mod(x, x, n);
            if (x == n - 1) witness = false;
        }
        if (witness) return false;
    }
    return true;
}

// Jacobi symbol (a/n) for odd n > 0 by quadratic reciprocity (binary form).
int jacobi(uint64_t a, uint64_t n) {
    a %= n;
    int t = 1;
    while (a != 0) {
        while ((a & 1) == 0) {
            a >>= 1;
            uint64_t r = n & 7;
            if (r == 3 || r == 5) t = -t;
        }
        uint64_t tmp = a;
        a = n;
        n = tmp;
        if ((a & 3) == 3 && (n & 3) == 3) t = -t;
        a %= n;
    }
    return n == 1 ? t : 0;
}

// psi = g^((q-1)/2N) with g the least quadratic non-residue (Jacobi = -1).
// Returns 0 if q is not a prime = 1 mod 2N.
uint64_t root_2n(uint64_t q, uint32_t log2n) {
    uint64_t two_n = 2ull << log2n;
    if (!is_prime_u64(q) || q < 3 || (q - 1) % two_n) return 0;
    uint64_t g = 2;
    while (jacobi(g, q) != -1) ++g;
    uint64_t psi = pow_mod(g, (q - 1) / two_n, q);
    // psi^N must be -1: then the order of psi is exactly 2N
    if (pow_mod(psi, two_n / 2, q) != q - 1) return 0;
    return psi;
}

uint64_t shoup_of(uint64_t w, uint64_t q) { return (uint64_t)(((u128)w << 64) / q); }

// Shoup companions of many w for one q without a 128-bit division each:
// with c = floor(2^64 / q) and r0 = 2^64 mod q,
//   floor(w 2^64 / q) = w c + floor(w r0 / q),
// and floor(w r0 / q) is the Shoup quotient of w * r0 (r0' = floor(r0 2^64 / q)),
// exact after one correction step.  w c < 2^64 because w < q.
struct ShoupGen {
    uint64_t q, c, r0, r0p;
    explicit ShoupGen(uint64_t q_) : q(q_) {
        c = (uint64_t)(((u128)1 << 64) / q);
        r0 = (uint64_t)(((u128)1 << 64) % q);
        r0p = shoup_of(r0, q);
    }
    uint64_t operator()(uint64_t w) const {
        uint64_t Q = (uint64_t)(((u128)w * r0p) >> 64);
        uint64_t rem = w * r0 - Q * q;   // exact remainder + {0, q}
        if (rem >= q) ++Q;
        return w * c + Q;
    }
};

// a * w mod q for a fixed w in Shoup form (exact)
static inline uint64_t shoup_mulmod(uint64_t a, uint64_t w, uint64_t wp, uint64_t q) {
    uint64_t Q = (uint64_t)(((u128)a * wp) >> 64);
    uint64_t r = a * w - Q * q;
    return r >= q ? r - q : r;
}

static uint32_t brv(uint32_t x, uint32_t bits) {
    uint32_t r = 0;
    for (uint32_t i = 0; i < bits; ++i, x >>= 1) r = (r << 1) | (x & 1);
    return r;
}

static uint32_t bit_length(uint64_t x) { return x ? 64u - (uint32_t)__builtin_clzll(x) : 0u; }

int build_plan_host(PlanHost& h, uint32_t log2n, const uint64_t* moduli, uint32_t n_moduli,
                    uint32_t batch, uint32_t flags) {
    if (log2n < NTT_MIN_LOG2N || log2n > NTT_MAX_LOG2N) return NTT_ERR_ARG;
    if (!moduli || n_moduli == 0 || batch == 0) return NTT_ERR_ARG;
    if (flags & ~(NTT_FLAG_HOST_ONLY | NTT_FLAG_CHECK | NTT_FLAG_NATURAL_ORDER | NTT_FLAG_WORD32 |
                  NTT_FLAG_OTF_TWIDDLES))
        return NTT_ERR_ARG;
    const bool word32 = (flags & NTT_FLAG_WORD32) != 0;
    if (word32 && ((flags & NTT_FLAG_NATURAL_ORDER) || log2n > NTT_WORD32_MAX_LOG2N)) return NTT_ERR_UNSUPPORTED;
    if ((flags & NTT_FLAG_OTF_TWIDDLES) &&
        ((flags & (NTT_FLAG_NATURAL_ORDER | NTT_FLAG_WORD32)) || log2n < NTT_OTF_MIN_LOG2N))
        return NTT_ERR_UNSUPPORTED;
    const uint64_t n = 1ull << log2n;
    const u128 total = (u128)batch * n_moduli * n;
    if (total >= ((u128)1 << 40)) return NTT_ERR_ARG;
    if (word32 && (u128)batch * n_moduli >= ((u128)1 << 32)) return NTT_ERR_ARG;
    for (uint32_t l = 0; l < n_moduli; ++l) {
        uint64_t q = moduli[l];
        if (q >= (1ull << NTT_MAX_MODULUS_BITS)) return NTT_ERR_MODULUS_TOO_LARGE;
        if (word32 && q >= (1ull << NTT_WORD32_MAX_MODULUS_BITS)) return NTT_ERR_MODULUS_TOO_LARGE;
        if (!is_prime_u64(q)) return NTT_ERR_NOT_PRIME;
        if ((q - 1) % (2 * n)) return NTT_ERR_NOT_NTT_FRIENDLY;
    }
    h.log2n = log2n;
    h.n_moduli = n_moduli;
    h.batch = batch;
    h.flags = flags;
    h.rows = (uint64_t)batch * n_moduli;
    h.moduli.assign(moduli, moduli + n_moduli);
    h.psi.resize(n_moduli);
    h.fwd.resize((size_t)n_moduli * n);
    h.inv.resize((size_t)n_moduli * n);
    h.consts.resize(n_moduli);
    h.mc = 2;
    for (uint32_t l = 0; l < n_moduli; ++l) {
        if (moduli[l] >= (1ull << NTT_SMALL_MODULUS_BITS)) h.mc = 0;
        else if (moduli[l] >= (1ull << NTT_LAZY_MODULUS_BITS) && h.mc == 2) h.mc = 1;
    }
    std::vector<uint64_t> pw(n), pwi(n);
    std::vector<uint32_t> rev(n);
    for (uint64_t k = 0; k < n; ++k) rev[k] = brv((uint32_t)k, log2n);
    for (uint32_t l = 0; l < n_moduli; ++l) {
        const uint64_t q = moduli[l];
        // repeated moduli share their tables
        uint32_t same = l;
        for (uint32_t m = 0; m < l; ++m)
            if (moduli[m] == q) { same = m; break; }
        TwPair* f = &h.fwd[(size_t)l * n];
        TwPair* v = &h.inv[(size_t)l * n];
        if (same != l) {
            std::copy(&h.fwd[(size_t)same * n], &h.fwd[(size_t)same * n] + n, f);
            std::copy(&h.inv[(size_t)same * n], &h.inv[(size_t)same * n] + n, v);
            h.psi[l] = h.psi[same];
            h.consts[l] = h.consts[same];
            continue;
        }
        const uint64_t psi = root_2n(q, log2n);
        if (!psi) return NTT_ERR_NOT_NTT_FRIENDLY;
        const uint64_t psi_inv = pow_mod(psi, 2 * n - 1, q);
        h.psi[l] = psi;
        const uint64_t psi_p = shoup_of(psi, q), psi_inv_p = shoup_of(psi_inv, q);
        pw[0] = pwi[0] = 1;
        for (uint64_t i = 1; i < n; ++i) {
            pw[i] = shoup_mulmod(pw[i - 1], psi, psi_p, q);
            pwi[i] = shoup_mulmod(pwi[i - 1], psi_inv, psi_inv_p, q);
        }
        const ShoupGen sg(q);
        for (uint64_t k = 0; k < n; ++k) {
            const uint32_t b = rev[k];
            f[k].w = pw[b];
            f[k].wp = sg(pw[b]);
            v[k].w = pwi[b];
            v[k].wp = sg(pwi[b]);
        }
        LimbConst& c = h.consts[l];
        std::memset(&c, 0, sizeof(c));
        c.q = q;
        c.two_q = 2 * q;
        c.four_q = 4 * q;
        c.one_p = shoup_of(1, q);
        c.ninv = pow_mod(n % q, q - 2, q);
        c.ninv_p = shoup_of(c.ninv, q);
        c.w1ninv = mul_mod(v[1].w, c.ninv, q);
        c.w1ninv_p = shoup_of(c.w1ninv, q);
        {
            uint64_t inv = q;                      // q^-1 mod 2^64 by Newton: each step doubles the correct bits
            for (int it = 0; it < 6; ++it) inv *= 2 - q * inv;
            c.qn = 0 - inv;
        }
        c.bits = bit_length(q);
        c.mu = (uint64_t)(((u128)1 << (2 * c.bits)) / q);
        c.red2_m = (uint32_t)(((u128)1 << (32 + (c.bits > 18 ? c.bits - 18 : 0))) / q);
        {
            const uint32_t sh = c.bits > 25 ? c.bits - 25 : 0;
            c.red_m = (uint32_t)(((u128)1 << (32 + sh)) / q);
        }
        if (l + 1 < n_moduli) {      // Rescale drops the last modulus: its inverse mod q
            const uint64_t ql = moduli[n_moduli - 1] % q;
            c.rs_inv = ql ? pow_mod(ql, q - 2, q) : 0;
            c.rs_inv_p = shoup_of(c.rs_inv, q);
        }
    }
    // the inverse after Montgomery products: last-stage scale N^-1 2^64
    h.consts_mont = h.consts;
    for (LimbConst& c : h.consts_mont) {
        const uint64_t r = (uint64_t)(((u128)1 << 64) % c.q);
        c.ninv = mul_mod(c.ninv, r, c.q);
        c.ninv_p = shoup_of(c.ninv, c.q);
        c.w1ninv = mul_mod(c.w1ninv, r, c.q);
        c.w1ninv_p = shoup_of(c.w1ninv, c.q);
    }
    if (flags & NTT_FLAG_OTF_TWIDDLES) {
        // per limb: psi^(+-lo), lo < 2^LO, then psi^(+-hi 2^LO); table entry
        // k of the full tables holds the power brv(k), so power e sits at brv(e)
        const int LO = otf_lo_bits((int)log2n);
        const uint32_t per = otf_entries((int)log2n);
        h.otf_fwd.resize((size_t)n_moduli * per);
        h.otf_inv.resize((size_t)n_moduli * per);
        for (uint32_t l = 0; l < n_moduli; ++l) {
            const TwPair* f = &h.fwd[(size_t)l * n];
            const TwPair* v = &h.inv[(size_t)l * n];
            for (uint32_t i = 0; i < per; ++i) {
                const uint32_t e = i < (1u << LO) ? i : (i - (1u << LO)) << LO;
                h.otf_fwd[(size_t)l * per + i] = f[rev[e]];
                h.otf_inv[(size_t)l * per + i] = v[rev[e]];
            }
        }
    }
    if (word32) {      // 32-bit tables: w' = floor(w 2^32 / q)
        auto sp32 = [](uint64_t w, uint64_t q) { return (uint32_t)((w << 32) / q); };
        h.fwd32.resize(h.fwd.size());
        h.inv32.resize(h.inv.size());
        for (size_t k = 0; k < h.fwd.size(); ++k) {
            const uint64_t q = moduli[k >> log2n];
            // N = 1024 tables are stored with each stage >= 5 transposed (the
            // one-warp-per-row kernel's order, tw1024_perm)
            const size_t pos = log2n == 10 ? ((k >> 10) << 10) + tw1024_perm((uint32_t)(k & 1023)) : k;
            h.fwd32[pos] = Tw32{(uint32_t)h.fwd[k].w, sp32(h.fwd[k].w, q)};
            h.inv32[pos] = Tw32{(uint32_t)h.inv[k].w, sp32(h.inv[k].w, q)};
        }
        h.consts32.resize(n_moduli);
        for (uint32_t l = 0; l < n_moduli; ++l) {
            const LimbConst& c = h.consts[l];
            LimbConst32& d = h.consts32[l];
            d.q = (uint32_t)c.q;
            d.two_q = (uint32_t)c.two_q;
            d.ninv = (uint32_t)c.ninv;
            d.ninv_p = sp32(c.ninv, c.q);
            d.w1ninv = (uint32_t)c.w1ninv;
            d.w1ninv_p = sp32(c.w1ninv, c.q);
            d.mu = (uint64_t)(((u128)1 << 64) / c.q);
        }
    }
    return NTT_OK;
}

// ---- RNS basis conversion constants (rns.cuh layout) ----

// Fills the constant block; validates the moduli (odd primes < 2^62,
// pairwise distinct within and across the two bases).
int bconv_constants(const uint64_t* q_from, uint32_t L, const uint64_t* p_to, uint32_t K,
                    std::vector<uint64_t>& w, uint32_t& chunk) {
    if (!q_from || !p_to || L == 0 || K == 0 || L > NTT_BCONV_MAX_MODULI || K > NTT_BCONV_MAX_MODULI)
        return NTT_ERR_ARG;
    std::vector<uint64_t> all(q_from, q_from + L);
    all.insert(all.end(), p_to, p_to + K);
    for (uint64_t m : all) {
        if (m >= (1ull << 62)) return NTT_ERR_MODULUS_TOO_LARGE;
        if (m < 3 || !is_prime_u64(m)) return NTT_ERR_NOT_PRIME;
    }
    for (uint32_t i = 0; i < L; ++i)
        for (uint32_t k = i + 1; k < L; ++k)
            if (q_from[i] == q_from[k]) return NTT_ERR_ARG;
    for (uint32_t j = 0; j < K; ++j)
        for (uint32_t k = j + 1; k < K; ++k)
            if (p_to[j] == p_to[k]) return NTT_ERR_ARG;
    w.assign((size_t)3 * L + 4 * K + (size_t)L * K, 0);
    uint64_t* q = w.data();
    uint64_t *qhi = q + L, *qhi_p = q + 2 * L, *p = q + 3 * L;
    uint64_t *p_one = p + K, *r64 = p + 2 * K, *r64_p = p + 3 * K, *c = p + 4 * K;
    uint64_t maxq = 0, maxp = 0;
    for (uint32_t i = 0; i < L; ++i) {
        q[i] = q_from[i];
        maxq = std::max(maxq, q[i]);
        // Qhat_i mod q_i, then its inverse (q_i prime: a^(q-2))
        uint64_t h = 1;
        for (uint32_t k = 0; k < L; ++k)
            if (k != i) h = mul_mod(h, q_from[k] % q[i], q[i]);
        qhi[i] = pow_mod(h, q[i] - 2, q[i]);
        qhi_p[i] = shoup_of(qhi[i], q[i]);
    }
    for (uint32_t j = 0; j < K; ++j) {
        p[j] = p_to[j];
        maxp = std::max(maxp, p[j]);
        p_one[j] = shoup_of(1, p[j]);
        r64[j] = (uint64_t)(((u128)1 << 64) % p[j]);
        r64_p[j] = shoup_of(r64[j], p[j]);
        for (uint32_t i = 0; i < L; ++i) {
            uint64_t h = 1;
            for (uint32_t k = 0; k < L; ++k)
                if (k != i) h = mul_mod(h, q_from[k] % p[j], p[j]);
            c[(size_t)i * K + j] = h;
        }
    }
    // terms of one 128-bit sum: chunk * (maxq - 1) * (maxp - 1) < 2^128
    const u128 term = (u128)(maxq - 1) * (maxp - 1);
    const u128 n = ~(u128)0 / (term ? term : 1);
    chunk = (uint32_t)std::min<u128>(n, (u128)(L + 1));
    return chunk >= 2 ? NTT_OK : NTT_ERR_ARG;
}

}  // namespace nttgb
