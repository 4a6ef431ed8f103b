// 32-bit-word transform for moduli below 2^30 (the TFHE-size primes, Sec.
// II-B mentions 32-bit TFHE moduli): coefficients and twiddles are uint32,
// a Shoup product is one 32-bit low multiply, one 32-bit high multiply and
// one more low multiply (against ~20 multiply-pipe slots for the 64-bit
// butterfly), and Harvey's bounds fit because 4q < 2^32.
//
// One kernel per transform, one whole row per tile (N <= 2^12), 8
// coefficients per thread: the tile geometry (pass layout, swizzle, twiddle
// indices) is the one of the 64-bit tile kernels (ntt_tile.cuh), applied to
// 32-bit words.  Host and device, like the 64-bit phases.
#pragma once
#include "ntt_tile.cuh"

namespace nttgb {

struct alignas(8) Tw32 {
    uint32_t w, wp;             // wp = floor(w 2^32 / q)
};

struct LimbConst32 {
    uint32_t q, two_q;
    uint32_t ninv, ninv_p;      // N^-1 and its Shoup form
    uint32_t w1ninv, w1ninv_p;  // psi^{-brv(1)} N^-1 and its Shoup form
    uint64_t mu;                // floor(2^64 / q): Barrett constant of the pointwise product
};

struct Args32 {
    const uint32_t* in;
    uint32_t* out;
    const Tw32* tw;             // [n_moduli][N]
    const LimbConst32* lc;      // [n_moduli]
    int* status;
    uint32_t row_begin, n_rows; // rows of this launch (plan layout)
    uint32_t n_moduli, check;
    uint64_t mod_magic;         // ceil(2^64 / n_moduli)
};

NTT_HD uint32_t mulhi32(uint32_t a, uint32_t b) {
#if defined(__CUDA_ARCH__)
    return __umulhi(a, b);
#else
    return (uint32_t)(((uint64_t)a * b) >> 32);
#endif
}

// y w mod q lazily, in [0, 2q) for any y < 2^32
NTT_HD uint32_t shoup32(uint32_t y, uint32_t w, uint32_t wp, uint32_t q) { return y * w - mulhi32(y, wp) * q; }
// x in [0, 2m) -> [0, m) as min(x, x - m): for x < m the difference wraps
// above 2^31 > x, so one subtraction and one unsigned minimum do it
// (In the transform kernels this form measured 7 % faster than compare and
// select; in a loop of nothing but butterflies the compare form is faster:
// probe kind 8.)
NTT_HD uint32_t csub32(uint32_t x, uint32_t m) {
#if defined(__CUDA_ARCH__)
    return umin(x, x - m);
#else
    const uint32_t d = x - m;
    return d < x ? d : x;
#endif
}

// Harvey CT: [0, 4q) -> [0, 4q)
NTT_HD void ct32(uint32_t& X, uint32_t& Y, Tw32 w, uint32_t q, uint32_t two_q) {
    const uint32_t x = csub32(X, two_q);
    const uint32_t t = shoup32(Y, w.w, w.wp, q);
    X = x + t;
    Y = x - t + two_q;
}

// Harvey GS: [0, 2q) -> [0, 2q); the stage-0 variant folds N^-1 in
NTT_HD void gs32(uint32_t& X, uint32_t& Y, Tw32 w, uint32_t q, uint32_t two_q) {
    const uint32_t s = csub32(X + Y, two_q);
    const uint32_t d = X - Y + two_q;
    Y = shoup32(d, w.w, w.wp, q);
    X = s;
}

NTT_HD void gs32_scaled(uint32_t& X, uint32_t& Y, const LimbConst32& c) {
    const uint32_t s = X + Y, d = X - Y + c.two_q;   // [0, 4q)
    X = shoup32(s, c.ninv, c.ninv_p, c.q);
    Y = shoup32(d, c.w1ninv, c.w1ninv_p, c.q);
}

NTT_HD Tw32 load_tw32(const Tw32* tw, uint32_t k) {
#if defined(__CUDA_ARCH__)
    const uint2 v = __ldg(reinterpret_cast<const uint2*>(tw) + k);
    return Tw32{v.x, v.y};
#else
    return tw[k];
#endif
}

// Shared-memory slot of tile element e for 32-bit words: 32 four-byte banks,
// so the higher 5-bit groups of e are XOR-folded into its low 5 bits (the
// 64-bit tiles fold 4-bit groups onto 16 eight-byte bank pairs).  A bijection,
// linear over GF(2), and swz32(e + 1) = swz32(e) ^ 1 for even e.
NTT_HD constexpr uint32_t swz32(uint32_t e) { return e ^ (((e >> 5) ^ (e >> 10)) & 31u); }

// The thread layout of pass P with the lane-bit exchanges that make its
// accesses conflict-free: the 5 lane bits land on e-bits of distinct
// residues mod 5.
template <class C, int P>
struct Pass32Geom {
    using Gm = PassGeom<C, P>;
    static constexpr uint64_t SWAPS = pass_swaps_g(Gm::PE, Gm::r, C::LOGT, 5);
    static NTT_HD constexpr uint32_t et(uint32_t t) {
        return spread(SWAPS ? swap_thread_bits_g(t, SWAPS) : t, Gm::PE, Gm::r);
    }
};

// one whole row per tile: C = TileCfg<LOGN, 0, LOGN, 0, LOGT, 3, TPC, INV, 1, 2> for the geometry
template <class C>
struct Regs32 {
    uint32_t x[C::R];
};

struct Loc32 {
    uint32_t row, limb;
    bool valid;
};

template <class C>
NTT_HD Loc32 locate32(const Args32& a, uint32_t cta, int tin) {
    Loc32 L;
    const uint32_t r = cta * (uint32_t)C::TPC + (uint32_t)tin;
    L.valid = r < a.n_rows;
    L.row = a.row_begin + (L.valid ? r : 0u);
    const uint32_t rq = a.n_moduli == 1 ? L.row : fdiv32(L.row, a.mod_magic, a.n_moduli);
    L.limb = a.n_moduli == 1 ? 0u : L.row - rq * a.n_moduli;
    return L;
}

// global -> registers (pair layout: thread t holds k = 2t + 2iT and k + 1)
// -> swizzled shared memory
template <class C>
NTT_HD void load32(Regs32<C>& st, const Args32& a, const Loc32& L, int t, uint32_t* sm) {
    if (!L.valid) return;
    const uint32_t* src = a.in + ((uint64_t)L.row << C::LOGN);
    const uint32_t q = a.lc[L.limb].q;
    bool bad = false;
#pragma unroll
    for (int i = 0; i < C::R / 2; ++i) {
        const uint32_t k = 2u * (uint32_t)t + 2u * (uint32_t)i * C::T;
        NTT_GMEM_CHECK(k + 1, 1u << C::LOGN);
#if defined(__CUDA_ARCH__)
        const uint2 v = *reinterpret_cast<const uint2*>(src + k);
        st.x[2 * i] = v.x;
        st.x[2 * i + 1] = v.y;
#else
        st.x[2 * i] = src[k];
        st.x[2 * i + 1] = src[k + 1];
#endif
        bad |= st.x[2 * i] >= q || st.x[2 * i + 1] >= q;
    }
    if (a.check && bad) record_status(a.status, NTT_STATUS_RANGE);
    const uint32_t b = swz32(2u * (uint32_t)t);
#pragma unroll
    for (int i = 0; i < C::R / 2; ++i) {
        const uint32_t c = swz32(2u * (uint32_t)i * C::T);
        NTT_SMEM_CHECK(b ^ c, C::E);
        sm[b ^ c] = st.x[2 * i];
        sm[(b ^ c) ^ 1u] = st.x[2 * i + 1];
    }
}

// pass P: read its registers, run its fused stages, write them back
template <class C, int P>
NTT_HD void pass32(Regs32<C>& st, const Args32& a, const Loc32& L, int t, uint32_t* sm) {
    if (!L.valid) return;
    using Gm = PassGeom<C, P>;
    using G32 = Pass32Geom<C, P>;
    constexpr int S_LO = Gm::S_LO, r = Gm::r, GS = Gm::GS;
    const uint32_t et = G32::et((uint32_t)t);
    const uint32_t b = swz32(et);
#pragma unroll
    for (int j = 0; j < C::R; ++j) {
        const uint32_t addr = b ^ swz32(Gm::ej(j));
        NTT_SMEM_CHECK(addr, C::E);
        st.x[j] = sm[addr];
    }
    const LimbConst32 lc = a.lc[L.limb];
    const Tw32* tw = a.tw + ((uint64_t)L.limb << C::LOGN);
    constexpr int SH = C::LOGN - S_LO;
    const uint32_t pre_t = place<C>(et) >> SH;
#pragma unroll
    for (int gi = 0; gi < Gm::G; ++gi) {
        const uint32_t pre = pre_t | (place<C>(Gm::ej(gi * GS)) >> SH);
        uint32_t* x = st.x + gi * GS;
        if (!C::INV) {
#pragma unroll
            for (int v = 0; v < r; ++v) {
                const int s = S_LO + v;
                const int d = 1 << (r - 1 - v);
                const uint32_t k0 = (1u << s) + (pre << v);
#pragma unroll
                for (int jl = 0; jl < GS; ++jl) {
                    if (jl & d) continue;
                    const uint32_t k = k0 + ((uint32_t)jl >> (r - v));
                    NTT_GMEM_CHECK(k, 1u << C::LOGN);
                    ct32(x[jl], x[jl + d], load_tw32(tw, k), lc.q, lc.two_q);
                }
            }
        } else {
#pragma unroll
            for (int v = r - 1; v >= 0; --v) {
                const int s = S_LO + v;
                const int d = 1 << (r - 1 - v);
                const uint32_t k0 = (1u << s) + (pre << v);
#pragma unroll
                for (int jl = 0; jl < GS; ++jl) {
                    if (jl & d) continue;
                    if (s == 0) {
                        gs32_scaled(x[jl], x[jl + d], lc);
                    } else {
                        const uint32_t k = k0 + ((uint32_t)jl >> (r - v));
                        NTT_GMEM_CHECK(k, 1u << C::LOGN);
                        gs32(x[jl], x[jl + d], load_tw32(tw, k), lc.q, lc.two_q);
                    }
                }
            }
        }
    }
#pragma unroll
    for (int j = 0; j < C::R; ++j) {
        const uint32_t addr = b ^ swz32(Gm::ej(j));
        sm[addr] = st.x[j];
    }
}

// shared memory -> canonical -> global
template <class C>
NTT_HD void store32(const Args32& a, const Loc32& L, int t, const uint32_t* sm) {
    if (!L.valid) return;
    uint32_t* dst = a.out + ((uint64_t)L.row << C::LOGN);
    const uint32_t q = a.lc[L.limb].q, two_q = a.lc[L.limb].two_q;
    const uint32_t b = swz32(2u * (uint32_t)t);
#pragma unroll
    for (int i = 0; i < C::R / 2; ++i) {
        const uint32_t c = swz32(2u * (uint32_t)i * C::T);
        uint32_t x = sm[b ^ c], y = sm[(b ^ c) ^ 1u];
        if (!C::INV) {          // [0, 4q) -> [0, q)
            x = csub32(csub32(x, two_q), q);
            y = csub32(csub32(y, two_q), q);
        } else {                // [0, 2q) -> [0, q)
            x = csub32(x, q);
            y = csub32(y, q);
        }
        const uint32_t k = 2u * (uint32_t)t + 2u * (uint32_t)i * C::T;
        NTT_GMEM_CHECK(k + 1, 1u << C::LOGN);
#if defined(__CUDA_ARCH__)
        *reinterpret_cast<uint2*>(dst + k) = make_uint2(x, y);
#else
        dst[k] = x;
        dst[k + 1] = y;
#endif
    }
}

// c = a b mod q for a, b < q < 2^30: p = a b < 2^60, p - floor(p mu / 2^64) q in [0, 2q)
NTT_HD uint32_t mulmod32(uint32_t x, uint32_t y, const LimbConst32& c) {
    const uint64_t p = (uint64_t)x * y;
    return csub32((uint32_t)(p - mulhi64(p, c.mu) * c.q), c.q);
}

// ---- N = 1024: one warp per row, two passes of five stages ----
// Lane t holds 32 coefficients.  Layout A: x[j] = element t + 32 j (lane bits
// = e-bits 0..4, registers = e-bits 5..9), which a coalesced load or store
// of consecutive words gives directly; stages 0..4 pair registers j and
// j + 2^(4 - s), with twiddle 2^s + (j >> (5 - s)) shared by all lanes.
// Layout B: x[j] = element 32 t + j (registers = e-bits 0..4); stages 5..9
// pair j and j + 2^(9 - s) with twiddle 2^s + t 2^(s - 5) + (j >> (10 - s)).
// The plan stores the N = 1024 tables with each stage s >= 5 transposed,
// entry 2^s + t 2^(s - 5) + i at 2^s + 32 i + t, so the 32 lanes' twiddles
// of one load are consecutive words.  The two layouts meet in shared
// memory through slot(e) = e ^ ((e >> 5) & 31): both the lanes of a layout-A
// access (e-bits 0..4 = t) and of a layout-B access (e = 32 t + j) hit 32
// distinct banks.  Only the row's own warp touches the row's words, so
// __syncwarp orders the exchanges.
NTT_HD constexpr uint32_t slot1024(uint32_t e) { return e ^ ((e >> 5) & 31u); }
NTT_HD constexpr uint32_t tw1024_pos(uint32_t s, uint32_t t, uint32_t i) { return (1u << s) + 32u * i + t; }

// table position of canonical entry k of a N = 1024 table (the transpose above)
NTT_HD constexpr uint32_t tw1024_perm(uint32_t k) {
    uint32_t s = 0;
    while ((2u << s) <= k) ++s;
    if (s < 5) return k;
    const uint32_t o = k - (1u << s), per = 1u << (s - 5);
    return tw1024_pos(s, o / per, o % per);
}

struct Row1024 {
    uint32_t x[32];
};

// row of warp w of CTA cta (four rows per CTA)
NTT_HD Loc32 locate1024(const Args32& a, uint32_t cta, int w) {
    Loc32 L;
    const uint32_t r = cta * 4u + (uint32_t)w;
    L.valid = r < a.n_rows;
    L.row = a.row_begin + (L.valid ? r : 0u);
    const uint32_t rq = a.n_moduli == 1 ? L.row : fdiv32(L.row, a.mod_magic, a.n_moduli);
    L.limb = a.n_moduli == 1 ? 0u : L.row - rq * a.n_moduli;
    return L;
}

// Twiddle entry k of a N = 1024 phase: from the CTA's shared-memory copy of
// the table when the launch has a single modulus (SMTW), else from global
// memory through the read-only path.
template <bool SMTW>
NTT_HD Tw32 tw1024(const Tw32* tws, const Tw32* tw, uint32_t k) {
    if (SMTW) {
        NTT_SMEM_CHECK(k, 1024);
        return tws[k];
    }
    return load_tw32(tw, k);
}

// forward, phase 2: layout B from shared memory, stages 5..9, canonical,
// back to shared memory in place (each lane rewrites only the words it read)
template <bool SMTW = false>
NTT_HD void w1024_fwd_b(Row1024& r, const Args32& a, const Loc32& L, int t, uint32_t* sm,
                        const Tw32* tws = nullptr) {
    if (!L.valid) return;
    const LimbConst32 lc = a.lc[L.limb];
    const Tw32* tw = a.tw + ((uint64_t)L.limb << 10);
#pragma unroll
    for (int j = 0; j < 32; ++j) r.x[j] = sm[slot1024(32 * t + j)];
#pragma unroll
    for (int s = 5; s < 10; ++s) {
        const int d = 1 << (9 - s);
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            if (j & d) continue;
            NTT_GMEM_CHECK(tw1024_pos(s, t, (uint32_t)j >> (10 - s)), 1024);
            ct32(r.x[j], r.x[j + d], tw1024<SMTW>(tws, tw, tw1024_pos(s, t, (uint32_t)j >> (10 - s))), lc.q, lc.two_q);
        }
    }
#pragma unroll
    for (int j = 0; j < 32; ++j) sm[slot1024(32 * t + j)] = csub32(csub32(r.x[j], lc.two_q), lc.q);
}

// store phase (both directions' forward output / the inverse's input
// transpose): shared memory in layout A -> consecutive words of the row
NTT_HD void w1024_store(const Args32& a, const Loc32& L, int t, const uint32_t* sm) {
    if (!L.valid) return;
    uint32_t* dst = a.out + ((uint64_t)L.row << 10);
#pragma unroll
    for (int j = 0; j < 32; ++j) dst[t + 32 * j] = sm[slot1024(t + 32 * j)];
}

// inverse, phase 2: layout B, GS stages 9..5, back in place
template <bool SMTW = false>
NTT_HD void w1024_inv_b(Row1024& r, const Args32& a, const Loc32& L, int t, uint32_t* sm,
                        const Tw32* tws = nullptr) {
    if (!L.valid) return;
    const LimbConst32 lc = a.lc[L.limb];
    const Tw32* tw = a.tw + ((uint64_t)L.limb << 10);
#pragma unroll
    for (int j = 0; j < 32; ++j) r.x[j] = sm[slot1024(32 * t + j)];
#pragma unroll
    for (int s = 9; s >= 5; --s) {
        const int d = 1 << (9 - s);
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            if (j & d) continue;
            gs32(r.x[j], r.x[j + d], tw1024<SMTW>(tws, tw, tw1024_pos(s, t, (uint32_t)j >> (10 - s))), lc.q, lc.two_q);
        }
    }
#pragma unroll
    for (int j = 0; j < 32; ++j) sm[slot1024(32 * t + j)] = r.x[j];
}

// inverse, phase 3: layout A, GS stages 4..0 (stage 0 with N^-1), canonical, coalesced store
template <bool SMTW = false>
NTT_HD void w1024_inv_c(Row1024& r, const Args32& a, const Loc32& L, int t, const uint32_t* sm,
                        const Tw32* tws = nullptr) {
    if (!L.valid) return;
    const LimbConst32 lc = a.lc[L.limb];
    const Tw32* tw = a.tw + ((uint64_t)L.limb << 10);
#pragma unroll
    for (int j = 0; j < 32; ++j) r.x[j] = sm[slot1024(t + 32 * j)];
#pragma unroll
    for (int s = 4; s >= 0; --s) {
        const int d = 16 >> s;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            if (j & d) continue;
            if (s == 0)
                gs32_scaled(r.x[j], r.x[j + d], lc);
            else
                gs32(r.x[j], r.x[j + d], tw1024<SMTW>(tws, tw, (1u << s) + ((uint32_t)j >> (5 - s))), lc.q, lc.two_q);
        }
    }
    uint32_t* dst = a.out + ((uint64_t)L.row << 10);
#pragma unroll
    for (int j = 0; j < 32; ++j) dst[t + 32 * j] = csub32(r.x[j], lc.q);
}

// ---- N = 1024, persistent warps with the next rows' loads in flight ----
// A warp walks a list of rows (forward or inverse, one per quad of the
// combined row space).  Row k lands in landing buffer k mod 2 in natural
// order through 16-byte cp.async copies issued two rows ahead; the compute
// phases then read it from shared memory, so the loads of the next row
// overlap the butterflies of this one.  Layout A reads of the natural order
// (word t + 32 j, lane t) hit 32 distinct banks.  The warp's work buffer
// holds the slot layout of the phases above.

NTT_HD void async_commit() {
#if defined(__CUDA_ARCH__)
    asm volatile("cp.async.commit_group;" ::: "memory");
#endif
}

// waits until at most one committed group of this thread is pending
NTT_HD void async_wait_prev() {
#if defined(__CUDA_ARCH__)
    asm volatile("cp.async.wait_group 1;" ::: "memory");
#endif
}

// row L of a (1024 words) -> landing buffer, lane t copying words
// 4 (t + 32 i) .. 4 (t + 32 i) + 3 (512 contiguous bytes per copy round)
NTT_HD void w1024_prefetch(const Args32& a, const Loc32& L, int t, uint32_t* land) {
    if (!L.valid) return;
    const uint32_t* src = a.in + ((uint64_t)L.row << 10);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const uint32_t w = 4u * ((uint32_t)t + 32u * (uint32_t)i);
        NTT_GMEM_CHECK(w + 3, 1024);
        NTT_SMEM_CHECK(w + 3, 1024);
        async_copy16(land + w, src + w);
    }
}

// forward, phase 1 from the landing buffer: layout A, range check, stages 0..4
template <bool SMTW = false>
NTT_HD void w1024_fwd_a_land(Row1024& r, const Args32& a, const Loc32& L, int t, const uint32_t* land,
                             const Tw32* tws = nullptr) {
    if (!L.valid) return;
    const LimbConst32 lc = a.lc[L.limb];
    const Tw32* tw = a.tw + ((uint64_t)L.limb << 10);
#pragma unroll
    for (int j = 0; j < 32; ++j) {
        NTT_SMEM_CHECK(t + 32 * j, 1024);
        r.x[j] = land[t + 32 * j];
    }
    if (a.check) {      // the range check costs its compares only when asked for
        bool bad = false;
#pragma unroll
        for (int j = 0; j < 32; ++j) bad |= r.x[j] >= lc.q;
        if (bad) record_status(a.status, NTT_STATUS_RANGE);
    }
#pragma unroll
    for (int s = 0; s < 5; ++s) {
        const int d = 16 >> s;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            if (j & d) continue;
            ct32(r.x[j], r.x[j + d], tw1024<SMTW>(tws, tw, (1u << s) + ((uint32_t)j >> (5 - s))), lc.q, lc.two_q);
        }
    }
}

// layout A registers -> the work buffer's slot layout
NTT_HD void w1024_write_a(const Row1024& r, const Loc32& L, int t, uint32_t* work) {
    if (!L.valid) return;
#pragma unroll
    for (int j = 0; j < 32; ++j) {
        NTT_SMEM_CHECK(slot1024(t + 32 * j), 1024);
        work[slot1024(t + 32 * j)] = r.x[j];
    }
}

// inverse, phase 1 from the landing buffer: range check, natural -> slot layout
NTT_HD void w1024_inv_a_land(const Args32& a, const Loc32& L, int t, const uint32_t* land, uint32_t* work) {
    if (!L.valid) return;
    const uint32_t q = a.lc[L.limb].q;
    bool bad = false;
#pragma unroll
    for (int j = 0; j < 32; ++j) {
        NTT_SMEM_CHECK(t + 32 * j, 1024);
        const uint32_t v = land[t + 32 * j];
        if (a.check) bad |= v >= q;
        work[slot1024(t + 32 * j)] = v;
    }
    if (bad) record_status(a.status, NTT_STATUS_RANGE);
}

// The row list of warp w of CTA `cta` in a grid of `grid` CTAs: its k-th row
// is row w of quad cta + k grid of the combined space (quads [0, quads_i)
// inverse rows of ai, the rest forward rows of af).
struct W1024Pick {
    bool live;      // the quad exists
    bool inv;
    Loc32 L;
};
NTT_HD W1024Pick w1024_pick(const Args32& af, const Args32& ai, uint32_t quads_i, uint32_t quads, uint32_t cta,
                            uint32_t grid, uint32_t k, int w) {
    W1024Pick p;
    const uint64_t qd = (uint64_t)cta + (uint64_t)k * grid;
    p.live = qd < quads;
    p.inv = qd < quads_i;
    const uint32_t qq = p.live ? (uint32_t)qd : 0u;
    p.L = p.inv ? locate1024(ai, qq, w) : locate1024(af, qq - quads_i, w);
    p.L.valid = p.L.valid && p.live;
    return p;
}

// the 32-bit configuration of a ring size: 8 coefficients per thread (or the
// whole row for N <= 8), passes of up to 3 stages, 128-thread CTAs (one row
// per CTA at N = 1024, so that a batch of a few hundred rows still spreads
// over every SM)
template <int LOGN, bool INV>
struct Cfg32Sel {
    static constexpr int LOGT = LOGN > 3 ? LOGN - 3 : 0;
    static constexpr int TPC = (128 >> LOGT) > 0 ? (128 >> LOGT) : 1;
    using C = TileCfg<LOGN, 0, LOGN, 0, LOGT, 3, TPC, INV, 1, 2>;
};

}  // namespace nttgb
