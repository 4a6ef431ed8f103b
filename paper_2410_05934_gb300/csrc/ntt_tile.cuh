// Tile phases of the batched negacyclic NTT kernels (arxiv 2410.05934,
// Sec. II-D Eq. 1 for what is computed; Sec. V for the fused-stage idea).
//
// A transform of one row runs its log2 N butterfly stages in one or two
// kernels.  A kernel performs the contiguous stage range [S0, S1) on "tiles":
// sets of elements that those stages only mix among themselves.  With
// A = S1 - S0 and LOGLO = LOGN - S1, a tile is
//     g(e) = (hi << (LOGN - S0)) | (a << LOGLO) | (lo_base + p),
//     e = (a << LOGP) | p,   a in [0, 2^A),  p in [0, 2^LOGP)
// i.e. 2^A "active" positions times 2^LOGP adjacent passive columns.  A
// single-kernel schedule has S0 = 0, S1 = LOGN, LOGP = 0 (one row per tile);
// a two-kernel schedule runs a column kernel over [0, SPLIT) then a row
// kernel over [SPLIT, LOGN) (the PCS/OSSP split of Sec. V-C/V-D becomes a
// kernel boundary here).
//
// Each tile lives in shared memory; 2^LOGT threads own it, R = E / 2^LOGT
// elements each.  Stages are fused in groups of up to LOGRP ("passes",
// the thread-aggregation idea of Sec. V-B with radix 2^LOGRP per thread): a
// pass loads a thread's R elements from shared memory into registers, runs
// its stages there with no synchronisation, and writes them back.
//
// Two kernel forms share these phases:
//   - direct: each CTA loads its tiles with 16-byte loads into registers and
//     stores them swizzled;
//   - pipelined (PIPE): a persistent CTA streams its tile groups through two
//     shared-memory buffers with bulk asynchronous copies (cp.async.bulk +
//     mbarrier), so the next group's data and twiddles arrive while the
//     current group computes; data land in natural order and are re-laid
//     out into the swizzled order before the first pass.
//
// Every phase is a function of (thread, its register state, shared memory,
// global memory) with barriers only between phases, so the same code runs on
// the host as an emulation (see emulate.cpp), thread by thread.
//
// Twiddle table (one per modulus, N entries of {w, w'}): entry k = 2^s + i is
// psi^{brv(k)} (forward) or psi^{-brv(k)} (inverse) for stage s, group i.
// A butterfly of stage s on element index g uses k = 2^s + (g >> (LOGN - s)).
#pragma once
#include <stdint.h>
#include "ntt_arith.cuh"

#if !defined(__CUDA_ARCH__)
#include <cstdio>
#include <cstdlib>
#include <cstring>
#endif

namespace nttgb {

struct alignas(16) TwPair {
    uint64_t w, wp;
};

struct LimbConst {
    uint64_t q, two_q, four_q;
    uint64_t one_p;             // floor(2^64 / q): Shoup form of 1
    uint64_t ninv, ninv_p;      // N^-1 mod q and its Shoup form
    uint64_t w1ninv, w1ninv_p;  // psi^{-brv(1)} N^-1 and its Shoup form (last GS stage)
    uint64_t mu;                // Barrett constant floor(2^(2 bits) / q)
    uint64_t rs_inv, rs_inv_p;  // q_last^-1 mod q and its Shoup form (Rescale; 0 for the last limb)
    uint32_t bits;              // bit length of q
    uint32_t red_m;             // floor(2^(32 + red_sh) / q), red_sh = max(bits - 25, 0): reduce_65q
    uint64_t qn;                // -q^-1 mod 2^64: Montgomery products of the fused operators, whose
                                // inverse runs on a copy of the constants with ninv, w1ninv times 2^64
    uint32_t red2_m;            // floor(2^(32 + max(bits - 18, 0)) / q): reduce_lazy
    uint32_t pad_;
};

// Modulus classes: 0 = any q < 2^62 (exact Shoup quotient, Harvey bounds),
// 1 = q < 2^57 (approximate quotient, 4q-wide lazy bounds, no conditional
// subtraction in the forward transform).
#define NTT_SMALL_MODULUS_BITS 57
// 2 = q < 2^50: as class 1, and the inverse's kernels of at most 11 stages
// skip the conditional subtraction of the GS sum (values grow at most 2x per
// stage), ending a kernel that is not the last with one reduce_lazy.
#define NTT_LAZY_MODULUS_BITS 50

#ifndef NTT_MUL_MAX_MAPPED
#define NTT_MUL_MAX_MAPPED 32     // polynomials of one ntt_inverse_mul call with index maps
#endif

struct TileArgs {
    const uint64_t* in;
    uint64_t* out;
    const TwPair* tw;       // [n_moduli][N]
    const LimbConst* lc;    // [n_moduli]
    int* status;            // device status word (may be null)
    uint64_t row_begin;     // first row (plan layout) of this launch
    uint64_t n_tiles;       // tiles covered by this launch
    uint32_t n_moduli;
    uint32_t check;         // verify canonical inputs (first kernel only)
    uint32_t fast32;        // tile and row indices below 2^32: use the reciprocal below
    uint64_t mod_magic;     // ceil(2^64 / n_moduli)  (n_moduli >= 2)
    // source mode: 0 = read `in`;
    // 1 (first kernel of an inverse) = CKKS tensor product, row r = k * n_moduli + l
    //   computes d_k of limb l from in = [a0; a1] and in_b = [b0; b1] (each
    //   [2][n_moduli][N], NTT domain): d0 = a0 b0, d1 = a0 b1 + a1 b0, d2 = a1 b1;
    // 2 (forward) = Rescale by the modulus aux_q: row r = p * n_moduli + i of
    //   the output reads the coefficients w of the dropped limb of polynomial p
    //   from in (row p) and transforms c = (h - [w + h]_aux_q) mod q_i,
    //   h = floor(aux_q / 2); the last kernel adds row p * (n_moduli + 1) + i
    //   of in_b (the NTT-domain input) and multiplies by aux_q^-1 mod q_i
    uint32_t src_mode;
    const uint64_t* in_b;
    uint64_t aux_q;
    // natural order (full-row tiles only): the forward's last kernel stores
    // A[brv(j)] at j, the inverse's first kernel takes its input that way
    uint32_t nat;
    // source mode 3 (first kernel of an inverse) = pointwise product: row
    // p * n_moduli + l reads row a_map[p] * n_moduli + l of `in` and row
    // b_map[p] * n_moduli + l of `in_b` (with has_map = 0: polynomial p of
    // both) and transforms their product mod q_l
    uint32_t has_map;
    uint8_t a_map[NTT_MUL_MAX_MAPPED], b_map[NTT_MUL_MAX_MAPPED];
    // on-the-fly twiddles (MODE 3): per limb otf_entries(LOGN) pairs, first
    // psi^(+-lo) for lo < 2^otf_lo_bits, then psi^(+-hi 2^otf_lo_bits)
    const TwPair* otf;
    // rows of `in` skipped between two input rows of the first kernel (source
    // mode 0): row r reads in + r (1 + in_skip) N, e.g. every L-th row of a
    // multi-limb layout; the other kernels and `out` stay contiguous
    uint32_t in_skip;
};

// on-the-fly twiddle tables of a ring of 2^logn: e = hi 2^lo_bits + lo
NTT_HD constexpr int otf_lo_bits(int logn) { return (logn + 1) / 2; }
NTT_HD constexpr uint32_t otf_entries(int logn) {
    return (1u << otf_lo_bits(logn)) + (1u << (logn - otf_lo_bits(logn)));
}

// floor(n / d) for n < 2^32 and 2 <= d < 2^32 from M = ceil(2^64 / d):
// n M / 2^64 exceeds n / d by less than n / 2^64 < 2^-32, while a non-integer
// n / d is at least 1/d > 2^-32 below the next integer, so the floor is
// exact; the 32 x 64-bit product is taken in two halves.
NTT_HD uint32_t fdiv32(uint32_t n, uint64_t M, uint32_t d) {
    if (d == 1) return n;
    const uint32_t mh = (uint32_t)(M >> 32), ml = (uint32_t)M;
#if defined(__CUDA_ARCH__)
    const uint64_t t = (uint64_t)n * mh + __umulhi(n, ml);
#else
    const uint64_t t = (uint64_t)n * mh + (((uint64_t)n * ml) >> 32);
#endif
    return (uint32_t)(t >> 32);
}

inline uint64_t fdiv_magic(uint64_t d) {
    return d < 2 ? 0 : (uint64_t)((((unsigned __int128)1 << 64) + d - 1) / d);
}

#define NTT_STATUS_RANGE (-8)
#define NTT_STATUS_TIMEOUT (-7)

// Swizzled shared-memory slot of tile element e: XOR-folds the higher 4-bit
// groups of e into its low 4 bits, which spreads the strided accesses of the
// later passes over the 16 eight-byte bank pairs.  A bijection on every
// 16-aligned block, hence on the tile.  It is linear over GF(2):
// swz(a ^ b) = swz(a) ^ swz(b), which the phases use to split an address
// into a per-thread part and a compile-time part.
NTT_HD constexpr uint32_t swz(uint32_t e) {
    return e ^ (((e >> 4) ^ (e >> 8) ^ (e >> 12)) & 15u);
}

// Places the bits of x around an r-bit hole at position pe (linear in x).
// the low `bits` bits of k reversed
NTT_HD uint32_t brv_bits(uint32_t k, int bits) {
#if defined(__CUDA_ARCH__)
    return bits == 0 ? 0u : __brev(k) >> (32 - bits);
#else
    uint32_t r = 0;
    for (int i = 0; i < bits; ++i) r |= ((k >> i) & 1u) << (bits - 1 - i);
    return r;
#endif
}

NTT_HD constexpr uint32_t spread(uint32_t x, int pe, int r) {
    return ((x >> pe) << (pe + r)) | (x & ((1u << pe) - 1));
}

// MODE: 0 = direct form (twiddles staged in shared memory when they fit),
//       1 = pipelined form, 2 = direct form reading twiddles through the
//           read-only path (no staging; the table stays in L1 when a batch
//           shares one modulus), 3 = direct form with on-the-fly twiddles:
//           psi^(+-e), e = brv(k), is applied as two Shoup products with
//           entries lo = e mod 2^OTF_LO and hi = e >> OTF_LO of two small
//           per-limb tables (TileArgs.otf).
// Kernel forms of a two-kernel schedule entry (its PIPE field): below 4 both
// kernels use it; A | B << 2 with B != 0 gives the column kernel form A and
// the row kernel form B.
constexpr int form_col(int f) { return f & 3; }
constexpr int form_row(int f) { return f < 4 ? f : (f >> 2) & 3; }

template <int LOGN_, int S0_, int S1_, int LOGP_, int LOGT_, int LOGRP_, int TPC_, bool INV_,
          int MC_ = 0, int MODE_ = 0>
struct TileCfg {
    static constexpr int LOGN = LOGN_, S0 = S0_, S1 = S1_, LOGP = LOGP_, LOGT = LOGT_;
    static constexpr int TPC = TPC_;
    static constexpr bool INV = INV_;
    static constexpr int MC = MC_;
    static constexpr int MODE = MODE_;
    static constexpr bool PIPE = MODE_ == 1;
    // class-2 inverse kernels run their GS stages without subtractions
    static constexpr bool LAZY_GS = MC_ == 2 && INV_ && S1_ - S0_ <= 11;
    static constexpr int A = S1 - S0;
    static constexpr int LOGLO = LOGN - S1;
    static constexpr int LOGE = A + LOGP;
    static constexpr int LOGR = LOGE - LOGT;
    static constexpr int R = 1 << LOGR;
    static constexpr int T = 1 << LOGT;
    static constexpr int E = 1 << LOGE;
    static constexpr int THREADS = T * TPC;
    static constexpr int RP = LOGRP_ < LOGR ? LOGRP_ : LOGR;   // stages per full pass
    static constexpr int NPASS = (A + RP - 1) / RP;
    static constexpr int LOGTPR = LOGN - LOGE;                 // log2 tiles per row
    static constexpr int LOGLOBLK = LOGLO - LOGP;
    // the first kernel of a transform reads the caller's (canonical) input,
    // the last writes canonical output
    static constexpr bool FIRST = INV ? (S1 == LOGN) : (S0 == 0);
    static constexpr bool LAST = INV ? (S0 == 0) : (S1 == LOGN);
    // Twiddles of a tile: stages [S0, S1) of one "hi" block need 2^(s-S0)
    // entries each, 2^A - 1 in all; they are staged in shared memory next to
    // the tile (always when pipelined, else when both fit comfortably) or
    // read through the read-only path.
    static constexpr size_t DATA_BYTES = sizeof(uint64_t) * (size_t)E;
    static constexpr size_t TW_BYTES = 16 * ((size_t)1 << A);
    static constexpr bool TWS = PIPE || (MODE_ == 0 && (DATA_BYTES + TW_BYTES) * TPC <= 160 * 1024);
    static constexpr size_t TILE_BYTES = DATA_BYTES + (TWS ? TW_BYTES : 0);
    static constexpr size_t TILE_WORDS = TILE_BYTES / sizeof(uint64_t);
    static constexpr int NBUF = PIPE ? 2 : 1;
    static constexpr size_t BUF_BYTES = TILE_BYTES * TPC;
    static constexpr size_t BUF_WORDS = BUF_BYTES / sizeof(uint64_t);
    static constexpr size_t BAR_OFFSET = BUF_BYTES * NBUF;      // mbarriers after the buffers
    static constexpr size_t SMEM_BYTES = BAR_OFFSET + (PIPE ? 16 : 0);
    // bulk copies of one tile: contiguous runs of 2^LOGP elements (one run
    // for row tiles) plus one run of twiddles per stage
    static constexpr int RUNS = LOGLO == 0 ? 1 : (1 << A);
    static constexpr uint32_t RUN_BYTES = (uint32_t)(LOGLO == 0 ? DATA_BYTES : (8u << LOGP));
    static constexpr int COPIES = RUNS + A;
    static constexpr uint32_t TILE_TX_BYTES = (uint32_t)(DATA_BYTES + 16u * ((1u << A) - 1));

    static_assert(A >= 1 && A <= LOGN, "stage range");
    static_assert(LOGLO >= LOGP, "passive columns must fit below the active bits");
    static_assert(LOGLO == 0 || LOGP >= 1, "column tiles need >= 2 adjacent columns");
    static_assert(LOGR >= 1, "each thread needs an element pair");
    static_assert(RP >= 1, "pass width");
    static_assert(SMEM_BYTES <= 227 * 1024, "shared memory per CTA");
};

// stage range [s_lo, s_lo + r) of pass p, passes numbered from the top index
// bits down (forward runs p = 0..NPASS-1, inverse runs p = NPASS-1..0)
template <class C>
NTT_HD void pass_range(int p, int& s_lo, int& r) {
    s_lo = C::S0 + p * C::RP;
    int rem = C::S1 - s_lo;
    r = rem < C::RP ? rem : C::RP;
}

struct TileLoc {
    uint64_t row;
    uint64_t rowq;      // row / n_moduli (polynomial index)
    uint32_t limb;
    uint32_t hi;
    uint32_t gbase;     // g(0): the tile's hi and lo_base bits
    int32_t tw_off;     // words from this tile's slot to the slot holding its twiddles
    bool valid;
};

// Tile order: tile = row * 2^LOGTPR + tau (tau = hi block, then lo block).
template <class C>
NTT_HD TileLoc locate(const TileArgs& a, uint64_t tile) {
    TileLoc L;
    L.valid = tile < a.n_tiles;
    uint64_t tl = L.valid ? tile : 0;
    const uint32_t tau = (uint32_t)(tl & ((1ull << C::LOGTPR) - 1));
    if (a.fast32) {
        const uint32_t row = (uint32_t)a.row_begin + (uint32_t)(tl >> C::LOGTPR);
        const uint32_t rq = fdiv32(row, a.mod_magic, a.n_moduli);
        L.row = row;
        L.rowq = rq;
        L.limb = row - rq * a.n_moduli;
    } else {
        L.row = a.row_begin + (tl >> C::LOGTPR);
        L.rowq = L.row / a.n_moduli;
        L.limb = (uint32_t)(L.row - L.rowq * a.n_moduli);
    }
    L.hi = tau >> C::LOGLOBLK;
    uint32_t lo_base = (tau & ((1u << C::LOGLOBLK) - 1)) << C::LOGP;
    L.gbase = (L.hi << (C::LOGN - C::S0)) | lo_base;
    L.tw_off = 0;
    return L;
}

// Twiddle leader of tile slot tin in group g: the first slot of the group
// that lies in the same run of tiles with equal (limb, hi); only leaders
// stage twiddles, the others read them from the leader's slot.  Runs in tile
// order: the 2^LOGLOBLK tiles of one hi block of a row, or all tiles when
// every tile has the same limb and hi (one modulus and a kernel starting at
// stage 0, e.g. a single-modulus batch of short polynomials).
template <class C>
NTT_HD int tw_leader(const TileArgs& a, uint64_t g, int tin) {
    const uint64_t t = g * C::TPC + tin;
    uint64_t start;
    if (a.n_moduli == 1 && C::S0 == 0) {
        start = 0;
    } else {
        start = t & ~((1ull << C::LOGLOBLK) - 1);
    }
    const uint64_t first = g * C::TPC;
    return (int)((start > first ? start : first) - first);
}

template <class C>
NTT_HD TileLoc locate_in_group(const TileArgs& a, uint64_t g, int tin) {
    TileLoc L = locate<C>(a, g * C::TPC + tin);
    if (C::TWS && C::TPC > 1 && L.valid) L.tw_off = (tw_leader<C>(a, g, tin) - tin) * (int32_t)C::TILE_WORDS;
    return L;
}

// bits of the row-local index g contributed by tile element e (linear in e):
// g(e) = gbase | place(e)
template <class C>
NTT_HD constexpr uint32_t place(uint32_t e) {
    return ((e >> C::LOGP) << C::LOGLO) | (e & ((1u << C::LOGP) - 1));
}

template <class C>
NTT_HD uint32_t gidx(const TileLoc& L, uint32_t e) {
    return L.gbase | place<C>(e);
}

#if defined(__CUDA_ARCH__)
#define NTT_SMEM_CHECK(i, n) ((void)0)
#define NTT_GMEM_CHECK(i, n) ((void)0)
#else
#define NTT_SMEM_CHECK(i, n)                                                          \
    do {                                                                              \
        if ((uint64_t)(i) >= (uint64_t)(n)) {                                         \
            fprintf(stderr, "emulation: smem index %llu >= %llu at %s:%d\n",          \
                    (unsigned long long)(i), (unsigned long long)(n), __FILE__, __LINE__); \
            abort();                                                                  \
        }                                                                             \
    } while (0)
#define NTT_GMEM_CHECK(i, n) NTT_SMEM_CHECK(i, n)
#endif

NTT_HD TwPair load_tw(const TwPair* tw, uint32_t k) {
#if defined(__CUDA_ARCH__)
    ulonglong2 v = __ldg(reinterpret_cast<const ulonglong2*>(tw) + k);
    return TwPair{v.x, v.y};
#else
    return tw[k];
#endif
}

NTT_HD void load_pair(const uint64_t* p, uint64_t& x, uint64_t& y) {
#if defined(__CUDA_ARCH__)
    ulonglong2 v = *reinterpret_cast<const ulonglong2*>(p);
    x = v.x;
    y = v.y;
#else
    x = p[0];
    y = p[1];
#endif
}

NTT_HD void store_pair(uint64_t* p, uint64_t x, uint64_t y) {
#if defined(__CUDA_ARCH__)
    *reinterpret_cast<ulonglong2*>(p) = make_ulonglong2(x, y);
#else
    p[0] = x;
    p[1] = y;
#endif
}

NTT_HD void record_status(int* status, int code) {
    if (!status) return;
#if defined(__CUDA_ARCH__)
    atomicCAS(status, 0, code);
#else
    if (*status == 0) *status = code;
#endif
}

NTT_HD uint32_t floor_log2(uint32_t x) {
#if defined(__CUDA_ARCH__)
    return 31u - (uint32_t)__clz(x);
#else
    return 31u - (uint32_t)__builtin_clz(x);
#endif
}

// Asynchronous 16-byte global -> shared copies (cp.async, completed by
// async_wait_all before the barrier that publishes the shared memory).  The
// host emulation copies at once.
NTT_HD void async_copy16(void* dst_smem, const void* src) {
#if defined(__CUDA_ARCH__)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst_smem)),
                 "l"(src)
                 : "memory");
#else
    memcpy(dst_smem, src, 16);
#endif
}

NTT_HD void async_wait_all() {
#if defined(__CUDA_ARCH__)
    asm volatile("cp.async.wait_all;" ::: "memory");
#endif
}

// Per-thread register state carried between phases.
template <class C>
struct TileRegs {
    uint64_t x[C::R];
};

// ---- load (direct form): global -> registers, 16-byte coalesced pairs ----
// Thread t holds the pairs e = 2 (t + i T) = 2t ^ 2iT (disjoint bits), so
// g(e) = (gbase | place(2t)) + place(2iT) with a compile-time second term.
template <class C>
NTT_HD void load_direct(TileRegs<C>& st, const TileArgs& a, const TileLoc& L, int t, uint64_t* sm) {
    if (!L.valid) return;
    if (C::TWS && L.tw_off == 0) {
        // the tile's 2^A - 1 twiddles: slot i <-> stage S0 + d, d = floor(log2(i + 1)),
        // copied asynchronously so that they arrive while the data loads below are in
        // flight (the caller waits with async_wait_all before its barrier)
        const TwPair* tw = a.tw + ((uint64_t)L.limb << C::LOGN);
        TwPair* tws = reinterpret_cast<TwPair*>(sm + C::E);
#pragma unroll 4
        for (uint32_t i = (uint32_t)t; i < (1u << C::A) - 1; i += C::T) {
            const uint32_t d = floor_log2(i + 1);
            const uint32_t k = (1u << (C::S0 + d)) + (L.hi << d) + (i + 1 - (1u << d));
            NTT_GMEM_CHECK(k, 1u << C::LOGN);
            async_copy16(&tws[i], tw + k);
        }
    }
    const uint32_t gt = L.gbase | place<C>(2u * (uint32_t)t);
    const uint64_t q = a.lc[L.limb].q;
    if (C::FIRST && C::INV && a.src_mode == 1) {
        // CKKS tensor product of the limb: rows (0|1) * n_moduli + limb of a and b
        const LimbConst lc = a.lc[L.limb];
        const uint64_t lrow = (uint64_t)L.limb << C::LOGN, step = (uint64_t)a.n_moduli << C::LOGN;
        const uint64_t* a0 = a.in + lrow + gt;
        const uint64_t* b0 = a.in_b + lrow + gt;
        const uint32_t k = (uint32_t)L.rowq;    // 0, 1 or 2
#pragma unroll
        for (int i = 0; i < C::R / 2; ++i) {
            const uint32_t off = place<C>(2u * (uint32_t)i * C::T);
            NTT_GMEM_CHECK(gt + off + 1, 1u << C::LOGN);
            uint64_t x0, x1, y0, y1, u0, u1, v0, v1;
            if (k == 0) {
                load_pair(a0 + off, x0, x1);
                load_pair(b0 + off, y0, y1);
            } else if (k == 2) {
                load_pair(a0 + step + off, x0, x1);
                load_pair(b0 + step + off, y0, y1);
            } else {
                load_pair(a0 + off, x0, x1);
                load_pair(b0 + step + off, y0, y1);
                load_pair(a0 + step + off, u0, u1);
                load_pair(b0 + off, v0, v1);
            }
            // Montgomery products (x y 2^-64 in [0, 2q)); the inverse's last
            // stage multiplies by 2^64 again.  A sum of two stays below 4q,
            // the small-modulus class's input bound; the exact class folds it.
            uint64_t r0 = mont_mul(x0, y0, lc.q, lc.qn);
            uint64_t r1 = mont_mul(x1, y1, lc.q, lc.qn);
            if (k == 1) {
                r0 += mont_mul(u0, v0, lc.q, lc.qn);
                r1 += mont_mul(u1, v1, lc.q, lc.qn);
                if (C::MC == 0) {
                    r0 = csub(r0, lc.two_q);
                    r1 = csub(r1, lc.two_q);
                }
            }
            st.x[2 * i] = r0;
            st.x[2 * i + 1] = r1;
        }
        return;
    }
    if (C::FIRST && !C::INV && a.src_mode == 2) {
        // Rescale: c = (h - [w + h]_aux_q) mod q from the dropped limb's coefficients
        const LimbConst lc = a.lc[L.limb];
        const uint64_t h = a.aux_q >> 1;
        const uint64_t hq = csub(shoup_mul(h, 1, lc.one_p, lc.q), lc.q);
        const uint64_t* w = a.in + (L.rowq << C::LOGN) + gt;
#pragma unroll
        for (int i = 0; i < C::R / 2; ++i) {
            const uint32_t off = place<C>(2u * (uint32_t)i * C::T);
            NTT_GMEM_CHECK(gt + off + 1, 1u << C::LOGN);
            uint64_t w0, w1;
            load_pair(w + off, w0, w1);
            const uint64_t r0 = csub(w0 + h, a.aux_q), r1 = csub(w1 + h, a.aux_q);   // w, h < aux_q
            const uint64_t m0 = csub(shoup_mul(r0, 1, lc.one_p, lc.q), lc.q);
            const uint64_t m1 = csub(shoup_mul(r1, 1, lc.one_p, lc.q), lc.q);
            st.x[2 * i] = hq >= m0 ? hq - m0 : hq + (lc.q - m0);
            st.x[2 * i + 1] = hq >= m1 ? hq - m1 : hq + (lc.q - m1);
        }
        return;
    }
    if (C::FIRST && C::INV && a.src_mode == 3) {
        const LimbConst lc = a.lc[L.limb];
        const uint64_t pa = a.has_map ? a.a_map[L.rowq] : L.rowq, pb = a.has_map ? a.b_map[L.rowq] : L.rowq;
        const uint64_t* x = a.in + ((pa * a.n_moduli + L.limb) << C::LOGN) + gt;
        const uint64_t* y = a.in_b + ((pb * a.n_moduli + L.limb) << C::LOGN) + gt;
#pragma unroll
        for (int i = 0; i < C::R / 2; ++i) {
            const uint32_t off = place<C>(2u * (uint32_t)i * C::T);
            NTT_GMEM_CHECK(gt + off + 1, 1u << C::LOGN);
            uint64_t x0, x1, y0, y1;
            load_pair(x + off, x0, x1);
            load_pair(y + off, y0, y1);
            // Montgomery products x y 2^-64 in [0, 2q), inside every class's
            // GS input bound; the inverse's last stage multiplies by 2^64 again
            st.x[2 * i] = mont_mul(x0, y0, lc.q, lc.qn);
            st.x[2 * i + 1] = mont_mul(x1, y1, lc.q, lc.qn);
        }
        return;
    }
    const uint64_t* src =
        (C::FIRST ? a.in + ((L.row * (1ull + a.in_skip)) << C::LOGN) : a.out + (L.row << C::LOGN)) + gt;
    bool bad = false;
#pragma unroll
    for (int i = 0; i < C::R / 2; ++i) {
        const uint32_t off = place<C>(2u * (uint32_t)i * C::T);
        NTT_GMEM_CHECK(gt + off + 1, 1u << C::LOGN);
        load_pair(src + off, st.x[2 * i], st.x[2 * i + 1]);
        if (C::FIRST) bad |= st.x[2 * i] >= q || st.x[2 * i + 1] >= q;
    }
    if (C::FIRST && a.check && bad) record_status(a.status, NTT_STATUS_RANGE);
}

// registers (pair layout of load_direct / relayout_read) -> swizzled shared memory
template <class C>
NTT_HD void write_pairs_swizzled(const TileRegs<C>& st, const TileLoc& L, int t, uint64_t* sm) {
    if (!L.valid) return;
    const uint32_t b = swz(2u * (uint32_t)t);
#pragma unroll
    for (int i = 0; i < C::R / 2; ++i) {
        const uint32_t c = swz(2u * (uint32_t)i * C::T);
        NTT_SMEM_CHECK(b ^ c, C::E);
        NTT_SMEM_CHECK(b ^ c ^ 1u, C::E);
        sm[b ^ c] = st.x[2 * i];
        sm[(b ^ c) ^ 1u] = st.x[2 * i + 1];   // swz(e + 1) = swz(e) ^ 1 for even e
    }
}

// ---- bit-reversal permutation of whole rows, tile by tile ----
// With K = min(5, log2n / 2) and M = log2n - 2K, row index (a, b, c) (a and
// c of K bits, b of M bits, a most significant) moves to (brv(c), brv(b),
// brv(a)): tile b (all a, c) becomes tile brv(b), transposed with both
// coordinates reversed.  Loads and stores run along c (contiguous).
struct BrvGeom {
    int K, M;
};
NTT_HD BrvGeom brv_geom(int log2n) {
    BrvGeom g;
    g.K = log2n / 2 < 5 ? log2n / 2 : 5;
    g.M = log2n - 2 * g.K;
    return g;
}
#define NTT_BRV_PITCH 33    // 2^5 + 1 words per tile row in shared memory

// tile b of row `src` -> sm (threads tid, tid + nthreads, ...)
NTT_HD void brv_tile_load(const uint64_t* src, BrvGeom g, uint32_t b, int tid, int nthreads, uint64_t* sm) {
    const uint32_t side = 1u << g.K;
    for (uint32_t idx = (uint32_t)tid; idx < side * side; idx += (uint32_t)nthreads) {
        const uint32_t a = idx >> g.K, c = idx & (side - 1);
        const uint64_t j = ((uint64_t)a << (g.M + g.K)) | ((uint64_t)b << g.K) | c;
        NTT_SMEM_CHECK(a * NTT_BRV_PITCH + c, NTT_BRV_PITCH * 32);
        sm[a * NTT_BRV_PITCH + c] = src[j];
    }
}

// sm (tile b) -> its place in row `dst`: tile brv(b), position (a2, c2)
// takes the element loaded at (brv(c2), brv(a2))
NTT_HD void brv_tile_store(uint64_t* dst, BrvGeom g, uint32_t b, int tid, int nthreads, const uint64_t* sm) {
    const uint32_t side = 1u << g.K, b2 = brv_bits(b, g.M);
    for (uint32_t idx = (uint32_t)tid; idx < side * side; idx += (uint32_t)nthreads) {
        const uint32_t a2 = idx >> g.K, c2 = idx & (side - 1);
        const uint32_t a = brv_bits(c2, g.K), c = brv_bits(a2, g.K);
        const uint64_t j = ((uint64_t)a2 << (g.M + g.K)) | ((uint64_t)b2 << g.K) | c2;
        NTT_SMEM_CHECK(a * NTT_BRV_PITCH + c, NTT_BRV_PITCH * 32);
        dst[j] = sm[a * NTT_BRV_PITCH + c];
    }
}

// The first kernel's registers -> shared memory.  A full-row tile of an
// inverse transform whose input is in natural order (a.nat) places element
// j of the row at tile position brv(j); everything else uses the pair layout.
template <class C>
NTT_HD void write_input_tile(const TileRegs<C>& st, const TileArgs& a, const TileLoc& L, int t, uint64_t* sm) {
    if (C::FIRST && C::INV && C::A == C::LOGN && a.nat) {
        if (!L.valid) return;
#pragma unroll
        for (int i = 0; i < C::R / 2; ++i) {
            const uint32_t k = 2u * (uint32_t)t + 2u * (uint32_t)i * C::T;
            const uint32_t e0 = brv_bits(k, C::LOGN), e1 = brv_bits(k + 1, C::LOGN);
            NTT_SMEM_CHECK(swz(e0), C::E);
            NTT_SMEM_CHECK(swz(e1), C::E);
            sm[swz(e0)] = st.x[2 * i];
            sm[swz(e1)] = st.x[2 * i + 1];
        }
        return;
    }
    write_pairs_swizzled<C>(st, L, t, sm);
}

// natural-order shared memory (pipelined staging) -> registers in the pair
// layout; checks canonical inputs for the first kernel of a transform
template <class C>
NTT_HD void relayout_read(TileRegs<C>& st, const TileArgs& a, const TileLoc& L, int t, const uint64_t* sm) {
    if (!L.valid) return;
    const uint64_t q = a.lc[L.limb].q;
    bool bad = false;
#pragma unroll
    for (int i = 0; i < C::R / 2; ++i) {
        const uint32_t e = 2u * ((uint32_t)t + (uint32_t)i * C::T);
        NTT_SMEM_CHECK(e + 1, C::E);
        load_pair(sm + e, st.x[2 * i], st.x[2 * i + 1]);
        if (C::FIRST) bad |= st.x[2 * i] >= q || st.x[2 * i + 1] >= q;
    }
    if (C::FIRST && a.check && bad) record_status(a.status, NTT_STATUS_RANGE);
}

// The two factors of twiddle entry k (= psi^(+-e), e = brv(k)) from a
// limb's on-the-fly tables: lo = psi^(+-(e mod 2^LO)), hi = psi^(+-(e >> LO) 2^LO).
template <class C>
NTT_HD void otf_twiddle(const TwPair* otf, uint32_t k, TwPair& lo, TwPair& hi) {
    constexpr int LO = otf_lo_bits(C::LOGN);
    const uint32_t e = brv_bits(k, C::LOGN);
    NTT_GMEM_CHECK(k, 1u << C::LOGN);
    NTT_GMEM_CHECK((1u << LO) + (e >> LO), otf_entries(C::LOGN));
    lo = load_tw(otf, e & ((1u << LO) - 1));
    hi = load_tw(otf, (1u << LO) + (e >> LO));
}

// Thread-bit exchanges of a pass.  Thread bit i of a pass with lowest e-bit
// PE and r stages sits at e-bit i (i < PE) or i + r.  The 16 lanes of a
// half-warp differ in thread bits 0..3, and swz folds e-bit k onto bank pair
// k mod 4 of a 64-bit word, so those four bits must land on e-bits of
// distinct residues mod 4 for a conflict-free access.  Where they do not,
// a lane bit is exchanged with a higher thread bit of a missing residue
// (any bijection of the threads is valid: each pass reads and writes through
// shared memory).  Up to four exchanges (i | j << 4 per byte, 0 = none).
NTT_HD constexpr uint32_t pass_swaps(int pe, int r, int logt) {
    int pos[32] = {};
    for (int i = 0; i < logt; ++i) pos[i] = i < pe ? i : i + r;
    uint32_t packed = 0, used = 0;
    int ns = 0;
    const int lim = logt < 4 ? logt : 4;
    for (int i = 0; i < lim; ++i) {
        if (used & (1u << (pos[i] & 3))) {
            for (int j = 4; j < logt; ++j) {
                bool ok = !(used & (1u << (pos[j] & 3)));
                for (int k = i + 1; k < lim; ++k) ok = ok && (pos[j] & 3) != (pos[k] & 3);
                if (ok) {
                    const int tmp = pos[i];
                    pos[i] = pos[j];
                    pos[j] = tmp;
                    packed |= (uint32_t)(i | (j << 4)) << (8 * ns);
                    ++ns;
                    break;
                }
            }
        }
        used |= 1u << (pos[i] & 3);
    }
    return packed;
}

// t with the recorded exchanges applied (last first, so thread bit i ends at
// the e-bit chosen for it)
NTT_HD constexpr uint32_t swap_thread_bits(uint32_t t, uint32_t packed) {
    int n = 0;
    while (n < 4 && ((packed >> (8 * n)) & 0xffu)) ++n;
    for (int s = n - 1; s >= 0; --s) {
        const uint32_t p = (packed >> (8 * s)) & 0xffu;
        const uint32_t i = p & 15u, j = p >> 4;
        const uint32_t d = ((t >> i) ^ (t >> j)) & 1u;
        t ^= (d << i) | (d << j);
    }
    return t;
}

// The same exchange search for G bank-index bits (a word's bank is the XOR of
// its e-bits' residues mod G after a G-bit fold, and 2^G lanes access at
// once): G = 5 for 32-bit words, whose 32 lanes of a warp hit the 32 banks.
// Up to 8 exchanges (i | j << 4 per byte).
NTT_HD constexpr uint64_t pass_swaps_g(int pe, int r, int logt, int g) {
    int pos[32] = {};
    for (int i = 0; i < logt; ++i) pos[i] = i < pe ? i : i + r;
    uint64_t packed = 0;
    uint32_t used = 0;
    int ns = 0;
    const int lim = logt < g ? logt : g;
    for (int i = 0; i < lim; ++i) {
        if (used & (1u << (pos[i] % g))) {
            for (int j = g; j < logt; ++j) {
                bool ok = !(used & (1u << (pos[j] % g)));
                for (int k = i + 1; k < lim; ++k) ok = ok && (pos[j] % g) != (pos[k] % g);
                if (ok) {
                    const int tmp = pos[i];
                    pos[i] = pos[j];
                    pos[j] = tmp;
                    packed |= (uint64_t)(i | (j << 4)) << (8 * ns);
                    ++ns;
                    break;
                }
            }
        }
        used |= 1u << (pos[i] % g);
    }
    return packed;
}

NTT_HD constexpr uint32_t swap_thread_bits_g(uint32_t t, uint64_t packed) {
    int n = 0;
    while (n < 8 && ((packed >> (8 * n)) & 0xffu)) ++n;
    for (int s = n - 1; s >= 0; --s) {
        const uint32_t p = (uint32_t)(packed >> (8 * s)) & 0xffu;
        const uint32_t i = p & 15u, j = p >> 4;
        const uint32_t d = ((t >> i) ^ (t >> j)) & 1u;
        t ^= (d << i) | (d << j);
    }
    return t;
}

// ---- passes: one fused group of r stages in registers ----
template <class C, int P>
struct PassGeom {
    static constexpr int S_LO = C::S0 + P * C::RP;
    static constexpr int REM = C::S1 - S_LO;
    static constexpr int r = REM < C::RP ? REM : C::RP;
    static constexpr int PE = C::LOGP + C::S1 - S_LO - r;   // e-bit of the pass's lowest bit
    static constexpr int G = C::R >> r;                     // independent groups per thread
    static constexpr int GS = 1 << r;                       // elements per group
    static constexpr uint32_t SWAPS = pass_swaps(PE, r, C::LOGT);
    // e of register j, minus the thread's contribution et(t)
    static NTT_HD constexpr uint32_t ej(int j) {
        return spread(((uint32_t)j >> r) << C::LOGT, PE, r) | (((uint32_t)j & (GS - 1)) << PE);
    }
    // the thread's contribution to its elements' e in this pass
    static NTT_HD constexpr uint32_t et(uint32_t t) {
        return spread(SWAPS ? swap_thread_bits(t, SWAPS) : t, PE, r);
    }
};

template <class C, int P>
NTT_HD void pass_read(TileRegs<C>& st, const TileLoc& L, int t, const uint64_t* sm) {
    if (!L.valid) return;
    using Gm = PassGeom<C, P>;
    const uint32_t b = swz(Gm::et((uint32_t)t));
#pragma unroll
    for (int j = 0; j < C::R; ++j) {
        const uint32_t addr = b ^ swz(Gm::ej(j));
        NTT_SMEM_CHECK(addr, C::E);
        st.x[j] = sm[addr];
    }
}

template <class C, int P>
NTT_HD void pass_write(const TileRegs<C>& st, const TileLoc& L, int t, uint64_t* sm) {
    if (!L.valid) return;
    using Gm = PassGeom<C, P>;
    const uint32_t b = swz(Gm::et((uint32_t)t));
#pragma unroll
    for (int j = 0; j < C::R; ++j) {
        const uint32_t addr = b ^ swz(Gm::ej(j));
        sm[addr] = st.x[j];
    }
}

template <class C, int P>
NTT_HD void pass_compute(TileRegs<C>& st, const TileArgs& a, const TileLoc& L, int t, const uint64_t* sm) {
    if (!L.valid) return;
    using Gm = PassGeom<C, P>;
    constexpr int S_LO = Gm::S_LO, r = Gm::r, GS = Gm::GS;
    const LimbConst lc = a.lc[L.limb];
    const TwPair* tw = a.tw + ((uint64_t)L.limb << C::LOGN);
    const TwPair* tws = reinterpret_cast<const TwPair*>(sm + C::E + L.tw_off);
    const TwPair* otf = C::MODE == 3 ? a.otf + (uint64_t)L.limb * otf_entries(C::LOGN) : nullptr;
    // row-local index bits above the pass: (g >> (LOGN - S_LO)) = hi part | pre_t | pre(gi)
    constexpr int SH = C::LOGN - S_LO;
    const uint32_t pre_t = place<C>(Gm::et((uint32_t)t)) >> SH;
    const uint32_t hi_part = L.hi << (S_LO - C::S0);
#pragma unroll
    for (int gi = 0; gi < Gm::G; ++gi) {
        const uint32_t pre = pre_t | (place<C>(Gm::ej(gi * GS)) >> SH);
        uint64_t* x = st.x + gi * GS;
        if (!C::INV) {
#pragma unroll
            for (int v = 0; v < r; ++v) {
                const int s = S_LO + v;
                const int d = 1 << (r - 1 - v);
                const int dd = s - C::S0;
                // butterfly jl uses table entry k0 + (jl >> (r - v)), staged at slot0 + (jl >> (r - v))
                const uint32_t slot0 = ((1u << dd) - 1) + (pre << v);
                const uint32_t k0 = (1u << s) + ((hi_part | pre) << v);
#pragma unroll
                for (int jl = 0; jl < GS; ++jl) {
                    if (jl & d) continue;
                    const uint32_t off = (uint32_t)jl >> (r - v);
                    TwPair w;
                    if (C::TWS) {
                        NTT_SMEM_CHECK(slot0 + off, (1u << C::A) - 1);
                        w = tws[slot0 + off];
                    } else if (C::MODE == 3) {
                        // psi^e = psi^lo psi^(hi 2^LO): Y times the first factor here,
                        // the butterfly's product supplies the second
                        TwPair w_lo;
                        otf_twiddle<C>(otf, k0 + off, w_lo, w);
                        x[jl + d] = C::MC >= 1 ? shoup_mul_approx(x[jl + d], w_lo.w, w_lo.wp, lc.q)
                                               : shoup_mul(x[jl + d], w_lo.w, w_lo.wp, lc.q);
                    } else {
                        NTT_GMEM_CHECK(k0 + off, 1u << C::LOGN);
                        w = load_tw(tw, k0 + off);
                    }
                    if (C::MC >= 1)
                        ct_butterfly_small(x[jl], x[jl + d], w.w, w.wp, lc.q, lc.four_q);
                    else
                        ct_butterfly(x[jl], x[jl + d], w.w, w.wp, lc.q, lc.two_q);
                }
            }
        } else {
#pragma unroll
            for (int v = r - 1; v >= 0; --v) {
                const int s = S_LO + v;
                const int d = 1 << (r - 1 - v);
                const int dd = s - C::S0;
                const uint32_t slot0 = ((1u << dd) - 1) + (pre << v);
                const uint32_t k0 = (1u << s) + ((hi_part | pre) << v);
#pragma unroll
                for (int jl = 0; jl < GS; ++jl) {
                    if (jl & d) continue;
                    if (s == 0) {
                        if (C::LAZY_GS)
                            gs_butterfly_scaled_lazy(x[jl], x[jl + d], lc.ninv, lc.ninv_p, lc.w1ninv,
                                                     lc.w1ninv_p, lc.q, lc.four_q << (C::S1 - 1));
                        else if (C::MC >= 1)
                            gs_butterfly_scaled_small(x[jl], x[jl + d], lc.ninv, lc.ninv_p, lc.w1ninv,
                                                      lc.w1ninv_p, lc.q, lc.four_q);
                        else
                            gs_butterfly_scaled(x[jl], x[jl + d], lc.ninv, lc.ninv_p, lc.w1ninv,
                                                lc.w1ninv_p, lc.q, lc.two_q);
                    } else {
                        const uint32_t off = (uint32_t)jl >> (r - v);
                        TwPair w, w_hi{0, 0};
                        if (C::TWS) {
                            NTT_SMEM_CHECK(slot0 + off, (1u << C::A) - 1);
                            w = tws[slot0 + off];
                        } else if (C::MODE == 3) {
                            otf_twiddle<C>(otf, k0 + off, w, w_hi);
                        } else {
                            NTT_GMEM_CHECK(k0 + off, 1u << C::LOGN);
                            w = load_tw(tw, k0 + off);
                        }
                        if (C::LAZY_GS)     // the kernel's (S1 - 1 - s)-th stage: values below 4q 2^(S1 - 1 - s)
                            gs_butterfly_lazy(x[jl], x[jl + d], w.w, w.wp, lc.q, lc.four_q << (C::S1 - 1 - s));
                        else if (C::MC >= 1)
                            gs_butterfly_small(x[jl], x[jl + d], w.w, w.wp, lc.q, lc.four_q);
                        else
                            gs_butterfly(x[jl], x[jl + d], w.w, w.wp, lc.q, lc.two_q);
                        if (C::MODE == 3)   // the difference times the second factor: still [0, 2q) / [0, 4q)
                            x[jl + d] = C::MC >= 1 ? shoup_mul_approx(x[jl + d], w_hi.w, w_hi.wp, lc.q)
                                                   : shoup_mul(x[jl + d], w_hi.w, w_hi.wp, lc.q);
                    }
                }
            }
        }
    }
}

// ---- store: swizzled shared -> global, canonical when this kernel ends the transform ----
template <class C>
NTT_HD void store_tile(const TileArgs& a, const TileLoc& L, int t, const uint64_t* sm) {
    if (!L.valid) return;
    const uint32_t gt = L.gbase | place<C>(2u * (uint32_t)t);
    uint64_t* dst = a.out + (L.row << C::LOGN) + gt;
    const uint64_t q = a.lc[L.limb].q, two_q = a.lc[L.limb].two_q;
    const uint32_t b = swz(2u * (uint32_t)t);
    const bool nat = C::LAST && !C::INV && C::A == C::LOGN && a.nat;
#pragma unroll
    for (int i = 0; i < C::R / 2; ++i) {
        const uint32_t c = swz(2u * (uint32_t)i * C::T);
        uint64_t x, y;
        if (nat) {      // output j holds tile position brv(j)
            const uint32_t k = 2u * (uint32_t)t + 2u * (uint32_t)i * C::T;
            const uint32_t s0 = swz(brv_bits(k, C::LOGN)), s1 = swz(brv_bits(k + 1, C::LOGN));
            NTT_SMEM_CHECK(s0, C::E);
            NTT_SMEM_CHECK(s1, C::E);
            x = sm[s0];
            y = sm[s1];
        } else {
            x = sm[b ^ c];
            y = sm[(b ^ c) ^ 1u];
        }
        if (C::LAZY_GS && !C::LAST) {      // [0, 2^(A + 2) q) -> [0, 3q), the next kernel's input bound
            const LimbConst& lc = a.lc[L.limb];
            x = reduce_lazy(x, lc.red2_m, lc.bits, q);
            y = reduce_lazy(y, lc.red2_m, lc.bits, q);
        }
        if (C::LAST) {
            if (C::MC >= 1 && !C::INV) {  // [0, 65q) -> [0, q)
                const LimbConst& lc = a.lc[L.limb];
                x = reduce_65q(x, lc.red_m, lc.bits, q);
                y = reduce_65q(y, lc.red_m, lc.bits, q);
            } else if (C::MC >= 1 || !C::INV) {  // [0, 4q) -> [0, q)
                x = csub(csub(x, two_q), q);
                y = csub(csub(y, two_q), q);
            } else {        // [0, 2q) -> [0, q)
                x = csub(x, q);
                y = csub(y, q);
            }
        }
        const uint32_t off = place<C>(2u * (uint32_t)i * C::T);
        NTT_GMEM_CHECK(gt + off + 1, 1u << C::LOGN);
        if (C::LAST && !C::INV && a.src_mode == 2) {
            // Rescale: (x_i + c) * aux_q^-1 with x_i the NTT-domain input row p * (n_moduli + 1) + i
            const LimbConst& lc = a.lc[L.limb];
            uint64_t u, v;
            load_pair(a.in_b + ((L.row + L.rowq) << C::LOGN) + gt + off, u, v);
            x = csub(shoup_mul(csub(x + u, q), lc.rs_inv, lc.rs_inv_p, q), q);
            y = csub(shoup_mul(csub(y + v, q), lc.rs_inv, lc.rs_inv_p, q), q);
        }
        store_pair(dst + off, x, y);
    }
}

// ---- pipelined form: the bulk copies of one tile ----
// Copy c of a tile: c < RUNS -> data run c (natural order in shared memory);
// else the twiddles of stage S0 + (c - RUNS) into their slots.
struct CopyDesc {
    const void* src;
    uint32_t dst_word;    // offset in the tile's shared-memory words
    uint32_t bytes;
};

template <class C>
NTT_HD CopyDesc tile_copy(const TileArgs& a, const TileLoc& L, int c) {
    CopyDesc d;
    if (c < C::RUNS) {
        const uint64_t* src =
            C::FIRST ? a.in + ((L.row * (1ull + a.in_skip)) << C::LOGN) : a.out + (L.row << C::LOGN);
        d.src = src + (L.gbase | ((uint32_t)c << C::LOGLO));
        d.dst_word = (uint32_t)c << C::LOGP;
        d.bytes = C::RUN_BYTES;
    } else {
        const uint32_t dd = (uint32_t)(c - C::RUNS);
        const TwPair* tw = a.tw + ((uint64_t)L.limb << C::LOGN);
        d.src = tw + (1u << (C::S0 + dd)) + (L.hi << dd);
        d.dst_word = C::E + 2u * ((1u << dd) - 1);
        d.bytes = 16u << dd;
    }
    return d;
}

// Tile slot `tin` of a pipeline buffer last held group g_prev's tile; when
// that tile had the same (limb, hi), its twiddles are still in place and are
// not copied again (all tiles of a single-modulus batch share them).
template <class C>
NTT_HD bool twiddles_reusable(const TileArgs& a, uint64_t g, uint64_t g_prev, bool have_prev, int tin) {
    if (!have_prev) return false;
    const TileLoc P = locate_in_group<C>(a, g_prev, tin);
    const TileLoc L = locate<C>(a, g * C::TPC + tin);
    return P.valid && P.tw_off == 0 && L.valid && P.limb == L.limb && P.hi == L.hi;
}

// Whether tile slot tin of group g needs its twiddles copied: only leaders
// hold twiddles, and a leader skips the copy when they are still in place.
template <class C>
NTT_HD bool twiddles_needed(const TileArgs& a, uint64_t g, uint64_t g_prev, bool have_prev, int tin) {
    const TileLoc L = locate_in_group<C>(a, g, tin);
    if (!L.valid || L.tw_off != 0) return false;
    return !twiddles_reusable<C>(a, g, g_prev, have_prev, tin);
}

}  // namespace nttgb
