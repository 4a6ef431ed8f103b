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
// pass loads a thread's R elements from shared memory into registers,
// runs its stages there with no synchronisation, and writes them back.
// Phases are separated only by __syncthreads(), and every phase is a pure
// function of (thread, shared memory, global memory), so the same code also
// runs on the host as an emulation (see ntt_emulate.cpp).
//
// Twiddle table (one per modulus, N entries of {w, w'}): entry k = 2^s + i is
// psi^{brv(k)} (forward) or psi^{-brv(k)} (inverse) for stage s, group i.
// A butterfly of stage s on element index g uses k = 2^s + (g >> (LOGN - s)).
#pragma once
#include <stdint.h>
#include "ntt_arith.cuh"

#if !defined(__CUDA_ARCH__)
#include <cassert>
#include <cstdio>
#include <cstdlib>
#endif

namespace nttgb {

struct TwPair {
    uint64_t w, wp;
};

struct LimbConst {
    uint64_t q, two_q;
    uint64_t ninv, ninv_p;      // N^-1 mod q and its Shoup form
    uint64_t w1ninv, w1ninv_p;  // psi^{-brv(1)} N^-1 and its Shoup form (last GS stage)
    uint64_t mu;                // Barrett constant floor(2^(2 bits) / q)
    uint32_t bits, pad_;
};

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
};

#define NTT_STATUS_RANGE (-8)

// Swizzled shared-memory slot of tile element e: XOR-folds the higher 4-bit
// groups of e into its low 4 bits, which spreads the strided accesses of the
// later passes over the 16 eight-byte bank pairs.  A bijection on every
// 16-aligned block, hence on the tile.
NTT_HD uint32_t swz(uint32_t e) {
    uint32_t h = e >> 4;
    return e ^ ((h ^ (h >> 4) ^ (h >> 8)) & 15u);
}

template <int LOGN_, int S0_, int S1_, int LOGP_, int LOGT_, int LOGRP_, int TPC_, bool INV_>
struct TileCfg {
    static constexpr int LOGN = LOGN_, S0 = S0_, S1 = S1_, LOGP = LOGP_, LOGT = LOGT_;
    static constexpr int TPC = TPC_;
    static constexpr bool INV = INV_;
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
    static constexpr size_t SMEM_BYTES = sizeof(uint64_t) * (size_t)E * TPC;

    static_assert(A >= 1 && A <= LOGN, "stage range");
    static_assert(LOGLO >= LOGP, "passive columns must fit below the active bits");
    static_assert(LOGLO == 0 || LOGP >= 1, "column tiles need >= 2 adjacent columns");
    static_assert(LOGR >= 1, "each thread needs an element pair");
    static_assert(RP >= 1, "pass width");
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
    uint32_t limb;
    uint32_t hi;
    uint32_t lo_base;
    bool valid;
};

template <class C>
NTT_HD TileLoc locate(const TileArgs& a, uint64_t tile) {
    TileLoc L;
    L.valid = tile < a.n_tiles;
    uint64_t tl = L.valid ? tile : 0;
    uint64_t row_local = tl >> C::LOGTPR;
    uint32_t tau = (uint32_t)(tl & ((1ull << C::LOGTPR) - 1));
    L.row = a.row_begin + row_local;
    L.limb = (uint32_t)(L.row % a.n_moduli);
    L.hi = tau >> C::LOGLOBLK;
    L.lo_base = (tau & ((1u << C::LOGLOBLK) - 1)) << C::LOGP;
    return L;
}

// global index (within the row) of tile element e
template <class C>
NTT_HD uint32_t gidx(const TileLoc& L, uint32_t e) {
    uint32_t a = e >> C::LOGP;
    uint32_t p = e & ((1u << C::LOGP) - 1);
    return ((uint32_t)L.hi << (C::LOGN - C::S0)) | (a << C::LOGLO) | (L.lo_base + p);
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

// ---- phase 1: global -> shared (16-byte pairs, coalesced) ----
template <class C>
NTT_HD void phase_load(const TileArgs& a, const TileLoc& L, int t, uint64_t* sm) {
    if (!L.valid) return;
    const uint64_t* src = (C::FIRST ? a.in : a.out) + (L.row << C::LOGN);
    const uint64_t q = a.lc[L.limb].q;
#pragma unroll
    for (int i = 0; i < C::R / 2; ++i) {
        uint32_t k = (uint32_t)t + (uint32_t)i * C::T;
        uint32_t e = 2 * k;
        uint32_t g = gidx<C>(L, e);
        NTT_GMEM_CHECK(g + 1, 1u << C::LOGN);
        uint64_t x, y;
        load_pair(src + g, x, y);
        if (C::FIRST && a.check && (x >= q || y >= q)) record_status(a.status, NTT_STATUS_RANGE);
        NTT_SMEM_CHECK(swz(e), C::E);
        NTT_SMEM_CHECK(swz(e + 1), C::E);
        sm[swz(e)] = x;
        sm[swz(e + 1)] = y;
    }
}

// tile element held in register j of thread t during a pass over e-bits [pe, pe + r)
template <class C>
NTT_HD uint32_t pass_elem(int t, int j, int pe, int r) {
    uint32_t jlo = (uint32_t)j & ((1u << r) - 1);
    uint32_t jhi = (uint32_t)j >> r;
    uint32_t other = (uint32_t)t | (jhi << C::LOGT);
    uint32_t low = other & ((1u << pe) - 1);
    uint32_t high = other >> pe;
    return (high << (pe + r)) | (jlo << pe) | low;
}

// ---- phase 2..: one fused group of r stages in registers ----
template <class C, int P>
NTT_HD void phase_pass(const TileArgs& a, const TileLoc& L, int t, uint64_t* sm) {
    if (!L.valid) return;
    constexpr int S_LO = C::S0 + P * C::RP;
    constexpr int REM = C::S1 - S_LO;
    constexpr int r = REM < C::RP ? REM : C::RP;
    // e-bit position of the pass's lowest bit
    constexpr int PE = C::LOGP + C::S1 - S_LO - r;
    constexpr int G = C::R >> r;        // independent groups per thread
    constexpr int GS = 1 << r;          // elements per group
    const LimbConst lc = a.lc[L.limb];
    const TwPair* tw = a.tw + ((uint64_t)L.limb << C::LOGN);
    uint64_t x[C::R];
#pragma unroll
    for (int j = 0; j < C::R; ++j) {
        uint32_t e = pass_elem<C>(t, j, PE, r);
        NTT_SMEM_CHECK(swz(e), C::E);
        x[j] = sm[swz(e)];
    }
#pragma unroll
    for (int gi = 0; gi < G; ++gi) {
        uint32_t e0 = pass_elem<C>(t, gi * GS, PE, r);
        uint32_t prefix = gidx<C>(L, e0) >> (C::LOGN - S_LO);
        if (!C::INV) {
#pragma unroll
            for (int v = 0; v < r; ++v) {
                const int s = S_LO + v;
                const int d = 1 << (r - 1 - v);
#pragma unroll
                for (int jl = 0; jl < GS; ++jl) {
                    if (jl & d) continue;
                    uint32_t k = (1u << s) + (prefix << v) + ((uint32_t)jl >> (r - v));
                    NTT_GMEM_CHECK(k, 1u << C::LOGN);
                    TwPair w = load_tw(tw, k);
                    ct_butterfly(x[gi * GS + jl], x[gi * GS + jl + d], w.w, w.wp, lc.q, lc.two_q);
                }
            }
        } else {
#pragma unroll
            for (int v = r - 1; v >= 0; --v) {
                const int s = S_LO + v;
                const int d = 1 << (r - 1 - v);
#pragma unroll
                for (int jl = 0; jl < GS; ++jl) {
                    if (jl & d) continue;
                    if (s == 0) {
                        gs_butterfly_scaled(x[gi * GS + jl], x[gi * GS + jl + d], lc.ninv, lc.ninv_p,
                                            lc.w1ninv, lc.w1ninv_p, lc.q, lc.two_q);
                    } else {
                        uint32_t k = (1u << s) + (prefix << v) + ((uint32_t)jl >> (r - v));
                        NTT_GMEM_CHECK(k, 1u << C::LOGN);
                        TwPair w = load_tw(tw, k);
                        gs_butterfly(x[gi * GS + jl], x[gi * GS + jl + d], w.w, w.wp, lc.q, lc.two_q);
                    }
                }
            }
        }
    }
#pragma unroll
    for (int j = 0; j < C::R; ++j) {
        uint32_t e = pass_elem<C>(t, j, PE, r);
        sm[swz(e)] = x[j];
    }
}

// ---- last phase: shared -> global, canonical when this kernel ends the transform ----
template <class C>
NTT_HD void phase_store(const TileArgs& a, const TileLoc& L, int t, const uint64_t* sm) {
    if (!L.valid) return;
    uint64_t* dst = a.out + (L.row << C::LOGN);
    const uint64_t q = a.lc[L.limb].q, two_q = a.lc[L.limb].two_q;
#pragma unroll
    for (int i = 0; i < C::R / 2; ++i) {
        uint32_t k = (uint32_t)t + (uint32_t)i * C::T;
        uint32_t e = 2 * k;
        uint32_t g = gidx<C>(L, e);
        uint64_t x = sm[swz(e)], y = sm[swz(e + 1)];
        if (C::LAST) {
            if (!C::INV) {  // [0, 4q) -> [0, q)
                x = csub(csub(x, two_q), q);
                y = csub(csub(y, two_q), q);
            } else {        // [0, 2q) -> [0, q)
                x = csub(x, q);
                y = csub(y, q);
            }
        }
        NTT_GMEM_CHECK(g + 1, 1u << C::LOGN);
        store_pair(dst + g, x, y);
    }
}

}  // namespace nttgb
