// Host emulation of the tile NTT kernels, built as a separate library
// (libntt_gb300_emu.so) that the CPU test suite loads.  It runs the very
// same phase functions as the CUDA kernels (ntt_tile.cuh), CTA by CTA and
// thread by thread, with every shared- and global-memory index checked, so
// index arithmetic and pass layouts can be verified without a GPU.  It is
// never used by the product library.
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "ntt_internal.h"
#include "ntt_batch_cfgs.h"
#include "ntt_launch.h"
#include "ntt_schedules.h"
#include "tfhe_cmux.cuh"
#include "rns.cuh"

namespace nttgb {

template <class C, int I>
static void emu_passes(std::vector<TileRegs<C>>& st, const TileArgs& a, const std::vector<TileLoc>& L,
                       uint64_t* buf) {
    if constexpr (I < C::NPASS) {
        constexpr int P = C::INV ? (C::NPASS - 1 - I) : I;
        for (int tid = 0; tid < C::THREADS; ++tid) {
            const int tin = tid >> C::LOGT, t = tid & (C::T - 1);
            uint64_t* sm = buf + (size_t)tin * C::TILE_WORDS;
            pass_read<C, P>(st[tid], L[tin], t, sm);
            pass_compute<C, P>(st[tid], a, L[tin], t, sm);
            pass_write<C, P>(st[tid], L[tin], t, sm);
        }
        emu_passes<C, I + 1>(st, a, L, buf);
    }
}

// Structural checks of a config: every pass, the load/store phases and the
// swizzle touch each tile element exactly once (no races between threads of
// one phase), the tiles of a row partition it, and the bulk copies of a tile
// cover its data and twiddle words exactly once.
template <class C>
static bool verify_cfg() {
    std::vector<int> seen(C::E);
    for (int e = 0; e < C::E; ++e) {
        uint32_t s = swz((uint32_t)e);
        if (s >= (uint32_t)C::E || seen[s]++) return false;
    }
    for (int p = 0; p < C::NPASS; ++p) {
        int s_lo, r;
        pass_range<C>(p, s_lo, r);
        const int pe = C::LOGP + C::S1 - s_lo - r;
        std::fill(seen.begin(), seen.end(), 0);
        for (int t = 0; t < C::T; ++t)
            for (int j = 0; j < C::R; ++j) {
                uint32_t jlo = (uint32_t)j & ((1u << r) - 1), jhi = (uint32_t)j >> r;
                const uint32_t tt = swap_thread_bits((uint32_t)t, pass_swaps(pe, r, C::LOGT));
                uint32_t e = spread(tt | (jhi << C::LOGT), pe, r) | (jlo << pe);
                if (e >= (uint32_t)C::E || seen[e]++) return false;
            }
    }
    std::fill(seen.begin(), seen.end(), 0);
    for (int t = 0; t < C::T; ++t)
        for (int i = 0; i < C::R / 2; ++i) {
            uint32_t e = 2 * ((uint32_t)t + (uint32_t)i * C::T);
            if (e + 1 >= (uint32_t)C::E || seen[e]++ || seen[e + 1]++) return false;
        }
    std::vector<int> row(1u << C::LOGN);
    TileArgs a{};
    a.n_tiles = 1ull << C::LOGTPR;
    a.n_moduli = 1;
    for (uint64_t tile = 0; tile < a.n_tiles; ++tile) {
        TileLoc L = locate<C>(a, tile);
        for (int e = 0; e < C::E; ++e) {
            uint32_t g = gidx<C>(L, (uint32_t)e);
            if (g >= (1u << C::LOGN) || row[g]++) return false;
        }
    }
    if (C::PIPE) {
        // copy coverage on a fake row: words [0, E) data, [E, E + 2(2^A - 1)) twiddles
        std::vector<int> words(C::TILE_WORDS);
        TileArgs b{};
        static uint64_t fake[2];
        b.in = b.out = fake;
        b.tw = reinterpret_cast<const TwPair*>(fake);
        b.n_tiles = 1;
        b.n_moduli = 1;
        TileLoc L = locate<C>(b, 0);
        uint32_t bytes = 0;
        for (int c = 0; c < C::COPIES; ++c) {
            CopyDesc d = tile_copy<C>(b, L, c);
            if (d.bytes % 16 || d.dst_word % 2) return false;
            for (uint32_t w = 0; w < d.bytes / 8; ++w)
                if (d.dst_word + w >= C::TILE_WORDS || words[d.dst_word + w]++) return false;
            bytes += d.bytes;
        }
        if (bytes != C::TILE_TX_BYTES) return false;
    }
    return true;
}

template <class C>
static TileArgs emu_args(const PlanDev& p, const uint64_t* in, uint64_t* out, uint64_t row_begin,
                         uint64_t n_rows) {
    TileArgs a;
    a.in = in;
    a.out = out;
    a.tw = C::INV ? p.inv : p.fwd;
    a.lc = p.lc;
    a.status = p.status;
    a.row_begin = row_begin;
    a.n_tiles = n_rows << C::LOGTPR;
    a.n_moduli = p.n_moduli;
    a.check = p.check;
    // the 32-bit reciprocal path whenever it applies, like the launcher
    a.fast32 = (row_begin + n_rows < (1ull << 32) && a.n_tiles < (1ull << 32)) ? 1u : 0u;
    a.mod_magic = fdiv_magic(a.n_moduli);
    a.src_mode = p.src_mode;
    a.in_b = p.in_b;
    a.aux_q = p.aux_q;
    a.nat = p.nat;
    a.has_map = p.has_map;
    for (int i = 0; i < NTT_MUL_MAX_MAPPED; ++i) {
        a.a_map[i] = p.a_map[i];
        a.b_map[i] = p.b_map[i];
    }
    a.otf = C::INV ? p.otf_inv : p.otf_fwd;
    a.in_skip = p.in_skip;
    return a;
}

// the phases after the data sit in a buffer (direct form: swizzled already)
template <class C>
static void emu_compute_store(const TileArgs& a, const std::vector<TileLoc>& L, uint64_t* buf,
                              std::vector<TileRegs<C>>& st) {
    emu_passes<C, 0>(st, a, L, buf);
    for (int tid = 0; tid < C::THREADS; ++tid) {
        const int tin = tid >> C::LOGT, t = tid & (C::T - 1);
        store_tile<C>(a, L[tin], t, buf + (size_t)tin * C::TILE_WORDS);
    }
}

template <class C>
static int emu_kernel(const PlanDev& p, const uint64_t* in, uint64_t* out, uint64_t row_begin,
                      uint64_t n_rows) {
    if (!verify_cfg<C>()) return NTT_ERR_UNSUPPORTED;
    if (C::PIPE && C::FIRST && p.src_mode) return NTT_ERR_UNSUPPORTED;   // direct form only
    const TileArgs a = emu_args<C>(p, in, out, row_begin, n_rows);
    const uint64_t groups = (a.n_tiles + C::TPC - 1) / C::TPC;
    std::vector<TileRegs<C>> st(C::THREADS);
    std::vector<TileLoc> L(C::TPC);
    if (!C::PIPE) {
        std::vector<uint64_t> sm(C::BUF_WORDS, 0xdeadbeefdeadbeefull);
        for (uint64_t g = 0; g < groups; ++g) {
            for (int tin = 0; tin < C::TPC; ++tin) L[tin] = locate_in_group<C>(a, g, tin);
            for (int tid = 0; tid < C::THREADS; ++tid) {
                const int tin = tid >> C::LOGT, t = tid & (C::T - 1);
                uint64_t* sm_t = sm.data() + (size_t)tin * C::TILE_WORDS;
                load_direct<C>(st[tid], a, L[tin], t, sm_t);
                write_input_tile<C>(st[tid], a, L[tin], t, sm_t);
            }
            emu_compute_store<C>(a, L, sm.data(), st);
        }
        return NTT_OK;
    }
    // pipelined form: a small pseudo-grid of persistent CTAs so that every
    // CTA walks several groups and the buffers (and twiddle reuse) rotate
    const uint64_t grid = groups < 3 ? groups : 3;
    for (uint64_t cta = 0; cta < grid; ++cta) {
        std::vector<uint64_t> sm(2 * C::BUF_WORDS, 0xdeadbeefdeadbeefull);
        uint32_t it = 0;
        for (uint64_t g = cta; g < groups; g += grid, ++it) {
            const int b = it & 1;
            uint64_t* buf = sm.data() + (size_t)b * C::BUF_WORDS;
            // the bulk copies that the kernel issues for this group
            const bool have_prev = it >= 2;
            const uint64_t g_prev = have_prev ? g - 2 * grid : 0;
            uint32_t expect = 0, copied = 0;
            for (int tin = 0; tin < C::TPC; ++tin) {
                const TileLoc T0 = locate<C>(a, g * C::TPC + tin);
                if (!T0.valid) continue;
                expect += (uint32_t)C::DATA_BYTES;
                if (twiddles_needed<C>(a, g, g_prev, have_prev, tin))
                    expect += (uint32_t)(C::TILE_TX_BYTES - C::DATA_BYTES);
            }
            for (int c = 0; c < C::TPC * C::COPIES; ++c) {
                const int tin = c / C::COPIES, cc = c % C::COPIES;
                const TileLoc T0 = locate<C>(a, g * C::TPC + tin);
                if (!T0.valid) continue;
                if (cc >= C::RUNS && !twiddles_needed<C>(a, g, g_prev, have_prev, tin)) continue;
                const CopyDesc d = tile_copy<C>(a, T0, cc);
                uint64_t* dst = buf + (size_t)tin * C::TILE_WORDS + d.dst_word;
                NTT_SMEM_CHECK((size_t)tin * C::TILE_WORDS + d.dst_word + d.bytes / 8 - 1, C::BUF_WORDS);
                memcpy(dst, d.src, d.bytes);
                copied += d.bytes;
            }
            if (copied != expect) return NTT_ERR_UNSUPPORTED;
            for (int tin = 0; tin < C::TPC; ++tin) L[tin] = locate_in_group<C>(a, g, tin);
            for (int tid = 0; tid < C::THREADS; ++tid) {
                const int tin = tid >> C::LOGT, t = tid & (C::T - 1);
                relayout_read<C>(st[tid], a, L[tin], t, buf + (size_t)tin * C::TILE_WORDS);
            }
            for (int tid = 0; tid < C::THREADS; ++tid) {
                const int tin = tid >> C::LOGT, t = tid & (C::T - 1);
                write_input_tile<C>(st[tid], a, L[tin], t, buf + (size_t)tin * C::TILE_WORDS);
            }
            emu_compute_store<C>(a, L, buf, st);
        }
    }
    return NTT_OK;
}

template <int LOGN, int LOGT, int LOGRP, int TPC, int PIPE, bool INV>
static int emu_s1(const PlanDev& p, const uint64_t* in, uint64_t* out, uint64_t rb, uint64_t nr) {
    if (INV && p.mc == 2)     // class 2 differs from class 1 only in the inverse (as the launcher)
        return emu_kernel<TileCfg<LOGN, 0, LOGN, 0, LOGT, LOGRP, TPC, INV, INV ? 2 : 1, PIPE>>(p, in, out, rb, nr);
    if (p.mc >= 1)
        return emu_kernel<TileCfg<LOGN, 0, LOGN, 0, LOGT, LOGRP, TPC, INV, 1, PIPE>>(p, in, out, rb, nr);
    return emu_kernel<TileCfg<LOGN, 0, LOGN, 0, LOGT, LOGRP, TPC, INV, 0, PIPE>>(p, in, out, rb, nr);
}

template <int LOGN, int SPLIT, int LOGP, int LOGTA, int LOGRPA, int TPCA, int LOGTB, int LOGRPB,
          int TPCB, int PIPE, bool INV, int MC>
static int emu_s2_mc(const PlanDev& p, const uint64_t* in, uint64_t* out, uint64_t rb, uint64_t nr) {
    using CA = TileCfg<LOGN, 0, SPLIT, LOGP, LOGTA, LOGRPA, TPCA, INV, MC, form_col(PIPE)>;
    using CB = TileCfg<LOGN, SPLIT, LOGN, 0, LOGTB, LOGRPB, TPCB, INV, MC, form_row(PIPE)>;
    int rc;
    if (!INV) {
        rc = emu_kernel<CA>(p, in, out, rb, nr);
        if (!rc) rc = emu_kernel<CB>(p, in, out, rb, nr);
    } else {
        rc = emu_kernel<CB>(p, in, out, rb, nr);
        if (!rc) rc = emu_kernel<CA>(p, in, out, rb, nr);
    }
    return rc;
}

template <int LOGN, int SPLIT, int LOGP, int LOGTA, int LOGRPA, int TPCA, int LOGTB, int LOGRPB,
          int TPCB, int PIPE, bool INV>
static int emu_s2(const PlanDev& p, const uint64_t* in, uint64_t* out, uint64_t rb, uint64_t nr) {
    if (INV && p.mc == 2)
        return emu_s2_mc<LOGN, SPLIT, LOGP, LOGTA, LOGRPA, TPCA, LOGTB, LOGRPB, TPCB, PIPE, INV, INV ? 2 : 1>(p, in, out, rb, nr);
    if (p.mc >= 1)
        return emu_s2_mc<LOGN, SPLIT, LOGP, LOGTA, LOGRPA, TPCA, LOGTB, LOGRPB, TPCB, PIPE, INV, 1>(p, in, out, rb, nr);
    return emu_s2_mc<LOGN, SPLIT, LOGP, LOGTA, LOGRPA, TPCA, LOGTB, LOGRPB, TPCB, PIPE, INV, 0>(p, in, out, rb, nr);
}

typedef int (*EmuFn)(const PlanDev&, const uint64_t*, uint64_t*, uint64_t, uint64_t);
struct EmuEntry {
    uint32_t log2n;
    EmuFn fwd, inv;
    uint32_t kernels;
};
#define NTT_EMU_S1(LOGN, LOGT, LOGRP, TPC, PIPE) \
    {LOGN, &emu_s1<LOGN, LOGT, LOGRP, TPC, PIPE, false>, &emu_s1<LOGN, LOGT, LOGRP, TPC, PIPE, true>, 1},
#define NTT_EMU_S2(LOGN, SPLIT, LOGP, LOGTA, LOGRPA, TPCA, LOGTB, LOGRPB, TPCB, PIPE)          \
    {LOGN, &emu_s2<LOGN, SPLIT, LOGP, LOGTA, LOGRPA, TPCA, LOGTB, LOGRPB, TPCB, PIPE, false>,   \
     &emu_s2<LOGN, SPLIT, LOGP, LOGTA, LOGRPA, TPCA, LOGTB, LOGRPB, TPCB, PIPE, true>, 2},
static const EmuEntry g_emu[] = {NTT_SCHEDULES_ALL(NTT_EMU_S1, NTT_EMU_S2)};
static const int g_emu_count = (int)(sizeof(g_emu) / sizeof(g_emu[0]));

static const EmuEntry* emu_find(uint32_t log2n, uint32_t id) {
    uint32_t seen = 0;
    for (int i = 0; i < g_emu_count; ++i) {
        if (g_emu[i].log2n != log2n) continue;
        if (seen == id) return &g_emu[i];
        ++seen;
    }
    return nullptr;
}

// the mixed-batch kernel's per-N configurations, direct form
#define NTT_EMU_BATCH_SINGLE(LOGN, LOGT, LOGRP, TPC, MODE) \
    {LOGN, &emu_s1<LOGN, LOGT, LOGRP, TPC, MODE, false>, &emu_s1<LOGN, LOGT, LOGRP, TPC, MODE, true>, 1},
#define NTT_EMU_BATCH_SPLIT(LOGN, SPLIT, LOGP, LOGTA, LOGRPA, TPCA, LOGTB, LOGRPB, TPCB, MODE)        \
    {LOGN, &emu_s2<LOGN, SPLIT, LOGP, LOGTA, LOGRPA, TPCA, LOGTB, LOGRPB, TPCB, MODE, false>,      \
     &emu_s2<LOGN, SPLIT, LOGP, LOGTA, LOGRPA, TPCA, LOGTB, LOGRPB, TPCB, MODE, true>, 2},
static const EmuEntry g_emu_batch[] = {NTT_BATCH_CONFIGS(NTT_EMU_BATCH_SINGLE, NTT_EMU_BATCH_SPLIT)};
// the on-the-fly-twiddle configurations (NTT_FLAG_OTF_TWIDDLES plans)
static const EmuEntry g_emu_otf[] = {NTT_OTF_CONFIGS(NTT_EMU_S1, NTT_EMU_S2)};

struct EmuPlan {
    PlanHost h;
    int status = 0;
};

// The 32-bit kernel of ntt32.cu, CTA by CTA and pass by pass.
template <class C, int I>
static void emu_passes32(std::vector<Regs32<C>>& st, const Args32& a, const std::vector<Loc32>& L,
                         std::vector<uint32_t>& sm) {
    if constexpr (I < C::NPASS) {
        constexpr int P = C::INV ? (C::NPASS - 1 - I) : I;
        for (int tid = 0; tid < C::THREADS; ++tid) {
            const int tin = tid >> C::LOGT, t = tid & (C::T - 1);
            pass32<C, P>(st[tid], a, L[tin], t, sm.data() + (size_t)tin * C::E);
        }
        emu_passes32<C, I + 1>(st, a, L, sm);
    }
}

// The N = 1024 kernel: persistent CTAs of four warps walking their row lists
// with two landing buffers per warp (a small pseudo-grid of 3 CTAs, so that
// warps take several rows and the buffers rotate), every phase for all 128
// threads before the next (the kernel's __syncwarp points); the 16-byte
// copies of a prefetch land at once, where the kernel's would land by the
// wait two rows later.
template <bool SMTW>
static int emu_w1024_rows_t(const Args32& af, const Args32& ai, uint64_t f_rows, uint64_t i_rows) {
    const uint32_t quads_i = (uint32_t)((i_rows + 3) / 4), quads = quads_i + (uint32_t)((f_rows + 3) / 4);
    const uint32_t grid = quads < 3 ? quads : 3;
    std::vector<Row1024> r(128);
    // the CTA's shared-memory copies of the two tables (single modulus)
    std::vector<Tw32> tf(SMTW ? 1024 : 0), ti(SMTW ? 1024 : 0);
    if (SMTW) {
        memcpy(tf.data(), af.tw, 1024 * sizeof(Tw32));
        memcpy(ti.data(), ai.tw, 1024 * sizeof(Tw32));
    }
    for (uint32_t cta = 0; cta < grid; ++cta) {
        std::vector<uint32_t> sm(4 * 3 * 1024, 0xdeadbeefu);
        auto land = [&](int w, uint32_t k) { return sm.data() + w * 3072 + (k & 1) * 1024; };
        auto work = [&](int w) { return sm.data() + w * 3072 + 2048; };
        W1024Pick cur[4], nxt[4], after[4];
        for (int w = 0; w < 4; ++w) {
            cur[w] = w1024_pick(af, ai, quads_i, quads, cta, grid, 0, w);
            nxt[w] = w1024_pick(af, ai, quads_i, quads, cta, grid, 1, w);
        }
        for (int tid = 0; tid < 128; ++tid) {
            const int w = tid >> 5, t = tid & 31;
            w1024_prefetch(cur[w].inv ? ai : af, cur[w].L, t, land(w, 0));
            w1024_prefetch(nxt[w].inv ? ai : af, nxt[w].L, t, land(w, 1));
        }
        for (uint32_t k = 0; cur[0].live; ++k) {
            for (int w = 0; w < 4; ++w) after[w] = w1024_pick(af, ai, quads_i, quads, cta, grid, k + 2, w);
            auto each = [&](auto&& phase) {
                for (int tid = 0; tid < 128; ++tid) phase(r[tid], tid >> 5, tid & 31);
            };
            const bool inv = cur[0].inv;     // one quad per CTA and step: the same direction in every warp
            const Args32& a = inv ? ai : af;
            if (!inv) {
                each([&](Row1024& x, int w, int t) { w1024_fwd_a_land<SMTW>(x, a, cur[w].L, t, land(w, k), tf.data()); });
                each([&](Row1024&, int w, int t) { w1024_prefetch(after[w].inv ? ai : af, after[w].L, t, land(w, k)); });
                each([&](Row1024& x, int w, int t) { w1024_write_a(x, cur[w].L, t, work(w)); });
                each([&](Row1024& x, int w, int t) { w1024_fwd_b<SMTW>(x, a, cur[w].L, t, work(w), tf.data()); });
                each([&](Row1024&, int w, int t) { w1024_store(a, cur[w].L, t, work(w)); });
            } else {
                each([&](Row1024&, int w, int t) { w1024_inv_a_land(a, cur[w].L, t, land(w, k), work(w)); });
                each([&](Row1024&, int w, int t) { w1024_prefetch(after[w].inv ? ai : af, after[w].L, t, land(w, k)); });
                each([&](Row1024& x, int w, int t) { w1024_inv_b<SMTW>(x, a, cur[w].L, t, work(w), ti.data()); });
                each([&](Row1024& x, int w, int t) { w1024_inv_c<SMTW>(x, a, cur[w].L, t, work(w), ti.data()); });
            }
            for (int w = 0; w < 4; ++w) {
                cur[w] = nxt[w];
                nxt[w] = after[w];
            }
        }
    }
    return NTT_OK;
}

static int emu_w1024_rows(const Args32& af, const Args32& ai, uint64_t f_rows, uint64_t i_rows) {
    if (af.n_moduli == 1 && ai.n_moduli == 1) return emu_w1024_rows_t<true>(af, ai, f_rows, i_rows);
    return emu_w1024_rows_t<false>(af, ai, f_rows, i_rows);
}

template <bool INV>
static int emu_ntt32_w1024(const Args32& a) {
    return INV ? emu_w1024_rows(a, a, 0, a.n_rows) : emu_w1024_rows(a, a, a.n_rows, 0);
}

template <int LOGN, bool INV>
static int emu_ntt32(const Args32& a) {
    if constexpr (LOGN == 10) return emu_ntt32_w1024<INV>(a);
    using C = typename Cfg32Sel<LOGN, INV>::C;
    if (!verify_cfg<C>()) return NTT_ERR_UNSUPPORTED;
    const uint32_t ctas = (a.n_rows + C::TPC - 1) / C::TPC;
    std::vector<Regs32<C>> st(C::THREADS);
    std::vector<Loc32> L(C::TPC);
    std::vector<uint32_t> sm((size_t)C::E * C::TPC, 0xdeadbeefu);
    for (uint32_t cta = 0; cta < ctas; ++cta) {
        for (int tin = 0; tin < C::TPC; ++tin) L[tin] = locate32<C>(a, cta, tin);
        for (int tid = 0; tid < C::THREADS; ++tid) {
            const int tin = tid >> C::LOGT, t = tid & (C::T - 1);
            load32<C>(st[tid], a, L[tin], t, sm.data() + (size_t)tin * C::E);
        }
        emu_passes32<C, 0>(st, a, L, sm);
        for (int tid = 0; tid < C::THREADS; ++tid) {
            const int tin = tid >> C::LOGT, t = tid & (C::T - 1);
            store32<C>(a, L[tin], t, sm.data() + (size_t)tin * C::E);
        }
    }
    return NTT_OK;
}

// The CMux kernel of tfhe.cu, CTA by CTA: every step between two barriers
// runs for all threads before the next one starts.
template <int LOGN, int MC>
static int emu_cmux(const CmuxArgs& c, const TileArgs& af, const TileArgs& ai) {
    using K = CmuxCfg<LOGN, MC>;
    using F = typename K::F;
    using I = typename K::I;
    if (!verify_cfg<F>() || !verify_cfg<I>()) return NTT_ERR_UNSUPPORTED;
    std::vector<uint64_t> smem(K::SMEM_BYTES / sizeof(uint64_t), 0xdeadbeefdeadbeefull);
    std::vector<CmuxRegs<K>> cr(K::THREADS);
    std::vector<TileRegs<F>> sf(K::THREADS);
    std::vector<TileRegs<I>> si(K::THREADS);
    std::vector<TileLoc> L(1);
    L[0].row = 0;
    L[0].rowq = 0;
    L[0].limb = 0;
    L[0].hi = 0;
    L[0].gbase = 0;
    L[0].tw_off = 0;
    L[0].valid = true;
    const LimbConst lc = af.lc[0];
    for (uint64_t ct = 0; ct < c.n_ct; ++ct) {
        for (int tid = 0; tid < K::THREADS; ++tid)
            cmux_load<K>(cr[tid], c, ct, tid >> K::LOGT, tid & (K::T - 1), smem.data());
        for (uint32_t j = 0; j < c.levels; ++j) {
            for (int tid = 0; tid < K::THREADS; ++tid) {
                const int s = tid >> K::LOGT, t = tid & (K::T - 1);
                cmux_digits<K>(sf[tid], cr[tid], j, c);
                write_pairs_swizzled<F>(sf[tid], L[0], t, smem.data() + (size_t)s * K::N);
            }
            for (int s = 0; s < 2; ++s) {
                std::vector<TileRegs<F>> part(sf.begin() + s * K::T, sf.begin() + (s + 1) * K::T);
                emu_passes<F, 0>(part, af, L, smem.data() + (size_t)s * K::N);
                std::copy(part.begin(), part.end(), sf.begin() + s * K::T);
            }
            for (int tid = 0; tid < K::THREADS; ++tid) {
                const int s = tid >> K::LOGT, t = tid & (K::T - 1);
                cmux_mac<K>(c, lc, (uint32_t)s * c.levels + j, s, t, smem.data());
            }
        }
        for (int tid = 0; tid < K::THREADS; ++tid) {
            const int s = tid >> K::LOGT, t = tid & (K::T - 1);
            cmux_inverse_input<K>(si[tid], lc, s, t, smem.data());
        }
        for (int tid = 0; tid < K::THREADS; ++tid) {
            const int s = tid >> K::LOGT, t = tid & (K::T - 1);
            write_pairs_swizzled<I>(si[tid], L[0], t, smem.data() + (size_t)s * K::N);
        }
        for (int s = 0; s < 2; ++s) {
            std::vector<TileRegs<I>> part(si.begin() + s * K::T, si.begin() + (s + 1) * K::T);
            emu_passes<I, 0>(part, ai, L, smem.data() + (size_t)s * K::N);
        }
        for (int tid = 0; tid < K::THREADS; ++tid) {
            const int s = tid >> K::LOGT, t = tid & (K::T - 1);
            cmux_store<K>(c, lc, ct, s, t, smem.data() + (size_t)s * K::N);
        }
    }
    return NTT_OK;
}

}  // namespace nttgb

using namespace nttgb;

extern "C" {

// Host-only plan for the emulation (same validation and tables as ntt_plan).
int nttemu_plan(void** out, uint32_t log2n, const uint64_t* moduli, uint32_t n_moduli,
                uint32_t batch, uint32_t flags) {
    if (!out) return NTT_ERR_ARG;
    EmuPlan* p = new (std::nothrow) EmuPlan();
    if (!p) return NTT_ERR_NOMEM;
    int rc = build_plan_host(p->h, log2n, moduli, n_moduli, batch, flags);
    if (rc) {
        delete p;
        return rc;
    }
    *out = p;
    return NTT_OK;
}

int nttemu_plan_destroy(void* plan) {
    delete static_cast<EmuPlan*>(plan);
    return NTT_OK;
}

int nttemu_schedule_count(uint32_t log2n) {
    int c = 0;
    for (int i = 0; i < g_emu_count; ++i) c += g_emu[i].log2n == log2n;
    return c;
}

// the bit-reversal pass of two-kernel natural-order transforms, with the
// kernel's tile functions (256 pseudo-threads per tile)
static void emu_bitrev_rows(const uint64_t* in, uint64_t* out, uint64_t row_begin, uint64_t n_rows, uint32_t log2n) {
    const BrvGeom g = brv_geom((int)log2n);
    std::vector<uint64_t> sm(2 * NTT_BRV_PITCH * 32, 0xdeadbeefdeadbeefull);
    const bool in_place = in == out;
    for (uint64_t u = 0; u < (n_rows << g.M); ++u) {
        const uint64_t base = (row_begin + (u >> g.M)) << log2n;
        const uint32_t b = (uint32_t)(u & ((1ull << g.M) - 1)), b2 = brv_bits(b, g.M);
        if (in_place) {
            if (b > b2) continue;
            for (int tid = 0; tid < 256; ++tid) {
                brv_tile_load(in + base, g, b, tid, 256, sm.data());
                if (b2 != b) brv_tile_load(in + base, g, b2, tid, 256, sm.data() + NTT_BRV_PITCH * 32);
            }
            for (int tid = 0; tid < 256; ++tid) {
                brv_tile_store(out + base, g, b, tid, 256, sm.data());
                if (b2 != b) brv_tile_store(out + base, g, b2, tid, 256, sm.data() + NTT_BRV_PITCH * 32);
            }
        } else {
            for (int tid = 0; tid < 256; ++tid) brv_tile_load(in + base, g, b, tid, 256, sm.data());
            for (int tid = 0; tid < 256; ++tid) brv_tile_store(out + base, g, b, tid, 256, sm.data());
        }
    }
}

// Runs schedule `sched` of the plan's N over rows [row_begin, row_begin + n_rows)
// (natural order when the plan has NTT_FLAG_NATURAL_ORDER, as ntt_forward does).
int nttemu_transform(void* plan, uint32_t sched, int inverse, const uint64_t* in, uint64_t* out,
                     uint64_t row_begin, uint64_t n_rows) {
    EmuPlan* p = static_cast<EmuPlan*>(plan);
    if (!p || !in || !out) return NTT_ERR_ARG;
    if (row_begin > p->h.rows || n_rows > p->h.rows - row_begin) return NTT_ERR_ARG;
    const EmuEntry* e = emu_find(p->h.log2n, sched);
    if (!e) return NTT_ERR_ARG;
    PlanDev d;
    d.fwd = p->h.fwd.data();
    d.inv = p->h.inv.data();
    d.lc = p->h.consts.data();
    d.status = &p->status;
    d.n_moduli = p->h.n_moduli;
    d.check = (p->h.flags & NTT_FLAG_CHECK) ? 1u : 0u;
    d.mc = p->h.mc;
    d.src_mode = 0;
    d.in_b = nullptr;
    d.aux_q = 0;
    d.nat = 0;
    d.has_map = 0;
    if (p->h.flags & NTT_FLAG_OTF_TWIDDLES) {     // its own configuration, like ntt_forward
        d.otf_fwd = p->h.otf_fwd.data();
        d.otf_inv = p->h.otf_inv.data();
        for (const EmuEntry& o : g_emu_otf)
            if (o.log2n == p->h.log2n) return (inverse ? o.inv : o.fwd)(d, in, out, row_begin, n_rows);
        return NTT_ERR_UNSUPPORTED;
    }
    const EmuFn fn = inverse ? e->inv : e->fwd;
    if (!(p->h.flags & NTT_FLAG_NATURAL_ORDER)) return fn(d, in, out, row_begin, n_rows);
    if (e->kernels == 1) {
        d.nat = 1;
        return fn(d, in, out, row_begin, n_rows);
    }
    if (!inverse) {
        const int rc = fn(d, in, out, row_begin, n_rows);
        if (rc) return rc;
        emu_bitrev_rows(out, out, row_begin, n_rows, p->h.log2n);
        return NTT_OK;
    }
    emu_bitrev_rows(in, out, row_begin, n_rows, p->h.log2n);
    return fn(d, out, out, row_begin, n_rows);
}

// Runs the mixed-batch kernel's configuration for the plan's N.
int nttemu_batch_transform(void* plan, int inverse, const uint64_t* in, uint64_t* out) {
    EmuPlan* p = static_cast<EmuPlan*>(plan);
    if (!p || !in || !out) return NTT_ERR_ARG;
    for (const EmuEntry& e : g_emu_batch) {
        if (e.log2n != p->h.log2n) continue;
        PlanDev d;
        d.fwd = p->h.fwd.data();
        d.inv = p->h.inv.data();
        d.lc = p->h.consts.data();
        d.status = &p->status;
        d.n_moduli = p->h.n_moduli;
        d.check = (p->h.flags & NTT_FLAG_CHECK) ? 1u : 0u;
        d.mc = p->h.mc;
        d.src_mode = 0;
        d.in_b = nullptr;
        d.aux_q = 0;
        d.nat = 0;
        d.has_map = 0;
    d.nat = 0;
        return (inverse ? e.inv : e.fwd)(d, in, out, 0, p->h.rows);
    }
    return NTT_ERR_UNSUPPORTED;
}

// Tensor product + inverse transform (ntt_hmul_tensor) with schedule `sched`:
// a, b are [2][n_moduli][N] in the NTT domain, out is [3][n_moduli][N].
int nttemu_hmul_tensor(void* plan, uint32_t sched, const uint64_t* a, const uint64_t* b, uint64_t* out) {
    EmuPlan* p = static_cast<EmuPlan*>(plan);
    if (!p || !a || !b || !out) return NTT_ERR_ARG;
    const EmuEntry* e = emu_find(p->h.log2n, sched);
    if (!e) return NTT_ERR_ARG;
    PlanDev d;
    d.fwd = p->h.fwd.data();
    d.inv = p->h.inv.data();
    d.lc = p->h.consts_mont.data();   // Montgomery products (see capi)
    d.status = &p->status;
    d.n_moduli = p->h.n_moduli;
    d.check = 0;
    d.mc = p->h.mc;
    d.src_mode = 1;
    d.in_b = b;
    d.aux_q = 0;
    d.nat = 0;
    d.has_map = 0;
    return e->inv(d, a, out, 0, 3ull * p->h.n_moduli);
}

// Pointwise product with the kernel's arithmetic (Barrett).
int nttemu_pointwise(void* plan, const uint64_t* a, const uint64_t* b, uint64_t* c, uint64_t n_rows) {
    EmuPlan* p = static_cast<EmuPlan*>(plan);
    if (!p || n_rows > p->h.rows) return NTT_ERR_ARG;
    const uint64_t n = 1ull << p->h.log2n;
    for (uint64_t r = 0; r < n_rows; ++r) {
        const LimbConst& m = p->h.consts[r % p->h.n_moduli];
        for (uint64_t j = 0; j < n; ++j)
            c[r * n + j] = barrett_mulmod(a[r * n + j], b[r * n + j], m.q, m.mu, m.bits);
    }
    return NTT_OK;
}

// tfhe_external_product (rot == NULL) / tfhe_cmux_rotate on the host, with the
// same argument rules as the C ABI.
int nttemu_tfhe_cmux(void* plan, const uint64_t* in, const uint32_t* rot, const uint64_t* key, uint32_t levels,
                     uint32_t log2_base, uint64_t* out, uint64_t n_ct) {
    EmuPlan* p = static_cast<EmuPlan*>(plan);
    if (!p || !in || !key || !out || p->h.n_moduli != 1) return NTT_ERR_ARG;
    if (p->h.log2n < NTT_TFHE_MIN_LOG2N || p->h.log2n > NTT_TFHE_MAX_LOG2N) return NTT_ERR_UNSUPPORTED;
    const uint64_t q = p->h.moduli[0];
    const uint32_t sigma = 63u - (uint32_t)__builtin_clzll(q);
    if (levels < 1 || levels > NTT_TFHE_MAX_LEVELS || log2_base < 1 || levels * log2_base > 32 ||
        levels * log2_base > sigma)
        return NTT_ERR_ARG;
    // the key in the Shoup form that tfhe_key_prepare produces
    std::vector<TwPair> kp((size_t)4 * levels << p->h.log2n);
    for (size_t i = 0; i < kp.size(); ++i)
        kp[i] = TwPair{key[i], (uint64_t)(((unsigned __int128)key[i] << 64) / q)};
    CmuxArgs c;
    c.in = in;
    c.rot = rot;
    c.key = kp.data();
    c.out = out;
    c.status = &p->status;
    c.q = q;
    c.half_q = q >> 1;
    c.m = (uint64_t)(((unsigned __int128)1 << (64 + sigma)) / q);
    c.n_ct = n_ct;
    c.sigma = sigma;
    c.levels = levels;
    c.log2_base = log2_base;
    c.check = (p->h.flags & NTT_FLAG_CHECK) ? 1u : 0u;
    TileArgs af{};
    af.lc = p->h.consts.data();
    af.status = &p->status;
    af.n_moduli = 1;
    TileArgs ai = af;
    af.tw = p->h.fwd.data();
    ai.tw = p->h.inv.data();
    const bool small = p->h.mc != 0;
    if (p->h.log2n == 10) return small ? emu_cmux<10, 1>(c, af, ai) : emu_cmux<10, 0>(c, af, ai);
    return small ? emu_cmux<11, 1>(c, af, ai) : emu_cmux<11, 0>(c, af, ai);
}

// A NTT_FLAG_WORD32 plan's transform (ntt_forward / ntt_inverse on uint32
// rows) or pointwise product on the host.
int nttemu_transform32(void* plan, int inverse, const uint32_t* in, uint32_t* out, uint64_t row_begin,
                       uint64_t n_rows) {
    EmuPlan* p = static_cast<EmuPlan*>(plan);
    if (!p || !in || !out || !(p->h.flags & NTT_FLAG_WORD32)) return NTT_ERR_ARG;
    if (row_begin > p->h.rows || n_rows > p->h.rows - row_begin) return NTT_ERR_ARG;
    Args32 a;
    a.in = in;
    a.out = out;
    a.tw = inverse ? p->h.inv32.data() : p->h.fwd32.data();
    a.lc = p->h.consts32.data();
    a.status = &p->status;
    a.row_begin = (uint32_t)row_begin;
    a.n_rows = (uint32_t)n_rows;
    a.n_moduli = p->h.n_moduli;
    a.check = (p->h.flags & NTT_FLAG_CHECK) ? 1u : 0u;
    a.mod_magic = fdiv_magic(p->h.n_moduli);
#define NTT_EMU32_CASE(LOGN) \
    case LOGN: return inverse ? emu_ntt32<LOGN, true>(a) : emu_ntt32<LOGN, false>(a);
    switch (p->h.log2n) {
        NTT_EMU32_CASE(1) NTT_EMU32_CASE(2) NTT_EMU32_CASE(3) NTT_EMU32_CASE(4) NTT_EMU32_CASE(5)
        NTT_EMU32_CASE(6) NTT_EMU32_CASE(7) NTT_EMU32_CASE(8) NTT_EMU32_CASE(9) NTT_EMU32_CASE(10)
        NTT_EMU32_CASE(11) NTT_EMU32_CASE(12)
        default: return NTT_ERR_UNSUPPORTED;
    }
#undef NTT_EMU32_CASE
}

// ntt_forward_inverse of two N = 1024 32-bit-word plans: one pseudo-grid
// over the inverse rows of iplan and the forward rows of fplan
int nttemu_forward_inverse32(void* fplan, const uint32_t* fin, uint32_t* fout, void* iplan, const uint32_t* iin,
                             uint32_t* iout) {
    EmuPlan* pf = static_cast<EmuPlan*>(fplan);
    EmuPlan* pi = static_cast<EmuPlan*>(iplan);
    if (!pf || !pi || !fin || !fout || !iin || !iout) return NTT_ERR_ARG;
    if (!(pf->h.flags & NTT_FLAG_WORD32) || !(pi->h.flags & NTT_FLAG_WORD32) || pf->h.log2n != 10 ||
        pi->h.log2n != 10)
        return NTT_ERR_ARG;
    auto args = [](EmuPlan* p, bool inverse, const uint32_t* in, uint32_t* out) {
        Args32 a;
        a.in = in;
        a.out = out;
        a.tw = inverse ? p->h.inv32.data() : p->h.fwd32.data();
        a.lc = p->h.consts32.data();
        a.status = &p->status;
        a.row_begin = 0;
        a.n_rows = (uint32_t)p->h.rows;
        a.n_moduli = p->h.n_moduli;
        a.check = (p->h.flags & NTT_FLAG_CHECK) ? 1u : 0u;
        a.mod_magic = fdiv_magic(p->h.n_moduli);
        return a;
    };
    return emu_w1024_rows(args(pf, false, fin, fout), args(pi, true, iin, iout), pf->h.rows, pi->h.rows);
}

int nttemu_pointwise32(void* plan, const uint32_t* x, const uint32_t* y, uint32_t* c, uint64_t n_rows) {
    EmuPlan* p = static_cast<EmuPlan*>(plan);
    if (!p || !(p->h.flags & NTT_FLAG_WORD32) || n_rows > p->h.rows) return NTT_ERR_ARG;
    const uint64_t n = 1ull << p->h.log2n;
    for (uint64_t r = 0; r < n_rows; ++r)
        for (uint64_t j = 0; j < n; ++j)
            c[r * n + j] = mulmod32(x[r * n + j], y[r * n + j], p->h.consts32[r % p->h.n_moduli]);
    return NTT_OK;
}

// ntt_inverse_mul on the host with schedule `sched` (direct-form first kernel)
int nttemu_inverse_mul(void* plan, uint32_t sched, const uint64_t* a, const uint32_t* a_poly, const uint64_t* b,
                       const uint32_t* b_poly, uint64_t* out) {
    EmuPlan* p = static_cast<EmuPlan*>(plan);
    if (!p || !a || !b || !out) return NTT_ERR_ARG;
    const EmuEntry* e = emu_find(p->h.log2n, sched);
    if (!e) return NTT_ERR_ARG;
    PlanDev d;
    d.fwd = p->h.fwd.data();
    d.inv = p->h.inv.data();
    d.lc = p->h.consts_mont.data();   // Montgomery products (see capi)
    d.status = &p->status;
    d.n_moduli = p->h.n_moduli;
    d.check = 0;
    d.mc = p->h.mc;
    d.src_mode = 3;
    d.in_b = b;
    d.aux_q = 0;
    d.nat = 0;
    d.has_map = 0;
    if (a_poly || b_poly) {
        if (!a_poly || !b_poly || p->h.batch > NTT_MUL_MAX_MAPPED) return NTT_ERR_ARG;
        for (uint32_t k = 0; k < p->h.batch; ++k) {
            d.a_map[k] = (uint8_t)a_poly[k];
            d.b_map[k] = (uint8_t)b_poly[k];
        }
        d.has_map = 1;
    }
    return e->inv(d, a, out, 0, p->h.rows);
}

// ntt_rescale on the host with schedule `sched` for both transforms (its
// first forward kernel must be in the direct form).
int nttemu_rescale(void* plan, uint32_t sched, const uint64_t* in, uint64_t* out, uint64_t* work, uint32_t n_polys) {
    EmuPlan* p = static_cast<EmuPlan*>(plan);
    if (!p || !in || !out || !work) return NTT_ERR_ARG;
    const uint32_t L = p->h.n_moduli;
    if (L < 2 || n_polys == 0 || n_polys > p->h.batch) return NTT_ERR_ARG;
    for (uint32_t i = 0; i + 1 < L; ++i)
        if (p->h.consts[i].rs_inv == 0) return NTT_ERR_ARG;
    const EmuEntry* e = emu_find(p->h.log2n, sched);
    if (!e) return NTT_ERR_ARG;
    const size_t n = (size_t)1 << p->h.log2n;
    PlanDev last;
    last.fwd = p->h.fwd.data() + (size_t)(L - 1) * n;
    last.inv = p->h.inv.data() + (size_t)(L - 1) * n;
    last.lc = p->h.consts.data() + (L - 1);
    last.status = &p->status;
    last.n_moduli = 1;
    last.check = 0;
    last.mc = p->h.consts[L - 1].q < (1ull << NTT_SMALL_MODULUS_BITS) ? 1u : 0u;
    last.src_mode = 0;
    last.in_b = nullptr;
    last.aux_q = 0;
    last.nat = 0;
    last.has_map = 0;
    last.in_skip = L - 1;       // the dropped limb's rows, read in place
    int rc = e->inv(last, in + (size_t)(L - 1) * n, work, 0, n_polys);
    if (rc) return rc;
    PlanDev d = last;
    d.in_skip = 0;
    d.fwd = p->h.fwd.data();
    d.inv = p->h.inv.data();
    d.lc = p->h.consts.data();
    d.n_moduli = L - 1;
    d.mc = 1;
    for (uint32_t i = 0; i + 1 < L; ++i)
        if (p->h.consts[i].q >= (1ull << NTT_SMALL_MODULUS_BITS)) d.mc = 0;
    d.src_mode = 2;
    d.in_b = in;
    d.aux_q = p->h.moduli[L - 1];
    return e->fwd(d, work, out, 0, (uint64_t)n_polys * (L - 1));
}

// ntt_bconv on the host: the kernel's per-coefficient arithmetic over
// in [n_polys][L][n] -> out [n_polys][K][n].
int nttemu_bconv(const uint64_t* q_from, uint32_t L, const uint64_t* p_to, uint32_t K, const uint64_t* in,
                 uint64_t* out, uint64_t n, uint64_t n_polys) {
    std::vector<uint64_t> w;
    uint32_t chunk = 0;
    int rc = bconv_constants(q_from, L, p_to, K, w, chunk);
    if (rc) return rc;
    const BconvView v = bconv_view(w.data(), L, K, chunk);
    std::vector<uint64_t> a(L);
    for (uint64_t poly = 0; poly < n_polys; ++poly)
        for (uint64_t k = 0; k < n; ++k) {
            for (uint32_t i = 0; i < L; ++i) a[i] = bconv_a(v, i, in[(poly * L + i) * n + k]);
            auto get = [&](int, uint32_t i) { return a[i]; };
            auto cij = [&](uint32_t i, uint32_t j) { return w[3 * L + 4 * K + (size_t)i * K + j]; };
            // the kernel's split: warp w of 4 takes outputs [K w / 4, K (w + 1) / 4) in runs of 4, 2, 1
            for (uint32_t w = 0; w < 4; ++w) {
                uint32_t j = K * w / 4;
                const uint32_t j_hi = K * (w + 1) / 4;
                for (; j + 4 <= j_hi; j += 4) {
                    uint64_t y[1][4];
                    bconv_y<4, 1>(v, j, get, cij, y);
                    for (int u = 0; u < 4; ++u) out[(poly * K + j + u) * n + k] = y[0][u];
                }
                for (; j + 2 <= j_hi; j += 2) {
                    uint64_t y[1][2];
                    bconv_y<2, 1>(v, j, get, cij, y);
                    for (int u = 0; u < 2; ++u) out[(poly * K + j + u) * n + k] = y[0][u];
                }
                for (; j < j_hi; ++j) {
                    uint64_t y[1][1];
                    bconv_y<1, 1>(v, j, get, cij, y);
                    out[(poly * K + j) * n + k] = y[0][0];
                }
            }
        }
    return NTT_OK;
}

// reduce_65q with the plan's constants of one limb, on n values (x < 65 q)
int nttemu_reduce_65q(void* plan, uint32_t limb, const uint64_t* x, uint64_t* out, uint64_t n) {
    EmuPlan* p = static_cast<EmuPlan*>(plan);
    if (!p || limb >= p->h.n_moduli) return NTT_ERR_ARG;
    const LimbConst& c = p->h.consts[limb];
    for (uint64_t i = 0; i < n; ++i) out[i] = reduce_65q(x[i], c.red_m, c.bits, c.q);
    return NTT_OK;
}

// The bounded-wait test kernel of ntt_debug_bounded_wait on a host model of
// its mbarrier: one expected arrival that announces 16 transaction bytes; the
// phase completes once the arrival has happened and the announced bytes have
// all been delivered.  With `deliver` the 16-byte copy of the plan's first
// forward twiddle pair lands before the wait; without, nothing delivers, the
// wait gives up after `spin_limit` rounds and the status records the timeout.
int nttemu_debug_bounded_wait(void* plan, uint32_t deliver, uint32_t spin_limit, uint64_t* out) {
    EmuPlan* p = static_cast<EmuPlan*>(plan);
    if (!p || spin_limit == 0 || spin_limit > NTT_DEBUG_SPIN_LIMIT_MAX || p->h.fwd.empty()) return NTT_ERR_ARG;
    struct {
        uint32_t arrivals_left;
        int64_t tx;
        uint32_t phase;
    } bar{1, 0, 0};
    auto settle = [&]() {
        if (bar.arrivals_left == 0 && bar.tx == 0) bar.phase ^= 1u;
    };
    uint64_t buf[2] = {0, 0};
    bar.tx += 16;             // arrive.expect_tx(16)
    bar.arrivals_left -= 1;
    settle();
    if (deliver) {            // the bulk copy completes its bytes
        buf[0] = p->h.fwd[0].w;
        buf[1] = p->h.fwd[0].wp;
        bar.tx -= 16;
        settle();
    }
    bool ok = false;
    for (uint32_t i = 0; i < spin_limit && !ok; ++i) ok = bar.phase != 0;   // try_wait.parity 0
    if (!ok) {
        if (p->status == 0) p->status = NTT_STATUS_TIMEOUT;
        return NTT_OK;
    }
    if (out) {
        out[0] = buf[0];
        out[1] = buf[1];
    }
    return NTT_OK;
}

int nttemu_status(void* plan) {
    EmuPlan* p = static_cast<EmuPlan*>(plan);
    int s = p->status;
    p->status = 0;
    return s;
}

}  // extern "C"
