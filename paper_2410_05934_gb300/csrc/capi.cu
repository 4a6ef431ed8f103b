// C ABI of the NTT library (declared in include/ntt_gb300.h): argument
// checks, plan lifetime, schedule table and dispatch to the kernel launchers.
// Host code only; the kernels live in kernels_*.cu.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <new>

#include "ntt_gb300.h"
#include "ntt_internal.h"
#include "ntt_launch.h"
#include "ntt_schedules.h"

namespace nttgb {

// ---- schedule table (order = NTT_SCHEDULES_ALL) ----
struct SchedParams {
    int kind;       // 1 = single kernel, 2 = column + row kernels
    int v[9];
    int pipe;
};

#define NTT_ENTRY_S1(LOGN, LOGT, LOGRP, TPC, PIPE)                          \
    {LOGN, 1, nullptr, &launch_s1<LOGN, LOGT, LOGRP, TPC, PIPE, false>,     \
     &launch_s1<LOGN, LOGT, LOGRP, TPC, PIPE, true>},
#define NTT_ENTRY_S2(LOGN, SPLIT, LOGP, LOGTA, LOGRPA, TPCA, LOGTB, LOGRPB, TPCB, PIPE)       \
    {LOGN, 2, nullptr,                                                                       \
     &launch_s2<LOGN, SPLIT, LOGP, LOGTA, LOGRPA, TPCA, LOGTB, LOGRPB, TPCB, PIPE, false>,    \
     &launch_s2<LOGN, SPLIT, LOGP, LOGTA, LOGRPA, TPCA, LOGTB, LOGRPB, TPCB, PIPE, true>},
static const SchedEntry g_table[] = {NTT_SCHEDULES_ALL(NTT_ENTRY_S1, NTT_ENTRY_S2)};

#define NTT_PARAM_S1(LOGN, LOGT, LOGRP, TPC, PIPE) {1, {LOGN, LOGT, LOGRP, TPC, 0, 0, 0, 0, 0}, PIPE},
#define NTT_PARAM_S2(LOGN, SPLIT, LOGP, LOGTA, LOGRPA, TPCA, LOGTB, LOGRPB, TPCB, PIPE) \
    {2, {LOGN, SPLIT, LOGP, LOGTA, LOGRPA, TPCA, LOGTB, LOGRPB, TPCB}, PIPE},
static const SchedParams g_params[] = {NTT_SCHEDULES_ALL(NTT_PARAM_S1, NTT_PARAM_S2)};

static const int g_count = (int)(sizeof(g_table) / sizeof(g_table[0]));

const SchedEntry* sched_table(int* count) {
    if (count) *count = g_count;
    return g_table;
}

static int sched_index(uint32_t log2n, uint32_t id) {
    uint32_t seen = 0;
    for (int i = 0; i < g_count; ++i) {
        if (g_table[i].log2n != log2n) continue;
        if (seen == id) return i;
        ++seen;
    }
    return -1;
}

int schedule_count(uint32_t log2n) {
    int c = 0;
    for (int i = 0; i < g_count; ++i) c += g_table[i].log2n == log2n;
    return c;
}

static const char* form_name(int f) {
    return f == 1 ? " pipelined" : (f == 2 ? " ro-twiddles" : (f == 3 ? " otf-twiddles" : ""));
}

static void sched_describe(int i, char* buf, size_t len) {
    const SchedParams& s = g_params[i];
    const int* v = s.v;
    if (s.kind == 1) {
        int r = v[0] - v[1];
        snprintf(buf, len, "1k%s: %d thr/row x %d coef, <=%d fused stages/pass, %d rows/CTA", form_name(s.pipe),
                 1 << v[1], 1 << r, v[2], v[3]);
    } else {
        int ra = v[1] + v[2] - v[3], rb = (v[0] - v[1]) - v[6];
        const int fa = form_col(s.pipe), fb = form_row(s.pipe);
        char form[48];
        if (fa == fb)
            snprintf(form, sizeof form, "%s", form_name(fa));
        else
            snprintf(form, sizeof form, " col%s row%s", fa ? form_name(fa) : " direct", form_name(fb));
        snprintf(buf, len,
                 "2k%s split %d+%d: col tile 2^%dx%d (%d thr x %d coef, <=%d/pass, %d/CTA); "
                 "row tile 2^%d (%d thr x %d coef, <=%d/pass, %d/CTA)",
                 form, v[1], v[0] - v[1], v[1], 1 << v[2], 1 << v[3], 1 << ra, v[4], v[5], v[0] - v[1],
                 1 << v[6], 1 << rb, v[7], v[8]);
    }
}

// Default choice before any tuning: per N and batch size, the schedule that
// won most often in the GB300 timing sweep of the autotuner (1100 random
// shapes, every candidate timed): small batches prefer short per-row tiles
// and the two-kernel split only pays once there are enough rows.
uint32_t default_schedule(uint32_t log2n, uint64_t rows) {
    switch (log2n) {
        case 10: return rows < 64 ? 6u : (rows < 256 ? 0u : 7u);      // 256 thr x 4 / 128 thr x 8 / read-only
        case 11: return rows < 128 ? 0u : 5u;                         // staged twiddles / read-only twiddles
        case 12: return rows < 64 ? 0u : 5u;
        case 13: return rows < 64 ? 3u : (rows < 1024 ? 4u : 5u);     // column + row kernels (6 + 7)
        case 14: return rows < 64 ? 4u : (rows < 256 ? 5u : 6u);      // column + row kernels (7 + 7)
        case 15: return rows < 4 ? 3u : (rows < 16 ? 6u : (rows < 64 ? 5u : 6u));
        case 16: return rows < 4 ? 6u : (rows < 16 ? 5u : (rows < 64 ? 1u : 5u));
        default: return 0u;
    }
}

static PlanDev plan_dev(const ntt_plan_s* p) {
    PlanDev d;
    d.fwd = p->d_fwd;
    d.inv = p->d_inv;
    d.lc = p->d_consts;
    d.status = p->d_status;
    d.n_moduli = p->h.n_moduli;
    d.check = (p->h.flags & NTT_FLAG_CHECK) ? 1u : 0u;
    d.mc = p->h.mc;
    d.src_mode = 0;
    d.in_b = nullptr;
    d.aux_q = 0;
    d.nat = 0;
    d.has_map = 0;
    return d;
}

static bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

static int check_device(const ntt_plan_s* p) {
    if (p->h.flags & NTT_FLAG_HOST_ONLY) return NTT_ERR_ARG;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return NTT_ERR_CUDA;
    return dev == p->device ? NTT_OK : NTT_ERR_ARG;
}

static bool word32(const ntt_plan_s* p) { return (p->h.flags & NTT_FLAG_WORD32) != 0; }

static Plan32Dev plan32_dev(const ntt_plan_s* p) {
    Plan32Dev d;
    d.fwd = p->d_fwd32;
    d.inv = p->d_inv32;
    d.lc = p->d_consts32;
    d.status = p->d_status;
    d.n_moduli = p->h.n_moduli;
    d.check = (p->h.flags & NTT_FLAG_CHECK) ? 1u : 0u;
    return d;
}

static bool natural(const ntt_plan_s* p) { return (p->h.flags & NTT_FLAG_NATURAL_ORDER) != 0; }
static bool otf(const ntt_plan_s* p) { return (p->h.flags & NTT_FLAG_OTF_TWIDDLES) != 0; }

// The on-the-fly-twiddle configuration of each N (ntt_schedules.h): the
// geometry of the measured default schedule with every kernel in form 3.
struct OtfEntry {
    uint32_t log2n;
    LaunchFn fwd, inv;
};
#define NTT_OTF_ENTRY_S1(LOGN, LOGT, LOGRP, TPC, PIPE) \
    {LOGN, &launch_s1<LOGN, LOGT, LOGRP, TPC, PIPE, false>, &launch_s1<LOGN, LOGT, LOGRP, TPC, PIPE, true>},
#define NTT_OTF_ENTRY_S2(LOGN, SPLIT, LOGP, LOGTA, LOGRPA, TPCA, LOGTB, LOGRPB, TPCB, PIPE)              \
    {LOGN, &launch_s2<LOGN, SPLIT, LOGP, LOGTA, LOGRPA, TPCA, LOGTB, LOGRPB, TPCB, PIPE, false>,         \
     &launch_s2<LOGN, SPLIT, LOGP, LOGTA, LOGRPA, TPCA, LOGTB, LOGRPB, TPCB, PIPE, true>},
static const OtfEntry g_otf[] = {NTT_OTF_CONFIGS(NTT_OTF_ENTRY_S1, NTT_OTF_ENTRY_S2)};

static const OtfEntry* otf_entry(uint32_t log2n) {
    for (const OtfEntry& e : g_otf)
        if (e.log2n == log2n) return &e;
    return nullptr;
}

// Two-kernel schedules end each of their kernels with a partly filled wave,
// which for batches of a few million coefficients is a visible share of the
// transform.  Such batches are issued as two halves of their rows: the first
// on the caller's stream, the second on the plan's side stream, forked from
// and joined back to the caller's stream through events (so the call keeps
// stream order, also under graph capture).  The first half's second kernel
// then runs beside the second half's first kernel and fills its tail.
#ifndef NTT_SPLIT_MIN_COEFFS
#define NTT_SPLIT_MIN_COEFFS (3ull << 20)
#endif
#ifndef NTT_SPLIT_MAX_COEFFS
#define NTT_SPLIT_MAX_COEFFS (1ull << 26)
#endif
static int launch_rows(ntt_plan_s* p, int idx, LaunchFn fn, const PlanDev& d, const uint64_t* in, uint64_t* out,
                       uint64_t row_begin, uint64_t n_rows, void* stream) {
    const uint64_t coeffs = n_rows << p->h.log2n;
    if (!p->side || g_params[idx].kind != 2 || n_rows < 2 || coeffs < NTT_SPLIT_MIN_COEFFS ||
        coeffs > NTT_SPLIT_MAX_COEFFS)
        return fn(d, in, out, row_begin, n_rows, stream, &p->last_launches);
    std::lock_guard<std::mutex> lock(p->split_mu);
    cudaStream_t st = (cudaStream_t)stream, side = (cudaStream_t)p->side;
    const cudaEvent_t fork = (cudaEvent_t)p->ev_fork, join = (cudaEvent_t)p->ev_join;
    if (cudaEventRecord(fork, st) != cudaSuccess || cudaStreamWaitEvent(side, fork, 0) != cudaSuccess)
        return NTT_ERR_CUDA;
    const uint64_t h = n_rows / 2;
    int rc = fn(d, in, out, row_begin, h, stream, &p->last_launches);
    if (rc == NTT_OK) rc = fn(d, in, out, row_begin + h, n_rows - h, p->side, &p->last_launches);
    // joined even after a failed launch, so the caller's stream never runs
    // ahead of work already queued on the side stream
    if (cudaEventRecord(join, side) != cudaSuccess || cudaStreamWaitEvent(st, join, 0) != cudaSuccess)
        return NTT_ERR_CUDA;
    return rc;
}

static int transform(ntt_plan_t plan, bool inverse, const uint64_t* in, uint64_t* out,
                     uint64_t row_begin, uint64_t n_rows, void* stream) {
    if (!plan || !in || !out) return NTT_ERR_ARG;
    if (!aligned16(in) || !aligned16(out)) return NTT_ERR_ALIGN;
    if (row_begin > plan->h.rows || n_rows > plan->h.rows - row_begin) return NTT_ERR_ARG;
    int rc = check_device(plan);
    if (rc) return rc;
    int idx = sched_index(plan->h.log2n, plan->schedule);
    if (idx < 0) return NTT_ERR_UNSUPPORTED;
    plan->last_launches = 0;
    if (n_rows == 0) return NTT_OK;
    if (word32(plan))
        return launch_ntt32(plan32_dev(plan), inverse, reinterpret_cast<const uint32_t*>(in),
                            reinterpret_cast<uint32_t*>(out), row_begin, n_rows, plan->h.log2n, stream,
                            &plan->last_launches);
    PlanDev d = plan_dev(plan);
    if (otf(plan)) {     // its own configuration; the plan's schedule id does not apply
        const OtfEntry* oe = otf_entry(plan->h.log2n);
        if (!oe) return NTT_ERR_UNSUPPORTED;
        d.otf_fwd = plan->d_otf_fwd;
        d.otf_inv = plan->d_otf_inv;
        return (inverse ? oe->inv : oe->fwd)(d, in, out, row_begin, n_rows, stream, &plan->last_launches);
    }
    const SchedEntry& e = g_table[idx];
    const LaunchFn fn = inverse ? e.inv : e.fwd;
    if (!natural(plan)) return launch_rows(plan, idx, fn, d, in, out, row_begin, n_rows, stream);
    // natural order: a one-kernel schedule holds whole rows and permutes in
    // shared memory; two-kernel schedules add a bit-reversal pass over HBM
    if (g_params[idx].kind == 1) {
        d.nat = 1;
        return fn(d, in, out, row_begin, n_rows, stream, &plan->last_launches);
    }
    if (!inverse) {
        rc = fn(d, in, out, row_begin, n_rows, stream, &plan->last_launches);
        if (rc) return rc;
        return launch_bitrev_rows(out, out, row_begin, n_rows, plan->h.log2n, stream, &plan->last_launches);
    }
    rc = launch_bitrev_rows(in, out, row_begin, n_rows, plan->h.log2n, stream, &plan->last_launches);
    if (rc) return rc;
    return fn(d, out, out, row_begin, n_rows, stream, &plan->last_launches);
}

static void free_device(ntt_plan_s* p) {
    if (p->d_fwd) cudaFree(p->d_fwd);
    if (p->d_inv) cudaFree(p->d_inv);
    if (p->d_consts) cudaFree(p->d_consts);
    if (p->d_consts_mont) cudaFree(p->d_consts_mont);
    p->d_consts_mont = nullptr;
    if (p->d_status) cudaFree(p->d_status);
    if (p->d_fwd32) cudaFree(p->d_fwd32);
    if (p->d_inv32) cudaFree(p->d_inv32);
    if (p->d_consts32) cudaFree(p->d_consts32);
    if (p->d_otf_fwd) cudaFree(p->d_otf_fwd);
    if (p->d_otf_inv) cudaFree(p->d_otf_inv);
    p->d_otf_fwd = p->d_otf_inv = nullptr;
    p->d_fwd = p->d_inv = nullptr;
    p->d_consts = nullptr;
    p->d_status = nullptr;
    p->d_fwd32 = p->d_inv32 = nullptr;
    p->d_consts32 = nullptr;
    if (p->ev_fork) cudaEventDestroy((cudaEvent_t)p->ev_fork);
    if (p->ev_join) cudaEventDestroy((cudaEvent_t)p->ev_join);
    if (p->side) cudaStreamDestroy((cudaStream_t)p->side);     // released once its work has finished
    p->ev_fork = p->ev_join = p->side = nullptr;
}



}  // namespace nttgb

using namespace nttgb;

extern "C" {

int ntt_plan(ntt_plan_t* out, uint32_t log2n, const uint64_t* moduli, uint32_t n_moduli,
             uint32_t batch, uint32_t flags) {
    if (!out) return NTT_ERR_ARG;
    *out = nullptr;
    ntt_plan_s* p = new (std::nothrow) ntt_plan_s();
    if (!p) return NTT_ERR_NOMEM;
    int rc;
    try {
        rc = build_plan_host(p->h, log2n, moduli, n_moduli, batch, flags);
    } catch (const std::bad_alloc&) {
        rc = NTT_ERR_NOMEM;
    }
    if (rc) {
        delete p;
        return rc;
    }
    p->schedule = default_schedule(log2n, p->h.rows);
    if (!(flags & NTT_FLAG_HOST_ONLY) && (flags & NTT_FLAG_WORD32)) {
        const size_t tw_bytes = p->h.fwd32.size() * sizeof(Tw32);
        const size_t lc_bytes = p->h.consts32.size() * sizeof(LimbConst32);
        bool ok = cudaGetDevice(&p->device) == cudaSuccess &&
                  cudaMalloc(&p->d_fwd32, tw_bytes) == cudaSuccess &&
                  cudaMalloc(&p->d_inv32, tw_bytes) == cudaSuccess &&
                  cudaMalloc(&p->d_consts32, lc_bytes) == cudaSuccess &&
                  cudaMalloc(&p->d_status, sizeof(int)) == cudaSuccess &&
                  cudaMemcpy(p->d_fwd32, p->h.fwd32.data(), tw_bytes, cudaMemcpyHostToDevice) == cudaSuccess &&
                  cudaMemcpy(p->d_inv32, p->h.inv32.data(), tw_bytes, cudaMemcpyHostToDevice) == cudaSuccess &&
                  cudaMemcpy(p->d_consts32, p->h.consts32.data(), lc_bytes, cudaMemcpyHostToDevice) == cudaSuccess &&
                  cudaMemset(p->d_status, 0, sizeof(int)) == cudaSuccess;
        if (!ok) {
            free_device(p);
            delete p;
            cudaGetLastError();
            return NTT_ERR_CUDA;
        }
        std::vector<TwPair>().swap(p->h.fwd);
        std::vector<TwPair>().swap(p->h.inv);
        std::vector<Tw32>().swap(p->h.fwd32);
        std::vector<Tw32>().swap(p->h.inv32);
    } else if (!(flags & NTT_FLAG_HOST_ONLY)) {
        const size_t tw_bytes = p->h.fwd.size() * sizeof(TwPair);
        const size_t lc_bytes = p->h.consts.size() * sizeof(LimbConst);
        bool ok = cudaGetDevice(&p->device) == cudaSuccess &&
                  cudaMalloc(&p->d_fwd, tw_bytes) == cudaSuccess &&
                  cudaMalloc(&p->d_inv, tw_bytes) == cudaSuccess &&
                  cudaMalloc(&p->d_consts, lc_bytes) == cudaSuccess &&
                  cudaMalloc(&p->d_consts_mont, lc_bytes) == cudaSuccess &&
                  cudaMalloc(&p->d_status, sizeof(int)) == cudaSuccess &&
                  cudaMemcpy(p->d_fwd, p->h.fwd.data(), tw_bytes, cudaMemcpyHostToDevice) == cudaSuccess &&
                  cudaMemcpy(p->d_inv, p->h.inv.data(), tw_bytes, cudaMemcpyHostToDevice) == cudaSuccess &&
                  cudaMemcpy(p->d_consts, p->h.consts.data(), lc_bytes, cudaMemcpyHostToDevice) == cudaSuccess &&
                  cudaMemcpy(p->d_consts_mont, p->h.consts_mont.data(), lc_bytes, cudaMemcpyHostToDevice) ==
                      cudaSuccess &&
                  cudaMemset(p->d_status, 0, sizeof(int)) == cudaSuccess;
        if (ok && otf(p)) {
            const size_t otf_bytes = p->h.otf_fwd.size() * sizeof(TwPair);
            ok = cudaMalloc(&p->d_otf_fwd, otf_bytes) == cudaSuccess &&
                 cudaMalloc(&p->d_otf_inv, otf_bytes) == cudaSuccess &&
                 cudaMemcpy(p->d_otf_fwd, p->h.otf_fwd.data(), otf_bytes, cudaMemcpyHostToDevice) == cudaSuccess &&
                 cudaMemcpy(p->d_otf_inv, p->h.otf_inv.data(), otf_bytes, cudaMemcpyHostToDevice) == cudaSuccess;
        }
        if (ok) {
            cudaStream_t side = nullptr;
            cudaEvent_t fork = nullptr, join = nullptr;
            ok = cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking) == cudaSuccess;
            p->side = side;
            ok = ok && cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) == cudaSuccess;
            p->ev_fork = fork;
            ok = ok && cudaEventCreateWithFlags(&join, cudaEventDisableTiming) == cudaSuccess;
            p->ev_join = join;
        }
        if (!ok) {
            free_device(p);
            delete p;
            cudaGetLastError();
            return NTT_ERR_CUDA;
        }
        // the device copies are authoritative; drop the host tables
        std::vector<TwPair>().swap(p->h.fwd);
        std::vector<TwPair>().swap(p->h.inv);
    }
    *out = p;
    return NTT_OK;
}

int ntt_plan_destroy(ntt_plan_t plan) {
    if (!plan) return NTT_ERR_ARG;
    free_device(plan);
    delete plan;
    return NTT_OK;
}

int ntt_plan_root(ntt_plan_t plan, uint32_t limb, uint64_t* psi) {
    if (!plan || !psi || limb >= plan->h.n_moduli) return NTT_ERR_ARG;
    *psi = plan->h.psi[limb];
    return NTT_OK;
}

int ntt_plan_shape(ntt_plan_t plan, uint32_t* log2n, uint32_t* n_moduli, uint32_t* batch,
                   uint64_t* rows) {
    if (!plan) return NTT_ERR_ARG;
    if (log2n) *log2n = plan->h.log2n;
    if (n_moduli) *n_moduli = plan->h.n_moduli;
    if (batch) *batch = plan->h.batch;
    if (rows) *rows = plan->h.rows;
    return NTT_OK;
}

int ntt_forward(ntt_plan_t plan, const uint64_t* d_in, uint64_t* d_out, void* cuda_stream) {
    return transform(plan, false, d_in, d_out, 0, plan ? plan->h.rows : 0, cuda_stream);
}

int ntt_inverse(ntt_plan_t plan, const uint64_t* d_in, uint64_t* d_out, void* cuda_stream) {
    return transform(plan, true, d_in, d_out, 0, plan ? plan->h.rows : 0, cuda_stream);
}

int ntt_forward_inverse(ntt_plan_t fwd_plan, const uint64_t* d_fwd_in, uint64_t* d_fwd_out,
                        ntt_plan_t inv_plan, const uint64_t* d_inv_in, uint64_t* d_inv_out, void* cuda_stream) {
    if (!fwd_plan || !inv_plan || !d_fwd_in || !d_fwd_out || !d_inv_in || !d_inv_out) return NTT_ERR_ARG;
    if (fwd_plan->h.log2n != inv_plan->h.log2n || word32(fwd_plan) != word32(inv_plan)) return NTT_ERR_ARG;
    const uint64_t word = word32(fwd_plan) ? 4 : 8;
    const uint64_t fb = (fwd_plan->h.rows << fwd_plan->h.log2n) * word, ib = (inv_plan->h.rows << inv_plan->h.log2n) * word;
    auto overlap = [](const void* a, uint64_t na, const void* b, uint64_t nb) {
        const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
        return na && nb && x < y + nb && y < x + na;
    };
    if (overlap(d_fwd_in, fb, d_inv_in, ib) || overlap(d_fwd_in, fb, d_inv_out, ib) ||
        overlap(d_fwd_out, fb, d_inv_in, ib) || overlap(d_fwd_out, fb, d_inv_out, ib))
        return NTT_ERR_ARG;
    if (!word32(fwd_plan)) {
        // one grid per kernel phase with N's grouped configuration, when both
        // plans are bit-reversed, table-twiddle plans of one modulus class
        const uint32_t log2n = fwd_plan->h.log2n;
        const int phases = grouped_phases(log2n);
        if (phases > 0 && fwd_plan->h.mc == inv_plan->h.mc && !natural(fwd_plan) && !natural(inv_plan) &&
            !otf(fwd_plan) && !otf(inv_plan)) {
            if (!aligned16(d_fwd_in) || !aligned16(d_fwd_out) || !aligned16(d_inv_in) || !aligned16(d_inv_out))
                return NTT_ERR_ALIGN;
            int rc = check_device(fwd_plan);
            if (!rc) rc = check_device(inv_plan);
            if (rc) return rc;
            fwd_plan->last_launches = 0;
            inv_plan->last_launches = 0;
            int* status[2] = {fwd_plan->d_status, inv_plan->d_status};
            const uint32_t check[2] = {(fwd_plan->h.flags & NTT_FLAG_CHECK) ? 1u : 0u,
                                       (inv_plan->h.flags & NTT_FLAG_CHECK) ? 1u : 0u};
            for (int ph = 0; ph < phases; ++ph) {
                GroupSeg seg[2];
                uint64_t groups[2];
                for (int k = 0; k < 2; ++k) {     // 0: forward, 1: inverse
                    const ntt_plan_s* p = k ? inv_plan : fwd_plan;
                    uint32_t ltpr = 0, tpc = 1;
                    rc = grouped_geometry(log2n, ph, k == 1, &ltpr, &tpc);
                    if (rc) return rc;
                    GroupSeg& g = seg[k];
                    g.in = ph == 0 ? (k ? d_inv_in : d_fwd_in) : (k ? d_inv_out : d_fwd_out);
                    g.out = k ? d_inv_out : d_fwd_out;
                    g.tw = k ? p->d_inv : p->d_fwd;
                    g.lc = p->d_consts;
                    g.n_tiles = p->h.rows << ltpr;
                    g.n_moduli = p->h.n_moduli;
                    g.inverse = (uint32_t)k;
                    g.fast32 = (p->h.rows < (1ull << 32) && g.n_tiles < (1ull << 32)) ? 1u : 0u;
                    g.mod_magic = fdiv_magic(p->h.n_moduli);
                    g.pad = 0;
                    groups[k] = (g.n_tiles + tpc - 1) / tpc;
                }
                seg[1].group_begin = 0;
                seg[0].group_begin = groups[1];     // the inverse rows' CTAs first
                rc = launch_pair(log2n, fwd_plan->h.mc, ph, seg[0], seg[1], groups[0] + groups[1], status, check,
                                 cuda_stream);
                if (rc) return rc;
                ++fwd_plan->last_launches;
            }
            return NTT_OK;
        }
        const int rc = transform(fwd_plan, false, d_fwd_in, d_fwd_out, 0, fwd_plan->h.rows, cuda_stream);
        return rc ? rc : transform(inv_plan, true, d_inv_in, d_inv_out, 0, inv_plan->h.rows, cuda_stream);
    }
    if (!aligned16(d_fwd_in) || !aligned16(d_fwd_out) || !aligned16(d_inv_in) || !aligned16(d_inv_out))
        return NTT_ERR_ALIGN;
    int rc = check_device(fwd_plan);
    if (!rc) rc = check_device(inv_plan);
    if (rc) return rc;
    fwd_plan->last_launches = 0;
    inv_plan->last_launches = 0;
    return launch_ntt32_fwd_inv(plan32_dev(fwd_plan), reinterpret_cast<const uint32_t*>(d_fwd_in),
                                reinterpret_cast<uint32_t*>(d_fwd_out), fwd_plan->h.rows, plan32_dev(inv_plan),
                                reinterpret_cast<const uint32_t*>(d_inv_in), reinterpret_cast<uint32_t*>(d_inv_out),
                                inv_plan->h.rows, fwd_plan->h.log2n, cuda_stream, &fwd_plan->last_launches);
}

int ntt_forward_rows(ntt_plan_t plan, const uint64_t* d_in, uint64_t* d_out, uint64_t row_begin,
                     uint64_t n_rows, void* cuda_stream) {
    return transform(plan, false, d_in, d_out, row_begin, n_rows, cuda_stream);
}

int ntt_inverse_rows(ntt_plan_t plan, const uint64_t* d_in, uint64_t* d_out, uint64_t row_begin,
                     uint64_t n_rows, void* cuda_stream) {
    return transform(plan, true, d_in, d_out, row_begin, n_rows, cuda_stream);
}

int ntt_hmul_tensor(ntt_plan_t plan, const uint64_t* d_a, const uint64_t* d_b, uint64_t* d_out,
                    void* cuda_stream) {
    if (!plan || !d_a || !d_b || !d_out) return NTT_ERR_ARG;
    if (!aligned16(d_a) || !aligned16(d_b) || !aligned16(d_out)) return NTT_ERR_ALIGN;
    if (natural(plan) || word32(plan)) return NTT_ERR_UNSUPPORTED;
    int rc = check_device(plan);
    if (rc) return rc;
    // the tensor product runs in the direct form of the inverse's first kernel
    // (the row kernel of a two-kernel schedule)
    auto inverse_first_pipelined = [](int k) {
        return (g_params[k].kind == 1 ? g_params[k].pipe : form_row(g_params[k].pipe)) == 1;
    };
    int idx = sched_index(plan->h.log2n, plan->schedule);
    if (idx < 0 || inverse_first_pipelined(idx)) {
        idx = -1;
        for (uint32_t id = 0; (int)id < schedule_count(plan->h.log2n); ++id) {
            const int k = sched_index(plan->h.log2n, id);
            if (!inverse_first_pipelined(k)) {
                idx = k;
                break;
            }
        }
        if (idx < 0) return NTT_ERR_UNSUPPORTED;
    }
    plan->last_launches = 0;
    PlanDev d = plan_dev(plan);
    d.src_mode = 1;
    d.in_b = d_b;
    d.lc = plan->d_consts_mont;     // Montgomery products: the last stage scales by N^-1 2^64
    return launch_rows(plan, idx, g_table[idx].inv, d, d_a, d_out, 0, 3ull * plan->h.n_moduli, cuda_stream);
}

int ntt_inverse_mul(ntt_plan_t plan, const uint64_t* d_a, const uint32_t* a_poly, uint32_t a_polys,
                    const uint64_t* d_b, const uint32_t* b_poly, uint32_t b_polys, uint64_t* d_out, void* cuda_stream) {
    if (!plan || !d_a || !d_b || !d_out) return NTT_ERR_ARG;
    if (!aligned16(d_a) || !aligned16(d_b) || !aligned16(d_out)) return NTT_ERR_ALIGN;
    if (natural(plan) || word32(plan)) return NTT_ERR_UNSUPPORTED;
    const uint32_t batch = plan->h.batch;
    PlanDev d = plan_dev(plan);
    if (a_poly || b_poly) {
        if (!a_poly || !b_poly || batch > NTT_MUL_MAX_MAPPED) return NTT_ERR_ARG;
        for (uint32_t p = 0; p < batch; ++p) {
            if (a_poly[p] >= a_polys || b_poly[p] >= b_polys) return NTT_ERR_ARG;
            d.a_map[p] = (uint8_t)a_poly[p];
            d.b_map[p] = (uint8_t)b_poly[p];
        }
        d.has_map = 1;
    } else if (a_polys < batch || b_polys < batch) {
        return NTT_ERR_ARG;
    }
    int rc = check_device(plan);
    if (rc) return rc;
    // the product is formed in the inverse's first kernel: a direct form
    auto inverse_first_pipelined = [](int k) {
        return (g_params[k].kind == 1 ? g_params[k].pipe : form_row(g_params[k].pipe)) == 1;
    };
    int idx = sched_index(plan->h.log2n, plan->schedule);
    if (idx < 0 || inverse_first_pipelined(idx)) {
        idx = -1;
        for (uint32_t id = 0; (int)id < schedule_count(plan->h.log2n); ++id) {
            const int k = sched_index(plan->h.log2n, id);
            if (!inverse_first_pipelined(k)) {
                idx = k;
                break;
            }
        }
        if (idx < 0) return NTT_ERR_UNSUPPORTED;
    }
    plan->last_launches = 0;
    d.src_mode = 3;
    d.in_b = d_b;
    d.lc = plan->d_consts_mont;     // Montgomery products: the last stage scales by N^-1 2^64
    return launch_rows(plan, idx, g_table[idx].inv, d, d_a, d_out, 0, plan->h.rows, cuda_stream);
}

int ntt_rescale(ntt_plan_t plan, const uint64_t* d_in, uint64_t* d_out, uint64_t* d_work, uint32_t n_polys,
                void* cuda_stream) {
    if (!plan || !d_in || !d_out || !d_work) return NTT_ERR_ARG;
    if (!aligned16(d_in) || !aligned16(d_out) || !aligned16(d_work)) return NTT_ERR_ALIGN;
    const uint32_t L = plan->h.n_moduli;
    if (L < 2) return NTT_ERR_ARG;
    if (natural(plan) || word32(plan)) return NTT_ERR_UNSUPPORTED;
    if (n_polys == 0) n_polys = plan->h.batch;
    if (n_polys > plan->h.batch) return NTT_ERR_ARG;
    for (uint32_t i = 0; i + 1 < L; ++i)
        if (plan->h.consts[i].rs_inv == 0) return NTT_ERR_ARG;     // the last modulus repeats an earlier one
    int rc = check_device(plan);
    if (rc) return rc;
    plan->last_launches = 0;
    const uint32_t log2n = plan->h.log2n;
    const size_t n = (size_t)1 << log2n;
    // 1. the dropped limb's rows (every L-th row of d_in, read in place by the
    //    first kernel) back to coefficients under the dropped modulus, into
    //    the work buffer, on the default schedule for that many rows
    const int inv_idx = sched_index(log2n, default_schedule(log2n, n_polys));
    int idx = sched_index(log2n, plan->schedule);
    if (idx < 0 || inv_idx < 0) return NTT_ERR_UNSUPPORTED;
    PlanDev last = plan_dev(plan);
    last.fwd = plan->d_fwd + (size_t)(L - 1) * n;
    last.inv = plan->d_inv + (size_t)(L - 1) * n;
    last.lc = plan->d_consts + (L - 1);
    last.n_moduli = 1;
    last.check = 0;
    last.mc = plan->h.consts[L - 1].q < (1ull << NTT_SMALL_MODULUS_BITS) ? 1u : 0u;
    last.in_skip = L - 1;
    rc = g_table[inv_idx].inv(last, d_in + (size_t)(L - 1) * n, d_work, 0, n_polys, cuda_stream,
                              &plan->last_launches);
    if (rc) return rc;
    // 2. forward transform of c = (h - [w + h]) mod q_i with the Rescale
    //    epilogue, over the n_polys x (L - 1) output rows (direct-form first kernel)
    auto forward_first_pipelined = [](int k) { return (g_params[k].kind == 1 ? g_params[k].pipe
                                                                          : form_col(g_params[k].pipe)) == 1; };
    if (forward_first_pipelined(idx)) {
        idx = -1;
        for (uint32_t id = 0; (int)id < schedule_count(log2n); ++id) {
            const int k = sched_index(log2n, id);
            if (!forward_first_pipelined(k)) {
                idx = k;
                break;
            }
        }
        if (idx < 0) return NTT_ERR_UNSUPPORTED;
    }
    PlanDev d = plan_dev(plan);
    d.n_moduli = L - 1;
    d.check = 0;
    d.mc = 1;
    for (uint32_t i = 0; i + 1 < L; ++i)
        if (plan->h.consts[i].q >= (1ull << NTT_SMALL_MODULUS_BITS)) d.mc = 0;
    d.src_mode = 2;
    d.in_b = d_in;
    d.aux_q = plan->h.moduli[L - 1];
    return launch_rows(plan, idx, g_table[idx].fwd, d, d_work, d_out, 0, (uint64_t)n_polys * (L - 1), cuda_stream);
}

int poly_mul_pointwise(ntt_plan_t plan, const uint64_t* d_a, const uint64_t* d_b, uint64_t* d_c,
                       uint32_t n_polys, void* cuda_stream) {
    if (!plan || !d_a || !d_b || !d_c) return NTT_ERR_ARG;
    if (!aligned16(d_a) || !aligned16(d_b) || !aligned16(d_c)) return NTT_ERR_ALIGN;
    if (n_polys == 0) n_polys = plan->h.batch;
    if (n_polys > plan->h.batch) return NTT_ERR_ARG;
    int rc = check_device(plan);
    if (rc) return rc;
    plan->last_launches = 0;
    if (word32(plan))
        return launch_pointwise32(plan32_dev(plan), plan->h.log2n, reinterpret_cast<const uint32_t*>(d_a),
                                  reinterpret_cast<const uint32_t*>(d_b), reinterpret_cast<uint32_t*>(d_c),
                                  (uint64_t)n_polys * plan->h.n_moduli, cuda_stream, &plan->last_launches);
    PlanDev d = plan_dev(plan);
    return launch_pointwise(d, plan->h.log2n, d_a, d_b, d_c, 0,
                            (uint64_t)n_polys * plan->h.n_moduli, cuda_stream,
                            &plan->last_launches);
}

int ntt_schedule_count(uint32_t log2n) {
    if (log2n < NTT_MIN_LOG2N || log2n > NTT_MAX_LOG2N) return NTT_ERR_ARG;
    return schedule_count(log2n);
}

int ntt_schedule_name(uint32_t log2n, uint32_t id, char* buf, size_t len) {
    int i = sched_index(log2n, id);
    if (i < 0 || !buf || len == 0) return NTT_ERR_ARG;
    sched_describe(i, buf, len);
    return NTT_OK;
}

int ntt_default_schedule(uint32_t log2n, uint64_t rows) {
    if (log2n < NTT_MIN_LOG2N || log2n > NTT_MAX_LOG2N) return NTT_ERR_ARG;
    return (int)default_schedule(log2n, rows);
}

int ntt_schedule_params(uint32_t log2n, uint32_t id, int32_t* params, uint32_t n) {
    int i = sched_index(log2n, id);
    if (i < 0 || !params || n < 11) return NTT_ERR_ARG;
    params[0] = g_params[i].kind;
    params[1] = g_params[i].pipe;
    for (int k = 0; k < 9; ++k) params[2 + k] = g_params[i].v[k];
    return NTT_OK;
}

int ntt_plan_set_schedule(ntt_plan_t plan, uint32_t id) {
    if (!plan) return NTT_ERR_ARG;
    if (sched_index(plan->h.log2n, id) < 0) return NTT_ERR_ARG;
    plan->schedule = id;
    return NTT_OK;
}

int ntt_plan_get_schedule(ntt_plan_t plan, uint32_t* id) {
    if (!plan || !id) return NTT_ERR_ARG;
    *id = plan->schedule;
    return NTT_OK;
}

int ntt_status(ntt_plan_t plan, void* cuda_stream) {
    if (!plan) return NTT_ERR_ARG;
    int rc = check_device(plan);
    if (rc) return rc;
    int host = 0;
    if (cudaStreamSynchronize((cudaStream_t)cuda_stream) != cudaSuccess) return NTT_ERR_CUDA;
    if (cudaMemcpy(&host, plan->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return NTT_ERR_CUDA;
    if (host && cudaMemset(plan->d_status, 0, sizeof(int)) != cudaSuccess) return NTT_ERR_CUDA;
    return host;
}

int ntt_plan_last_launches(ntt_plan_t plan, uint32_t* launches) {
    if (!plan || !launches) return NTT_ERR_ARG;
    *launches = plan->last_launches;
    return NTT_OK;
}

int ntt_debug_bounded_wait(ntt_plan_t plan, uint32_t deliver, uint32_t spin_limit, uint64_t* d_out,
                           void* cuda_stream) {
    if (!plan || spin_limit == 0 || spin_limit > NTT_DEBUG_SPIN_LIMIT_MAX) return NTT_ERR_ARG;
    int rc = check_device(plan);
    if (rc) return rc;
    if (!plan->d_fwd || (d_out && !aligned16(d_out))) return NTT_ERR_ARG;
    return launch_debug_bounded_wait(plan->d_fwd, deliver, spin_limit, plan->d_status, d_out, cuda_stream);
}

int ntt_bench_butterflies(uint64_t q, uint32_t kind, uint32_t blocks, uint32_t threads,
                          uint32_t iters, uint64_t* d_sink, void* cuda_stream) {
    if (q < 3 || q >= (1ull << NTT_MAX_MODULUS_BITS) || kind > 8 || (kind == 6 && (q & 1) == 0) ||
        ((kind == 2 || kind == 3) && q >= (1ull << NTT_SMALL_MODULUS_BITS)) ||
        (kind == 7 && q >= (1ull << NTT_LAZY_MODULUS_BITS)) ||
        ((kind == 5 || kind == 8) && q >= (1ull << NTT_WORD32_MAX_MODULUS_BITS)) || blocks == 0 ||
        threads == 0 || threads > 256 || !d_sink)
        return NTT_ERR_ARG;
    if (kind == 8) return launch_bench_bfly32_cmp(q, blocks, threads, iters, d_sink, cuda_stream);
    return launch_bench_bfly(q, kind, blocks, threads, iters, d_sink, cuda_stream);
}

const char* ntt_strerror(int code) {
    switch (code) {
        case NTT_OK: return "ok";
        case NTT_ERR_ARG: return "invalid argument";
        case NTT_ERR_NOT_PRIME: return "modulus is not prime";
        case NTT_ERR_NOT_NTT_FRIENDLY: return "modulus is not 1 mod 2N";
        case NTT_ERR_MODULUS_TOO_LARGE: return "modulus is not below 2^62";
        case NTT_ERR_ALIGN: return "device pointer not 16-byte aligned";
        case NTT_ERR_CUDA: return "CUDA runtime error";
        case NTT_ERR_TIMEOUT: return "bounded device wait timed out";
        case NTT_ERR_RANGE: return "input coefficient not below its modulus";
        case NTT_ERR_NOMEM: return "out of memory";
        case NTT_ERR_UNSUPPORTED: return "schedule unsupported for this shape";
        default: return "unknown error";
    }
}

const char* ntt_version(void) { return "ntt_gb300 0.1 sm_103a"; }

}  // extern "C"
