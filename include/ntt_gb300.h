/*
 * ntt_gb300.h -- C ABI of the batched negacyclic NTT library (sm_103a).
 *
 * What the library computes (arxiv 2410.05934, Sec. II-D, Eq. 1): for
 * polynomials of R_q = Z_q[x]/(x^N + 1) held in RNS form (one row of N
 * uint64 coefficients per (polynomial, modulus) pair),
 *
 *   forward  NTT_{no->bo}^{CT,psi}:  A[j] = sum_i a[i] psi^(i (2 brv(j) + 1))  mod q
 *   inverse  INTT_{bo->no}^{GS,psi^-1}: a[i] = N^-1 sum_j A[j] psi^(-i (2 brv(j) + 1))  mod q
 *   pointwise (the (.) of Eq. 1):    c[j] = a[j] b[j] mod q
 *
 * so that INTT(NTT(a) (.) NTT(b)) = a b mod (x^N + 1, q).  psi is the
 * primitive 2N-th root of unity required by Eq. 1; the library fixes it as
 * psi = g^((q-1)/2N) with g the least quadratic non-residue mod q (the paper
 * leaves the choice open; any fixed choice permutes nothing else).
 * Forward outputs are in bit-reversed order (the CT no->bo form of Eq. 1),
 * inverse outputs in natural order.  All results are canonical in [0, q)
 * and bit-exact: there is no approximation anywhere.
 *
 * Conventions shared by every entry point:
 *  - Return 0 on success or a negative NTT_ERR_* code; ntt_strerror() names it.
 *  - Device pointers are caller-owned CUDA device memory, 16-byte aligned.
 *    Calls are asynchronous on the given stream (a cudaStream_t passed as
 *    void*, NULL = legacy default stream).  Launch errors are returned at
 *    once; errors detected inside kernels are read with ntt_status().  The
 *    transform and CMux kernels are launched with programmatic stream
 *    serialization: a kernel may be scheduled while the previous kernel of
 *    the stream finishes, but reads nothing before that kernel has completed
 *    and its writes are visible, so stream order holds as for plain launches
 *    (and a caller's own launches, without that attribute, wait as usual).
 *  - Inputs must be canonical (< q of their row); with NTT_FLAG_CHECK the
 *    kernels verify this and report NTT_ERR_RANGE through ntt_status().
 *  - Data layout: [batch][n_moduli][N] uint64, row r = b * n_moduli + l uses
 *    modulus l.  in == out is allowed (in-place); other overlap is not.
 *  - A plan owns its twiddle tables (device memory) and is immutable after
 *    creation except for its schedule and status word; do not destroy a plan
 *    while work using it is in flight or while another thread uses it.
 */
#ifndef NTT_GB300_H
#define NTT_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ---- */
#define NTT_OK                    0
#define NTT_ERR_ARG              -1  /* bad size, null pointer, bad flag, bad index   */
#define NTT_ERR_NOT_PRIME        -2  /* a modulus failed the primality test           */
#define NTT_ERR_NOT_NTT_FRIENDLY -3  /* a modulus is not 1 mod 2N                     */
#define NTT_ERR_MODULUS_TOO_LARGE -4 /* a modulus is >= 2^62                          */
#define NTT_ERR_ALIGN            -5  /* a device pointer is not 16-byte aligned       */
#define NTT_ERR_CUDA             -6  /* a CUDA runtime call failed                    */
#define NTT_ERR_TIMEOUT          -7  /* a bounded device-side wait ran out            */
#define NTT_ERR_RANGE            -8  /* NTT_FLAG_CHECK found an input >= q            */
#define NTT_ERR_NOMEM            -9  /* host or device allocation failed              */
#define NTT_ERR_UNSUPPORTED      -10 /* schedule not available for this shape         */

/* ---- plan flags ---- */
#define NTT_FLAG_HOST_ONLY  1u  /* build and validate on the host only: no device
                                   memory, compute entry points return NTT_ERR_ARG */
#define NTT_FLAG_CHECK      2u  /* kernels check inputs < q (status word)          */
#define NTT_FLAG_NATURAL_ORDER 4u /* the NTT domain in natural order: ntt_forward
                                   writes A_nat[j] = a(psi^(2j + 1)), ntt_inverse
                                   reads that order (see ntt_forward)             */
#define NTT_FLAG_WORD32     8u  /* 32-bit words: every modulus < 2^30, N <= 2^12;
                                   ntt_forward / ntt_inverse(_rows) and
                                   poly_mul_pointwise read and write uint32
                                   coefficients (same layout); the fused
                                   operators and natural order are not offered */
#define NTT_FLAG_OTF_TWIDDLES 16u /* on-the-fly twiddles (N >= 2^10): ntt_forward /
                                   ntt_inverse(_rows) form each twiddle
                                   psi^(+-brv(k)) as the product of two entries of
                                   per-limb tables of 2^ceil(n/2) + 2^floor(n/2)
                                   pairs (n = log2 N) instead of reading an
                                   N-entry table: one more Shoup product per
                                   butterfly, ~1/128 of the twiddle bytes at
                                   N = 2^16.  Same results bit for bit; the fused
                                   operators keep the stored tables; not with
                                   NTT_FLAG_NATURAL_ORDER or NTT_FLAG_WORD32 */
#define NTT_OTF_MIN_LOG2N 10
#define NTT_WORD32_MAX_LOG2N 12
#define NTT_WORD32_MAX_MODULUS_BITS 30

#define NTT_MIN_LOG2N 1
#define NTT_MAX_LOG2N 16
#define NTT_MAX_MODULUS_BITS 62

typedef struct ntt_plan_s* ntt_plan_t;

/*
 * ntt_plan -- validate (N = 2^log2n, moduli[0..n_moduli), batch) and build
 * the twiddle tables of Sec. II-D (powers of psi in bit-reversed order, in
 * Shoup form w' = floor(w 2^64 / q)), then copy them to the current device.
 *   log2n     in [NTT_MIN_LOG2N, NTT_MAX_LOG2N]
 *   moduli    host array, each a prime q < 2^62 with q = 1 mod 2N
 *   n_moduli  >= 1;  batch >= 1;  batch * n_moduli * N < 2^40
 *   flags     NTT_FLAG_*
 * On success *out receives a plan the caller releases with ntt_plan_destroy.
 * Errors: ARG, NOT_PRIME, NOT_NTT_FRIENDLY, MODULUS_TOO_LARGE, NOMEM, CUDA.
 */
int ntt_plan(ntt_plan_t* out, uint32_t log2n, const uint64_t* moduli, uint32_t n_moduli,
             uint32_t batch, uint32_t flags);
int ntt_plan_destroy(ntt_plan_t plan);

/* psi of modulus `limb` (the root every transform of this plan uses). */
int ntt_plan_root(ntt_plan_t plan, uint32_t limb, uint64_t* psi);

/* Shape queries: N, n_moduli, batch, and rows = batch * n_moduli. */
int ntt_plan_shape(ntt_plan_t plan, uint32_t* log2n, uint32_t* n_moduli, uint32_t* batch,
                   uint64_t* rows);

/*
 * Forward NTT (CT, natural -> bit-reversed, Sec. II-D Eq. 1) of all
 * batch * n_moduli rows: d_in -> d_out (may alias).  The inverse is the GS
 * bit-reversed -> natural transform with psi^-1, scaled by N^-1, so that
 * ntt_inverse(ntt_forward(a)) = a.
 * With NTT_FLAG_NATURAL_ORDER the NTT domain is in natural order instead:
 * the forward writes A[brv(j)] = a(psi^(2j + 1)) at j and the inverse reads
 * that order.  One-kernel schedules (N <= 2^12) permute inside the tile at no
 * extra memory traffic; two-kernel schedules add one bit-reversal pass over
 * the rows (one more kernel launch).  The fused operators (ntt_hmul_tensor,
 * ntt_rescale, tfhe_*, ntt_batch_execute_static) take bit-reversed plans only
 * and return NTT_ERR_UNSUPPORTED for natural-order ones.
 * Row split: on a two-kernel schedule, a call of 64-bit words over 3 * 2^20
 * to 2^26 coefficients (ntt_forward / ntt_inverse / their _rows forms on
 * bit-reversed table-twiddle plans, ntt_inverse_mul, ntt_hmul_tensor and the
 * forward of ntt_rescale) issues the first half of its rows on cuda_stream
 * and the second half on a side stream the plan owns, forked from and
 * joined back to cuda_stream through events: the call keeps stream order
 * (work queued after it on cuda_stream sees both halves) and is valid under
 * CUDA graph capture, where it records a fork and a join.  Host threads that
 * share one plan are serialised while they enqueue such a call, and their
 * second halves run in order on the plan's side stream.
 */
int ntt_forward(ntt_plan_t plan, const uint64_t* d_in, uint64_t* d_out, void* cuda_stream);
int ntt_inverse(ntt_plan_t plan, const uint64_t* d_in, uint64_t* d_out, void* cuda_stream);

/*
 * Both directions of one step at once (Sec. IV-A batches the independent
 * transforms of one iteration into one launch; config: the 3780 digit NTTs
 * and 1260 accumulator INTTs of a blind-rotation step): the forward of
 * fwd_plan's rows d_fwd_in -> d_fwd_out and the inverse of inv_plan's rows
 * d_inv_in -> d_inv_out, with the same results as ntt_forward followed by
 * ntt_inverse.  The two transforms run concurrently: in one launch for
 * 32-bit-word plans at N = 1024; for 64-bit plans of one modulus class in
 * one grid per kernel phase (one launch for N <= 2^12, two above) on the
 * N's grouped configuration (the one of NTT_BATCH_GROUPED, not the plans'
 * schedules); otherwise (natural-order or on-the-fly-twiddle plans, 32-bit
 * words at other N, different classes) one after the other on the stream.
 * Errors found in the kernels go to each plan's own status word.  Both
 * plans must have the same N and word size.  Each transform may work in
 * place, but no buffer of one transform may overlap a buffer of the other
 * (NTT_ERR_ARG).  Layout, alignment and ownership as ntt_forward.
 */
int ntt_forward_inverse(ntt_plan_t fwd_plan, const uint64_t* d_fwd_in, uint64_t* d_fwd_out,
                        ntt_plan_t inv_plan, const uint64_t* d_inv_in, uint64_t* d_inv_out, void* cuda_stream);

/*
 * Row-range variants: transform rows [row_begin, row_begin + n_rows) of the
 * plan's layout; d_in / d_out point at the FIRST ROW OF THE PLAN (row 0), so
 * a multi-device caller can give each device a disjoint range of one buffer
 * layout.  Errors: ARG when the range leaves [0, rows).
 */
int ntt_forward_rows(ntt_plan_t plan, const uint64_t* d_in, uint64_t* d_out, uint64_t row_begin,
                     uint64_t n_rows, void* cuda_stream);
int ntt_inverse_rows(ntt_plan_t plan, const uint64_t* d_in, uint64_t* d_out, uint64_t row_begin,
                     uint64_t n_rows, void* cuda_stream);

/*
 * Pointwise product (the (.) of Eq. 1): d_c[r][j] = d_a[r][j] * d_b[r][j]
 * mod q_l(r) over n_polys * n_moduli rows (n_polys = 0 means the plan's
 * batch).  Row r uses modulus r mod n_moduli.  d_c may alias d_a or d_b.
 */
/*
 * Pointwise product fused into the inverse transform (Eq. 1's
 * INTT(NTT(a) (.) NTT(b)), the CKKS cross products of a ciphertext
 * multiplication): for every output polynomial p < batch and limb l,
 *   out[p][l] = INTT( a[a_poly[p]][l] (.) b[b_poly[p]][l] )  mod q_l,
 * the product formed while the inverse's first kernel loads its tile (no
 * product buffer, no extra launch).
 *   d_a, d_b     NTT-domain polynomials [a_polys][n_moduli][N] and
 *                [b_polys][n_moduli][N], canonical; may alias each other
 *   a_poly, b_poly  host arrays of `batch` polynomial indices (< a_polys,
 *                < b_polys), at most NTT_MUL_MAX_MAPPED entries; both NULL =
 *                polynomial p of each (then a_polys, b_polys >= batch)
 *   d_out        [batch][n_moduli][N]; must not overlap d_a or d_b
 * Errors: ARG (bad index or count), ALIGN, UNSUPPORTED (natural-order or
 * 32-bit plans), CUDA.
 */
#define NTT_MUL_MAX_MAPPED 32
int ntt_inverse_mul(ntt_plan_t plan, const uint64_t* d_a, const uint32_t* a_poly, uint32_t a_polys,
                    const uint64_t* d_b, const uint32_t* b_poly, uint32_t b_polys, uint64_t* d_out,
                    void* cuda_stream);

/*
 * CKKS Rescale of NTT-domain ciphertext limbs (Sec. II-A: after a
 * multiplication the scale is brought back to Delta and one level is
 * dropped): for the plan's moduli q_0 .. q_(L-1) and every polynomial,
 *   out_i = round(X / q_(L-1)) mod q_i,  i < L - 1,
 * X the integer with residues in_0 .. in_(L-1) (coefficient by coefficient),
 * computed as INTT of the last limb, then per remaining limb a forward NTT of
 * c = (h - [w + h]_{q_(L-1)}) mod q_i (h = floor(q_(L-1) / 2), w the last
 * limb's coefficients) fused with (in_i + NTT(c)) * q_(L-1)^-1 mod q_i.
 *   d_in    [n_polys][L][N] NTT domain (bit-reversed order), canonical
 *   d_out   [n_polys][L-1][N] NTT domain; must not overlap d_in or d_work
 *   d_work  [n_polys][N] caller-owned scratch (the last limb's coefficients)
 *   n_polys 0 = the plan's batch; at most the plan's batch
 * The plan needs L >= 2 and a last modulus distinct from the others.  The
 * INTT reads the last limb's rows of d_in in place (on the default schedule
 * for n_polys rows) and the forward runs on the plan's schedule: two to four
 * kernel launches on cuda_stream.
 * Errors: ARG, ALIGN, UNSUPPORTED, CUDA.
 */
int ntt_rescale(ntt_plan_t plan, const uint64_t* d_in, uint64_t* d_out, uint64_t* d_work, uint32_t n_polys,
                void* cuda_stream);

int poly_mul_pointwise(ntt_plan_t plan, const uint64_t* d_a, const uint64_t* d_b, uint64_t* d_c,
                       uint32_t n_polys, void* cuda_stream);

/*
 * Fused CKKS ciphertext multiplication core (Sec. II-A HMUL; Eq. 1 applied to
 * the tensor product of two ciphertexts): given ciphertexts a = (a0, a1) and
 * b = (b0, b1) already in the NTT domain (each [2][n_moduli][N]), computes
 *   d0 = INTT(a0 (.) b0),  d1 = INTT(a0 (.) b1 + a1 (.) b0),  d2 = INTT(a1 (.) b1)
 * into d_out ([3][n_moduli][N], coefficient domain).  The products are formed
 * inside the first kernel of the inverse transform (no separate pointwise
 * pass).  d_out must not overlap d_a or d_b.  Uses the plan's tables and
 * moduli (its batch is not used); if the plan's schedule is a pipelined one,
 * the first direct-form schedule of N is used instead.
 */
int ntt_hmul_tensor(ntt_plan_t plan, const uint64_t* d_a, const uint64_t* d_b, uint64_t* d_out,
                    void* cuda_stream);

/*
 * Schedules (Sec. V-D: the split of the log2 N stages into fused groups and
 * kernel passes, threads per polynomial, polynomials per CTA).  Each N has a
 * small fixed list of candidate schedules; ntt_plan picks a default, an
 * autotuner or cost model may override it.  Bit-exact results do not depend
 * on the schedule.
 *   ntt_schedule_count(log2n)              -> number of candidates (>= 1)
 *   ntt_schedule_name(log2n, id, buf, len) -> human-readable description
 *   ntt_plan_set_schedule / get_schedule   -> choose / read the plan's choice
 */
int ntt_schedule_count(uint32_t log2n);
int ntt_schedule_name(uint32_t log2n, uint32_t id, char* buf, size_t len);
int ntt_plan_set_schedule(ntt_plan_t plan, uint32_t id);
/* The schedule ntt_plan picks by default for N = 2^log2n and `rows` rows. */
int ntt_default_schedule(uint32_t log2n, uint64_t rows);
/* Raw parameters of a schedule: params[0] = kernels (1 or 2), params[1] =
 * kernel form (0 direct, 1 pipelined, 2 read-only-cache twiddles; for two
 * kernels A | B << 2 with B != 0 = column form A, row form B), params[2..10] = the nine numbers of its S1/S2 entry
 * (S1: LOGN, LOGT, LOGRP, TPC, 0...; S2: LOGN, SPLIT, LOGP, LOGTA, LOGRPA,
 * TPCA, LOGTB, LOGRPB, TPCB).  n must be >= 11. */
int ntt_schedule_params(uint32_t log2n, uint32_t id, int32_t* params, uint32_t n);
int ntt_plan_get_schedule(ntt_plan_t plan, uint32_t* id);

/*
 * Device status word of the plan: 0 or the first NTT_ERR_* a kernel recorded
 * (RANGE under NTT_FLAG_CHECK, TIMEOUT from a bounded wait).  Synchronises
 * `cuda_stream`, returns the status and clears it.
 */
int ntt_status(ntt_plan_t plan, void* cuda_stream);

/* Number of kernel launches the most recent call on this plan issued. */
int ntt_plan_last_launches(ntt_plan_t plan, uint32_t* launches);

/*
 * Integer-pipe peak probe (the denominator of the "alu" roofline): launches
 * blocks x threads threads, each running `iters` rounds of 8 independent
 * butterflies in registers with the exact arithmetic of the transform
 * kernels (kind 0: Harvey CT forward butterfly, kind 1: Harvey GS inverse
 * butterfly, both for any q < 2^62; kinds 2 and 3: the forward and inverse
 * butterflies of the small-modulus class, q < 2^57; kind 4: a 64 x 64 ->
 * 128-bit multiply-accumulate, the inner step of ntt_bconv, counted as one
 * operation; kind 5: the 32-bit forward butterfly of NTT_FLAG_WORD32 plans,
 * q < 2^30; kind 6: a Montgomery product (R = 2^64, odd q < 2^62), the
 * pointwise product formed inside ntt_inverse_mul and ntt_hmul_tensor;
 * kind 7: the inverse butterfly of moduli below 2^50, whose sum is not
 * reduced; kind 8: the 32-bit forward butterfly with its conditional
 * subtraction as compare and select, which a loop of independent
 * butterflies runs faster than kind 5's subtract-and-minimum form, while the
 * transform kernels are faster with the latter: the higher of kinds 5 and 8
 * is the 32-bit roofline denominator).  Total operations = blocks * threads
 * * iters * 8; time it with events on `cuda_stream`.
 * d_sink (blocks * threads uint64, caller-owned) only defeats dead-code
 * elimination.  Not part of the paper: a measurement aid.
 */
int ntt_bench_butterflies(uint64_t q, uint32_t kind, uint32_t blocks, uint32_t threads,
                          uint32_t iters, uint64_t* d_sink, void* cuda_stream);

/*
 * Test aid for the bounded device-side waits.  The paper has no counterpart:
 * its kernels synchronise with barriers that have no time limit, while every
 * wait of this library on an mbarrier (the pipelined transform form) gives
 * up after a fixed number of rounds, records NTT_ERR_TIMEOUT and returns, so
 * that a lost copy leaves the context usable.  This call makes that path
 * observable without any fault.
 * Launches one CTA of 32 threads that arms an mbarrier for 16 bytes and
 * waits on it with the same bounded wait, for at most `spin_limit` try_wait
 * rounds (1 .. NTT_DEBUG_SPIN_LIMIT_MAX; each round suspends the warp for a
 * hardware-chosen interval).
 *  - deliver != 0: one 16-byte bulk copy of the plan's first forward twiddle
 *    pair {w, w'} completes the barrier; the pair is written to d_out
 *    (2 uint64, caller-owned device memory, 16-byte aligned; may be NULL).
 *  - deliver == 0: no copy is issued, the wait runs out, and the kernel
 *    records NTT_ERR_TIMEOUT in the plan's status word (read and cleared by
 *    ntt_status).  Nothing is in flight when the CTA returns.
 * Errors: NTT_ERR_ARG for a NULL, host-only or 32-bit-word plan, a spin limit
 * out of range or a misaligned d_out; NTT_ERR_CUDA if the launch fails.
 * Asynchronous on cuda_stream.
 */
#define NTT_DEBUG_SPIN_LIMIT_MAX (1u << 22)
int ntt_debug_bounded_wait(ntt_plan_t plan, uint32_t deliver, uint32_t spin_limit, uint64_t* d_out,
                           void* cuda_stream);

/*
 * Uneven mixed batches (Sec. IV-A's batching of many independent transforms
 * into one launch, applied to whole requests): many requests of different N,
 * limb count, polynomial count and direction run in ONE persistent kernel
 * launch that pulls (request, row-range) work items from an atomic queue,
 * largest items first.  Each request has layout [n_polys][n_moduli][N] and
 * uses moduli_pool[moduli_offset .. moduli_offset + n_moduli).
 *   log2n          in [NTT_BATCH_MIN_LOG2N, NTT_MAX_LOG2N]
 *   inverse        0 forward, 1 inverse
 *   schedule       0: the request's rows are work items of the persistent
 *                  kernel.  s + 1 (s < ntt_schedule_count(log2n)): the
 *                  request runs instead as its own launch sequence with
 *                  schedule s of its N, on one of up to four branches that
 *                  fork from and join the caller's stream around the
 *                  persistent kernel (all in the same CUDA graph; the k-th
 *                  scheduled request goes to branch k mod 4).  Meant
 *                  for requests large enough to fill the GPU by themselves,
 *                  whose tuned schedule beats the batch kernel's fixed tiles.
 *   in / out       caller-owned device buffers (may alias), 16-byte aligned
 * ntt_batch_plan validates the requests, builds the twiddle tables of every
 * (N, pool modulus) pair the batch uses, and uploads the work-item list; the
 * batch plan owns those tables, the item list, the queue counter and (with
 * scheduled requests) up to four more streams and five events.  With
 * NTT_BATCH_GRAPH, execution captures [reset counter, kernel] (and the
 * scheduled requests' launches) into a CUDA graph on first use and replays
 * it afterwards.
 * ntt_batch_update replaces the requests' in/out pointers (same shapes),
 * enqueued on `cuda_stream` so the next execution (or graph replay) sees
 * them; with scheduled requests the graph is captured again on the next
 * execution, since their pointers are kernel arguments.  ntt_batch_execute_plain is the comparison arm: one launch sequence
 * per request on the same tables (schedules[i] per request, or the default
 * schedule of its N when schedules is NULL).
 * NTT_BATCH_GROUPED replaces the persistent kernel by grouped launches: the
 * unscheduled requests of one N, forward and inverse alike, are segments of
 * one grid per kernel phase of that N's configuration (one launch for N <=
 * 2^12, two above), CTA b working on the segment whose range of tile groups
 * holds b; the grids of different N go to the branches (N group k on branch
 * k mod 4 after the scheduled requests) so that their last waves overlap.
 * The same tables, pointers and results as the persistent form.
 * Errors: ARG, NOT_PRIME, NOT_NTT_FRIENDLY, MODULUS_TOO_LARGE, ALIGN,
 * UNSUPPORTED (log2n below NTT_BATCH_MIN_LOG2N), NOMEM, CUDA.
 */
#define NTT_BATCH_MIN_LOG2N 10
#define NTT_BATCH_GRAPH 1u
#define NTT_BATCH_GROUPED 4u

typedef struct {
    uint32_t log2n;
    uint32_t n_moduli;
    uint32_t n_polys;
    uint32_t moduli_offset;
    uint32_t inverse;
    uint32_t schedule;
    const uint64_t* in;
    uint64_t* out;
} ntt_request_t;

typedef struct ntt_batch_s* ntt_batch_t;

int ntt_batch_plan(ntt_batch_t* out, const ntt_request_t* reqs, uint32_t n_reqs,
                   const uint64_t* moduli_pool, uint32_t pool_len, uint32_t flags);
int ntt_batch_update(ntt_batch_t batch, const ntt_request_t* reqs, uint32_t n_reqs, void* cuda_stream);
int ntt_batch_execute(ntt_batch_t batch, void* cuda_stream);
int ntt_batch_execute_plain(ntt_batch_t batch, const uint32_t* schedules, void* cuda_stream);
int ntt_batch_destroy(ntt_batch_t batch);
/* Device status word of the batch (as ntt_status): synchronises, returns, clears. */
int ntt_batch_status(ntt_batch_t batch, void* cuda_stream);
/* Work items of the persistent kernel, kernels run by the last execution
 * (graph replays included), and coefficients per execution. */
int ntt_batch_info(ntt_batch_t batch, uint64_t* items, uint32_t* last_launches, uint64_t* coefficients);

/*
 * Schedule cost model kernels (the switch-point / fused-stage choice of
 * Sec. V-D, learned from measured timings): an FP32 MLP
 * NTT_MLP_IN -> 64 -> 64 -> NTT_MLP_OUT with ReLU hidden layers that maps a
 * transform shape (log2 N, limbs, batch, modulus bits; scaled features) to
 * the predicted log-time of every candidate schedule of that N.
 *   d_params  NTT_MLP_PARAMS floats: W1[64][IN], b1[64], W2[64][64], b2[64],
 *             W3[OUT][64], b3[OUT] (row-major)
 *   d_x       [batch][NTT_MLP_IN] features
 *   d_act     [batch][NTT_MLP_ACTS]: h1[64], h2[64], y[OUT] (written by forward)
 *   d_target, d_mask  [batch][NTT_MLP_OUT]: target log-times, 1/0 validity
 *   mask_count        sum of d_mask (the loss is the masked mean squared error)
 *   d_grad    NTT_MLP_PARAMS floats (written), d_work caller-owned scratch of
 *             batch * (NTT_MLP_ACTS + 1) floats, d_loss one float or NULL
 * ntt_mlp_adam applies one Adam step (bias-corrected, step >= 1) in place.
 * All device pointers are caller-owned; calls are asynchronous on the stream.
 */
#define NTT_MLP_IN 4
#define NTT_MLP_HIDDEN 64
#define NTT_MLP_OUT 12
#define NTT_MLP_PARAMS (NTT_MLP_HIDDEN * NTT_MLP_IN + NTT_MLP_HIDDEN + NTT_MLP_HIDDEN * NTT_MLP_HIDDEN + \
                        NTT_MLP_HIDDEN + NTT_MLP_OUT * NTT_MLP_HIDDEN + NTT_MLP_OUT)
#define NTT_MLP_ACTS (2 * NTT_MLP_HIDDEN + NTT_MLP_OUT)

int ntt_mlp_forward(const float* d_params, const float* d_x, uint32_t batch, float* d_act, void* cuda_stream);
int ntt_mlp_backward(const float* d_params, const float* d_x, const float* d_act, const float* d_target,
                     const float* d_mask, uint32_t batch, float mask_count, float* d_grad, float* d_work,
                     float* d_loss, void* cuda_stream);
int ntt_mlp_adam(float* d_params, const float* d_grad, float* d_m, float* d_v, uint32_t n, float lr,
                 float beta1, float beta2, float eps, uint32_t step, void* cuda_stream);

/*
 * Allocation-free execution of a mixed batch (no counterpart in the paper:
 * this is an interface for callers that cannot call cudaMalloc, e.g. code
 * that owns all device memory through its own allocator and reserves it at
 * start-up, plugin interfaces of host frameworks, or request paths where the
 * implicit device synchronisation of cudaMalloc is not acceptable).
 *
 * Runs the same persistent mixed-batch kernel as ntt_batch_execute, but the
 * kernel's scratch memory (work-queue counter and request descriptors) lives
 * in one file-scope __device__ array of NTT_STATIC_SCRATCH_BYTES that every
 * device loading the library holds until process exit.  The call allocates
 * no device memory; twiddle tables come from plans the caller created
 * earlier (ntt_plan, at a time when it could allocate).
 *   reqs[i].plan     a plan with N >= 2^NTT_BATCH_MIN_LOG2N on the current device
 *   reqs[i].n_polys  polynomials of the plan's layout to transform (0 = its batch)
 *   reqs[i].inverse  0 forward, 1 inverse
 *   reqs[i].in/out   device buffers [n_polys][n_moduli][N], 16-byte aligned, may alias
 * n_reqs must be in [1, NTT_STATIC_MAX_REQUESTS]; more is rejected with
 * NTT_ERR_ARG before anything is enqueued.  Range errors (NTT_FLAG_CHECK
 * plans) go to each request's plan status word (ntt_status).
 * The first call on a device sets that device up (it looks up the array's
 * device address with cudaGetSymbolAddress and the kernel's occupancy), so
 * make that first call outside any stream capture.  Every call reuses the
 * same array and overwrites what the previous call left there (the queue
 * counter is cleared on the stream at the start of each call); calls whose
 * executions overlap on the GPU (different streams without ordering, or
 * concurrent host threads) race on it and must be serialised by the caller.
 */
#define NTT_STATIC_SCRATCH_BYTES (64 * 1024)
#define NTT_STATIC_MAX_REQUESTS 816

typedef struct {
    ntt_plan_t plan;
    uint32_t n_polys;
    uint32_t inverse;
    const uint64_t* in;
    uint64_t* out;
} ntt_plan_request_t;

int ntt_batch_execute_static(const ntt_plan_request_t* reqs, uint32_t n_reqs, void* cuda_stream);

/*
 * TFHE external product and CMux step, batched over n_ct RLWE ciphertexts
 * that share one RGSW key: the batched CMux gate of Sec. IV-A (all
 * ciphertexts of one blind-rotation iteration use the same key RGSW(s_i));
 * blind rotation itself (Sec. II-B) repeats the CMux step once per LWE
 * coefficient.  One kernel launch, no scratch memory: each ciphertext is
 * decomposed, transformed, multiplied with the key and transformed back on
 * one SM.  The plan must hold one modulus q (prime, q = 1 mod 2N, q < 2^62)
 * and N = 2^10 or 2^11; it supplies the twiddle tables and the status word.
 *   d_in, d_acc   [n_ct][2][N] RLWE ciphertexts (B(x), A(x)), canonical
 *   d_rot         [n_ct] exponents a of x^a, taken mod 2N (CMux only)
 *   d_key         [2 levels][2][N] RGSW rows in the NTT domain (the forward
 *                 transform's bit-reversed order) as {w, floor(w 2^64 / q)}
 *                 pairs (16 bytes per entry), made once per key by
 *                 tfhe_key_prepare from canonical values; row i * levels + j
 *                 multiplies digit level j of input polynomial i
 *   levels, log2_base  the gadget B = 2^log2_base, l = levels:
 *                 1 <= l <= NTT_TFHE_MAX_LEVELS, l * log2_base <= 32, B^l < q
 *   d_out         [n_ct][2][N]; may be the same buffer as d_in / d_acc, no
 *                 other overlap.  d_in, d_acc, d_key, d_out 16-byte aligned.
 * Decomposition (the gadget over a prime q; the paper does not spell it out):
 * t = round(v B^l / q) mod B^l written with signed digits e_0..e_(l-1) in
 * [-B/2, B/2), e_0 most significant, each digit taken mod q.
 *   tfhe_external_product: out_c = sum_{i, j} e_j(d_i) * K[i l + j][c]
 *   tfhe_cmux_rotate:      out = acc + K [x] (x^a acc - acc)
 * with products in Z_q[x]/(x^N + 1).  Asynchronous on cuda_stream; n_ct = 0
 * launches nothing and does not look at the data pointers.
 * Errors: ARG (plan with several moduli, bad gadget, null pointers), ALIGN,
 * UNSUPPORTED (N), CUDA; with NTT_FLAG_CHECK plans a non-canonical input is
 * reported as NTT_ERR_RANGE through ntt_status.
 */
#define NTT_TFHE_MIN_LOG2N 10
#define NTT_TFHE_MAX_LOG2N 11
#define NTT_TFHE_MAX_LEVELS 8

/* d_key [2 levels][2][N] canonical -> d_key_shoup [2 levels][2][N][2] (one
 * kernel launch; NTT_FLAG_CHECK plans report keys >= q as NTT_ERR_RANGE). */
int tfhe_key_prepare(ntt_plan_t plan, const uint64_t* d_key, uint32_t levels, uint64_t* d_key_shoup,
                     void* cuda_stream);
int tfhe_external_product(ntt_plan_t plan, const uint64_t* d_in, const uint64_t* d_key, uint32_t levels,
                          uint32_t log2_base, uint64_t* d_out, uint64_t n_ct, void* cuda_stream);
int tfhe_cmux_rotate(ntt_plan_t plan, const uint64_t* d_acc, const uint32_t* d_rot, const uint64_t* d_key,
                     uint32_t levels, uint32_t log2_base, uint64_t* d_out, uint64_t n_ct, void* cuda_stream);

/*
 * RNS basis conversion (BConv), the CKKS key-switching operator beside the
 * NTT (Sec. III, Phase 1): residues of X modulo Q = q_0 ... q_(L-1) become
 * residues modulo p_0 ... p_(K-1),
 *   y_j = sum_i [x_i Qhat_i^-1]_{q_i} Qhat_i  mod p_j,   Qhat_i = Q / q_i,
 * the fast conversion, equal to X + alpha Q (mod p_j) for one integer
 * 0 <= alpha < L.  Coefficient domain, element by element.
 *   ntt_bconv_plan  precomputes the constants on the host and copies them to
 *                   the current device (the plan owns them); every modulus
 *                   an odd prime < 2^62, distinct within each basis,
 *                   1 <= L, K <= NTT_BCONV_MAX_MODULI
 *   ntt_bconv       d_in [n_polys][L][2^log2n] -> d_out [n_polys][K][2^log2n]
 *                   (device, 16-byte aligned, not overlapping; log2n >= 1);
 *                   inputs may be any 64-bit values (each x_i is reduced mod
 *                   q_i on the way)
 * Errors: ARG, NOT_PRIME, MODULUS_TOO_LARGE, ALIGN, NOMEM, CUDA.
 */
#define NTT_BCONV_MAX_MODULI 64
typedef struct ntt_bconv_s* ntt_bconv_t;

int ntt_bconv_plan(ntt_bconv_t* out, const uint64_t* q_from, uint32_t L, const uint64_t* p_to, uint32_t K);
int ntt_bconv(ntt_bconv_t bconv, const uint64_t* d_in, uint64_t* d_out, uint32_t log2n, uint64_t n_polys,
              void* cuda_stream);
int ntt_bconv_destroy(ntt_bconv_t bconv);

const char* ntt_strerror(int code);

/* Library version string ("ntt_gb300 <major>.<minor> sm_103a"). */
const char* ntt_version(void);

#ifdef __cplusplus
}
#endif

#endif /* NTT_GB300_H */
