/*
 * CPU oracle for the negacyclic NTT path -- TEST INFRASTRUCTURE ONLY.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg may
 * load this library.  It is deliberately plain and slow: every transform is
 * the O(N^2) definition written out with 128-bit integer products, so that a
 * reader can check it against the paper by eye.  It shares no code with the
 * CUDA path (no headers, no tables, no helpers).
 *
 * What it computes (arxiv 2410.05934, Sec. II-D, Eq. 1):
 *   ring R_q = Z_q[x]/(x^N + 1), psi a primitive 2N-th root of unity mod q.
 *   forward  NTT_{no->bo}^{CT,psi}:   A[j] = sum_i a[i] * psi^(i*(2*brv(j)+1))
 *            (evaluation of a(x) at the odd powers of psi, listed in
 *            bit-reversed order, which is what the Cooley-Tukey
 *            natural-in / bit-reversed-out transform of Eq. 1 produces)
 *   inverse  INTT_{bo->no}^{GS,psi^-1}: a[i] = N^-1 * sum_j A[j] * psi^(-i*(2*brv(j)+1))
 *   product  c = INTT(NTT(a) (.) NTT(b)) = a*b mod (x^N+1, q)       (Eq. 1)
 *   schoolbook  c_k = sum_{i+j=k} a_i b_j - sum_{i+j=k+N} a_i b_j   (mod q)
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *   - psi: g = smallest integer >= 2 with g^((q-1)/2) != 1 (a quadratic
 *     non-residue), psi = g^((q-1)/(2N)).  Then psi^N = -1 by Euler's
 *     criterion, so psi has order exactly 2N.
 *   - outputs are canonical residues in [0, q).
 *
 * Parity pins (tests/test_oracle_pins.py): brute-force root search for tiny q,
 * the convolution theorem against numpy's exact object-dtype convolution,
 * special vectors (delta, x, constants), order of psi via sympy, primality via
 * sympy, INTT(NTT(a)) = a.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

typedef unsigned __int128 u128;

/* ---- scalar arithmetic: the plain definitions ---- */

uint64_t oracle_mulmod(uint64_t a, uint64_t b, uint64_t q) {
    return (uint64_t)(((u128)a * (u128)b) % q);
}

uint64_t oracle_addmod(uint64_t a, uint64_t b, uint64_t q) {
    return (uint64_t)(((u128)a + (u128)b) % q);
}

uint64_t oracle_submod(uint64_t a, uint64_t b, uint64_t q) {
    return (uint64_t)(((u128)a + (u128)q - (u128)(b % q)) % q);
}

uint64_t oracle_powmod(uint64_t a, uint64_t e, uint64_t q) {
    uint64_t r = 1 % q, base = a % q;
    while (e) {
        if (e & 1) r = oracle_mulmod(r, base, q);
        base = oracle_mulmod(base, base, q);
        e >>= 1;
    }
    return r;
}

/* Deterministic Miller-Rabin: the first twelve primes as bases decide every
 * n < 3.3e24, so in particular every 64-bit n. */
int oracle_is_prime(uint64_t n) {
    static const uint64_t bases[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return 0;
    for (int i = 0; i < 12; i++) {
        if (n == bases[i]) return 1;
        if (n % bases[i] == 0) return 0;
    }
    uint64_t d = n - 1;
    int s = 0;
    while ((d & 1) == 0) { d >>= 1; s++; }
    for (int i = 0; i < 12; i++) {
        uint64_t x = oracle_powmod(bases[i], d, n);
        if (x == 1 || x == n - 1) continue;
        int composite = 1;
        for (int r = 1; r < s; r++) {
            x = oracle_mulmod(x, x, n);
            if (x == n - 1) { composite = 0; break; }
        }
        if (composite) return 0;
    }
    return 1;
}

/* psi for (q, N): returns 0 when q is not a prime with q = 1 mod 2N. */
uint64_t oracle_psi(uint64_t q, uint32_t log2n) {
    uint64_t two_n = (uint64_t)2 << log2n;
    if (!oracle_is_prime(q) || (q - 1) % two_n != 0) return 0;
    uint64_t g = 2;
    while (oracle_powmod(g, (q - 1) / 2, q) == 1) g++;
    return oracle_powmod(g, (q - 1) / two_n, q);
}

uint32_t oracle_bitrev(uint32_t j, uint32_t log2n) {
    uint32_t r = 0;
    for (uint32_t b = 0; b < log2n; b++)
        if (j & (1u << b)) r |= 1u << (log2n - 1 - b);
    return r;
}

/* Table of psi^k for k in [0, 2N): since psi^(2N) = 1 every exponent in the
 * definitions can be taken mod 2N. */
static uint64_t* psi_powers(uint64_t psi, uint32_t log2n, uint64_t q) {
    uint64_t two_n = (uint64_t)2 << log2n;
    uint64_t* pw = (uint64_t*)malloc(sizeof(uint64_t) * two_n);
    if (!pw) return NULL;
    pw[0] = 1 % q;
    for (uint64_t k = 1; k < two_n; k++) pw[k] = oracle_mulmod(pw[k - 1], psi, q);
    return pw;
}

/* ---- one-polynomial transforms, straight from the definitions ---- */

/* A[j] for the listed output indices j (all N of them when idx == NULL). */
int oracle_ntt_forward_at(const uint64_t* a, uint32_t log2n, uint64_t q, uint64_t psi,
                          const uint32_t* idx, uint32_t n_idx, uint64_t* out) {
    uint64_t n = (uint64_t)1 << log2n, two_n = 2 * n;
    uint64_t* pw = psi_powers(psi, log2n, q);
    if (!pw) return -1;
    uint32_t count = idx ? n_idx : (uint32_t)n;
    for (uint32_t t = 0; t < count; t++) {
        uint32_t j = idx ? idx[t] : t;
        uint64_t odd = 2 * (uint64_t)oracle_bitrev(j, log2n) + 1;
        uint64_t acc = 0;
        for (uint64_t i = 0; i < n; i++) {
            uint64_t e = (i * odd) % two_n;
            acc = oracle_addmod(acc, oracle_mulmod(a[i] % q, pw[e], q), q);
        }
        out[t] = acc;
    }
    free(pw);
    return 0;
}

/* a[i] for the listed coefficient indices i (all N of them when idx == NULL). */
int oracle_ntt_inverse_at(const uint64_t* A, uint32_t log2n, uint64_t q, uint64_t psi,
                          const uint32_t* idx, uint32_t n_idx, uint64_t* out) {
    uint64_t n = (uint64_t)1 << log2n, two_n = 2 * n;
    uint64_t* pw = psi_powers(psi, log2n, q);
    if (!pw) return -1;
    /* N^-1 = N^(q-2) by Fermat (q prime). */
    uint64_t n_inv = oracle_powmod(n % q, q - 2, q);
    uint32_t count = idx ? n_idx : (uint32_t)n;
    for (uint32_t t = 0; t < count; t++) {
        uint64_t i = idx ? idx[t] : t;
        uint64_t acc = 0;
        for (uint64_t j = 0; j < n; j++) {
            uint64_t odd = 2 * (uint64_t)oracle_bitrev((uint32_t)j, log2n) + 1;
            /* psi^(-e) = psi^(2N - e mod 2N) */
            uint64_t e = (two_n - (i * odd) % two_n) % two_n;
            acc = oracle_addmod(acc, oracle_mulmod(A[j] % q, pw[e], q), q);
        }
        out[t] = oracle_mulmod(acc, n_inv, q);
    }
    free(pw);
    return 0;
}

void oracle_pointwise(const uint64_t* a, const uint64_t* b, uint64_t* c, uint64_t n, uint64_t q) {
    for (uint64_t i = 0; i < n; i++) c[i] = oracle_mulmod(a[i] % q, b[i] % q, q);
}

/* c = a * b mod (x^N + 1, q): x^N = -1 folds the upper half back with a minus sign. */
void oracle_negacyclic_schoolbook(const uint64_t* a, const uint64_t* b, uint64_t* c,
                                  uint32_t log2n, uint64_t q) {
    uint64_t n = (uint64_t)1 << log2n;
    for (uint64_t k = 0; k < n; k++) c[k] = 0;
    for (uint64_t i = 0; i < n; i++) {
        for (uint64_t j = 0; j < n; j++) {
            uint64_t p = oracle_mulmod(a[i] % q, b[j] % q, q);
            uint64_t k = i + j;
            if (k < n) c[k] = oracle_addmod(c[k], p, q);
            else       c[k - n] = oracle_submod(c[k - n], p, q);
        }
    }
}

/* Selected coefficients c_k (k in idx) of a * b mod (x^N + 1, q), each from
 * its O(N) defining sum: c_k = sum_{i<=k} a_i b_{k-i} - sum_{i>k} a_i b_{N+k-i}. */
void oracle_negacyclic_schoolbook_at(const uint64_t* a, const uint64_t* b, uint32_t log2n, uint64_t q,
                                     const uint32_t* idx, uint32_t n_idx, uint64_t* out) {
    uint64_t n = (uint64_t)1 << log2n;
    for (uint32_t t = 0; t < n_idx; t++) {
        uint64_t k = idx[t], acc = 0;
        for (uint64_t i = 0; i < n; i++) {
            if (i <= k) acc = oracle_addmod(acc, oracle_mulmod(a[i] % q, b[k - i] % q, q), q);
            else        acc = oracle_submod(acc, oracle_mulmod(a[i] % q, b[n + k - i] % q, q), q);
        }
        out[t] = acc;
    }
}

/* ---- many rows over host threads (rows are independent) ---- */

typedef struct {
    int inverse;
    const uint64_t* in;
    uint64_t* out;
    uint32_t rows, log2n;
    const uint64_t* q_row;
    const uint64_t* psi_row;
    const uint32_t* idx;     /* per-row sampled indices, rows*n_idx, or NULL */
    uint32_t n_idx;
    uint32_t next;           /* next row to take (protected by mu) */
    pthread_mutex_t mu;
    int err;
} rows_job;

static void* rows_worker(void* arg) {
    rows_job* job = (rows_job*)arg;
    uint64_t n = (uint64_t)1 << job->log2n;
    for (;;) {
        pthread_mutex_lock(&job->mu);
        uint32_t r = job->next++;
        pthread_mutex_unlock(&job->mu);
        if (r >= job->rows) break;
        const uint64_t* src = job->in + (uint64_t)r * n;
        const uint32_t* idx = job->idx ? job->idx + (uint64_t)r * job->n_idx : NULL;
        uint64_t* dst = job->out + (uint64_t)r * (job->idx ? job->n_idx : n);
        int rc = job->inverse
            ? oracle_ntt_inverse_at(src, job->log2n, job->q_row[r], job->psi_row[r], idx, job->n_idx, dst)
            : oracle_ntt_forward_at(src, job->log2n, job->q_row[r], job->psi_row[r], idx, job->n_idx, dst);
        if (rc) job->err = rc;
    }
    return NULL;
}

/* Transforms `rows` rows of N coefficients.  Row r uses modulus q_row[r] and
 * root psi_row[r].  With idx != NULL only n_idx outputs per row are computed
 * (row r's indices are idx[r*n_idx ...]) and out holds rows*n_idx values. */
int oracle_transform_rows(int inverse, const uint64_t* in, uint64_t* out, uint32_t rows,
                          uint32_t log2n, const uint64_t* q_row, const uint64_t* psi_row,
                          const uint32_t* idx, uint32_t n_idx, int nthreads) {
    rows_job job;
    job.inverse = inverse; job.in = in; job.out = out; job.rows = rows; job.log2n = log2n;
    job.q_row = q_row; job.psi_row = psi_row; job.idx = idx; job.n_idx = n_idx;
    job.next = 0; job.err = 0;
    pthread_mutex_init(&job.mu, NULL);
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    pthread_t th[256];
    for (int t = 0; t < nthreads; t++) pthread_create(&th[t], NULL, rows_worker, &job);
    for (int t = 0; t < nthreads; t++) pthread_join(th[t], NULL);
    pthread_mutex_destroy(&job.mu);
    return job.err;
}

/* Output-parallel variant for few, long rows: the (row, output) pairs are
 * split over threads.  Same arithmetic as oracle_ntt_*_at. */
typedef struct {
    int inverse;
    const uint64_t* in;
    uint64_t* out;
    uint32_t rows, log2n;
    const uint64_t* q_row;
    const uint64_t* psi_row;
    uint32_t chunk;
    uint64_t next;
    pthread_mutex_t mu;
    int err;
} outs_job;

static void* outs_worker(void* arg) {
    outs_job* job = (outs_job*)arg;
    uint64_t n = (uint64_t)1 << job->log2n;
    /* tasks never straddle rows: task t covers row t / per_row */
    uint64_t per_row = (n + job->chunk - 1) / job->chunk;
    uint64_t total = (uint64_t)job->rows * per_row;
    uint32_t* idx = (uint32_t*)malloc(sizeof(uint32_t) * job->chunk);
    if (!idx) { job->err = -1; return NULL; }
    for (;;) {
        pthread_mutex_lock(&job->mu);
        uint64_t task = job->next++;
        pthread_mutex_unlock(&job->mu);
        if (task >= total) break;
        uint64_t r = task / per_row;
        uint64_t j0 = (task % per_row) * job->chunk;
        uint32_t cnt = job->chunk;
        if (j0 + cnt > n) cnt = (uint32_t)(n - j0);
        for (uint32_t t = 0; t < cnt; t++) idx[t] = (uint32_t)(j0 + t);
        const uint64_t* src = job->in + r * n;
        uint64_t* dst = job->out + r * n + j0;
        int rc = job->inverse
            ? oracle_ntt_inverse_at(src, job->log2n, job->q_row[r], job->psi_row[r], idx, cnt, dst)
            : oracle_ntt_forward_at(src, job->log2n, job->q_row[r], job->psi_row[r], idx, cnt, dst);
        if (rc) job->err = rc;
    }
    free(idx);
    return NULL;
}

int oracle_transform_rows_split(int inverse, const uint64_t* in, uint64_t* out, uint32_t rows,
                                uint32_t log2n, const uint64_t* q_row, const uint64_t* psi_row,
                                uint32_t chunk, int nthreads) {
    outs_job job;
    job.inverse = inverse; job.in = in; job.out = out; job.rows = rows; job.log2n = log2n;
    job.q_row = q_row; job.psi_row = psi_row; job.chunk = chunk ? chunk : 64;
    job.next = 0; job.err = 0;
    pthread_mutex_init(&job.mu, NULL);
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    pthread_t th[256];
    for (int t = 0; t < nthreads; t++) pthread_create(&th[t], NULL, outs_worker, &job);
    for (int t = 0; t < nthreads; t++) pthread_join(th[t], NULL);
    pthread_mutex_destroy(&job.mu);
    return job.err;
}
