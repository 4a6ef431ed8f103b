/*
 * Plain CPU radix-2 NTT -- the second, O(N log N) CPU BASELINE of bench.py
 * (TEST INFRASTRUCTURE ONLY, like the rest of oracle/).
 *
 * The O(N^2) definitions in ntt_oracle.c are what parity is checked against;
 * this file is the fairer CPU timing arm: the textbook iterative transforms
 * of Eq. 1 (Sec. II-D), one row at a time, rows spread over host threads.
 * It shares no code with the CUDA path.
 *
 *   forward  Cooley-Tukey, natural order in, bit-reversed order out, psi
 *            merged into the twiddles: stage m (m = 1, 2, 4, ..., N/2) pairs
 *            a[j] and a[j + t] (t = N / 2m) inside block i with the twiddle
 *            W[m + i] = psi^brv(m + i), brv over log2 N bits;
 *              (U, V) -> (U + V W, U - V W)  mod q
 *   inverse  Gentleman-Sande, bit-reversed in, natural out, twiddles
 *            psi^-brv(m + i), stages in the opposite order;
 *              (U, V) -> (U + V, (U - V) W)  mod q,  then every output x N^-1
 *
 * Twiddle products use Shoup's precomputed quotient w' = floor(w 2^64 / q):
 * for x, w < q, r = x w - floor(x w' / 2^64) q lies in [0, 2q), one
 * conditional subtraction gives x w mod q.  Every value stays canonical
 * ([0, q)) after each butterfly; q < 2^62.
 *
 * Pinned by tests/test_oracle_radix2.py against the O(N^2) definitions.
 */
#include <stdint.h>
#include <stdlib.h>
#include <pthread.h>

typedef unsigned __int128 u128;

uint64_t oracle_powmod(uint64_t a, uint64_t e, uint64_t q);
uint64_t oracle_psi(uint64_t q, uint32_t log2n);

static uint32_t rev_bits(uint32_t k, uint32_t bits) {
    uint32_t r = 0;
    for (uint32_t i = 0; i < bits; i++) r |= ((k >> i) & 1u) << (bits - 1 - i);
    return r;
}

static uint64_t shoup_of(uint64_t w, uint64_t q) { return (uint64_t)(((u128)w << 64) / q); }

static uint64_t mul_shoup(uint64_t x, uint64_t w, uint64_t wp, uint64_t q) {
    uint64_t quo = (uint64_t)(((u128)x * wp) >> 64);
    uint64_t r = x * w - quo * q;
    return r >= q ? r - q : r;
}

/* Tables of one modulus: fwd[k] = psi^brv(k), inv[k] = psi^-brv(k), k < N,
 * each followed by its Shoup quotient; n_inv = N^-1 mod q and its quotient. */
typedef struct {
    uint64_t q, n_inv, n_inv_p;
    uint64_t *fw, *fwp, *iw, *iwp;
} r2_tables;

static int r2_tables_make(r2_tables* t, uint64_t q, uint32_t log2n) {
    uint64_t n = (uint64_t)1 << log2n;
    t->q = q;
    t->fw = (uint64_t*)malloc(4 * n * sizeof(uint64_t));
    if (!t->fw) return -1;
    t->fwp = t->fw + n;
    t->iw = t->fw + 2 * n;
    t->iwp = t->fw + 3 * n;
    uint64_t psi = oracle_psi(q, log2n);
    if (!psi) { free(t->fw); t->fw = NULL; return -1; }
    uint64_t psi_inv = oracle_powmod(psi, 2 * n - 1, q);     /* psi^(2N - 1) = psi^-1 */
    uint64_t p = 1, pi = 1;
    /* powers in natural order, then placed at their bit-reversed slots */
    for (uint64_t e = 0; e < n; e++) {
        uint32_t k = rev_bits((uint32_t)e, log2n);
        t->fw[k] = p;
        t->iw[k] = pi;
        p = (uint64_t)(((u128)p * psi) % q);
        pi = (uint64_t)(((u128)pi * psi_inv) % q);
    }
    for (uint64_t k = 0; k < n; k++) {
        t->fwp[k] = shoup_of(t->fw[k], q);
        t->iwp[k] = shoup_of(t->iw[k], q);
    }
    t->n_inv = oracle_powmod(n % q, q - 2, q);
    t->n_inv_p = shoup_of(t->n_inv, q);
    return 0;
}

static void r2_forward(uint64_t* a, uint32_t log2n, const r2_tables* t) {
    uint64_t n = (uint64_t)1 << log2n, q = t->q, len = n;
    for (uint64_t m = 1; m < n; m <<= 1) {
        len >>= 1;                                   /* half-block length t */
        for (uint64_t i = 0; i < m; i++) {
            uint64_t w = t->fw[m + i], wp = t->fwp[m + i];
            uint64_t* x = a + 2 * i * len;
            for (uint64_t j = 0; j < len; j++) {
                uint64_t u = x[j];
                uint64_t v = mul_shoup(x[j + len], w, wp, q);
                uint64_t s = u + v;
                x[j] = s >= q ? s - q : s;
                x[j + len] = u >= v ? u - v : u + q - v;
            }
        }
    }
}

static void r2_inverse(uint64_t* a, uint32_t log2n, const r2_tables* t) {
    uint64_t n = (uint64_t)1 << log2n, q = t->q, len = 1;
    for (uint64_t m = n >> 1; m >= 1; m >>= 1) {
        for (uint64_t i = 0; i < m; i++) {
            uint64_t w = t->iw[m + i], wp = t->iwp[m + i];
            uint64_t* x = a + 2 * i * len;
            for (uint64_t j = 0; j < len; j++) {
                uint64_t u = x[j], v = x[j + len];
                uint64_t s = u + v;
                x[j] = s >= q ? s - q : s;
                x[j + len] = mul_shoup(u >= v ? u - v : u + q - v, w, wp, q);
            }
        }
        len <<= 1;
    }
    for (uint64_t k = 0; k < n; k++) a[k] = mul_shoup(a[k], t->n_inv, t->n_inv_p, q);
}

typedef struct {
    int inverse;
    const uint64_t* in;
    uint64_t* out;
    uint32_t rows, log2n, n_moduli;
    const r2_tables* tab;     /* n_moduli tables; row r uses r mod n_moduli */
    uint32_t next;
    pthread_mutex_t mu;
} r2_job;

static void* r2_worker(void* arg) {
    r2_job* job = (r2_job*)arg;
    uint64_t n = (uint64_t)1 << job->log2n;
    for (;;) {
        pthread_mutex_lock(&job->mu);
        uint32_t r = job->next++;
        pthread_mutex_unlock(&job->mu);
        if (r >= job->rows) break;
        uint64_t* dst = job->out + (uint64_t)r * n;
        const uint64_t* src = job->in + (uint64_t)r * n;
        for (uint64_t k = 0; k < n; k++) dst[k] = src[k];
        const r2_tables* t = &job->tab[r % job->n_moduli];
        if (job->inverse) r2_inverse(dst, job->log2n, t);
        else r2_forward(dst, job->log2n, t);
    }
    return NULL;
}

/* Transforms `rows` rows laid out [rows][N]; row r uses moduli[r % n_moduli]
 * (the [poly][limb][N] layout).  Tables are built once per modulus before the
 * rows run.  Inputs must be canonical.  Returns 0, or -1 on a bad argument or
 * allocation failure. */
int oracle_radix2_rows(int inverse, const uint64_t* in, uint64_t* out, uint32_t rows, uint32_t log2n,
                       const uint64_t* moduli, uint32_t n_moduli, int nthreads) {
    if (log2n < 1 || log2n > 20 || n_moduli == 0) return -1;
    r2_tables* tab = (r2_tables*)calloc(n_moduli, sizeof(r2_tables));
    if (!tab) return -1;
    int rc = 0;
    for (uint32_t l = 0; l < n_moduli && !rc; l++) {
        if (moduli[l] < 3 || moduli[l] >= ((uint64_t)1 << 62)) rc = -1;
        else rc = r2_tables_make(&tab[l], moduli[l], log2n);
    }
    if (!rc) {
        r2_job job;
        job.inverse = inverse; job.in = in; job.out = out; job.rows = rows; job.log2n = log2n;
        job.n_moduli = n_moduli; job.tab = tab; job.next = 0;
        pthread_mutex_init(&job.mu, NULL);
        if (nthreads < 1) nthreads = 1;
        if (nthreads > 256) nthreads = 256;
        pthread_t th[256];
        for (int t = 0; t < nthreads; t++) pthread_create(&th[t], NULL, r2_worker, &job);
        for (int t = 0; t < nthreads; t++) pthread_join(th[t], NULL);
        pthread_mutex_destroy(&job.mu);
    }
    for (uint32_t l = 0; l < n_moduli; l++) free(tab[l].fw);
    free(tab);
    return rc;
}
