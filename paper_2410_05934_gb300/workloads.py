"""Seeded synthetic inputs for the negacyclic NTT workloads.

This module holds no NTT arithmetic: it only draws coefficients and request
lists from a counter-based generator, so the CUDA path and the CPU oracle can
be fed identical inputs.  Generator (stated so either side can re-implement
it): for element index i of stream s under seed S,

    key(S, s)   = mix64(S * 0x9E3779B97F4A7C15 + s * 0xD1B54A32D192ED03 + 1)
    draw(i, t)  = mix64(key + (i + t * 2^40 + 1) * 0x9E3779B97F4A7C15)   (mod 2^64)

with mix64 the splitmix64 finaliser.  A value uniform in [0, q) takes the top
bit_length(q) bits of draw(i, 0), draw(i, 1), ... and keeps the first one
below q (rejection sampling, acceptance > 1/2 per try).

Workloads (the paper's parameter shapes, Sec. VI-A and VI-E):
  plain_n1024      N=1024, one 59-bit prime, 64 rows + 32 product pairs
  ckks_hmul_n65536 N=65536, 24 RNS limbs of 50-bit primes, 4 polynomials
                   (2 ciphertexts x 2 components) -> 96 rows
  tfhe_blind_rot   N=1024, one 62-bit prime, 3780 forward rows of signed
                   digits in [-128, 128) and 1260 inverse rows
  mixed_batch      200 requests, N in {2^10,2^12,2^14,2^16} (weights
                   .5/.2/.2/.1), limbs U{1..32}, polys U{1..64}
"""
import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
DELTA = np.uint64(0xD1B54A32D192ED03)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
ATTEMPT_STRIDE = 1 << 40

DEFAULT_SEED = 2410

# Largest prime below 2^59 with q = 1 mod 2048 (word-size TFHE/CKKS modulus).
Q59_N1024 = 576460752303421441
# Largest prime below 2^62 with q = 1 mod 2048 (64-bit TFHE modulus).
Q62_N1024 = 4611686018427365377
# The 48 largest primes below 2^50 with q = 1 mod 2^17, descending: NTT-friendly
# for every N <= 2^16.  A request with k limbs takes the first k.
POOL50 = [
    1125899903827969, 1125899902124033, 1125899887312897, 1125899886395393,
    1125899885740033, 1125899884167169, 1125899884036097, 1125899883642881,
    1125899883380737, 1125899882987521, 1125899879710721, 1125899877875713,
    1125899870404609, 1125899870011393, 1125899865948161, 1125899864506369,
    1125899862016001, 1125899861753857, 1125899859263489, 1125899852578817,
    1125899851530241, 1125899846025217, 1125899844714497, 1125899843665921,
    1125899842486273, 1125899842093057, 1125899841175553, 1125899840520193,
    1125899839602689, 1125899834490881, 1125899834228737, 1125899831345153,
    1125899831083009, 1125899828723713, 1125899823087617, 1125899822694401,
    1125899822432257, 1125899821907969, 1125899818762241, 1125899817582593,
    1125899816927233, 1125899810635777, 1125899806965761, 1125899804999681,
    1125899799887873, 1125899799232513, 1125899795955713, 1125899795562497,
]


def mix64(z):
    """splitmix64 finaliser on a numpy uint64 array (wrapping arithmetic)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def stream_key(seed, stream):
    with np.errstate(over="ignore"):
        k = np.uint64(seed) * GAMMA + np.uint64(stream) * DELTA + np.uint64(1)
    return mix64(k)


def draws(seed, stream, count, attempt=0, start=0):
    """Raw 64-bit draws for indices start..start+count-1 at a given attempt."""
    key = stream_key(seed, stream)
    i = np.arange(start, start + count, dtype=np.uint64)
    with np.errstate(over="ignore"):
        ctr = i + np.uint64(attempt * ATTEMPT_STRIDE + 1)
        return mix64(key + ctr * GAMMA)


def uniform_mod(seed, stream, count, q, start=0):
    """count values uniform in [0, q) by rejection on the top bits."""
    q = int(q)
    bits = q.bit_length()
    shift = np.uint64(64 - bits)
    out = draws(seed, stream, count, 0, start) >> shift
    bad = np.nonzero(out >= np.uint64(q))[0]
    attempt = 1
    while bad.size:
        redraw = draws(seed, stream, count, attempt, start)[bad] >> shift
        out[bad] = redraw
        bad = bad[redraw >= np.uint64(q)]
        attempt += 1
    return out


def signed_digits_mod(seed, stream, count, q, lo=-128, hi=128, start=0):
    """Signed digits uniform in [lo, hi) (hi-lo a power of two), reduced mod q."""
    span = hi - lo
    assert span & (span - 1) == 0
    bits = span.bit_length() - 1
    d = (draws(seed, stream, count, 0, start) >> np.uint64(64 - bits)).astype(np.int64) + lo
    out = d.astype(np.uint64)
    neg = d < 0
    out[neg] = (d[neg] + q).astype(np.uint64)
    return out


def rows_uniform(seed, stream, moduli_per_row, n):
    """One row of n values per modulus, row r uniform in [0, moduli_per_row[r])."""
    rows = len(moduli_per_row)
    out = np.empty((rows, n), dtype=np.uint64)
    for r, q in enumerate(moduli_per_row):
        out[r] = uniform_mod(seed, stream, n, q, start=r * n)
    return out


# ---- the workloads ----------------------------------------------------------

def plain_n1024(seed=DEFAULT_SEED):
    """64 rows at N=1024 under one 59-bit prime; product pairs (r, r+32)."""
    n, rows = 1024, 64
    x = rows_uniform(seed, 1, [Q59_N1024] * rows, n)
    return dict(log2n=10, moduli=[Q59_N1024], batch=rows, x=x)


def ckks_hmul_n65536(seed=DEFAULT_SEED, limbs=24, polys=4):
    """4 polynomials x 24 limbs at N=65536; layout [poly][limb][N]."""
    n = 1 << 16
    moduli = POOL50[:limbs]
    per_row = [moduli[l] for _ in range(polys) for l in range(limbs)]
    x = rows_uniform(seed, 2, per_row, n)
    return dict(log2n=16, moduli=moduli, batch=polys, x=x.reshape(polys, limbs, n))


def tfhe_blind_rotation(seed=DEFAULT_SEED, n_lwe=630, k1=2, levels=3):
    """Forward rows: n_lwe*k1*levels signed-digit polys; inverse rows: n_lwe*k1."""
    n = 1024
    fwd_rows, inv_rows = n_lwe * k1 * levels, n_lwe * k1
    fwd = signed_digits_mod(seed, 3, fwd_rows * n, Q62_N1024).reshape(fwd_rows, n)
    inv = uniform_mod(seed, 4, inv_rows * n, Q62_N1024).reshape(inv_rows, n)
    return dict(log2n=10, moduli=[Q62_N1024], fwd=fwd, inv=inv)


def tfhe_cmux(seed=DEFAULT_SEED, n_ct=1024, log2n=10, q=Q62_N1024, levels=3, steps=1):
    """Batched CMux steps: n_ct RLWE accumulators [n_ct][2][N] uniform mod q,
    rotation exponents [steps][n_ct] uniform in [0, 2N), and one RGSW key per
    step [steps][2 levels][2][N] uniform mod q (NTT domain)."""
    n = 1 << log2n
    acc = uniform_mod(seed, 6, n_ct * 2 * n, q).reshape(n_ct, 2, n)
    rot = (draws(seed, 7, steps * n_ct) >> np.uint64(64 - (log2n + 1))).astype(np.uint32).reshape(steps, n_ct)
    key = uniform_mod(seed, 8, steps * 2 * levels * 2 * n, q).reshape(steps, 2 * levels, 2, n)
    return dict(log2n=log2n, moduli=[q], levels=levels, acc=acc, rot=rot, key=key)


def ckks_bconv(seed=DEFAULT_SEED, log2n=16, L=24, K=24, polys=2):
    """Key-switching basis conversion of a ciphertext (hybrid key switching
    with one digit, ModUp): polys x L limbs over Q = POOL50[:L], converted to
    K special primes P = POOL50[L:L+K]; layout [poly][limb][N]."""
    n = 1 << log2n
    Q, P = POOL50[:L], POOL50[L:L + K]
    per_row = [Q[l] for _ in range(polys) for l in range(L)]
    x = rows_uniform(seed, 9, per_row, n)
    return dict(log2n=log2n, Q=Q, P=P, x=x.reshape(polys, L, n))


def mixed_requests(seed=DEFAULT_SEED, n_requests=200, max_limbs=32, max_polys=64,
                   log2ns=(10, 12, 14, 16), weights=(0.5, 0.2, 0.2, 0.1)):
    """The uneven request list: (log2n, limbs, polys) per request."""
    d = draws(seed, 5, 3 * n_requests)
    u = (d >> np.uint64(11)).astype(np.float64) / float(1 << 53)
    cum = np.cumsum(weights)
    reqs = []
    for r in range(n_requests):
        k = int(np.searchsorted(cum, u[3 * r], side="right"))
        k = min(k, len(log2ns) - 1)
        limbs = 1 + int(u[3 * r + 1] * max_limbs)
        polys = 1 + int(u[3 * r + 2] * max_polys)
        reqs.append((log2ns[k], min(limbs, max_limbs), min(polys, max_polys)))
    return reqs


def request_rows(seed, req_index, log2n, limbs, polys, pool=POOL50):
    """Coefficients of one mixed-batch request, layout [poly][limb][N]."""
    n = 1 << log2n
    per_row = [pool[l] for _ in range(polys) for l in range(limbs)]
    out = np.empty((len(per_row), n), dtype=np.uint64)
    for r, q in enumerate(per_row):
        out[r] = uniform_mod(seed, 1000 + req_index, n, q, start=r * n)
    return out


# ---- the same generator on a torch device (int64 arithmetic wraps mod 2^64) ----

def _s64(v):
    v = int(v) & 0xFFFFFFFFFFFFFFFF
    return v - (1 << 64) if v >= (1 << 63) else v


def _lsr(t, k):
    """logical right shift of int64 bit patterns"""
    return (t >> k) & ((1 << (64 - k)) - 1)


def mix64_torch(z):
    z = (z ^ _lsr(z, 30)) * _s64(_M1)
    z = (z ^ _lsr(z, 27)) * _s64(_M2)
    return z ^ _lsr(z, 31)


def uniform_mod_torch(seed, stream, count, q, start=0, device="cuda"):
    """uniform_mod on a torch device: identical values, returned as int64 bit patterns."""
    import torch
    q = int(q)
    shift = 64 - q.bit_length()
    key = int(stream_key(seed, stream))
    i = torch.arange(start, start + count, dtype=torch.int64, device=device)

    def draw(attempt):
        ctr = i + (attempt * ATTEMPT_STRIDE + 1)
        return _lsr(mix64_torch(ctr * _s64(GAMMA) + _s64(key)), shift)

    out = draw(0)
    attempt = 1
    bad = out >= q
    while bool(bad.any()):
        out = torch.where(bad, draw(attempt), out)
        bad = out >= q
        attempt += 1
    return out


def uniform_mod_torch_idx(seed, stream, idx, q):
    """uniform_mod at arbitrary element indices idx (int64 tensor)."""
    import torch
    q = int(q)
    shift = 64 - q.bit_length()
    key = int(stream_key(seed, stream))

    def draw(attempt):
        ctr = idx + (attempt * ATTEMPT_STRIDE + 1)
        return _lsr(mix64_torch(ctr * _s64(GAMMA) + _s64(key)), shift)

    out = draw(0)
    attempt = 1
    bad = out >= q
    while bool(bad.any()):
        out = torch.where(bad, draw(attempt), out)
        bad = out >= q
        attempt += 1
    return out


def request_rows_torch(seed, req_index, log2n, limbs, polys, pool=POOL50, device="cuda"):
    """request_rows on a torch device ([polys * limbs, N] int64 bit patterns),
    one vectorised draw per limb."""
    import torch
    n = 1 << log2n
    out = torch.empty((polys, limbs, n), dtype=torch.int64, device=device)
    j = torch.arange(n, dtype=torch.int64, device=device)
    p = torch.arange(polys, dtype=torch.int64, device=device)
    for l in range(limbs):
        idx = (p[:, None] * limbs + l) * n + j[None, :]
        out[:, l, :] = uniform_mod_torch_idx(seed, 1000 + req_index, idx, pool[l])
    return out.view(polys * limbs, n)
