"""Pins for the CPU oracle (Sec. II-D, Eq. 1): every check here comes from
something other than the oracle's own formulas -- brute-force root search,
sympy's number theory, numpy's exact convolution, the recursive structure of
the Cooley-Tukey bit-reversed output, and special vectors with closed forms.
"""
import random

import numpy as np
import pytest

from paper_2410_05934_gb300 import workloads as W

SMALL_CASES = [  # (q, log2n) with q = 1 mod 2N
    (17, 1), (17, 2), (17, 3), (97, 4), (257, 5), (257, 6), (7681, 8), (12289, 10),
]
BIG_PRIMES = [W.Q59_N1024, W.Q62_N1024, W.POOL50[0], W.POOL50[23]]


def _trial_division_is_prime(n):
    if n < 2:
        return False
    d = 2
    while d * d <= n:
        if n % d == 0:
            return False
        d += 1
    return True


def test_miller_rabin_matches_trial_division(oracle):
    for n in range(0, 20000):
        assert oracle.is_prime(n) == _trial_division_is_prime(n), n


def test_miller_rabin_hard_composites_and_sympy(oracle):
    sympy = pytest.importorskip("sympy")
    # Carmichael numbers and strong pseudoprimes to several small bases.
    for n in [561, 1105, 1729, 2465, 2821, 6601, 3215031751, 2152302898747,
              3474749660383, 341550071728321, 3825123056546413051]:
        assert not oracle.is_prime(n), n
    rng = random.Random(7)
    for _ in range(3000):
        n = rng.getrandbits(64) | 1
        assert oracle.is_prime(n) == sympy.isprime(n), n
    for q in BIG_PRIMES + W.POOL50:
        assert oracle.is_prime(q) and sympy.isprime(q)


def test_workload_primes_are_the_stated_ones():
    """The moduli are exactly 'the largest primes below 2^k with q = 1 mod 2N'."""
    sympy = pytest.importorskip("sympy")

    def largest(bits, step, count):
        q = ((1 << bits) - 1) // step * step + 1
        out = []
        while len(out) < count:
            if sympy.isprime(q):
                out.append(q)
            q -= step
        return out

    assert W.POOL50 == largest(50, 1 << 17, 48)
    assert [W.Q59_N1024] == largest(59, 2048, 1)
    assert [W.Q62_N1024] == largest(62, 2048, 1)
    assert all(q.bit_length() == 50 for q in W.POOL50)


def test_bitrev_is_string_reversal(oracle):
    for log2n in range(1, 12):
        for j in range(0, 1 << log2n, max(1, (1 << log2n) // 97)):
            assert oracle.bitrev(j, log2n) == int(format(j, "0%db" % log2n)[::-1], 2)


@pytest.mark.parametrize("q,log2n", SMALL_CASES + [(q, 10) for q in BIG_PRIMES] + [(W.POOL50[0], 16)])
def test_psi_has_order_2n_and_uses_least_nonresidue(oracle, q, log2n):
    sympy = pytest.importorskip("sympy")
    n = 1 << log2n
    psi = oracle.psi(q, log2n)
    assert sympy.n_order(psi, q) == 2 * n
    assert pow(psi, n, q) == q - 1
    g = 2
    while sympy.legendre_symbol(g, q) == 1:
        g += 1
    assert psi == pow(g, (q - 1) // (2 * n), q)


def test_psi_rejects_bad_moduli(oracle):
    assert oracle.psi(7681, 10) == 0          # 2N = 2048 does not divide 7680
    assert oracle.psi(7681 * 12289, 4) == 0   # composite
    assert oracle.psi(W.POOL50[0], 17) == 0   # 2^18 does not divide q-1


@pytest.mark.parametrize("q,log2n", [c for c in SMALL_CASES if c[1] <= 6])
def test_forward_is_evaluation_at_all_roots_of_xn_plus_1(oracle, q, log2n):
    """Brute force: scan Z_q for the roots of x^N = -1; NTT(a) must be exactly
    the multiset {a(r)} over those roots (no psi involved)."""
    n = 1 << log2n
    roots = [r for r in range(q) if pow(r, n, q) == q - 1]
    assert len(roots) == n
    rng = random.Random(q * 131 + log2n)
    for _ in range(4):
        a = [rng.randrange(q) for _ in range(n)]
        A = [int(v) for v in oracle.ntt_forward(a, q)]
        ev = [sum(c * pow(r, i, q) for i, c in enumerate(a)) % q for r in roots]
        assert sorted(A) == sorted(ev)


@pytest.mark.parametrize("q,log2n", SMALL_CASES + [(q, 10) for q in BIG_PRIMES])
def test_output_order_is_cooley_tukey_bit_reversed(oracle, q, log2n):
    """NTT(x)[j] lists the evaluation points.  The CT natural->bit-reversed
    transform starts at psi and setting bit b of the index multiplies the point
    by psi^(N/2^b) (b = 0 pairs r with -r)."""
    n = 1 << log2n
    psi = oracle.psi(q, log2n)
    x = np.zeros(n, dtype=np.uint64)
    x[1] = 1
    P = [int(v) for v in oracle.ntt_forward(x, q)]
    assert P[0] == psi
    for j in range(n):
        for b in range(log2n):
            if not (j >> b) & 1:
                assert P[j | (1 << b)] == P[j] * pow(psi, n >> b, q) % q
    assert all(P[2 * k + 1] == (q - P[2 * k]) % q for k in range(n // 2))


@pytest.mark.parametrize("q,log2n", SMALL_CASES + [(q, 10) for q in BIG_PRIMES])
def test_special_vectors(oracle, q, log2n):
    n = 1 << log2n
    delta = np.zeros(n, dtype=np.uint64)
    delta[0] = 1
    assert np.all(oracle.ntt_forward(delta, q) == 1)
    c = np.zeros(n, dtype=np.uint64)
    c[0] = q - 5
    assert np.all(oracle.ntt_forward(c, q) == q - 5)
    assert np.all(oracle.ntt_inverse(np.ones(n, dtype=np.uint64), q) == delta)
    rng = random.Random(11)
    a = [rng.randrange(q) for _ in range(n)]
    b = [rng.randrange(q) for _ in range(n)]
    al, be = rng.randrange(q), rng.randrange(q)
    lin = [(al * x + be * y) % q for x, y in zip(a, b)]
    A, B, L = (oracle.ntt_forward(v, q) for v in (a, b, lin))
    assert all(int(l) == (al * int(x) + be * int(y)) % q for l, x, y in zip(L, A, B))


def _numpy_negacyclic(a, b, q):
    """numpy's exact (object dtype) linear convolution folded by x^N = -1."""
    n = len(a)
    full = np.convolve(np.array(a, dtype=object), np.array(b, dtype=object))
    full = list(full) + [0]
    return [int((full[k] - full[k + n]) % q) for k in range(n)]


@pytest.mark.parametrize("q,log2n", SMALL_CASES + [(q, lg) for q in BIG_PRIMES for lg in (2, 7, 10)])
def test_convolution_theorem_and_schoolbook_vs_numpy(oracle, q, log2n):
    """Eq. 1: INTT(NTT(a) . NTT(b)) is a*b mod (x^N+1); checked against numpy."""
    n = 1 << log2n
    rng = random.Random(q ^ log2n)
    a = [rng.randrange(q) for _ in range(n)]
    b = [rng.randrange(q) for _ in range(n)]
    ref = _numpy_negacyclic(a, b, q)
    sb = [int(v) for v in oracle.schoolbook(a, b, q)]
    assert sb == ref
    c = oracle.ntt_inverse(oracle.pointwise(oracle.ntt_forward(a, q), oracle.ntt_forward(b, q), q), q)
    assert [int(v) for v in c] == ref


@pytest.mark.parametrize("q,log2n", SMALL_CASES + [(q, 10) for q in BIG_PRIMES])
def test_roundtrip(oracle, q, log2n):
    n = 1 << log2n
    rng = random.Random(5 * q + log2n)
    a = np.array([rng.randrange(q) for _ in range(n)], dtype=np.uint64)
    assert np.array_equal(oracle.ntt_inverse(oracle.ntt_forward(a, q), q), a)
    assert np.array_equal(oracle.ntt_forward(oracle.ntt_inverse(a, q), q), a)


@pytest.mark.parametrize("q,log2n", [(257, 4), (W.Q62_N1024, 10), (W.POOL50[5], 6)])
def test_negacyclic_sign(oracle, q, log2n):
    n = 1 << log2n
    a = np.zeros(n, dtype=np.uint64)
    b = np.zeros(n, dtype=np.uint64)
    a[n - 1] = 1
    b[1] = 1
    c = oracle.schoolbook(a, b, q)
    assert int(c[0]) == q - 1 and not np.any(c[1:])


def test_pointwise_vs_python_ints(oracle):
    rng = random.Random(3)
    for q in BIG_PRIMES:
        a = [rng.randrange(q) for _ in range(257)]
        b = [rng.randrange(q) for _ in range(257)]
        assert [int(v) for v in oracle.pointwise(a, b, q)] == [x * y % q for x, y in zip(a, b)]


def test_sampled_and_threaded_paths_agree(oracle):
    q = W.Q59_N1024
    x = W.rows_uniform(1, 9, [q] * 6, 256)
    full = np.stack([oracle.ntt_forward(r, q) for r in x])
    assert np.array_equal(oracle.transform_rows(x, [q] * 6, nthreads=3), full)
    assert np.array_equal(oracle.transform_rows(x, [q] * 6, nthreads=4, split=True, chunk=37), full)
    idx = np.array([[3, 200, 17]] * 6, dtype=np.uint32)
    assert np.array_equal(oracle.transform_rows(x, [q] * 6, idx=idx, nthreads=2), full[:, [3, 200, 17]])
    inv = np.stack([oracle.ntt_inverse(r, q) for r in full])
    assert np.array_equal(oracle.transform_rows(full, [q] * 6, inverse=True, nthreads=3), inv)
    assert np.array_equal(inv, x)


@pytest.mark.parametrize("q,log2n", [(257, 5), (W.Q62_N1024, 10), (W.POOL50[3], 8)])
def test_sampled_schoolbook_matches_numpy(oracle, q, log2n):
    n = 1 << log2n
    rng = random.Random(q + 17)
    a = [rng.randrange(q) for _ in range(n)]
    b = [rng.randrange(q) for _ in range(n)]
    ref = _numpy_negacyclic(a, b, q)
    idx = [0, 1, n // 2, n - 1, rng.randrange(n)]
    got = oracle.schoolbook_at(a, b, q, idx)
    assert [int(v) for v in got] == [ref[k] for k in idx]


def test_hand_derived_known_answers(oracle):
    """Values worked out by hand from the definition of Eq. 1 (tests/golden)."""
    from golden.load import negacyclic_q17
    ntt_cases, mul_cases = negacyclic_q17()
    assert len(ntt_cases) == 2 and len(mul_cases) == 2
    for q, log2n, psi, a, A in ntt_cases:
        assert oracle.psi(q, log2n) == psi
        assert oracle.ntt_forward(np.array(a, dtype=np.uint64), q).tolist() == A
        assert oracle.ntt_inverse(np.array(A, dtype=np.uint64), q).tolist() == a
    for q, log2n, a, b, c in mul_cases:
        a, b = np.array(a, dtype=np.uint64), np.array(b, dtype=np.uint64)
        assert oracle.schoolbook(a, b, q).tolist() == c
        prod = oracle.pointwise(oracle.ntt_forward(a, q), oracle.ntt_forward(b, q), q)
        assert oracle.ntt_inverse(prod, q).tolist() == c
