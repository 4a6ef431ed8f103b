"""Pins for the TFHE external-product / CMux oracle (Sec. II-B, Sec. IV-A):
exhaustive checks of the gadget decomposition against exact rational
rounding, the approximation bound it must meet, rotation against the
schoolbook product with a monomial, keys with a closed-form NTT (constants
and monomials, whose transform is psi-powers) that turn the external
product into an approximate identity or rotation, exact identities (zero
key, linearity in the key), and a brute-force tiny case with numpy's exact
convolution.  A second part plants plausible mistakes in a copy of the
oracle and checks that these pins catch each one."""
import math
import random
import types
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as O
from oracle import tfhe_oracle as T
from paper_2410_05934_gb300 import workloads as W

Q62 = W.Q62_N1024


def _round_fraction(fr):
    return math.floor(fr + Fraction(1, 2))


def _centered(x, q):
    x %= q
    return x - q if x > q // 2 else x


def _bound(q, log2_base, levels):
    """|sum_j e_j g_j - v| <= q / (2 B^l) + l B / 4 (rounding of t, and of each g_j)."""
    return q / (2 << (log2_base * levels)) + levels * (1 << log2_base) / 4


def _check_decomposition(t, v, q, log2_base, levels):
    base = 1 << log2_base
    e = t.decompose(v, q, log2_base, levels)
    assert len(e) == levels and all(-base // 2 <= d < base // 2 for d in e), (v, e)
    top = _round_fraction(Fraction(v << (log2_base * levels), q)) % (1 << (log2_base * levels))
    assert sum(d << (log2_base * (levels - 1 - j)) for j, d in enumerate(e)) % (1 << (log2_base * levels)) == top
    g = t.gadget(q, log2_base, levels)
    assert g == [_round_fraction(Fraction(q, 1 << (log2_base * (j + 1)))) for j in range(levels)]
    err = abs(_centered(sum(d * gj for d, gj in zip(e, g)) - v, q))
    assert err <= _bound(q, log2_base, levels), (v, e, err)


@pytest.mark.parametrize("q,log2_base,levels", [(7681, 2, 3), (12289, 3, 2), (7681, 4, 2), (12289, 1, 5)])
def test_decomposition_exhaustive_small_q(q, log2_base, levels):
    for v in range(q):
        _check_decomposition(T, v, q, log2_base, levels)


def test_decomposition_random_62_bit():
    rng = random.Random(5)
    for log2_base, levels in [(8, 3), (10, 2), (6, 4)]:
        for v in [0, 1, Q62 - 1, Q62 // 2, Q62 // 2 + 1] + [rng.randrange(Q62) for _ in range(3000)]:
            _check_decomposition(T, v, Q62, log2_base, levels)


def _monomial(n, k, q):
    """x^k for k in [0, 2N) as a coefficient vector."""
    p = [0] * n
    p[k % n] = 1 if k < n else q - 1
    return np.array(p, dtype=np.uint64)


def test_rotation_is_product_with_a_monomial():
    q, n = 12289, 16
    rng = np.random.default_rng(3)
    p = rng.integers(0, q, n).astype(np.uint64)
    for a in range(2 * n):
        assert T.rotate(p, a, q) == O.schoolbook(p, _monomial(n, a, q), q).tolist(), a
    assert T.rotate(T.rotate(p, 7, q), 2 * n - 7, q) == p.tolist()


def _gadget_key(n, q, log2_base, levels, b=0, scale=1):
    """NTT-domain rows of RGSW(scale * x^b) without noise: row i*l+j, column c
    is delta_(i,c) * g_j * scale * x^b; NTT(x^b)[k] = psi^(b (2 brv(k) + 1))."""
    log2n = n.bit_length() - 1
    psi = O.psi(q, log2n)
    mono = [pow(psi, b * (2 * O.bitrev(k, log2n) + 1), q) for k in range(n)]
    g = T.gadget(q, log2_base, levels)
    key = np.zeros((2 * levels, 2, n), dtype=np.uint64)
    for i in range(2):
        for j in range(levels):
            key[i * levels + j, i] = [(g[j] * scale * m) % q for m in mono]
    return key


@pytest.mark.parametrize("b", [0, 3, 21])
def test_external_product_with_gadget_key_is_approximate_rotation(b):
    q, n, log2_base, levels = Q62, 16, 8, 3
    rng = np.random.default_rng(b)
    d = rng.integers(0, q, (2, n), dtype=np.uint64)
    out = T.external_product(d, _gadget_key(n, q, log2_base, levels, b=b), q, log2_base, levels)
    bound = _bound(q, log2_base, levels)
    for c in range(2):
        want = T.rotate(d[c], b, q)
        for k in range(n):
            assert abs(_centered(int(out[c, k]) - want[k], q)) <= bound, (c, k)


def test_cmux_with_zero_key_is_identity_and_with_unit_key_rotates():
    q, n, log2_base, levels = Q62, 16, 8, 3
    rng = np.random.default_rng(9)
    acc = rng.integers(0, q, (2, n), dtype=np.uint64)
    zero = np.zeros((2 * levels, 2, n), dtype=np.uint64)
    unit = _gadget_key(n, q, log2_base, levels)
    bound = _bound(q, log2_base, levels)
    for a in (0, 1, 5, n, n + 3, 2 * n - 1):
        assert np.array_equal(T.cmux_rotate(acc, a, zero, q, log2_base, levels), acc)
        out = T.cmux_rotate(acc, a, unit, q, log2_base, levels)
        for c in range(2):
            want = T.rotate(acc[c], a, q)
            for k in range(n):
                assert abs(_centered(int(out[c, k]) - want[k], q)) <= bound, (a, c, k)


def test_external_product_is_linear_in_the_key():
    q, n, log2_base, levels = 12289, 8, 2, 3
    rng = np.random.default_rng(11)
    d = rng.integers(0, q, (2, n), dtype=np.uint64)
    k1 = rng.integers(0, q, (2 * levels, 2, n), dtype=np.uint64)
    k2 = rng.integers(0, q, (2 * levels, 2, n), dtype=np.uint64)
    s = ((k1.astype(object) + k2.astype(object)) % q).astype(np.uint64)
    lhs = T.external_product(d, s, q, log2_base, levels)
    rhs = (T.external_product(d, k1, q, log2_base, levels).astype(object)
           + T.external_product(d, k2, q, log2_base, levels).astype(object)) % q
    assert np.array_equal(lhs, rhs.astype(np.uint64))


def _negacyclic_numpy(a, b, q):
    n = len(a)
    full = np.convolve(np.array([int(x) for x in a], dtype=object), np.array([int(x) for x in b], dtype=object))
    out = full[:n].copy()
    out[:n - 1] -= full[n:]
    return [int(x) % q for x in out]


def test_external_product_brute_force_tiny():
    """N = 4, q = 17, B = 2, l = 2: digit rows times coefficient-domain key rows, by numpy."""
    q, n, log2_base, levels = 17, 4, 1, 2
    rng = np.random.default_rng(2)
    for _ in range(20):
        d = rng.integers(0, q, (2, n), dtype=np.uint64)
        key_coef = rng.integers(0, q, (2 * levels, 2, n), dtype=np.uint64)
        key_ntt = np.array([[O.ntt_forward(key_coef[p, c], q) for c in range(2)] for p in range(2 * levels)],
                           dtype=np.uint64)
        want = [[0] * n for _ in range(2)]
        for i in range(2):
            digs = [T.decompose(int(v), q, log2_base, levels) for v in d[i]]
            for j in range(levels):
                row = [dd[j] % q for dd in digs]
                for c in range(2):
                    prod = _negacyclic_numpy(row, key_coef[i * levels + j, c], q)
                    want[c] = [(x + y) % q for x, y in zip(want[c], prod)]
        assert T.external_product(d, key_ntt, q, log2_base, levels).tolist() == want


def test_sampled_outputs_match_full():
    q, n, log2_base, levels = Q62, 32, 8, 3
    rng = np.random.default_rng(4)
    acc = rng.integers(0, q, (2, n), dtype=np.uint64)
    key = rng.integers(0, q, (2 * levels, 2, n), dtype=np.uint64)
    full = T.cmux_rotate(acc, 37, key, q, log2_base, levels)
    idx = [0, 5, 31, 17]
    assert np.array_equal(T.cmux_rotate(acc, 37, key, q, log2_base, levels, idx=idx), full[:, idx])


# ---- planted mistakes: each must fail at least one pin ----------------------

def _mutant(**over):
    m = types.ModuleType("tfhe_mutant")
    for k in ("gadget", "decompose", "rotate", "digit_polys", "key_coefficients", "external_product",
              "cmux_rotate"):
        setattr(m, k, getattr(T, k))
    m.__dict__.update(over)
    # re-bind the helpers so that they call the mutant's functions
    for k in ("digit_polys", "external_product", "cmux_rotate"):
        f = getattr(T, k)
        setattr(m, k, types.FunctionType(f.__code__, m.__dict__ | {"np": np, "O": O}, k, f.__defaults__))
    return m


def _decompose_truncating(v, q, log2_base, levels):          # floor instead of round
    base = 1 << log2_base
    t = ((v << (log2_base * levels))) // q % (1 << (log2_base * levels))
    out = [0] * levels
    for j in reversed(range(levels)):
        e = t % base
        t //= base
        if e >= base // 2:
            e -= base
            t += 1
        out[j] = e
    return out


def _decompose_reversed(v, q, log2_base, levels):            # least significant digit first
    return list(reversed(T.decompose(v, q, log2_base, levels)))


def _decompose_unsigned(v, q, log2_base, levels):            # digits in [0, B)
    base = 1 << log2_base
    t = ((v << (log2_base * levels)) + q // 2) // q % (1 << (log2_base * levels))
    out = [0] * levels
    for j in reversed(range(levels)):
        out[j] = t % base
        t //= base
    return out


def _rotate_cyclic(p, a, q):                                 # x^N = +1
    n = len(p)
    out = [0] * n
    for m in range(n):
        out[(m + a) % n] = int(p[m]) % q
    return out


def _gadget_floor(q, log2_base, levels):                     # floor instead of round
    return [q >> (log2_base * (j + 1)) for j in range(levels)]


MUTANTS = {
    "truncating_decomposition": dict(decompose=_decompose_truncating),
    "reversed_digits": dict(decompose=_decompose_reversed),
    "unsigned_digits": dict(decompose=_decompose_unsigned),
    "cyclic_rotation": dict(rotate=_rotate_cyclic),
    "floor_gadget": dict(gadget=_gadget_floor),
}


def _pins(t):
    """Runs the pins against module t; returns the names of those that fail."""
    failed = []

    def run(name, fn):
        try:
            fn()
        except AssertionError:
            failed.append(name)

    run("exhaustive", lambda: [_check_decomposition(t, v, 7681, 2, 3) for v in range(7681)])
    run("62-bit", lambda: [_check_decomposition(t, v, Q62, 8, 3) for v in (1, Q62 // 3, Q62 - 2)])

    def rotation():
        p = np.random.default_rng(1).integers(0, 12289, 16).astype(np.uint64)
        for a in range(32):
            assert t.rotate(p, a, 12289) == O.schoolbook(p, _monomial(16, a, 12289), 12289).tolist()

    run("rotation", rotation)
    return failed


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistakes(name):
    assert _pins(T) == []
    m = _mutant(**MUTANTS[name])
    failed = _pins(m)
    if not failed:
        # the decomposition and rotation pins passed: the product-level pins must fail
        q, n, log2_base, levels = Q62, 16, 8, 3
        d = np.random.default_rng(0).integers(0, q, (2, n), dtype=np.uint64)
        out = m.external_product(d, _gadget_key(n, q, log2_base, levels, b=3), q, log2_base, levels)
        bound = _bound(q, log2_base, levels)
        ok = all(abs(_centered(int(out[c, k]) - T.rotate(d[c], 3, q)[k], q)) <= bound
                 for c in range(2) for k in range(n))
        assert not ok, name
