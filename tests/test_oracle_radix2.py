"""The O(N log N) CPU baseline (oracle/ntt_radix2.c) against the O(N^2)
definitions of Eq. 1 in oracle/ntt_oracle.c: every N up to 2^12 on tiny,
50-, 59- and 62-bit primes, sampled outputs at N = 2^16, round trips, the
[poly][limb] modulus layout and argument errors.  CPU only."""
import numpy as np
import pytest

from paper_2410_05934_gb300 import workloads as W
from oracle import oracle as O


def _prime(log2n, bits):
    """Largest prime below 2^bits with q = 1 mod 2^(log2n + 1)."""
    step = 1 << (log2n + 1)
    q = ((1 << bits) - 1) // step * step + 1
    while not O.is_prime(q):
        q -= step
    return q


@pytest.mark.parametrize("log2n", range(1, 13))
@pytest.mark.parametrize("bits", [17, 50, 59, 62])
def test_matches_definition(log2n, bits):
    if bits == 17 and log2n > 12:
        pytest.skip("no such prime")
    q = _prime(log2n, bits)
    rng = np.random.default_rng(log2n * 100 + bits)
    x = rng.integers(0, q, (3, 1 << log2n), dtype=np.uint64)
    x[0, :] = q - 1                                   # the largest residue everywhere
    fwd = O.radix2_rows(x, [q])
    assert np.array_equal(fwd, O.transform_rows(x, [q] * 3))
    inv = O.radix2_rows(x, [q], inverse=True)
    assert np.array_equal(inv, O.transform_rows(x, [q] * 3, inverse=True))
    assert np.array_equal(O.radix2_rows(fwd, [q], inverse=True), x)


def test_n65536_sampled_outputs_and_limb_layout():
    Q = W.POOL50[:3]
    per_row = [Q[r % 3] for r in range(6)]
    x = W.rows_uniform(11, 16, per_row, 1 << 16)
    fwd = O.radix2_rows(x, Q)
    rng = np.random.default_rng(16)
    idx = np.stack([np.concatenate([[0, 1, 65535], rng.integers(0, 1 << 16, 13)]) for _ in per_row]).astype(np.uint32)
    rows = np.arange(6)[:, None]
    assert np.array_equal(fwd[rows, idx], O.transform_rows(x, per_row, idx=idx))
    inv = O.radix2_rows(x, Q, inverse=True)
    assert np.array_equal(inv[rows, idx], O.transform_rows(x, per_row, inverse=True, idx=idx))
    assert np.array_equal(O.radix2_rows(fwd, Q, inverse=True), x)


def test_convolution_theorem():
    q, n = W.POOL50[0], 256
    rng = np.random.default_rng(3)
    a, b = (rng.integers(0, q, n, dtype=np.uint64) for _ in range(2))
    A, B = O.radix2_rows(np.stack([a, b]), [q])
    c = O.radix2_rows(O.pointwise(A, B, q)[None, :], [q], inverse=True)[0]
    assert np.array_equal(c, O.schoolbook(a, b, q))


def test_rejects_bad_moduli():
    x = np.zeros((1, 16), np.uint64)
    for q in [15, 97 * 2, (1 << 62) + 135, 2]:
        with pytest.raises(ValueError):
            O.radix2_rows(x, [q])
