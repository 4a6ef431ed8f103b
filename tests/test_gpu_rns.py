"""RNS basis conversion on the GPU (C ABI ntt_bconv) against the oracle's
definition: the key-switching shape (24 limbs -> 24 special primes) at
N = 2^16 on sampled coefficients, full rows at small N, 62-bit bases whose
128-bit sums fold, non-canonical inputs, empty calls and argument errors."""
import numpy as np
import pytest

from paper_2410_05934_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2410_05934_gb300 as ntt  # noqa: E402
from gpu_util import to_dev, to_host  # noqa: E402
from oracle import rns_oracle as RO  # noqa: E402


def test_key_switching_shape_sampled():
    w = W.ckks_bconv()
    Q, P, x = w["Q"], w["P"], w["x"]
    b = ntt.BConv(Q, P)
    out = torch.empty((x.shape[0], len(P), 1 << 16), dtype=torch.int64, device="cuda")
    b(to_dev(x), out, 16)
    got = to_host(out)
    rng = np.random.default_rng(1)
    idx = np.concatenate([[0, 1, 65535], rng.integers(0, 1 << 16, 61)])
    for p in range(x.shape[0]):
        assert np.array_equal(got[p][:, idx], RO.bconv(x[p][:, idx], Q, P)), p


@pytest.mark.parametrize("log2n,L,K", [(10, 5, 3), (12, 3, 40), (1, 2, 2)])
def test_full_rows_small(log2n, L, K):
    Q = W.POOL50[:L]
    P = W.POOL50[L:L + K] if L + K <= 48 else [W.Q62_N1024, W.Q59_N1024] + W.POOL50[L + 2:L + K]
    rng = np.random.default_rng(log2n)
    x = np.stack([np.array([rng.integers(0, q, 1 << log2n, dtype=np.uint64) for q in Q]) for _ in range(3)])
    out = torch.empty((3, K, 1 << log2n), dtype=torch.int64, device="cuda")
    ntt.BConv(Q, P)(to_dev(x), out, log2n)
    got = to_host(out)
    for p in range(3):
        assert np.array_equal(got[p], RO.bconv(x[p], Q, P))


def _primes_below(top, count):
    from oracle import oracle as O
    qs, c = [], top - 1
    while len(qs) < count:
        if O.is_prime(c):
            qs.append(c)
        c -= 2
    return qs


def test_largest_bases_many_steps():
    """64 -> 64 limbs (the largest bases, 64 KiB of shared memory per CTA) over
    more 64-coefficient steps than one wave of CTAs, with a ragged last step."""
    qs = _primes_below(1 << 50, 128)
    Q, P = qs[:64], qs[64:]
    log2n, polys = 5, 2051                      # 65632 coefficients: 1025.5 steps
    rng = np.random.default_rng(64)
    x = np.stack([np.array([rng.integers(0, q, 1 << log2n, dtype=np.uint64) for q in Q]) for _ in range(polys)])
    out = torch.empty((polys, 64, 1 << log2n), dtype=torch.int64, device="cuda")
    ntt.BConv(Q, P)(to_dev(x), out, log2n)
    got = to_host(out)
    for p in [0, 1, 1000, polys - 2, polys - 1]:
        assert np.array_equal(got[p], RO.bconv(x[p], Q, P)), p


def test_62_bit_bases_and_noncanonical_inputs():
    from oracle import oracle as O
    qs, c = [], (1 << 62) - 1
    while len(qs) < 43:
        if O.is_prime(c):
            qs.append(c)
        c -= 2
    Q, P = qs[:40], qs[40:]
    rng = np.random.default_rng(7)
    x = np.array([[rng.integers(0, 1 << 63, 256, dtype=np.uint64) | np.uint64(1 << 63) for _ in Q]])
    out = torch.empty((1, 3, 256), dtype=torch.int64, device="cuda")
    ntt.BConv(Q, P)(to_dev(x), out, 8)
    xr = np.array([[int(v) % q for v in row] for row, q in zip(x[0], Q)], dtype=np.uint64)
    assert np.array_equal(to_host(out)[0], RO.bconv(xr, Q, P))


def test_empty_call_and_errors():
    b = ntt.BConv(W.POOL50[:2], W.POOL50[2:3])
    x = torch.zeros((1, 2, 16), dtype=torch.int64, device="cuda")
    b(x, torch.empty((1, 1, 16), dtype=torch.int64, device="cuda"), 4, n_polys=0)
    for q, p, code in [([W.POOL50[0]] * 2, [W.POOL50[1]], -1), ([W.POOL50[0]], [15], -2),
                       ([W.POOL50[0]], [(1 << 62) + 135], -4), ([], [W.POOL50[1]], -1)]:
        with pytest.raises(ntt.NttError) as e:
            ntt.BConv(q, p)
        assert e.value.code == code, (q, p)


def test_rescale_ckks_shape_sampled():
    """2 polynomials x 24 limbs at N = 2^16 (NTT domain) -> 23 limbs."""
    from oracle import oracle as O
    n, Q = 1 << 16, W.POOL50[:24]
    w = W.ckks_hmul_n65536(limbs=24, polys=2)
    x = w["x"]                                   # treated as NTT-domain limbs
    plan = ntt.Plan(16, Q, 2)
    out = torch.empty((2, 23, n), dtype=torch.int64, device="cuda")
    work = torch.empty((2, n), dtype=torch.int64, device="cuda")
    plan.rescale(to_dev(x), out, work)
    assert plan.status() == 0
    got = to_host(out)
    idx = [0, 1, 4097, n - 1]
    for p in range(2):
        assert np.array_equal(got[p][:, idx], RO.rescale_ntt(x[p], Q, idx=idx)), p


@pytest.mark.parametrize("log2n", [10, 12, 14])
def test_rescale_full_rows_every_schedule(log2n):
    n = 1 << log2n
    Q = [W.POOL50[3], W.POOL50[1], W.POOL50[7], W.POOL50[0]]
    rng = np.random.default_rng(log2n)
    x = np.stack([np.array([rng.integers(0, q, n, dtype=np.uint64) for q in Q]) for _ in range(3)])
    want = [RO.rescale_ntt(x[p], Q) for p in range(3)] if log2n <= 12 else None
    idx = [0, 2, n // 2 + 1, n - 1]
    if want is None:
        want = [RO.rescale_ntt(x[p], Q, idx=idx) for p in range(3)]
    plan = ntt.Plan(log2n, Q, 3)
    xd = to_dev(x)
    for s in range(ntt.schedule_count(log2n)):
        plan.schedule = s                        # a pipelined first kernel falls back to a direct one
        out = torch.empty((3, 3, n), dtype=torch.int64, device="cuda")
        plan.rescale(xd, out, torch.empty((3, n), dtype=torch.int64, device="cuda"))
        got = to_host(out)
        for p in range(3):
            g = got[p] if log2n <= 12 else got[p][:, idx]
            assert np.array_equal(g, want[p]), (s, p)
    # two of the three polynomials only
    out = torch.zeros((3, 3, n), dtype=torch.int64, device="cuda")
    plan.rescale(xd, out, torch.empty((2, n), dtype=torch.int64, device="cuda"), n_polys=2)
    assert not to_host(out)[2].any()


def test_rescale_errors():
    x = torch.zeros((1, 2, 1024), dtype=torch.int64, device="cuda")
    w = torch.zeros((1, 1024), dtype=torch.int64, device="cuda")
    with pytest.raises(ntt.NttError):
        ntt.Plan(10, [W.POOL50[0]]).rescale(x[:, :1], torch.zeros((1, 1, 1024), dtype=torch.int64, device="cuda"), w)
    with pytest.raises(ntt.NttError):                      # last modulus repeats the first
        ntt.Plan(10, [W.POOL50[0], W.POOL50[0]]).rescale(x, torch.zeros((1, 1, 1024), dtype=torch.int64,
                                                                          device="cuda"), w)
