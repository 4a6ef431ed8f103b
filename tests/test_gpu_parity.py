"""Parity of the sm_103a kernels (through the C ABI) with the CPU oracle:
bit-exact on every schedule of every N, on the three fixed workloads at their
full sizes (sampled outputs where the O(N^2) oracle is too slow), and on the
edge cases (in-place, row ranges, empty launches, extreme values, maximum
sizes, range checking)."""
import numpy as np
import pytest

from paper_2410_05934_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2410_05934_gb300 as ntt  # noqa: E402
from gpu_util import to_dev, to_host  # noqa: E402


def _primes_below(bits, log2n, count):
    """The largest `count` primes below 2^bits that are 1 mod 2^(log2n + 1)."""
    from oracle import oracle as O
    step = 1 << (log2n + 1)
    q, out = ((1 << bits) - 1) // step * step + 1, []
    while len(out) < count:
        if O.is_prime(q):
            out.append(q)
        q -= step
    return out


def _moduli(log2n, cls="big"):
    """big: 59..62-bit moduli (exact-quotient class 0); mid: the largest below 2^57 (class 1,
    approximate quotients); small: 50-bit (class 2, also lazy inverse sums)."""
    if cls == "big":
        return [W.Q62_N1024, W.Q59_N1024] if log2n <= 10 else _primes_below(62, log2n, 2)
    if cls == "mid":
        return _primes_below(57, 16, 2)
    return [W.POOL50[0], W.POOL50[7]]


def _sample_idx(n, rows, k, seed):
    rng = np.random.default_rng(seed)
    base = np.array([0, 1, n // 2, n - 1], dtype=np.int64)
    return np.stack([np.concatenate([base, rng.integers(0, n, k)]) for _ in range(rows)]).astype(np.uint32)


@pytest.mark.parametrize("cls", ["big", "mid", "small"])
@pytest.mark.parametrize("log2n", range(1, 17))
def test_every_schedule_bit_exact(oracle, log2n, cls):
    n = 1 << log2n
    mods = _moduli(log2n, cls)
    batch = 3 if log2n > 12 else 5            # ragged: not a multiple of rows per CTA
    per_row = [mods[r % 2] for r in range(batch * 2)]
    x = W.rows_uniform(101, log2n, per_row, n)
    if log2n <= 11:
        idx = None
        ref = oracle.transform_rows(x, per_row)
        ref_inv = oracle.transform_rows(x, per_row, inverse=True)
    else:
        idx = _sample_idx(n, len(per_row), 28, log2n)
        ref = oracle.transform_rows(x, per_row, idx=idx)
        ref_inv = oracle.transform_rows(x, per_row, inverse=True, idx=idx)
    rows = np.arange(len(per_row))[:, None]
    plan = ntt.Plan(log2n, mods, batch)
    dx = to_dev(x)
    for s in range(ntt.schedule_count(log2n)):
        plan.schedule = s
        out = torch.empty_like(dx)
        plan.forward(dx, out)
        got = to_host(out)
        got = got if idx is None else got[rows, idx]
        assert np.array_equal(got, ref), "forward, schedule %d" % s
        back = torch.empty_like(dx)
        plan.inverse(out, back)
        assert np.array_equal(to_host(back), x), "round trip, schedule %d" % s
        inv = torch.empty_like(dx)
        plan.inverse(dx, inv)
        got = to_host(inv)
        got = got if idx is None else got[rows, idx]
        assert np.array_equal(got, ref_inv), "inverse, schedule %d" % s
        assert plan.status() == 0


def test_plain_n1024_workload(oracle):
    """64 rows at N=1024 (59-bit prime); 32 product pairs vs schoolbook."""
    w = W.plain_n1024()
    q, x = w["moduli"][0], w["x"]
    plan = ntt.Plan(10, [q], 64)
    dx = to_dev(x)
    A = torch.empty_like(dx)
    plan.forward(dx, A)
    assert np.array_equal(to_host(A), oracle.transform_rows(x, [q] * 64))
    pairs = ntt.Plan(10, [q], 32)
    C = torch.empty_like(A[:32])
    pairs.pointwise(A[:32].contiguous(), A[32:].contiguous(), C)
    pairs.inverse(C, C)
    c = to_host(C)
    for i in range(32):
        if i < 6:
            assert np.array_equal(c[i], oracle.schoolbook(x[i], x[32 + i], q)), i
        else:
            k = np.array([0, 1, 511, 1023, 3 * i], dtype=np.uint32)
            assert np.array_equal(c[i][k], oracle.schoolbook_at(x[i], x[32 + i], q, k)), i
    back = torch.empty_like(dx)
    plan.inverse(A, back)
    assert np.array_equal(to_host(back), x)


def test_ckks_hmul_n65536_workload(oracle):
    """The full CKKS-HMUL-shaped batch: 4 polys x 24 limbs at N=2^16, forward,
    the 4 cross products, inverse; sampled outputs on every row, one full
    O(N^2) row, the convolution identity at sampled coefficients."""
    w = W.ckks_hmul_n65536()
    mods, x = w["moduli"], w["x"]
    L, n = len(mods), 1 << 16
    per_row = [mods[r % L] for r in range(4 * L)]
    xr = x.reshape(4 * L, n)
    plan = ntt.Plan(16, mods, 4)
    dx = to_dev(xr)
    A = torch.empty_like(dx)
    plan.forward(dx, A)
    a_host = to_host(A)
    idx = _sample_idx(n, 4 * L, 12, 2)
    ref = oracle.transform_rows(xr, per_row, idx=idx)
    assert np.array_equal(a_host[np.arange(4 * L)[:, None], idx], ref)
    # one whole row by the O(N^2) definition
    full = oracle.transform_rows(xr[37:38], [per_row[37]], split=True, chunk=512)
    assert np.array_equal(a_host[37], full[0])
    # cross products a_i (.) b_j, i, j in {0, 1}, then the inverse
    limb_plan = ntt.Plan(16, mods, 1)
    Ap = A.view(4, L, n)
    prods = torch.empty((4, L, n), dtype=A.dtype, device=A.device)
    for k, (i, j) in enumerate([(0, 0), (0, 1), (1, 0), (1, 1)]):
        limb_plan.pointwise(Ap[i].contiguous(), Ap[2 + j].contiguous(), prods[k])
    plan.inverse(prods.view(4 * L, n), prods.view(4 * L, n))
    c = to_host(prods)
    for k, (i, j) in enumerate([(0, 0), (0, 1), (1, 0), (1, 1)]):
        for l in (0, 11, 23):
            kk = np.array([0, 1, 4097, n - 1], dtype=np.uint32)
            assert np.array_equal(c[k, l][kk], oracle.schoolbook_at(x[i, l], x[2 + j, l], mods[l], kk))
    # the same cross products formed inside the inverse's first kernel (the bench's step)
    fused = torch.empty_like(prods)
    plan.inverse_mul(A, A, fused, a_poly=[0, 0, 1, 1], b_poly=[2, 3, 2, 3])
    assert torch.equal(fused, prods)
    back = torch.empty_like(dx)
    plan.inverse(A, back)
    assert torch.equal(back, dx)


def test_tfhe_blind_rotation_workload(oracle):
    """3780 forward NTTs of signed digits + 1260 inverse NTTs (62-bit prime)."""
    w = W.tfhe_blind_rotation()
    q = w["moduli"][0]
    fwd, inv = w["fwd"], w["inv"]
    pf = ntt.Plan(10, [q], fwd.shape[0])
    pi = ntt.Plan(10, [q], inv.shape[0])
    df, di = to_dev(fwd), to_dev(inv)
    of, oi = torch.empty_like(df), torch.empty_like(di)
    pf.forward(df, of)
    pi.inverse(di, oi)
    gf, gi = to_host(of), to_host(oi)
    rows_f = np.arange(0, fwd.shape[0], 59)
    rows_i = np.arange(0, inv.shape[0], 41)
    assert np.array_equal(gf[rows_f], oracle.transform_rows(fwd[rows_f], [q] * len(rows_f)))
    assert np.array_equal(gi[rows_i], oracle.transform_rows(inv[rows_i], [q] * len(rows_i), inverse=True))
    idx = _sample_idx(1024, fwd.shape[0], 4, 3)
    assert np.array_equal(gf[np.arange(fwd.shape[0])[:, None], idx],
                          oracle.transform_rows(fwd, [q] * fwd.shape[0], idx=idx))


@pytest.mark.parametrize("log2n", [1, 4, 10, 14, 16])
def test_in_place_row_ranges_and_empty(oracle, log2n):
    n = 1 << log2n
    mods = _moduli(log2n)
    plan = ntt.Plan(log2n, mods, 3)
    per_row = [mods[r % 2] for r in range(6)]
    x = W.rows_uniform(9, 4, per_row, n)
    dx = to_dev(x)
    full = torch.empty_like(dx)
    plan.forward(dx, full)
    y = dx.clone()
    plan.forward(y)                                   # in place
    assert torch.equal(y, full)
    z = dx.clone()
    plan.forward_rows(z, z, 2, 3)
    assert torch.equal(z[2:5], full[2:5]) and torch.equal(z[:2], dx[:2]) and torch.equal(z[5:], dx[5:])
    plan.forward_rows(z, z, 6, 0)                     # empty range: no launch
    assert plan.last_launches() == 0
    from paper_2410_05934_gb300 import _native
    L = _native.load()
    assert L.ntt_forward_rows(plan.handle, z.data_ptr(), z.data_ptr(), 5, 2, None) == -1
    assert L.ntt_forward(plan.handle, z.data_ptr() + 8, z.data_ptr(), None) == -5


@pytest.mark.parametrize("q", [W.Q62_N1024, W.POOL50[0]])
def test_extreme_values(oracle, q):
    plan = ntt.Plan(10, [q], 4)
    x = np.zeros((4, 1024), dtype=np.uint64)
    x[1, :] = q - 1
    x[2, 0] = 1
    x[3, 1] = 1
    for s in range(ntt.schedule_count(10)):
        plan.schedule = s
        out = plan.forward(to_dev(x), torch.empty((4, 1024), dtype=torch.int64, device="cuda"))
        h = to_host(out)
        assert not h[0].any()
        assert np.array_equal(h[1], oracle.ntt_forward(x[1], q))
        assert np.all(h[2] == 1)
        assert np.array_equal(h[3], oracle.ntt_forward(x[3], q))


def test_range_check_reports_status():
    q = W.Q59_N1024
    plan = ntt.Plan(10, [q], 2, flags=ntt.NTT_FLAG_CHECK)
    x = np.zeros((2, 1024), dtype=np.uint64)
    d = to_dev(x)
    plan.forward(d, torch.empty_like(d))
    assert plan.status() == 0
    x[1, 500] = q
    d = to_dev(x)
    plan.forward(d, torch.empty_like(d))
    assert plan.status() == -8
    assert plan.status() == 0                        # cleared on read


def test_pointwise_against_oracle(oracle):
    for q, log2n in [(W.Q62_N1024, 10), (W.POOL50[0], 16), (W.Q59_N1024, 1)]:
        n = 1 << log2n
        plan = ntt.Plan(log2n, [q], 3)
        a = W.rows_uniform(3, 1, [q] * 3, n)
        b = W.rows_uniform(3, 2, [q] * 3, n)
        a[0, : min(n, 64)] = q - 1
        b[0, : min(n, 64)] = q - 1
        c = to_host(plan.pointwise(to_dev(a), to_dev(b), torch.empty((3, n), dtype=torch.int64, device="cuda")))
        for r in range(3):
            assert np.array_equal(c[r], oracle.pointwise(a[r], b[r], q))


def test_maximum_size_row_index_beyond_2_32(oracle):
    """2^16 rows of N = 2^16: 2^32 coefficients, so element offsets need 64 bits."""
    log2n, rows = 16, 1 << 16
    n = 1 << log2n
    q = W.POOL50[0]
    free, _ = torch.cuda.mem_get_info()
    if free < 40 * 2**30:
        pytest.skip("needs 40 GiB free")
    plan = ntt.Plan(log2n, [q], rows)
    d = torch.zeros((rows, n), dtype=torch.int64, device="cuda")
    pick = [0, 1, rows // 2 + 3, rows - 1]
    x = W.rows_uniform(77, 8, [q] * len(pick), n)
    for i, r in enumerate(pick):
        d[r] = to_dev(x[i])
    for s in range(ntt.schedule_count(log2n)):
        plan.schedule = s
        e = d.clone() if s == 0 else e.copy_(d)
        plan.forward(e)
        idx = _sample_idx(n, len(pick), 12, s)
        ref = oracle.transform_rows(x, [q] * len(pick), idx=idx)
        got = to_host(e[pick])
        assert np.array_equal(got[np.arange(len(pick))[:, None], idx], ref), s
        zero_rows = to_host(e[[2, rows // 2, rows - 2]])
        assert not zero_rows.any()
    del d, e
    torch.cuda.empty_cache()


def test_hmul_tensor_ckks_shape(oracle):
    """Fused CKKS tensor product + inverse at N=2^16, 24 limbs: d0, d1, d2 at
    sampled coefficients against the oracle's schoolbook products."""
    w = W.ckks_hmul_n65536()
    mods, x = w["moduli"], w["x"]
    L, n = len(mods), 1 << 16
    plan = ntt.Plan(16, mods, 4)
    dx = to_dev(x.reshape(4 * L, n))
    A = torch.empty_like(dx)
    plan.forward(dx, A)
    out = torch.empty((3 * L, n), dtype=torch.int64, device="cuda")
    plan.hmul_tensor(A[:2 * L].contiguous(), A[2 * L:].contiguous(), out)
    got = to_host(out)
    kk = np.array([0, 1, 12345, n - 1], dtype=np.uint32)
    for l in (0, 7, 23):
        q = mods[l]
        a0, a1, b0, b1 = x[0, l], x[1, l], x[2, l], x[3, l]
        d0 = oracle.schoolbook_at(a0, b0, q, kk)
        d1 = (oracle.schoolbook_at(a0, b1, q, kk).astype(object) + oracle.schoolbook_at(a1, b0, q, kk).astype(object)) % q
        d2 = oracle.schoolbook_at(a1, b1, q, kk)
        assert np.array_equal(got[l][kk], d0)
        assert np.array_equal(got[L + l][kk], np.array(d1, dtype=np.uint64))
        assert np.array_equal(got[2 * L + l][kk], d2)


def test_hand_derived_known_answers():
    """The kernels reproduce the hand-worked examples of tests/golden (q = 17)."""
    from golden.load import negacyclic_q17
    ntt_cases, mul_cases = negacyclic_q17()
    for q, log2n, psi, a, A in ntt_cases:
        p = ntt.Plan(log2n, [q], 1)
        assert p.root(0) == psi
        x = to_dev(np.array(a, dtype=np.uint64))
        y = torch.empty_like(x)
        p.forward(x, y)
        assert to_host(y).tolist() == A
        p.inverse(y, x)
        assert to_host(x).tolist() == a
        assert p.status() == 0
    for q, log2n, a, b, c in mul_cases:
        p = ntt.Plan(log2n, [q], 1)
        xa, xb = to_dev(np.array(a, dtype=np.uint64)), to_dev(np.array(b, dtype=np.uint64))
        p.forward(xa)
        p.forward(xb)
        p.pointwise(xa, xb, xa)
        p.inverse(xa)
        assert to_host(xa).tolist() == c


@pytest.mark.parametrize("log2n", [10, 13, 16])
def test_natural_order_plans(oracle, log2n):
    """NTT_FLAG_NATURAL_ORDER: forward output A[brv(j)] at j, inverse back,
    in place too; sampled against the oracle at N = 2^16."""
    n = 1 << log2n
    mods = _moduli(log2n, "small")
    x = W.rows_uniform(23, log2n, mods * 2, n)
    p = ntt.Plan(log2n, mods, 2, flags=4)
    d = to_dev(x)
    out = torch.empty_like(d)
    p.forward(d, out)
    got = to_host(out)
    rng = np.random.default_rng(log2n)
    idx = np.stack([np.concatenate([[0, 1, n - 1], rng.integers(0, n, 13)]) for _ in range(4)]).astype(np.uint32)
    brv = np.array([[oracle.bitrev(int(j), log2n) for j in row] for row in idx], dtype=np.uint32)
    ref = oracle.transform_rows(x, [mods[r % 2] for r in range(4)], idx=brv)
    assert np.array_equal(got[np.arange(4)[:, None], idx], ref)
    back = torch.empty_like(d)
    p.inverse(out, back)
    assert torch.equal(back, d)
    p.inverse(out)                                   # in place
    assert torch.equal(out, d)
    assert p.status() == 0


@pytest.mark.parametrize("log2n", [10, 12, 14])
def test_inverse_mul_every_schedule(oracle, log2n):
    """ntt_inverse_mul (the product formed in the inverse's first kernel) on
    every schedule, identity and cross-product maps, against the oracle."""
    n, mods = 1 << log2n, _moduli(log2n, "small")
    x = W.rows_uniform(41, log2n, mods * 4, n)              # 4 polys x 2 limbs, NTT domain
    per = [mods[r % 2] for r in range(8)]
    rows_a = [p * 2 + l for p in (0, 0, 1, 1) for l in range(2)]
    rows_b = [p * 2 + l for p in (2, 3, 2, 3) for l in range(2)]
    idx = _sample_idx(n, 8, 10, log2n)
    prod = np.array([oracle.pointwise(x[ra], x[rb], per[k]) for k, (ra, rb) in enumerate(zip(rows_a, rows_b))])
    want = oracle.transform_rows(prod, per, inverse=True, idx=idx)
    plan = ntt.Plan(log2n, mods, 4)
    d = to_dev(x)
    for s in range(ntt.schedule_count(log2n)):
        plan.schedule = s                           # a pipelined first kernel falls back to a direct one
        out = torch.empty_like(d)
        plan.inverse_mul(d, d, out, a_poly=[0, 0, 1, 1], b_poly=[2, 3, 2, 3])
        assert np.array_equal(to_host(out)[np.arange(8)[:, None], idx], want), s
    with pytest.raises(ntt.NttError):
        plan.inverse_mul(d, d, out, a_poly=[0, 0, 1, 4], b_poly=[2, 3, 2, 3])     # index out of range


def test_natural_order_plans_reject_fused_operators():
    q = W.Q62_N1024
    p = ntt.Plan(10, [q], 3, flags=4)
    z = torch.zeros((3, 1024), dtype=torch.int64, device="cuda")
    with pytest.raises(ntt.NttError) as e:
        p.hmul_tensor(z[:2], z[:2], torch.zeros((3, 1024), dtype=torch.int64, device="cuda"))
    assert e.value.code == -10
    with pytest.raises(ntt.NttError) as e:
        p.tfhe_external_product(torch.zeros((1, 2, 1024), dtype=torch.int64, device="cuda"),
                                torch.zeros((6, 2, 1024, 2), dtype=torch.int64, device="cuda"), 3, 8)
    assert e.value.code == -10


Q30 = [1073692673, 1073668097]   # the largest primes < 2^30 that are 1 mod 2^13


def _to_dev32(x):
    return torch.from_numpy(np.ascontiguousarray(x).astype(np.uint32).view(np.int32)).cuda()


def _to_host32(t):
    return t.cpu().numpy().view(np.uint32).astype(np.uint64)


@pytest.mark.parametrize("log2n", list(range(1, 13)))
def test_word32_plans(oracle, log2n):
    """NTT_FLAG_WORD32: uint32 rows, 30-bit primes, every N up to 2^12."""
    n = 1 << log2n
    x = W.rows_uniform(29, log2n, Q30 * 3, n)
    p = ntt.Plan(log2n, Q30, 3, flags=ntt.NTT_FLAG_WORD32)
    d = _to_dev32(x)
    out = torch.empty_like(d)
    p.forward(d, out)
    got = _to_host32(out)
    assert np.array_equal(got, oracle.transform_rows(x, Q30 * 3))
    back = torch.empty_like(d)
    p.inverse(out, back)
    assert torch.equal(back, d)
    prod = torch.empty_like(d)
    p.pointwise(out, out, prod)
    want = np.array([[int(a) * int(a) % Q30[r % 2] for a in got[r]] for r in range(6)], dtype=np.uint64)
    assert np.array_equal(_to_host32(prod), want)
    assert p.status() == 0


def test_word32_tfhe_shape_and_rules(oracle):
    """3780 rows at N = 1024 (the TFHE forward batch) sampled; range check; rules."""
    q = Q30[0]
    x = W.rows_uniform(31, 10, [q] * 3780, 1024)
    p = ntt.Plan(10, [q], 3780, flags=ntt.NTT_FLAG_WORD32)
    d = _to_dev32(x)
    p.forward(d)
    got = _to_host32(d)
    rows = np.array([0, 1, 1777, 3779])
    assert np.array_equal(got[rows], oracle.transform_rows(x[rows], [q] * 4))
    chk = ntt.Plan(10, [q], 1, flags=ntt.NTT_FLAG_WORD32 | ntt.NTT_FLAG_CHECK)
    bad = torch.zeros((1, 1024), dtype=torch.int32, device="cuda")
    bad[0, 9] = q
    chk.forward(bad)
    assert chk.status() == -8
    with pytest.raises(ntt.NttError):
        ntt.Plan(13, [Q30[0]], 1, flags=ntt.NTT_FLAG_WORD32)
    with pytest.raises(ntt.NttError):
        ntt.Plan(10, [W.POOL50[0]], 1, flags=ntt.NTT_FLAG_WORD32)
    with pytest.raises(ValueError):
        p.forward(torch.zeros((3780, 1024), dtype=torch.int64, device="cuda"))   # 64-bit buffer


def _prime_62(log2n):
    step = 1 << (log2n + 1)
    q = ((1 << 62) - 1) // step * step + 1
    from oracle import oracle as O
    while not O.is_prime(q):
        q -= step
    return q


@pytest.mark.parametrize("log2n", range(10, 17))
def test_otf_twiddle_plans(oracle, log2n):
    """NTT_FLAG_OTF_TWIDDLES on the GPU: the same bits as the stored-table
    plan (both modulus classes), oracle samples, the inverse, a row range."""
    n = 1 << log2n
    for mods in (W.POOL50[:3], [_prime_62(log2n), W.POOL50[2]]):
        rows = 3 * len(mods)
        per_row = [mods[r % len(mods)] for r in range(rows)]
        x = W.rows_uniform(43, log2n, per_row, n)
        otf = ntt.Plan(log2n, mods, 3, flags=ntt.NTT_FLAG_OTF_TWIDDLES)
        tab = ntt.Plan(log2n, mods, 3)
        d = to_dev(x)
        a, b = torch.empty_like(d), torch.empty_like(d)
        otf.forward(d, a)
        tab.forward(d, b)
        assert torch.equal(a, b)
        got = to_host(a)
        rng = np.random.default_rng(log2n)
        idx = np.stack([np.concatenate([[0, n - 1], rng.integers(0, n, 6)]) for _ in per_row]).astype(np.uint32)
        assert np.array_equal(got[np.arange(rows)[:, None], idx], oracle.transform_rows(x, per_row, idx=idx))
        otf.inverse(d, a)
        tab.inverse(d, b)
        assert torch.equal(a, b)
        back = torch.empty_like(d)
        otf.forward(d, a)
        otf.inverse(a, back)
        assert torch.equal(back, d)
        c = d.clone()
        otf.forward_rows(d, c, 1, rows - 2)
        assert torch.equal(c[1:rows - 1], a[1:rows - 1]) and torch.equal(c[0], d[0])
        assert otf.status() == 0
    for log2n_, flags in [(9, ntt.NTT_FLAG_OTF_TWIDDLES), (12, ntt.NTT_FLAG_OTF_TWIDDLES | ntt.NTT_FLAG_NATURAL_ORDER)]:
        with pytest.raises(ntt.NttError):
            ntt.Plan(log2n_, [W.POOL50[0]], 1, flags=flags)


@pytest.mark.parametrize("log2n", [12, 13, 16])
@pytest.mark.parametrize("cls", ["big", "mid", "small"])
def test_largest_residues_every_schedule(oracle, log2n, cls):
    """Inputs q - 1 (and q - 1 alternating with 0) with the largest primes of
    each modulus class drive every lazy bound to its largest value."""
    n = 1 << log2n
    mods = _moduli(log2n, cls)
    x = np.zeros((4, n), dtype=np.uint64)
    x[0, :] = mods[0] - 1
    x[1, :] = mods[1] - 1
    x[2, ::2] = mods[0] - 1
    x[3, 1::2] = mods[1] - 1
    per_row = [mods[r % 2] for r in range(4)]
    idx = _sample_idx(n, 4, 9, log2n)
    r = np.arange(4)[:, None]
    want = oracle.transform_rows(x, per_row, idx=idx)
    want_inv = oracle.transform_rows(x, per_row, inverse=True, idx=idx)
    plan = ntt.Plan(log2n, mods, 2)
    dx = to_dev(x)
    for s in range(ntt.schedule_count(log2n)):
        plan.schedule = s
        fwd, back, inv = torch.empty_like(dx), torch.empty_like(dx), torch.empty_like(dx)
        plan.forward(dx, fwd)
        assert np.array_equal(to_host(fwd)[r, idx], want), s
        plan.inverse(fwd, back)
        assert torch.equal(back, dx), s
        plan.inverse(dx, inv)
        assert np.array_equal(to_host(inv)[r, idx], want_inv), s


def test_word32_back_to_back_in_place(oracle):
    """In-place 32-bit transforms issued back to back with no host
    synchronisation (each launch may start while the previous finishes):
    forward, inverse, forward again equals the oracle's forward; one more
    inverse gives the input back."""
    q = Q30[0]
    x = W.rows_uniform(37, 10, [q] * 2048, 1024)
    p = ntt.Plan(10, [q], 2048, flags=ntt.NTT_FLAG_WORD32)
    d = _to_dev32(x)
    ref_in = d.clone()
    torch.cuda.synchronize()
    p.forward(d)
    p.inverse(d)
    p.forward(d)
    got = _to_host32(d)
    rows = np.array([0, 5, 1024, 2047])
    assert np.array_equal(got[rows], oracle.transform_rows(x[rows], [q] * 4))
    p.inverse(d)
    assert torch.equal(d, ref_in)
    assert p.status() == 0


def test_forward_inverse_word32_tfhe_batch(oracle):
    """ntt_forward_inverse on the blind-rotation shape with 32-bit words (3780
    digit rows forward, 1260 rows inverse, one launch) equals the oracle's
    forward and inverse definitions on sampled rows and the separate calls
    on every row; issued twice in a row in place, with no host
    synchronisation in between."""
    q = Q30[0]
    xf = W.signed_digits_mod(W.DEFAULT_SEED, 3, 3780 * 1024, q).reshape(3780, 1024)
    xi = W.uniform_mod(W.DEFAULT_SEED, 4, 1260 * 1024, q).reshape(1260, 1024)
    pf = ntt.Plan(10, [q], 3780, flags=ntt.NTT_FLAG_WORD32)
    pi = ntt.Plan(10, [q], 1260, flags=ntt.NTT_FLAG_WORD32)
    df, di = _to_dev32(xf), _to_dev32(xi)
    of, oi = torch.empty_like(df), torch.empty_like(di)
    ntt.forward_inverse(pf, df, di, pi, of, oi)
    assert pf.last_launches() == 1
    rf, ri = np.array([0, 1, 2000, 3779]), np.array([0, 7, 1259])
    assert np.array_equal(_to_host32(of)[rf], oracle.transform_rows(xf[rf], [q] * 4))
    assert np.array_equal(_to_host32(oi)[ri], oracle.transform_rows(xi[ri], [q] * 3, inverse=True))
    sf, si = torch.empty_like(df), torch.empty_like(di)
    pf.forward(df, sf)
    pi.inverse(di, si)
    assert torch.equal(of, sf) and torch.equal(oi, si)
    # twice in place, back to back: forward twice and inverse twice
    ntt.forward_inverse(pf, of, oi, pi)
    pf.forward(sf)
    pi.inverse(si)
    assert torch.equal(of, sf) and torch.equal(oi, si)
    assert pf.status() == 0 and pi.status() == 0


def test_forward_inverse_rules_and_64_bit(oracle):
    """64-bit plans of one modulus class run both transforms in one grid
    (one launch at N = 1024) with the oracle's results; overlapping buffers
    of the two transforms, different N and mixed word sizes are argument
    errors."""
    q = W.Q62_N1024
    x = W.rows_uniform(43, 10, [q] * 6, 1024)
    pf, pi = ntt.Plan(10, [q], 4), ntt.Plan(10, [q], 2)
    d = to_dev(x)
    f, i = torch.empty_like(d[:4]), torch.empty_like(d[4:])
    ntt.forward_inverse(pf, d[:4].contiguous(), d[4:].contiguous(), pi, f, i)
    assert pf.last_launches() == 1
    assert np.array_equal(to_host(f), oracle.transform_rows(x[:4], [q] * 4))
    assert np.array_equal(to_host(i), oracle.transform_rows(x[4:], [q] * 2, inverse=True))
    assert pf.status() == 0 and pi.status() == 0
    with pytest.raises(ntt.NttError):
        ntt.forward_inverse(pf, d[:4], d[2:4], pi)                 # inverse rows inside the forward's buffer
    with pytest.raises(ntt.NttError):
        ntt.forward_inverse(pf, f, i, ntt.Plan(11, [_prime_62(11)], 1),
                            out_inv=torch.empty((1, 2048), dtype=torch.int64, device="cuda"))
    p32 = ntt.Plan(10, [Q30[0]], 2, flags=ntt.NTT_FLAG_WORD32)
    with pytest.raises(ntt.NttError):
        ntt.forward_inverse(pf, f, torch.zeros((2, 1024), dtype=torch.int32, device="cuda"), p32)


@pytest.mark.parametrize("log2n", [12, 13, 16])
def test_forward_inverse_64_bit_two_phases_and_fallback(oracle, log2n):
    """64-bit ntt_forward_inverse at larger N (one grid per kernel phase: two
    launches from 2^13 up) on multi-limb plans with different row counts,
    against the separate calls and sampled oracle outputs; plans of
    different modulus classes fall back to the two calls in stream order."""
    n = 1 << log2n
    mods = [W.POOL50[0], W.POOL50[5]]
    xf = W.rows_uniform(51, log2n, mods * 3, n)       # 3 polys x 2 limbs
    xi = W.rows_uniform(52, log2n, mods * 2, n)       # 2 polys x 2 limbs
    pf, pi = ntt.Plan(log2n, mods, 3), ntt.Plan(log2n, mods, 2)
    df, di = to_dev(xf), to_dev(xi)
    of, oi = torch.empty_like(df), torch.empty_like(di)
    ntt.forward_inverse(pf, df, di, pi, of, oi)
    assert pf.last_launches() == (1 if log2n <= 12 else 2)
    sf, si = torch.empty_like(df), torch.empty_like(di)
    pf.forward(df, sf)
    pi.inverse(di, si)
    assert torch.equal(of, sf) and torch.equal(oi, si)
    idx = np.array([[0, 1, n // 2, n - 1]] * 2, dtype=np.uint32)
    assert np.array_equal(to_host(of)[[0, 5]][:, [0, 1, n // 2, n - 1]],
                          oracle.transform_rows(xf[[0, 5]], [mods[0], mods[1]], idx=idx))
    q62 = _prime_62(log2n)
    p62 = ntt.Plan(log2n, [q62], 2)
    x62 = W.rows_uniform(53, log2n, [q62] * 2, n)
    d62, o62 = to_dev(x62), torch.empty((2, n), dtype=torch.int64, device="cuda")
    ntt.forward_inverse(p62, d62, di, pi, o62, oi)     # class 0 forward, class 2 inverse
    assert torch.equal(oi, si)
    p62.forward(d62, sf[:2])
    assert torch.equal(o62, sf[:2])
    assert pf.status() == 0 and pi.status() == 0 and p62.status() == 0


@pytest.mark.gpu
def test_two_stream_row_split_parity_and_graph_capture(oracle):
    """A two-kernel batch inside the split window (N = 2^16, 48 rows: 3.1 M
    coefficients) runs as two row halves on the caller's stream and the
    plan's side stream: sampled outputs against the oracle, equality with
    row ranges below the window (issued unsplit), the inverse round trip,
    the fused-product inverse against pointwise + inverse, and the same
    transform captured in a CUDA graph and replayed."""
    log2n, n = 16, 1 << 16
    mods = [W.POOL50[i] for i in (0, 3, 7, 11)]
    polys = 12
    x = W.rows_uniform(61, log2n, mods * polys, n)
    plan = ntt.Plan(log2n, mods, polys)
    d = to_dev(x)
    out = torch.empty_like(d)
    plan.forward(d, out)
    assert plan.last_launches() == 4          # two halves x two kernels
    rows = [0, 5, 23, 24, 25, 47]
    idx = _sample_idx(n, len(rows), 6, 62)
    got = to_host(out)[rows][np.arange(len(rows))[:, None], idx]
    assert np.array_equal(got, oracle.transform_rows(x[rows], [mods[r % 4] for r in rows], idx=idx))
    parts = torch.empty_like(d)
    for r0 in range(0, 48, 12):               # 12 rows: 0.79 M coefficients, below the window
        plan.forward_rows(d, parts, r0, 12)
        assert plan.last_launches() == 2
    assert torch.equal(parts, out)
    back = torch.empty_like(d)
    plan.inverse(out, back)
    assert plan.last_launches() == 4 and torch.equal(back, d)
    b = to_dev(W.rows_uniform(63, log2n, mods * polys, n))
    fused = torch.empty_like(d)
    plan.inverse_mul(out, b, fused)
    prod = torch.empty_like(d)
    plan.pointwise(out, b, prod)
    ref = torch.empty_like(d)
    plan.inverse(prod, ref)
    assert torch.equal(fused, ref)
    g_out = torch.zeros_like(d)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        plan.forward(d, g_out)                # warm-up outside the capture
    torch.cuda.current_stream().wait_stream(side)
    g_out.zero_()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        plan.forward(d, g_out)
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(g_out, out)
    assert plan.status() == 0
