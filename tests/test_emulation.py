"""The CUDA kernels' phase functions run on the host (libntt_gb300_emu.so,
same source as the kernels, every memory index bounds-checked) and must be
bit-exact against the oracle for every schedule of every N."""
import numpy as np
import pytest

from paper_2410_05934_gb300 import workloads as W
import emu


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
        return _primes_below(57, max(log2n, 16), 2)
    return [W.POOL50[0], W.POOL50[7]]


@pytest.mark.parametrize("cls", ["big", "mid", "small"])
@pytest.mark.parametrize("log2n", range(1, 17))
def test_every_schedule_matches_oracle(oracle, log2n, cls):
    n = 1 << log2n
    mods = _moduli(log2n, cls)
    batch = 2
    plan = emu.EmuPlan(log2n, mods, batch)
    per_row = [mods[r % len(mods)] for r in range(batch * len(mods))]
    x = W.rows_uniform(31, log2n, per_row, n)
    if log2n <= 11:
        ref = oracle.transform_rows(x, per_row)
        idx = None
    else:
        rng = np.random.default_rng(log2n)
        idx = np.stack([np.concatenate([[0, 1, n // 2, n - 1], rng.integers(0, n, 12)])
                        for _ in per_row]).astype(np.uint32)
        ref = oracle.transform_rows(x, per_row, idx=idx)
    rows = np.arange(len(per_row))[:, None]
    for s in range(emu.schedule_count(log2n)):
        out = plan.transform(x, s)
        got = out if idx is None else out[rows, idx]
        assert np.array_equal(got, ref), "schedule %d" % s
        back = plan.transform(out, s, inverse=True)
        assert np.array_equal(back, x), "round trip, schedule %d" % s
        # inverse of arbitrary canonical data against the oracle inverse
        if idx is None:
            inv = plan.transform(x, s, inverse=True)
            assert np.array_equal(inv, oracle.transform_rows(x, per_row, inverse=True))


@pytest.mark.parametrize("log2n", [1, 5, 10, 16])
def test_in_place_and_row_ranges(oracle, log2n):
    n = 1 << log2n
    mods = _moduli(log2n)
    plan = emu.EmuPlan(log2n, mods, 3)
    per_row = [mods[r % 2] for r in range(6)]
    x = W.rows_uniform(5, 3, per_row, n)
    full = plan.transform(x, 0)
    y = x.copy()
    plan.transform(y, 0, out=y)            # in place
    assert np.array_equal(y, full)
    z = x.copy()
    plan.transform(z, 0, out=z, row_begin=2, n_rows=3)
    assert np.array_equal(z[2:5], full[2:5])
    assert np.array_equal(z[:2], x[:2]) and np.array_equal(z[5:], x[5:])


@pytest.mark.parametrize("q", [W.Q62_N1024, W.POOL50[0]])
def test_extreme_values(oracle, q):
    log2n = 10
    n = 1 << log2n
    plan = emu.EmuPlan(log2n, [q], 3)
    x = np.zeros((3, n), dtype=np.uint64)
    x[1, :] = q - 1
    x[2, 0] = 1
    for s in range(emu.schedule_count(log2n)):
        out = plan.transform(x, s)
        assert not out[0].any()
        assert np.array_equal(out[1], oracle.ntt_forward(x[1], q))
        assert np.all(out[2] == 1)
        assert np.array_equal(plan.transform(out, s, inverse=True), x)


def test_range_check_flag_reports_non_canonical_input():
    q = W.Q59_N1024
    plan = emu.EmuPlan(10, [q], 1, flags=2)
    x = np.zeros((1, 1024), dtype=np.uint64)
    plan.transform(x, 0)
    assert plan.status() == 0
    x[0, 77] = q
    plan.transform(x, 0)
    assert plan.status() == -8


def test_pointwise_barrett_matches_oracle(oracle):
    for q in [W.Q62_N1024, W.Q59_N1024, W.POOL50[0], 12289, 257]:
        log2n = 4 if q == 257 else 6
        n = 1 << log2n
        plan = emu.EmuPlan(log2n, [q], 4)
        a = W.rows_uniform(1, 1, [q] * 4, n)
        b = W.rows_uniform(1, 2, [q] * 4, n)
        a[0, :] = q - 1
        b[0, :] = q - 1
        c = plan.pointwise(a, b)
        for r in range(4):
            assert np.array_equal(c[r], oracle.pointwise(a[r], b[r], q))


@pytest.mark.parametrize("log2n,rows", [(8, 13), (10, 11), (12, 7), (16, 3)])
def test_single_modulus_batches(oracle, log2n, rows):
    """One modulus for all rows: the pipelined kernels keep a tile slot's
    twiddles across groups instead of copying them again."""
    q = W.POOL50[3]
    n = 1 << log2n
    plan = emu.EmuPlan(log2n, [q], rows)
    x = W.rows_uniform(17, log2n, [q] * rows, n)
    if log2n <= 12:
        ref = oracle.transform_rows(x, [q] * rows)
        idx = None
    else:
        idx = np.stack([np.array([0, 5, n // 3, n - 1])] * rows).astype(np.uint32)
        ref = oracle.transform_rows(x, [q] * rows, idx=idx)
    for s in range(emu.schedule_count(log2n)):
        out = plan.transform(x, s)
        got = out if idx is None else out[np.arange(rows)[:, None], idx]
        assert np.array_equal(got, ref), s
        assert np.array_equal(plan.transform(out, s, inverse=True), x), s


@pytest.mark.parametrize("log2n", range(10, 17))
def test_mixed_batch_configs_match_oracle(oracle, log2n):
    """The per-N tile configurations of the mixed-batch persistent kernel."""
    n = 1 << log2n
    mods = [W.POOL50[2], W.POOL50[9], W.POOL50[30]]
    plan = emu.EmuPlan(log2n, mods, 2)
    per_row = [mods[r % 3] for r in range(6)]
    x = W.rows_uniform(23, log2n, per_row, n)
    idx = np.stack([np.array([0, 1, 7, n // 2, n - 1]) for _ in per_row]).astype(np.uint32)
    out = plan.batch_transform(x)
    assert np.array_equal(out[np.arange(6)[:, None], idx], oracle.transform_rows(x, per_row, idx=idx))
    assert np.array_equal(plan.batch_transform(out, inverse=True), x)
    inv = plan.batch_transform(x, inverse=True)
    assert np.array_equal(inv[np.arange(6)[:, None], idx],
                          oracle.transform_rows(x, per_row, inverse=True, idx=idx))


def test_fast_division_is_exact():
    """The reciprocal division of tile/row indices (host build of the same code)."""
    import random
    rng = random.Random(1)
    ds = [2, 3, 5, 7, 24, 48, 1000, 3780, 65535, (1 << 31) - 1, (1 << 32) - 1]
    ns = [0, 1, 2, 3, (1 << 32) - 1, (1 << 31), 12345678] + [rng.getrandbits(32) for _ in range(2000)]
    for d in ds:
        M = ((1 << 64) + d - 1) // d
        for n in ns:
            mh, ml = M >> 32, M & 0xFFFFFFFF
            t = n * mh + ((n * ml) >> 32)
            assert (t >> 32) == n // d, (n, d)


@pytest.mark.parametrize("log2n", [10, 13, 16])
def test_hmul_tensor_matches_schoolbook(oracle, log2n):
    """Fused tensor product + inverse: d0 = a0 b0, d1 = a0 b1 + a1 b0,
    d2 = a1 b1 (negacyclic products, checked against the oracle's schoolbook
    coefficients), for every direct-form schedule of N."""
    n = 1 << log2n
    mods = [W.POOL50[1], W.POOL50[4]]
    L = len(mods)
    plan = emu.EmuPlan(log2n, mods, 4)
    per_row = [mods[r % L] for r in range(2 * L)]
    ca = W.rows_uniform(51, 1, per_row, n)       # a0 (L rows), a1 (L rows), coefficient domain
    cb = W.rows_uniform(51, 2, per_row, n)
    A = plan.transform(np.concatenate([ca, cb]), 0)    # forward NTT of a and b
    Aa, Ab = A[:2 * L], A[2 * L:]
    kk = np.array([0, 1, n // 2, n - 1], dtype=np.uint32)
    ref = {}
    for l, q in enumerate(mods):
        a0, a1, b0, b1 = ca[l], ca[L + l], cb[l], cb[L + l]
        d1 = (oracle.schoolbook_at(a0, b1, q, kk).astype(object) + oracle.schoolbook_at(a1, b0, q, kk).astype(object)) % q
        ref[l] = [oracle.schoolbook_at(a0, b0, q, kk), np.array(d1, dtype=np.uint64), oracle.schoolbook_at(a1, b1, q, kk)]
    tried = 0
    for s in range(emu.schedule_count(log2n)):
        try:
            out = plan.hmul_tensor(Aa, Ab, s)
        except ValueError:
            continue                                    # pipelined schedules: direct form only
        tried += 1
        for k in range(3):
            for l in range(L):
                assert np.array_equal(out[k * L + l][kk], ref[l][k]), (s, k, l)
    assert tried >= 1


@pytest.mark.parametrize("log2n,q", [(10, W.Q62_N1024), (10, W.POOL50[0]), (11, W.POOL50[3])])
def test_tfhe_cmux_and_external_product_match_oracle(log2n, q):
    """The CMux kernel's steps (decompose, NTT, MAC, exchange, INTT) on the
    host, against the schoolbook oracle of the external product and CMux."""
    from oracle import tfhe_oracle as TO
    n, levels, log2_base = 1 << log2n, 3, 8
    rng = np.random.default_rng(log2n + q % 7)
    d = rng.integers(0, q, (2, 2, n), dtype=np.uint64)
    key = rng.integers(0, q, (2 * levels, 2, n), dtype=np.uint64)
    rot = np.array([5, 2 * n - 3], dtype=np.uint32)
    plan = emu.EmuPlan(log2n, [q])
    kc = TO.key_coefficients(key, q)
    idx = [0, 1, 7, n // 2, n - 1]
    ep = plan.tfhe(d, key, levels, log2_base)
    cm = plan.tfhe(d, key, levels, log2_base, rot=rot)
    assert plan.status() == 0
    for c in range(2):
        assert np.array_equal(ep[c][:, idx], TO.external_product(d[c], key, q, log2_base, levels, key_coef=kc, idx=idx))
        assert np.array_equal(cm[c][:, idx], TO.cmux_rotate(d[c], int(rot[c]), key, q, log2_base, levels,
                                                            key_coef=kc, idx=idx))
    # in place, other gadgets, and a full-row comparison on one ciphertext
    for levels2, base2 in [(2, 10), (4, 6), (1, 16)]:
        key2 = rng.integers(0, q, (2 * levels2, 2, n), dtype=np.uint64)
        x = d.copy()
        plan.tfhe(x, key2, levels2, base2, rot=rot, out=x)
        assert np.array_equal(x[0], TO.cmux_rotate(d[0], int(rot[0]), key2, q, base2, levels2))


def test_tfhe_argument_rules():
    q = W.Q62_N1024
    plan = emu.EmuPlan(10, [q])
    d = np.zeros((1, 2, 1024), dtype=np.uint64)
    for levels, base in [(0, 8), (9, 3), (3, 11), (1, 33)]:
        with pytest.raises(ValueError):
            plan.tfhe(d, np.zeros((2 * max(levels, 1), 2, 1024), dtype=np.uint64), levels, base)
    with pytest.raises(ValueError):
        emu.EmuPlan(9, [q]).tfhe(d[:, :, :512], np.zeros((6, 2, 512), dtype=np.uint64), 3, 8)
    with pytest.raises(ValueError):
        emu.EmuPlan(10, [q, W.Q59_N1024]).tfhe(d, np.zeros((6, 2, 1024), dtype=np.uint64), 3, 8)
    # range check: a non-canonical coefficient sets the status word
    chk = emu.EmuPlan(10, [q], flags=2)
    bad = d.copy()
    bad[0, 1, 3] = q
    chk.tfhe(bad, np.zeros((6, 2, 1024), dtype=np.uint64), 3, 8)
    assert chk.status() == -8


@pytest.mark.parametrize("L,K", [(5, 3), (24, 24), (3, 40)])
def test_bconv_matches_oracle(L, K):
    """ntt_bconv's per-coefficient arithmetic (128-bit sums folded every
    `chunk` terms) against the oracle's definition, on 50- and 62-bit bases."""
    from oracle import rns_oracle as RO
    Q = W.POOL50[:L] if L <= 24 else W.POOL50[:L]
    P = W.POOL50[L:L + K] if L + K <= 48 else [W.Q62_N1024, W.Q59_N1024] + W.POOL50[L + 2:L + K]
    rng = np.random.default_rng(L * 100 + K)
    x = np.stack([np.array([rng.integers(0, q, 40, dtype=np.uint64) for q in Q]) for _ in range(2)])
    got = emu.bconv(x, Q, P)
    for p in range(2):
        assert np.array_equal(got[p], RO.bconv(x[p], Q, P))


def test_bconv_largest_bases():
    """64 -> 64 limbs: every output run length of the kernel's 4-warp split."""
    from oracle import rns_oracle as RO
    from oracle import oracle as O
    qs, c = [], (1 << 50) - 1
    while len(qs) < 128:
        if O.is_prime(c):
            qs.append(c)
        c -= 2
    rng = np.random.default_rng(9)
    for L, K in [(64, 64), (7, 6), (1, 1)]:
        Q, P = qs[:L], qs[64:64 + K]
        x = np.array([[rng.integers(0, q, 4, dtype=np.uint64) for q in Q]])
        assert np.array_equal(emu.bconv(x, Q, P)[0], RO.bconv(x[0], Q, P)), (L, K)


def test_bconv_62_bit_moduli_fold_the_accumulator():
    """62-bit primes on both sides: chunk = 16 terms, so 40 source limbs fold twice."""
    from oracle import rns_oracle as RO
    import sympy
    qs, c = [], (1 << 62) - 1
    while len(qs) < 43:
        if sympy.isprime(c):
            qs.append(c)
        c -= 2
    Q, P = qs[:40], qs[40:]
    rng = np.random.default_rng(3)
    x = np.array([[rng.integers(0, q, 8, dtype=np.uint64) for q in Q]])
    assert np.array_equal(emu.bconv(x, Q, P)[0], RO.bconv(x[0], Q, P))


def test_bconv_argument_rules():
    with pytest.raises(ValueError):
        emu.bconv(np.zeros((1, 2, 4), np.uint64), [W.POOL50[0], W.POOL50[0]], [W.POOL50[1]])   # repeated
    with pytest.raises(ValueError):
        emu.bconv(np.zeros((1, 1, 4), np.uint64), [W.POOL50[0]], [15])                          # not prime
    with pytest.raises(ValueError):
        emu.bconv(np.zeros((1, 1, 4), np.uint64), [W.POOL50[0]], [(1 << 62) + 135])             # too large


@pytest.mark.parametrize("log2n", [10, 12, 13])
def test_rescale_matches_oracle(log2n):
    """ntt_rescale's kernels (INTT of the dropped limb, forward transform with
    the Rescale load and epilogue) for every direct-form schedule of N,
    against the oracle's definition through the transform definitions."""
    from oracle import oracle as O
    from oracle import rns_oracle as RO
    Q = [W.POOL50[0], W.POOL50[5], W.POOL50[9]] if log2n > 10 else [W.Q62_N1024, W.POOL50[1], W.Q59_N1024]
    n = 1 << log2n
    rng = np.random.default_rng(log2n)
    x = np.stack([np.array([rng.integers(0, q, n, dtype=np.uint64) for q in Q]) for _ in range(2)])
    plan = emu.EmuPlan(log2n, Q, 2)
    want = [RO.rescale_ntt(x[p], Q) for p in range(2)]
    tried = 0
    for s in range(emu.schedule_count(log2n)):
        try:
            got = plan.rescale(x, s, 2)
        except ValueError:
            continue                                    # pipelined first kernel
        tried += 1
        for p in range(2):
            assert np.array_equal(got[p], want[p]), (s, p)
    assert tried >= 1 and plan.status() == 0


@pytest.mark.parametrize("log2n", [1, 3, 10, 12, 13, 14])
def test_natural_order_every_schedule(log2n):
    """NTT_FLAG_NATURAL_ORDER: the forward writes A[brv(j)] at j (fused into
    the store of one-kernel schedules, a tile bit-reversal pass otherwise) and
    the inverse reads that order back."""
    from oracle import oracle as O
    n = 1 << log2n
    q = W.POOL50[2] if log2n > 10 else W.Q62_N1024
    rng = np.random.default_rng(log2n)
    x = np.array([rng.integers(0, q, n, dtype=np.uint64) for _ in range(3)])
    brv = np.array([O.bitrev(j, log2n) for j in range(n)], dtype=np.int64)
    ref = O.transform_rows(x, [q] * 3)            # bit-reversed order
    want = ref[:, brv]
    plan = emu.EmuPlan(log2n, [q], 3, flags=4)
    for s in range(emu.schedule_count(log2n)):
        got = plan.transform(x, s)
        assert np.array_equal(got, want), s
        back = plan.transform(got, s, inverse=True)
        assert np.array_equal(back, x), s
        y = got.copy()
        plan.transform(y, s, inverse=True, out=y)   # in place (tile pairs swap)
        assert np.array_equal(y, x), s
    # a row range
    part = plan.transform(x, 0, row_begin=1, n_rows=1, out=np.zeros_like(x))
    assert np.array_equal(part[1], want[1]) and not part[0].any() and not part[2].any()


Q30 = [1073692673, 1073668097, 1073651713]   # the largest primes < 2^30 that are 1 mod 2^13


@pytest.mark.parametrize("log2n", list(range(1, 13)))
def test_word32_plans_match_oracle(log2n):
    """NTT_FLAG_WORD32: the 32-bit kernel's phases against the oracle (the
    same transform definition), plus the round trip and the pointwise product."""
    from oracle import oracle as O
    n = 1 << log2n
    mods = Q30[:2]
    rng = np.random.default_rng(log2n)
    x = np.array([rng.integers(0, mods[r % 2], n, dtype=np.uint64) for r in range(6)])
    plan = emu.EmuPlan(log2n, mods, 3, flags=8)
    got = plan.transform32(x.astype(np.uint32))
    assert np.array_equal(got.astype(np.uint64), O.transform_rows(x, [mods[r % 2] for r in range(6)]))
    assert np.array_equal(plan.transform32(got, inverse=True).astype(np.uint64), x)
    prod = plan.pointwise32(got, got[::-1].copy())
    want = np.array([[int(a) * int(b) % mods[r % 2] for a, b in zip(got[r], got[5 - r])] for r in range(6)],
                    dtype=np.uint64)
    assert np.array_equal(prod.astype(np.uint64), want)
    # extreme values and a row range
    top = np.array([[m - 1] * n for m in (mods * 3)[:6]], dtype=np.uint64)
    assert np.array_equal(plan.transform32(top.astype(np.uint32)).astype(np.uint64),
                          O.transform_rows(top, [mods[r % 2] for r in range(6)]))
    part = plan.transform32(x.astype(np.uint32), row_begin=3, n_rows=2)
    assert not part[:3].any() and not part[5].any() and np.array_equal(part[3:5], got[3:5])
    assert plan.status() == 0


def test_word32_plan_rules():
    with pytest.raises(ValueError):
        emu.EmuPlan(13, Q30[:1], 1, flags=8)                  # N > 2^12
    with pytest.raises(ValueError):
        emu.EmuPlan(10, [W.POOL50[0]], 1, flags=8)            # modulus >= 2^30
    with pytest.raises(ValueError):
        emu.EmuPlan(10, Q30[:1], 1, flags=8 | 4)              # natural order


@pytest.mark.parametrize("log2n", [4, 10, 13])
def test_inverse_mul_every_direct_schedule(log2n):
    """ntt_inverse_mul: the product formed in the inverse's first kernel, with
    the CKKS cross-product maps, equals INTT of the oracle's pointwise product."""
    from oracle import oracle as O
    n, mods = 1 << log2n, [W.POOL50[0], W.POOL50[4]]
    rng = np.random.default_rng(log2n)
    A = np.array([rng.integers(0, mods[r % 2], n, dtype=np.uint64) for r in range(8)])   # 4 polys x 2 limbs
    a_poly, b_poly = [0, 0, 1, 1], [2, 3, 2, 3]
    rows_a = [a_poly[k // 2] * 2 + k % 2 for k in range(8)]
    rows_b = [b_poly[k // 2] * 2 + k % 2 for k in range(8)]
    prod = np.array([O.pointwise(A[ra], A[rb], mods[k % 2]) for k, (ra, rb) in enumerate(zip(rows_a, rows_b))])
    want = O.transform_rows(prod, [mods[k % 2] for k in range(8)], inverse=True)
    plan = emu.EmuPlan(log2n, mods, 4)
    tried = 0
    for s in range(emu.schedule_count(log2n)):
        try:
            got = plan.inverse_mul(A, A, s, a_poly, b_poly)
        except ValueError:
            continue                                    # pipelined first kernel
        tried += 1
        assert np.array_equal(got, want), s
    assert tried >= 1
    # identity maps
    B = A[::-1].copy()[[6, 7, 4, 5, 2, 3, 0, 1]]
    got = plan.inverse_mul(A, B, 0)
    want2 = O.transform_rows(np.array([O.pointwise(A[r], B[r], mods[r % 2]) for r in range(8)]),
                             [mods[k % 2] for k in range(8)], inverse=True)
    assert np.array_equal(got, want2)


def test_forward_output_reduction_bounds():
    """The forward transform's last step in the small-modulus class maps
    x in [0, 65q) to x mod q with one estimated quotient and one conditional
    subtraction (reduce_65q): checked against x mod q for primes of every bit
    length 3..57 on the values where the estimate is tightest (multiples of q
    and their neighbours, 65q - 1, powers of two) and on random values."""
    from oracle import oracle as O
    rng = np.random.default_rng(65)
    qs = []
    for bits in range(3, 58):
        q = (1 << bits) - 3
        while q > (1 << (bits - 1)) and not (q % 4 == 1 and O.is_prime(q)):
            q -= 2
        if q > (1 << (bits - 1)):
            qs.append(q)
        qs.append(next(c for c in range((1 << (bits - 1)) + 1, 1 << bits, 4) if O.is_prime(c)))
    for q in qs:
        plan = emu.EmuPlan(1, [q], 1)
        top = 65 * q
        edges = [0, 1, q - 1, q, q + 1, top - 1, top - q, top - q - 1]
        edges += [k * q + d for k in range(1, 65) for d in (-1, 0, 1)]
        edges += [1 << b for b in range(64) if (1 << b) < top]
        edges += [(1 << b) - 1 for b in range(1, 64) if (1 << b) - 1 < top]
        x = np.array(edges + [int(v) for v in rng.integers(0, top, 2000, dtype=np.uint64)], dtype=np.uint64)
        want = np.array([int(v) % q for v in x], dtype=np.uint64)
        assert np.array_equal(plan.reduce_65q(0, x), want), q


def _prime_62(log2n):
    """Largest prime below 2^62 with q = 1 mod 2^(log2n + 1) (exact modulus class)."""
    from oracle import oracle as O
    step = 1 << (log2n + 1)
    q = ((1 << 62) - 1) // step * step + 1
    while not O.is_prime(q):
        q -= step
    return q


@pytest.mark.parametrize("log2n", range(10, 17))
@pytest.mark.parametrize("cls", ["small", "exact"])
def test_otf_twiddles_match_tables(oracle, log2n, cls):
    """NTT_FLAG_OTF_TWIDDLES: every twiddle formed from the two small tables
    gives the same bits as the stored-table transform and the oracle, both
    modulus classes, forward and inverse, on a ragged row range."""
    n = 1 << log2n
    mods = W.POOL50[:3] if cls == "small" else [_prime_62(log2n), W.POOL50[1]]
    rows = 2 * len(mods)
    per_row = [mods[r % len(mods)] for r in range(rows)]
    x = W.rows_uniform(41, log2n, per_row, n)
    x[0, :] = mods[0] - 1
    otf = emu.EmuPlan(log2n, mods, 2, flags=16)
    tab = emu.EmuPlan(log2n, mods, 2)
    fwd = otf.transform(x, 0)
    assert np.array_equal(fwd, tab.transform(x, 0))
    rng = np.random.default_rng(log2n)
    idx = np.stack([np.concatenate([[0, 1, n - 1], rng.integers(0, n, 9)]) for _ in per_row]).astype(np.uint32)
    r = np.arange(rows)[:, None]
    assert np.array_equal(fwd[r, idx], oracle.transform_rows(x, per_row, idx=idx))
    inv = otf.transform(x, 0, inverse=True)
    assert np.array_equal(inv, tab.transform(x, 0, inverse=True))
    assert np.array_equal(otf.transform(fwd, 0, inverse=True), x)
    part = otf.transform(x, 0, row_begin=1, n_rows=rows - 2)
    assert np.array_equal(part[1:rows - 1], fwd[1:rows - 1])
    assert otf.status() == 0


def test_otf_twiddle_plan_rules():
    for log2n, flags in [(9, 16), (12, 16 | 4), (10, 16 | 8)]:
        with pytest.raises(ValueError):
            emu.EmuPlan(log2n, [Q30[0] if flags & 8 else W.POOL50[0]], 1, flags=flags)


@pytest.mark.parametrize("log2n", [10, 13, 16])
def test_products_at_the_largest_residues(log2n):
    """The inverse's first kernel forms its products lazily (Barrett remainder
    in [0, 3q), a tensor-product sum folded into [0, 4q) in the small-modulus
    class): operands q - 1 everywhere give the largest remainders; the results
    must still equal the oracle's exact products transformed back."""
    from oracle import oracle as O
    n = 1 << log2n
    for mods in ([W.POOL50[0], W.POOL50[3]], [_prime_62(log2n), W.POOL50[3]]):
        A = np.array([np.full(n, mods[r % 2] - 1, dtype=np.uint64) for r in range(8)])
        A[1, ::3] = 1
        plan = emu.EmuPlan(log2n, mods, 4)
        a_poly, b_poly = [0, 0, 1, 1], [2, 3, 2, 3]
        rows_a = [a_poly[k // 2] * 2 + k % 2 for k in range(8)]
        rows_b = [b_poly[k // 2] * 2 + k % 2 for k in range(8)]
        prod = np.array([O.pointwise(A[ra], A[rb], mods[k % 2]) for k, (ra, rb) in enumerate(zip(rows_a, rows_b))])
        s = 5 if log2n >= 13 else 7
        got = plan.inverse_mul(A, A, s, a_poly, b_poly)
        idx = np.stack([np.concatenate([[0, 1, n - 1], np.arange(5, n, max(1, n // 24))[:24]])
                        for _ in range(8)]).astype(np.uint32)
        want = O.transform_rows(prod, [mods[k % 2] for k in range(8)], inverse=True, idx=idx)
        assert np.array_equal(got[np.arange(8)[:, None], idx], want)


@pytest.mark.parametrize("log2n", [12, 13, 16])
@pytest.mark.parametrize("cls", ["big", "mid", "small"])
def test_largest_residues_every_schedule(oracle, log2n, cls):
    """Inputs q - 1 (and q - 1 alternating with 0) drive every lazy bound to
    its largest value; with the largest primes of each modulus class every
    schedule must still give the oracle's outputs and round trip."""
    n = 1 << log2n
    mods = _moduli(log2n, cls)
    x = np.zeros((4, n), dtype=np.uint64)
    x[0, :] = mods[0] - 1
    x[1, :] = mods[1] - 1
    x[2, ::2] = mods[0] - 1
    x[3, 1::2] = mods[1] - 1
    per_row = [mods[r % 2] for r in range(4)]
    rng = np.random.default_rng(log2n)
    idx = np.stack([np.concatenate([[0, 1, n - 1], rng.integers(0, n, 9)]) for _ in per_row]).astype(np.uint32)
    r = np.arange(4)[:, None]
    want = oracle.transform_rows(x, per_row, idx=idx)
    want_inv = oracle.transform_rows(x, per_row, inverse=True, idx=idx)
    plan = emu.EmuPlan(log2n, mods, 2)
    for s in range(emu.schedule_count(log2n)):
        fwd = plan.transform(x, s)
        assert np.array_equal(fwd[r, idx], want), s
        assert np.array_equal(plan.transform(fwd, s, inverse=True), x), s
        assert np.array_equal(plan.transform(x, s, inverse=True)[r, idx], want_inv), s


@pytest.mark.parametrize("n_mod", [2, 1])
def test_word32_n1024_row_lists_and_forward_inverse(n_mod):
    """N = 1024 on 32-bit words: the persistent kernel's warps walk lists of
    several rows with two landing buffers (partial last quads included), in
    one direction and with forward and inverse rows in one grid
    (ntt_forward_inverse), against the oracle's definitions; with one
    modulus the twiddles come from the CTA's shared-memory copy."""
    from oracle import oracle as O
    mods = (Q30 * 2)[:2] if n_mod == 2 else [Q30[0]] * 2
    rng = np.random.default_rng(1024)
    xf = np.array([rng.integers(0, mods[r % 2], 1024, dtype=np.uint64) for r in range(30)])
    xi = np.array([rng.integers(0, mods[r % 2], 1024, dtype=np.uint64) for r in range(14)])
    pf = emu.EmuPlan(10, mods[:n_mod], 30 // n_mod, flags=8)
    pi = emu.EmuPlan(10, mods[:n_mod], 14 // n_mod, flags=8)
    want_f = O.transform_rows(xf, [mods[r % 2] for r in range(30)])
    want_i = O.transform_rows(xi, [mods[r % 2] for r in range(14)], inverse=True)
    assert np.array_equal(pf.transform32(xf.astype(np.uint32)).astype(np.uint64), want_f)
    assert np.array_equal(pi.transform32(xi.astype(np.uint32), inverse=True).astype(np.uint64), want_i)
    of, oi = pf.forward_inverse32(xf, pi, xi)
    assert np.array_equal(of.astype(np.uint64), want_f)
    assert np.array_equal(oi.astype(np.uint64), want_i)
    part = pf.transform32(xf.astype(np.uint32), row_begin=5, n_rows=19)
    assert not part[:5].any() and not part[24:].any() and np.array_equal(part[5:24].astype(np.uint64), want_f[5:24])
    assert pf.status() == 0 and pi.status() == 0
