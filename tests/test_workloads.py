"""The seeded input generators: the numpy and torch versions agree, values
are canonical and the request list has the stated distribution."""
import numpy as np
import pytest

from paper_2410_05934_gb300 import workloads as W


def test_torch_generator_matches_numpy():
    torch = pytest.importorskip("torch")
    for q in [W.POOL50[0], W.Q59_N1024, W.Q62_N1024, 12289]:
        a = W.uniform_mod(7, 3, 5000, q, start=11)
        b = W.uniform_mod_torch(7, 3, 5000, q, start=11, device="cpu").numpy().view(np.uint64)
        assert np.array_equal(a, b)
        assert int(a.max()) < q
    r1 = W.request_rows(3, 5, 10, 3, 2)
    r2 = W.request_rows_torch(3, 5, 10, 3, 2, device="cpu").numpy().view(np.uint64)
    assert np.array_equal(r1, r2)


def test_uniformity_and_digits():
    q = W.POOL50[0]
    x = W.uniform_mod(1, 1, 200000, q).astype(np.float64) / q
    assert abs(x.mean() - 0.5) < 0.01 and abs(x.var() - 1 / 12) < 0.005
    d = W.signed_digits_mod(1, 2, 100000, W.Q62_N1024)
    s = np.where(d > W.Q62_N1024 // 2, d.astype(object) - W.Q62_N1024, d.astype(object)).astype(np.int64)
    assert s.min() == -128 and s.max() == 127


def test_mixed_request_distribution():
    reqs = W.mixed_requests(n_requests=4000)
    ns = np.array([r[0] for r in reqs])
    for log2n, wgt in zip((10, 12, 14, 16), (0.5, 0.2, 0.2, 0.1)):
        assert abs((ns == log2n).mean() - wgt) < 0.03
    limbs = np.array([r[1] for r in reqs])
    polys = np.array([r[2] for r in reqs])
    assert limbs.min() == 1 and limbs.max() == 32 and polys.min() == 1 and polys.max() == 64
    assert W.mixed_requests() == W.mixed_requests()   # deterministic


def test_timing_records_follow_the_schedule_list():
    """A timing record only counts for the candidate list it was measured on."""
    from paper_2410_05934_gb300 import tune
    sig10, sig16 = tune.schedule_signature(10), tune.schedule_signature(16)
    assert sig10 != sig16 and len(sig10) == 12
    assert tune.schedule_signature(10) == sig10                   # stable
    recs = [dict(log2n=10, sig=sig10), dict(log2n=16, sig=sig10), dict(log2n=16), dict(log2n=16, sig=sig16)]
    assert tune.current_records(recs) == [recs[0], recs[3]]
