"""Mixed batches through the persistent kernel (C ABI ntt_batch_*): every
request's output matches the oracle, the CUDA-graph replay after a pointer
update and the plain per-request arm give the same bits, and argument errors
are reported before any launch."""
import numpy as np
import pytest

from paper_2410_05934_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2410_05934_gb300 as ntt  # noqa: E402
from gpu_util import to_dev, to_host  # noqa: E402

SHAPES = [  # (log2n, limbs, polys, offset, inverse)
    (10, 3, 5, 0, 0), (16, 2, 2, 4, 0), (12, 1, 7, 2, 1), (14, 5, 1, 0, 0), (11, 2, 3, 9, 1),
    (13, 4, 2, 1, 0), (15, 1, 3, 0, 1), (10, 1, 1, 30, 1), (16, 3, 1, 0, 1), (12, 6, 2, 3, 0),
]


def _make(seed, shapes=SHAPES, in_place=False):
    reqs, hosts = [], []
    for i, (log2n, limbs, polys, off, inv) in enumerate(shapes):
        x = W.request_rows(seed, i, log2n, limbs, polys, pool=W.POOL50[off:])
        d = to_dev(x)
        o = d if (in_place and i % 2) else torch.empty_like(d)
        reqs.append(dict(log2n=log2n, n_moduli=limbs, n_polys=polys, moduli_offset=off, inverse=inv,
                         **{"in": d, "out": o}))
        hosts.append(x)
    return reqs, hosts


def _check(oracle, reqs, hosts, shapes=SHAPES):
    for (log2n, limbs, polys, off, inv), r, x in zip(shapes, reqs, hosts):
        n = 1 << log2n
        got = to_host(r["out"])
        per_row = [W.POOL50[off + (k % limbs)] for k in range(limbs * polys)]
        rng = np.random.default_rng(log2n * 7 + off)
        idx = np.stack([np.concatenate([[0, n - 1], rng.integers(0, n, 6)]) for _ in per_row]).astype(np.uint32)
        ref = oracle.transform_rows(x, per_row, inverse=bool(inv), idx=idx)
        assert np.array_equal(got[np.arange(len(per_row))[:, None], idx], ref), (log2n, limbs, polys, inv)


def test_persistent_batch_matches_oracle(oracle):
    reqs, hosts = _make(1)
    b = ntt.Batch(reqs, W.POOL50, flags=0)
    b.execute()
    torch.cuda.synchronize()
    assert b.info()["last_launches"] == 1
    _check(oracle, reqs, hosts)
    assert b.status() == 0


def test_graph_replay_with_new_pointers_and_plain_arm(oracle):
    reqs, hosts = _make(2, in_place=True)
    saved = [r["in"].clone() for r in reqs]
    b = ntt.Batch(reqs, W.POOL50, flags=ntt.NTT_BATCH_GRAPH)
    b.execute()
    torch.cuda.synchronize()
    _check(oracle, reqs, hosts)
    outs_graph = [to_host(r["out"]).copy() for r in reqs]
    # replay on fresh buffers holding the same inputs
    reqs2 = [dict(r, **{"in": s.clone()}) for r, s in zip(reqs, saved)]
    for r in reqs2:
        r["out"] = torch.empty_like(r["in"])
    b.update(reqs2)
    b.execute()
    torch.cuda.synchronize()
    for o, r in zip(outs_graph, reqs2):
        assert np.array_equal(o, to_host(r["out"]))
    # the per-request arm over the same tables
    reqs3 = [dict(r, **{"in": s.clone()}) for r, s in zip(reqs, saved)]
    for r in reqs3:
        r["out"] = torch.empty_like(r["in"])
    b.update(reqs3)
    b.execute_plain()
    torch.cuda.synchronize()
    assert b.info()["last_launches"] >= len(reqs3)
    for o, r in zip(outs_graph, reqs3):
        assert np.array_equal(o, to_host(r["out"]))


def test_batch_argument_errors():
    d = torch.zeros((4, 1024), dtype=torch.int64, device="cuda")
    good = dict(log2n=10, n_moduli=2, n_polys=2, moduli_offset=0, inverse=0, **{"in": d, "out": d})
    for bad, code in [(dict(log2n=9), -10), (dict(moduli_offset=47), -1), (dict(inverse=2), -1),
                      (dict(n_polys=0), -1)]:
        with pytest.raises(ntt.NttError) as e:
            ntt.Batch([dict(good, **bad)], W.POOL50)
        assert e.value.code == code
    with pytest.raises(ntt.NttError) as e:
        ntt.Batch([dict(good, **{"in": d.data_ptr() + 8})], W.POOL50)
    assert e.value.code == -5
    with pytest.raises(ntt.NttError) as e:
        ntt.Batch([dict(good, n_moduli=1)], [7681])                      # not 1 mod 2048
    assert e.value.code == -3


def test_batch_range_check():
    q = W.POOL50[0]
    x = np.zeros((2, 1024), dtype=np.uint64)
    x[1, 3] = q
    d = to_dev(x)
    b = ntt.Batch([dict(log2n=10, n_moduli=1, n_polys=2, moduli_offset=0, inverse=0, **{"in": d,
                        "out": torch.empty_like(d)})], W.POOL50, flags=ntt.NTT_FLAG_CHECK)
    b.execute()
    assert b.status() == -8


def test_scheduled_requests_in_the_same_graph(oracle):
    """Requests with a schedule run as their own launches on a second graph
    branch; together with the persistent kernel's items they give the oracle's
    bits, also after a pointer update (the graph is captured again)."""
    reqs, hosts = _make(3)
    for i, r in enumerate(reqs):
        if i % 3 != 1:
            continue
        r["schedule"] = 1 + (i // 3) % ntt.schedule_count(r["log2n"])
    n_sched = sum(1 for r in reqs if r.get("schedule"))
    assert n_sched >= 3
    b = ntt.Batch(reqs, W.POOL50, flags=ntt.NTT_BATCH_GRAPH)
    b.execute()
    torch.cuda.synchronize()
    info = b.info()
    assert info["last_launches"] >= 1 + n_sched
    assert info["items"] > 0
    _check(oracle, reqs, hosts)
    outs = [to_host(r["out"]).copy() for r in reqs]
    reqs2 = [dict(r, **{"in": to_dev(h), "out": torch.empty_like(r["in"])}) for r, h in zip(reqs, hosts)]
    b.update(reqs2)
    b.execute()
    torch.cuda.synchronize()
    for o, r in zip(outs, reqs2):
        assert np.array_equal(o, to_host(r["out"]))
    # every request scheduled: no persistent kernel at all
    reqs3 = [dict(r, schedule=1, **{"in": to_dev(h), "out": torch.empty_like(r["in"])})
             for r, h in zip(reqs, hosts)]
    b3 = ntt.Batch(reqs3, W.POOL50, flags=0)
    assert b3.info()["items"] == 0
    b3.execute()
    torch.cuda.synchronize()
    for o, r in zip(outs, reqs3):
        assert np.array_equal(o, to_host(r["out"]))
    assert b.status() == 0 and b3.status() == 0


def test_scheduled_request_argument_error():
    d = torch.zeros((4, 1024), dtype=torch.int64, device="cuda")
    r = dict(log2n=10, n_moduli=2, n_polys=2, moduli_offset=0, inverse=0, **{"in": d, "out": d})
    with pytest.raises(ntt.NttError) as e:
        ntt.Batch([dict(r, schedule=ntt.schedule_count(10) + 1)], W.POOL50)
    assert e.value.code == -1


def test_full_mixed_batch_as_benchmarked(oracle):
    """The 200-request mixed batch at its full size (about 1.1 G coefficients)
    in the configuration the bench times: requests of >= 2^22 coefficients on
    their learned schedules on the second graph branch, the rest in the
    persistent kernel; sampled rows and outputs of every request."""
    from paper_2410_05934_gb300.costmodel import schedule_requests
    spec = W.mixed_requests(seed=W.DEFAULT_SEED)
    reqs = []
    for i, (log2n, limbs, polys) in enumerate(spec):
        x = W.request_rows_torch(W.DEFAULT_SEED, i, log2n, limbs, polys)
        reqs.append(dict(log2n=log2n, n_moduli=limbs, n_polys=polys, moduli_offset=0, inverse=0,
                         **{"in": x, "out": torch.empty_like(x)}))
    sreqs = schedule_requests(reqs, W.POOL50, 22)
    assert any(r["schedule"] for r in sreqs) and any(not r["schedule"] for r in sreqs)
    b = ntt.Batch(sreqs, W.POOL50, flags=ntt.NTT_BATCH_GRAPH)
    b.execute()
    b.execute()                                      # a graph replay gives the same bits
    torch.cuda.synchronize()
    assert b.status() == 0
    rng = np.random.default_rng(200)
    for i, (log2n, limbs, polys) in enumerate(spec):
        n, rows = 1 << log2n, limbs * polys
        pick = sorted(set([0, rows - 1] + rng.integers(0, rows, 1).tolist()))
        x = np.stack([W.uniform_mod(W.DEFAULT_SEED, 1000 + i, n, W.POOL50[r % limbs], start=r * n) for r in pick])
        idx = np.stack([np.concatenate([[0, n - 1], rng.integers(0, n, 4)]) for _ in pick]).astype(np.uint32)
        ref = oracle.transform_rows(x, [W.POOL50[r % limbs] for r in pick], idx=idx)
        got = to_host(sreqs[i]["out"][pick])
        assert np.array_equal(got[np.arange(len(pick))[:, None], idx], ref), (i, log2n, limbs, polys)
        sreqs[i]["in"] = sreqs[i]["out"] = None       # free as we go


@pytest.mark.parametrize("flags", [ntt.NTT_BATCH_GROUPED, ntt.NTT_BATCH_GROUPED | ntt.NTT_BATCH_GRAPH])
def test_grouped_batch_matches_oracle(oracle, flags):
    """Grouped launches: the requests of one N (both directions) are segments
    of one grid per kernel phase; every N from 2^10 to 2^16."""
    reqs, hosts = _make(5)
    b = ntt.Batch(reqs, W.POOL50, flags=flags)
    b.execute()
    torch.cuda.synchronize()
    phases = {10: 1, 11: 1, 12: 1, 13: 2, 14: 2, 15: 2, 16: 2}
    assert b.info()["last_launches"] == sum(phases[n] for n in {s[0] for s in SHAPES})
    assert b.info()["items"] == 0                      # no persistent-kernel work items
    _check(oracle, reqs, hosts)
    assert b.status() == 0


def test_grouped_replay_after_pointer_update_in_place(oracle):
    reqs, hosts = _make(6, in_place=True)
    saved = [r["in"].clone() for r in reqs]
    b = ntt.Batch(reqs, W.POOL50, flags=ntt.NTT_BATCH_GROUPED | ntt.NTT_BATCH_GRAPH)
    b.execute()
    torch.cuda.synchronize()
    _check(oracle, reqs, hosts)
    # new buffers with the original inputs, same shapes: the replay uses them
    for r, s in zip(reqs, saved):
        r["in"] = s.clone()
        r["out"] = torch.empty_like(s)
    b.update(reqs)
    b.execute()
    torch.cuda.synchronize()
    _check(oracle, reqs, hosts)
    assert b.status() == 0


def test_grouped_tfhe_batch_is_one_launch(oracle):
    """The TFHE blind-rotation-shaped batch (3780 forward + 1260 inverse rows
    at N = 1024, 62-bit prime) as one grouped launch."""
    w = W.tfhe_blind_rotation()
    q = w["moduli"][0]
    xf, xi = to_dev(w["fwd"]), to_dev(w["inv"])
    reqs = [dict(log2n=10, n_moduli=1, n_polys=xf.shape[0], moduli_offset=0, inverse=0,
                 **{"in": xf, "out": torch.empty_like(xf)}),
            dict(log2n=10, n_moduli=1, n_polys=xi.shape[0], moduli_offset=0, inverse=1,
                 **{"in": xi, "out": torch.empty_like(xi)})]
    b = ntt.Batch(reqs, [q], flags=ntt.NTT_BATCH_GROUPED | ntt.NTT_BATCH_GRAPH)
    b.execute()
    torch.cuda.synchronize()
    assert b.info()["last_launches"] == 1 and b.status() == 0
    for r, x, inv in ((reqs[0], w["fwd"], False), (reqs[1], w["inv"], True)):
        rows = np.array([0, 1, x.shape[0] // 2, x.shape[0] - 1])
        got = to_host(r["out"])[rows]
        assert np.array_equal(got, oracle.transform_rows(x[rows], [q] * len(rows), inverse=inv))


def test_full_mixed_batch_grouped(oracle):
    """The 200-request mixed batch at full size through grouped launches (one
    grid per N and phase, the four N on concurrent branches); sampled rows and
    outputs of every request."""
    spec = W.mixed_requests(seed=W.DEFAULT_SEED)
    reqs = []
    for i, (log2n, limbs, polys) in enumerate(spec):
        x = W.request_rows_torch(W.DEFAULT_SEED, i, log2n, limbs, polys)
        reqs.append(dict(log2n=log2n, n_moduli=limbs, n_polys=polys, moduli_offset=0, inverse=0,
                         **{"in": x, "out": torch.empty_like(x)}))
    b = ntt.Batch(reqs, W.POOL50, flags=ntt.NTT_BATCH_GROUPED | ntt.NTT_BATCH_GRAPH)
    b.execute()
    b.execute()
    torch.cuda.synchronize()
    assert b.status() == 0
    rng = np.random.default_rng(201)
    for i, (log2n, limbs, polys) in enumerate(spec):
        n, rows = 1 << log2n, limbs * polys
        pick = sorted(set([0, rows - 1] + rng.integers(0, rows, 1).tolist()))
        x = np.stack([W.uniform_mod(W.DEFAULT_SEED, 1000 + i, n, W.POOL50[r % limbs], start=r * n) for r in pick])
        idx = np.stack([np.concatenate([[0, n - 1], rng.integers(0, n, 4)]) for _ in pick]).astype(np.uint32)
        ref = oracle.transform_rows(x, [W.POOL50[r % limbs] for r in pick], idx=idx)
        got = to_host(reqs[i]["out"][pick])
        assert np.array_equal(got[np.arange(len(pick))[:, None], idx], ref), (i, log2n, limbs, polys)
        reqs[i]["in"] = reqs[i]["out"] = None
