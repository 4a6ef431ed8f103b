"""The batched TFHE CMux step and external product (C ABI tfhe_*) against
the schoolbook oracle: sampled outputs of many ciphertexts, full rows of a
few, both moduli classes and both ring sizes, other gadgets, in-place use,
a chain of blind-rotation steps, the zero key (exact identity), empty
batches, argument errors and the range check."""
import numpy as np
import pytest

from paper_2410_05934_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2410_05934_gb300 as ntt  # noqa: E402
from gpu_util import to_dev, to_host  # noqa: E402
from oracle import tfhe_oracle as TO  # noqa: E402


def _rot_dev(rot):
    return torch.from_numpy(np.ascontiguousarray(rot).astype(np.int32)).cuda()


@pytest.mark.parametrize("log2n,q", [(10, W.Q62_N1024), (10, W.POOL50[0]), (11, W.POOL50[5])])
def test_cmux_and_external_product_match_oracle(log2n, q):
    n, levels, log2_base = 1 << log2n, 3, 8
    w = W.tfhe_cmux(seed=11 + log2n, n_ct=48, log2n=log2n, q=q, levels=levels)
    acc, rot, key = w["acc"], w["rot"][0], w["key"][0]
    plan = ntt.Plan(log2n, [q])
    d_acc, d_key = to_dev(acc), plan.tfhe_key_prepare(to_dev(key), levels)
    out_ep = torch.empty_like(d_acc)
    out_cm = torch.empty_like(d_acc)
    plan.tfhe_external_product(d_acc, d_key, levels, log2_base, out=out_ep)
    plan.tfhe_cmux_rotate(d_acc, _rot_dev(rot), d_key, levels, log2_base, out=out_cm)
    assert plan.status() == 0 and plan.last_launches() == 1
    ep, cm = to_host(out_ep), to_host(out_cm)
    kc = TO.key_coefficients(key, q)
    rng = np.random.default_rng(log2n)
    for c in list(range(0, 48, 7)) + [47]:
        idx = sorted(set([0, n - 1] + rng.integers(0, n, 6).tolist()))
        assert np.array_equal(ep[c][:, idx], TO.external_product(acc[c], key, q, log2_base, levels, key_coef=kc,
                                                                 idx=idx)), c
        assert np.array_equal(cm[c][:, idx], TO.cmux_rotate(acc[c], int(rot[c]), key, q, log2_base, levels,
                                                            key_coef=kc, idx=idx)), c
    # full rows of one ciphertext
    assert np.array_equal(cm[3], TO.cmux_rotate(acc[3], int(rot[3]), key, q, log2_base, levels, key_coef=kc))


def test_gadgets_in_place_and_blind_rotation_chain():
    q, log2n, n = W.Q62_N1024, 10, 1024
    w = W.tfhe_cmux(seed=3, n_ct=5, log2n=log2n, q=q, levels=4, steps=3)
    plan = ntt.Plan(log2n, [q])
    for levels, log2_base in [(1, 16), (2, 10), (4, 6)]:
        key = w["key"][0][:2 * levels]
        x = to_dev(w["acc"])
        plan.tfhe_cmux_rotate(x, _rot_dev(w["rot"][0]), plan.tfhe_key_prepare(to_dev(key), levels), levels,
                              log2_base)                                                   # in place
        got = to_host(x)
        kc = TO.key_coefficients(key, q)
        for c in (0, 4):
            assert np.array_equal(got[c], TO.cmux_rotate(w["acc"][c], int(w["rot"][0][c]), key, q, log2_base,
                                                         levels, key_coef=kc)), (levels, c)
    # three blind-rotation steps, each with its own key and exponents
    levels, log2_base = 4, 6
    x = to_dev(w["acc"])
    ref = w["acc"][1].copy()
    for step in range(3):
        key = w["key"][step]
        plan.tfhe_cmux_rotate(x, _rot_dev(w["rot"][step]), plan.tfhe_key_prepare(to_dev(key), levels), levels,
                              log2_base)
        ref = TO.cmux_rotate(ref, int(w["rot"][step][1]), key, q, log2_base, levels)
    assert np.array_equal(to_host(x)[1], ref)
    assert plan.status() == 0


def test_zero_key_is_identity_and_empty_batch():
    q, log2n = W.POOL50[2], 11
    w = W.tfhe_cmux(seed=4, n_ct=300, log2n=log2n, q=q)
    plan = ntt.Plan(log2n, [q])
    x = to_dev(w["acc"])
    out = torch.empty_like(x)
    zero = plan.tfhe_key_prepare(torch.zeros((6, 2, 1 << log2n), dtype=torch.int64, device="cuda"), 3)
    plan.tfhe_cmux_rotate(x, _rot_dev(w["rot"][0]), zero, 3, 8, out=out)
    assert torch.equal(out, x)
    plan.tfhe_external_product(x[:0], zero, 3, 8, out=out[:0])
    assert plan.last_launches() == 0


def test_tfhe_argument_errors_and_range_check():
    q = W.Q62_N1024
    plan = ntt.Plan(10, [q])
    x = torch.zeros((2, 2, 1024), dtype=torch.int64, device="cuda")
    key = torch.zeros((18, 2, 1024, 2), dtype=torch.int64, device="cuda")
    for levels, base in [(0, 8), (9, 3), (3, 11), (1, 33)]:
        with pytest.raises(ntt.NttError) as e:
            plan.tfhe_external_product(x, key, levels, base)
        assert e.value.code == -1
    with pytest.raises(ntt.NttError) as e:
        ntt.Plan(12, [W.POOL50[0]]).tfhe_external_product(
            torch.zeros((1, 2, 4096), dtype=torch.int64, device="cuda"),
            torch.zeros((6, 2, 4096, 2), dtype=torch.int64, device="cuda"), 3, 8)
    assert e.value.code == -10
    with pytest.raises(ntt.NttError) as e:
        ntt.Plan(10, [q, W.Q59_N1024]).tfhe_external_product(x, key, 3, 8)
    assert e.value.code == -1
    chk = ntt.Plan(10, [q], flags=ntt.NTT_FLAG_CHECK)
    bad = x.clone()
    bad[1, 0, 5] = q
    chk.tfhe_external_product(bad, key, 3, 8, out=torch.empty_like(bad))
    assert chk.status() == -8
    badkey = torch.zeros((6, 2, 1024), dtype=torch.int64, device="cuda")
    badkey[3, 1, 7] = q
    chk.tfhe_key_prepare(badkey, 3)
    assert chk.status() == -8


def test_full_size_cmux_step_as_benchmarked():
    """One CMux step over the bench's 1024 accumulators (N = 1024, 62-bit q,
    B = 2^8, l = 3), in place, sampled ciphertexts against the oracle."""
    q, log2n, levels, log2_base = W.Q62_N1024, 10, 3, 8
    w = W.tfhe_cmux(n_ct=1024, steps=1, levels=levels)
    plan = ntt.Plan(log2n, [q])
    acc = to_dev(w["acc"])
    plan.tfhe_cmux_rotate(acc, _rot_dev(w["rot"][0]), plan.tfhe_key_prepare(to_dev(w["key"][0]), levels), levels,
                          log2_base)
    got = to_host(acc)
    kc = TO.key_coefficients(w["key"][0], q)
    rng = np.random.default_rng(5)
    for c in [0, 511, 1023] + rng.integers(0, 1024, 3).tolist():
        idx = sorted(set([0, 1023] + rng.integers(0, 1024, 6).tolist()))
        assert np.array_equal(got[c][:, idx], TO.cmux_rotate(w["acc"][c], int(w["rot"][0][c]), w["key"][0], q,
                                                             log2_base, levels, key_coef=kc, idx=idx)), c


def test_back_to_back_cmux_steps_match_the_oracle_chain():
    """Consecutive in-place CMux launches with nothing between them on the
    stream, as in a blind rotation: every key and rotation tensor is prepared
    first, then six steps are issued with no host synchronisation, so each
    launch may be scheduled while the previous one finishes (programmatic
    dependent launch) and must still read only its finished output.  600
    ciphertexts give more than one wave of CTAs per launch."""
    q, log2n, levels, log2_base, steps = W.Q62_N1024, 10, 3, 8, 6
    w = W.tfhe_cmux(seed=21, n_ct=600, log2n=log2n, q=q, levels=levels, steps=steps)
    plan = ntt.Plan(log2n, [q])
    keys = [plan.tfhe_key_prepare(to_dev(w["key"][s]), levels) for s in range(steps)]
    rots = [_rot_dev(w["rot"][s]) for s in range(steps)]
    x = to_dev(w["acc"])
    torch.cuda.synchronize()
    for s in range(steps):
        plan.tfhe_cmux_rotate(x, rots[s], keys[s], levels, log2_base)
    got = to_host(x)
    assert plan.status() == 0
    for c in (0, 599):
        ref = w["acc"][c].copy()
        for s in range(steps):
            ref = TO.cmux_rotate(ref, int(w["rot"][s][c]), w["key"][s], q, log2_base, levels)
        assert np.array_equal(got[c], ref), c
