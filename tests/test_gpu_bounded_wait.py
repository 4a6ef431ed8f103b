"""The bounded device-side wait runs out without any fault (C ABI
ntt_debug_bounded_wait): one CTA waits on an mbarrier that no copy
completes, gives up after the given number of rounds, records
NTT_ERR_TIMEOUT in the plan's status word and returns; the context stays
usable and later transforms still match the oracle.  A delivered 16-byte
bulk copy completes the same wait with the bytes it carried."""
import numpy as np
import pytest

from paper_2410_05934_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2410_05934_gb300 as ntt  # noqa: E402
from paper_2410_05934_gb300._native import NttError  # noqa: E402
from gpu_util import to_dev, to_host  # noqa: E402

NTT_ERR_ARG, NTT_ERR_TIMEOUT = -1, -7


def test_delivered_copy_completes_the_wait():
    q = W.Q59_N1024
    plan = ntt.Plan(10, [q], 1)
    out = torch.zeros(2, dtype=torch.int64, device="cuda")
    plan.debug_bounded_wait(True, 1 << 20, out)
    assert plan.status() == 0
    # entry 0 of the forward table: psi^0 = 1 with its Shoup form floor(2^64 / q)
    assert to_host(out).tolist() == [1, (1 << 64) // q]


def test_wait_runs_out_records_timeout_and_later_calls_match_the_oracle(oracle):
    q = W.Q59_N1024
    plan = ntt.Plan(10, [q], 4)
    out = torch.zeros(2, dtype=torch.int64, device="cuda")
    for limit in (1, 64):
        plan.debug_bounded_wait(False, limit, out)
        assert plan.status() == NTT_ERR_TIMEOUT
        assert plan.status() == 0                  # read and cleared
    assert to_host(out).tolist() == [0, 0]         # the timed-out kernel wrote nothing
    x = W.rows_uniform(5, 1, [q] * 4, 1 << 10)
    d = to_dev(x)
    y = torch.empty_like(d)
    plan.forward(d, y)
    assert np.array_equal(to_host(y), oracle.transform_rows(x, [q] * 4))
    back = torch.empty_like(d)
    plan.inverse(y, back)
    assert torch.equal(back, d)
    assert plan.status() == 0
    # and a delivered copy still completes the wait afterwards
    plan.debug_bounded_wait(True, 1 << 20, out)
    assert plan.status() == 0 and to_host(out).tolist() == [1, (1 << 64) // q]


def test_arguments_are_checked():
    plan = ntt.Plan(10, [W.Q59_N1024], 1)
    for limit in (0, (1 << 22) + 1):
        with pytest.raises(NttError) as e:
            plan.debug_bounded_wait(False, limit)
        assert e.value.code == NTT_ERR_ARG
    assert plan.status() == 0
