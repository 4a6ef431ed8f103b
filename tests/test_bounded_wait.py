"""The bounded-wait test aid on the host emulation (nttemu_debug_bounded_wait,
the model of the kernel behind ntt_debug_bounded_wait): a wait that nothing
completes gives up, records NTT_ERR_TIMEOUT in the plan's status word, and
leaves the plan usable; a delivered copy completes the wait with the bytes
it carried; limits out of range are rejected."""
import numpy as np

from paper_2410_05934_gb300 import workloads as W

import emu

NTT_ERR_ARG, NTT_ERR_TIMEOUT = -1, -7
SPIN_MAX = 1 << 22


def test_delivered_copy_completes_the_wait():
    q = W.Q59_N1024
    p = emu.EmuPlan(10, [q], 1)
    rc, out = p.debug_bounded_wait(True, 16)
    assert rc == 0 and p.status() == 0
    # entry 0 of the forward table is psi^0 = 1 in Shoup form {1, floor(2^64 / q)}
    assert out.tolist() == [1, (1 << 64) // q]


def test_wait_that_nothing_completes_times_out_and_the_plan_stays_usable(oracle):
    q = W.Q59_N1024
    p = emu.EmuPlan(10, [q], 2)
    rc, out = p.debug_bounded_wait(False, 64)
    assert rc == 0
    assert out.tolist() == [0, 0]                  # nothing was copied out
    assert p.status() == NTT_ERR_TIMEOUT
    assert p.status() == 0                         # read and cleared
    x = W.rows_uniform(3, 1, [q, q], 1 << 10)
    got = p.transform(x, 0)
    assert np.array_equal(got, oracle.transform_rows(x, [q, q]))
    assert p.status() == 0


def test_first_status_is_kept():
    p = emu.EmuPlan(10, [W.Q59_N1024], 1)
    for _ in range(3):
        assert p.debug_bounded_wait(False, 1)[0] == 0
    assert p.status() == NTT_ERR_TIMEOUT and p.status() == 0


def test_spin_limit_range():
    p = emu.EmuPlan(10, [W.Q59_N1024], 1)
    assert p.debug_bounded_wait(False, 0)[0] == NTT_ERR_ARG
    assert p.debug_bounded_wait(False, SPIN_MAX + 1)[0] == NTT_ERR_ARG
    assert p.debug_bounded_wait(True, SPIN_MAX)[0] == 0
    assert p.status() == 0
