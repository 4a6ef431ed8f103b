"""Host side of the C ABI, on the CPU: the library loads, exports every
symbol the header declares, validates plans and derives the same psi as the
oracle (independent code)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2410_05934_gb300 import build as B
from paper_2410_05934_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def ntt():
    B.build_product()
    import paper_2410_05934_gb300 as P
    return P


def header_functions():
    names = []
    inc = os.path.join(ROOT, "include")
    for h in os.listdir(inc):
        if h.endswith(".h"):
            src = open(os.path.join(inc, h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b(\w+)\s*\([^;]*\)\s*;", src, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_header_symbol(ntt):
    from paper_2410_05934_gb300 import _native
    L = _native.load()
    names = header_functions()
    assert len(names) >= 17
    for name in names:
        assert hasattr(L, name), name
    declared = {s[0] for s in _native.SIGNATURES}
    assert set(names) == declared


def test_version_and_strerror(ntt):
    from paper_2410_05934_gb300 import _native
    L = _native.load()
    assert b"sm_103a" in L.ntt_version()
    for code in range(-10, 1):
        assert L.ntt_strerror(code) not in (None, b"unknown error")


@pytest.mark.parametrize("args,code", [
    ((0, [W.Q59_N1024], 1, 1), -1),
    ((17, [W.POOL50[0]], 1, 1), -1),
    ((10, [], 1, 1), -1),
    ((10, [W.Q59_N1024], 0, 1), -1),
    ((10, [W.Q59_N1024], 1, 1 | 64), -1),
    ((10, [W.Q59_N1024 + 2048], 1, 1), -2),      # composite, still 1 mod 2048
    ((10, [1], 1, 1), -2),
    ((10, [7681], 1, 1), -3),
    ((16, [W.Q59_N1024], 1, 1), -3),
    ((10, [(1 << 62) + 1], 1, 1), -4),
    ((16, [W.POOL50[0]], 1 << 24, 1), -1),        # 2^40 coefficients
])
def test_plan_validation(ntt, args, code):
    with pytest.raises(ntt.NttError) as e:
        ntt.Plan(*args[:3], flags=args[3])
    assert e.value.code == code


def test_psi_matches_oracle(ntt, oracle):
    cases = [(log2n, q) for log2n in (1, 5, 10) for q in (W.Q59_N1024, W.Q62_N1024, 12289)]
    cases += [(log2n, q) for log2n in (11, 13, 16) for q in W.POOL50[:8]]
    for log2n, q in cases:
        p = ntt.Plan(log2n, [q], 1, flags=ntt.NTT_FLAG_HOST_ONLY)
        assert p.root(0) == oracle.psi(q, log2n)


def test_schedules_enumerate(ntt):
    for log2n in range(1, 17):
        c = ntt.schedule_count(log2n)
        assert c >= 1
        names = {ntt.schedule_name(log2n, i) for i in range(c)}
        assert len(names) == c
    p = ntt.Plan(16, W.POOL50[:2], 1, flags=ntt.NTT_FLAG_HOST_ONLY)
    p.schedule = 1
    assert p.schedule == 1
    with pytest.raises(ntt.NttError):
        p.schedule = 99


def test_compute_on_host_only_plan_is_rejected(ntt):
    from paper_2410_05934_gb300 import _native
    L = _native.load()
    p = ntt.Plan(10, [W.Q59_N1024], 1, flags=ntt.NTT_FLAG_HOST_ONLY)
    buf = ctypes.create_string_buffer(8 * 1024 + 16)
    addr = (ctypes.addressof(buf) + 15) & ~15
    assert L.ntt_forward(p.handle, addr, addr, None) == -1
    assert L.ntt_forward(p.handle, addr + 8, addr, None) == -5   # alignment checked first
    assert L.poly_mul_pointwise(p.handle, addr, addr, addr, 0, None) == -1
    assert L.ntt_forward(p.handle, None, addr, None) == -1


def test_forward_inverse_argument_rules_on_the_host(ntt):
    """ntt_forward_inverse rejects null plans and pointers, plans of different
    N or word size, and overlapping buffers of the two transforms before any
    device work (host-only plans reach no launch either)."""
    from paper_2410_05934_gb300 import _native
    L = _native.load()
    f = ntt.Plan(10, [W.Q59_N1024], 2, flags=ntt.NTT_FLAG_HOST_ONLY)
    i = ntt.Plan(10, [W.Q59_N1024], 1, flags=ntt.NTT_FLAG_HOST_ONLY)
    i11 = ntt.Plan(11, [4611686018427322369], 1, flags=ntt.NTT_FLAG_HOST_ONLY)   # a 62-bit prime = 1 mod 2^12
    buf = ctypes.create_string_buffer(8 * 4096 + 16)
    a = (ctypes.addressof(buf) + 15) & ~15
    b = a + 8 * 2048                              # after the forward's 2 rows
    assert L.ntt_forward_inverse(None, a, a, i.handle, b, b, None) == -1
    assert L.ntt_forward_inverse(f.handle, None, a, i.handle, b, b, None) == -1
    assert L.ntt_forward_inverse(f.handle, a, a, i11.handle, b, b, None) == -1      # different N
    assert L.ntt_forward_inverse(f.handle, a, a, i.handle, a + 8 * 1024, b, None) == -1   # overlap
    assert L.ntt_forward_inverse(f.handle, a, a, i.handle, b, b, None) == -1        # host-only plans


def test_twiddle_tables_and_shoup_companions(ntt, oracle):
    """Host tables of a plan (emulation library exposes none, so check through
    the emulator's transforms and directly through the oracle's root): every
    forward entry is psi^brv(k) and every companion floor(w 2^64 / q)."""
    import emu
    for log2n, q in [(10, W.Q62_N1024), (16, W.POOL50[5]), (4, 257)]:
        n = 1 << log2n
        plan = emu.EmuPlan(log2n, [q, q], 1)        # repeated modulus shares its tables
        x = W.rows_uniform(3, 3, [q, q], n)
        out = plan.transform(x, 0)
        for r in range(2):
            idx = np.array([0, 1, n - 1], dtype=np.uint32)
            assert np.array_equal(out[r][idx], oracle.ntt_forward(x[r], q, idx=idx))
