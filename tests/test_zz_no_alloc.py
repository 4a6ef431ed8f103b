"""The allocation-free entry point ntt_batch_execute_static, called through
the C ABI, gives the same results as the regular entry points.

That entry point exists for callers that cannot call cudaMalloc (they own
all device memory through their own allocator, or cannot afford the device
synchronisation of an allocation on their request path): its kernel keeps
its scratch (queue counter and request descriptors) in a file-scope device
array instead of allocated memory, so only the plans (created earlier) hold
device allocations.  This file is collected last so that, when it fails, a
run that stops at the first failure has already run every other test; it
also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

from paper_2410_05934_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2410_05934_gb300 import _native  # noqa: E402
import paper_2410_05934_gb300 as ntt  # noqa: E402

SHAPES = [(10, 2, 6), (12, 3, 2), (14, 1, 3), (16, 2, 2)]   # (log2n, limbs, polys)


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x).view(np.int64)).cuda()


def _requests(plans, ins, outs, inverse):
    arr = (_native.NttPlanRequest * len(plans))()
    for i, (p, x, o) in enumerate(zip(plans, ins, outs)):
        arr[i].plan = p.handle.value
        arr[i].n_polys = 0
        arr[i].inverse = inverse[i]
        arr[i].in_ = x.data_ptr()
        arr[i].out = o.data_ptr()
    return arr


def test_static_entry_point_matches_regular_entry_points():
    L = _native.load()
    stream = torch.cuda.current_stream()
    plans, ins = [], []
    for k, (log2n, limbs, polys) in enumerate(SHAPES):
        plans.append(ntt.Plan(log2n, W.POOL50[:limbs], polys))
        ins.append(_dev(W.request_rows(41, k, log2n, limbs, polys)))
    for call, inverse in enumerate(([0, 1, 0, 1], [1, 0, 1, 0])):   # two calls in a row
        outs = [torch.empty_like(x) for x in ins]
        reqs = _requests(plans, ins, outs, inverse)
        rc = L.ntt_batch_execute_static(reqs, len(plans), ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0, L.ntt_strerror(rc)
        for p, x, o, inv in zip(plans, ins, outs, inverse):
            ref = torch.empty_like(x)
            (p.inverse if inv else p.forward)(x, ref)
            torch.cuda.synchronize()
            assert torch.equal(o, ref), "call %d, N=2^%d" % (call, p.log2n)
            assert p.status() == 0


def test_static_entry_point_rejects_too_many_requests():
    L = _native.load()
    p = ntt.Plan(10, W.POOL50[:1], 1)
    x = torch.zeros((1, 1024), dtype=torch.int64, device="cuda")
    n = 817                                          # NTT_STATIC_MAX_REQUESTS + 1
    reqs = _requests([p] * n, [x] * n, [x] * n, [0] * n)
    assert L.ntt_batch_execute_static(reqs, n, None) == -1
    assert L.ntt_batch_execute_static(reqs, 0, None) == -1


def test_static_entry_point_allocates_no_device_memory():
    """The property the entry point exists for: once its per-device set-up has
    run (the first call), further calls leave the device's free memory and
    torch's allocated bytes exactly as they were."""
    L = _native.load()
    stream = torch.cuda.current_stream()
    plans, ins = [], []
    for k, (log2n, limbs, polys) in enumerate(SHAPES):
        plans.append(ntt.Plan(log2n, W.POOL50[:limbs], polys))
        ins.append(_dev(W.request_rows(43, k, log2n, limbs, polys)))
    outs = [torch.empty_like(x) for x in ins]
    reqs = _requests(plans, ins, outs, [0, 1, 1, 0])
    h = ctypes.c_void_p(stream.cuda_stream)
    assert L.ntt_batch_execute_static(reqs, len(plans), h) == 0     # set-up, kernel module loaded
    torch.cuda.synchronize()
    free0, alloc0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
    for _ in range(5):
        assert L.ntt_batch_execute_static(reqs, len(plans), h) == 0
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_allocated() == alloc0
    for p in plans:
        assert p.status() == 0
