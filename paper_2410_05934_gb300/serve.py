"""Poisson request stream over the transform path: latency and throughput.

Requests follow the uneven mixed-batch distribution (N in {2^10, 2^12, 2^14,
2^16} with weights .5/.2/.2/.1, limbs U{1..32}, polys U{1..64}; forward
transforms) and arrive as a Poisson process.  Two serving policies:

  per_request  every arrival is launched at once on one stream with the
               schedule the cost model (or the autotuner DB) picks;
  microbatch   arrivals are gathered for a window and each window runs as
               ONE persistent mixed-batch launch (the allocation-free entry
               point, so nothing is allocated on the request path).

Latency = completion of the request's kernel (CUDA event on the stream) minus
its arrival time, both on the host clock of the driver (the GPU clock is
aligned with a reference event recorded when the stream is idle).
"""
import ctypes
import math
import time

import numpy as np

from . import ntt as _ntt
from . import workloads as W
from ._native import NttPlanRequest, check, load


class RequestPool:
    """Device-resident inputs/outputs and plans for the request types."""

    def __init__(self, seed=W.DEFAULT_SEED, n_types=200):
        import torch
        from .costmodel import choose_schedule
        self.spec = W.mixed_requests(seed=seed, n_requests=n_types)
        self.x, self.y, self.plans, self.sched = [], [], {}, []
        maxpolys = {}
        for log2n, limbs, polys in self.spec:
            maxpolys[(log2n, limbs)] = max(maxpolys.get((log2n, limbs), 0), polys)
        for key, polys in maxpolys.items():
            self.plans[key] = _ntt.Plan(key[0], W.POOL50[:key[1]], polys)
        for i, (log2n, limbs, polys) in enumerate(self.spec):
            x = W.request_rows_torch(seed, i, log2n, limbs, polys)
            self.x.append(x)
            self.y.append(torch.empty_like(x))
            self.sched.append(choose_schedule(log2n, limbs, polys)[0])
        self.coef = [x.numel() for x in self.x]
        torch.cuda.synchronize()


def poisson_arrivals(rate, n, seed):
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, n))


def _wait_until(t0, t):
    while time.perf_counter() - t0 < t:
        pass


def serve(pool, rate=5000.0, n_requests=4000, policy="per_request", window_us=500.0, seed=1):
    """Runs one stream; returns latencies (s), throughput and counts."""
    import torch
    L = load()
    st = torch.cuda.current_stream()
    sp = ctypes.c_void_p(st.cuda_stream)
    arrivals = poisson_arrivals(rate, n_requests, seed)
    rng = np.random.default_rng(seed + 1)
    kinds = rng.integers(0, len(pool.spec), n_requests)
    ev = []          # (event, [request indices])
    torch.cuda.synchronize()
    ref = torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    ref.record(st)
    if policy == "per_request":
        for i in range(n_requests):
            _wait_until(t0, arrivals[i])
            k = int(kinds[i])
            log2n, limbs, polys = pool.spec[k]
            plan = pool.plans[(log2n, limbs)]
            plan.schedule = pool.sched[k]
            plan.forward_rows(pool.x[k], pool.y[k], 0, polys * limbs, stream=st)
            e = torch.cuda.Event(enable_timing=True)
            e.record(st)
            ev.append((e, [i]))
    elif policy == "microbatch":
        w = window_us * 1e-6
        i = 0
        t_win = w
        while i < n_requests:
            t_win = max(t_win, arrivals[i])
            t_win = math.ceil(t_win / w) * w
            _wait_until(t0, t_win)
            window = []
            while i < n_requests and arrivals[i] <= t_win and len(window) < 816:
                window.append(i)
                i += 1
            # one launch per window; a request type that repeats inside the
            # window starts a new launch so no two work items share an output
            groups, seen = [[]], set()
            for idx in window:
                k = int(kinds[idx])
                if k in seen:
                    groups.append([])
                    seen = set()
                groups[-1].append(idx)
                seen.add(k)
            for batch in groups:
                reqs = (NttPlanRequest * len(batch))()
                for j, idx in enumerate(batch):
                    k = int(kinds[idx])
                    log2n, limbs, polys = pool.spec[k]
                    reqs[j].plan = pool.plans[(log2n, limbs)].handle.value
                    reqs[j].n_polys = polys
                    reqs[j].inverse = 0
                    reqs[j].in_ = pool.x[k].data_ptr()
                    reqs[j].out = pool.y[k].data_ptr()
                check(L.ntt_batch_execute_static(reqs, len(batch), sp), "ntt_batch_execute_static")
                e = torch.cuda.Event(enable_timing=True)
                e.record(st)
                ev.append((e, batch))
            t_win += w
    else:
        raise ValueError(policy)
    torch.cuda.synchronize()
    t_end = time.perf_counter() - t0
    lat = np.zeros(n_requests)
    done_last = 0.0
    for e, idxs in ev:
        done = ref.elapsed_time(e) * 1e-3
        done_last = max(done_last, done)
        for idx in idxs:
            lat[idx] = done - arrivals[idx]
    coef = sum(pool.coef[int(k)] for k in kinds)
    return {
        "policy": policy, "rate": rate, "requests": n_requests, "launch_groups": len(ev),
        "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
        "mean_ms": float(lat.mean() * 1e3), "max_ms": float(lat.max() * 1e3),
        "throughput_coef_s": coef / done_last, "offered_coef_s": coef / arrivals[-1],
        "span_s": done_last, "host_s": t_end,
        "window_us": window_us if policy == "microbatch" else None,
    }
