"""Autotuner of the transform schedules (the switch-point / fused-stage choice
of Sec. V-D, decided here by measurement).

For a shape (log2 N, limbs, batch, modulus bits) every candidate schedule of
that N is timed with CUDA events on the launching stream (warm-up, then the
median of several repetitions; optional L2 flush between repetitions) for the
forward and the inverse transform.  Results go to a JSON-lines timing DB keyed
by (GPU name, library build, shape, direction, schedule) so that tuning
resumes where it stopped and the cost model can train on it.

    python -m paper_2410_05934_gb300.tune --shape 16,24,4 [--shape 10,1,5040]

The heuristic arm, the paper's SM-aware rule restated for these kernels, is
``costmodel.heuristic_choice``.
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import time

from . import ntt as _ntt
from . import workloads as W

DEFAULT_DB = os.environ.get("NTT_TUNE_DB", os.path.join(os.path.expanduser("~"), ".cache", "ntt_gb300",
                                                        "tune.jsonl"))


def moduli_for(log2n, limbs, bits=50):
    """`limbs` moduli of the requested size class: 50 -> the 50-bit pool (any
    N <= 2^16); 59 / 62 -> the 59- / 62-bit prime (N <= 1024), repeated."""
    if bits == 50:
        return W.POOL50[:limbs]
    if log2n > 10:
        raise ValueError("the 59/62-bit primes are NTT-friendly only up to N = 1024")
    return [W.Q59_N1024 if bits == 59 else W.Q62_N1024] * limbs


def build_stamp():
    from . import build as B
    try:
        return open(B.LIB + ".stamp").read().strip()[:16]
    except OSError:
        return "unknown"


def gpu_name():
    import torch
    return torch.cuda.get_device_name(torch.cuda.current_device())


class Timer:
    """Times plan.forward / plan.inverse per schedule on one buffer set."""

    def __init__(self, log2n, limbs, batch, bits=50, flush_l2=None, seed=1):
        import numpy as np
        import torch
        self.torch = torch
        self.log2n, self.limbs, self.batch = log2n, limbs, batch
        self.moduli = moduli_for(log2n, limbs, bits)
        self.plan = _ntt.Plan(log2n, self.moduli, batch)
        n = 1 << log2n
        rows = batch * limbs
        dev = torch.device("cuda", torch.cuda.current_device())
        # canonical inputs generated on the device (the smallest modulus bounds all rows)
        qmin = min(self.moduli)
        g = torch.Generator(device=dev)
        g.manual_seed(seed)
        self.x = torch.randint(0, qmin, (rows, n), dtype=torch.int64, device=dev, generator=g)
        self.y = torch.empty_like(self.x)
        nbytes = rows * n * 8
        self.flush_l2 = (nbytes < (256 << 20)) if flush_l2 is None else flush_l2
        self.flush = torch.empty(512 << 18, dtype=torch.int32, device=dev) if self.flush_l2 else None
        self.stream = torch.cuda.current_stream()
        del np

    def time(self, sched, inverse=False, reps=7, warmup=2):
        torch = self.torch
        self.plan.schedule = sched
        fn = self.plan.inverse if inverse else self.plan.forward
        for _ in range(warmup):
            fn(self.x, self.y)
        inner = _inner_count(torch, self.stream, lambda: fn(self.x, self.y))
        ms = []
        for r in range(reps):
            if self.flush is not None:
                self.flush.fill_(r)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(self.stream)
            for _ in range(inner):
                fn(self.x, self.y)
            b.record(self.stream)
            b.synchronize()
            ms.append(a.elapsed_time(b) / inner)
        return statistics.median(ms), min(ms), max(ms)

    def close(self):
        self.plan.close()
        del self.x, self.y, self.flush


_SIGS = {}


def schedule_signature(log2n):
    """Hash of N's candidate list (schedule names in id order).  A timing
    record holds for the list it was measured on: when the list of an N
    changes, its old records no longer say which schedule is which."""
    if log2n not in _SIGS:
        h = hashlib.sha256()
        for s in range(_ntt.schedule_count(log2n)):
            h.update(_ntt.schedule_name(log2n, s).encode() + b"\0")
        _SIGS[log2n] = h.hexdigest()[:12]
    return _SIGS[log2n]


def current_records(recs):
    """The records measured on the schedule lists this library has."""
    return [r for r in recs if r.get("sig") == schedule_signature(int(r["log2n"]))]


def load_db(path=DEFAULT_DB, current=False):
    """All records of a timing DB (JSON lines), or only the current ones."""
    recs = []
    if os.path.exists(path):
        with open(path) as f:
            for line in f:
                line = line.strip()
                if line:
                    try:
                        recs.append(json.loads(line))
                    except ValueError:
                        pass
    return current_records(recs) if current else recs


def _key(r):
    return (r["gpu"], r["build"], r.get("sig"), r["log2n"], r["limbs"], r["batch"], r["bits"], r["inverse"],
            r["sched"])


def tune_shape(log2n, limbs, batch, bits=50, db=DEFAULT_DB, reps=7, skip_done=True, directions=(False, True)):
    """Times every schedule of one shape; appends new records to the DB."""
    gpu, stamp = gpu_name(), build_stamp()
    done = {_key(r) for r in load_db(db)} if skip_done else set()
    timer = None
    out = []
    os.makedirs(os.path.dirname(db) or ".", exist_ok=True)
    try:
        for inverse in directions:
            for s in range(_ntt.schedule_count(log2n)):
                rec = dict(gpu=gpu, build=stamp, sig=schedule_signature(log2n), log2n=log2n, limbs=limbs,
                           batch=batch, bits=bits, inverse=bool(inverse), sched=s)
                if _key(rec) in done:
                    continue
                if timer is None:
                    timer = Timer(log2n, limbs, batch, bits)
                med, lo, hi = timer.time(s, inverse, reps=reps)
                rec.update(ms=med, ms_min=lo, ms_max=hi, t=time.time())
                out.append(rec)
                with open(db, "a") as f:
                    f.write(json.dumps(rec) + "\n")
    finally:
        if timer is not None:
            timer.close()
    return out


def best_from_db(log2n, limbs, batch, bits=50, inverse=False, db=DEFAULT_DB, recs=None):
    """Fastest recorded schedule for this exact shape, or None."""
    gpu, stamp = gpu_name(), build_stamp()
    recs = load_db(db) if recs is None else recs
    cands = [r for r in recs if r["gpu"] == gpu and r["build"] == stamp and r["log2n"] == log2n
             and r["limbs"] == limbs and r["batch"] == batch and r["bits"] == bits
             and r["inverse"] == bool(inverse)]
    if not cands:
        return None
    return min(cands, key=lambda r: r["ms"])["sched"]


def probe_peaks(iters=4000, reps=3):
    """Butterflies/s of the integer-pipe probe for each butterfly kind."""
    import torch
    from . import _native
    L = _native.load()
    dev = torch.device("cuda", torch.cuda.current_device())
    st = torch.cuda.current_stream()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sink = torch.empty(sms * 8 * 256, dtype=torch.int64, device=dev)
    out = {}
    for kind, q in [(0, W.POOL50[0]), (1, W.POOL50[0]), (2, W.POOL50[0]), (3, W.POOL50[0])]:
        best = 0.0
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            rc = L.ntt_bench_butterflies(q, kind, sms * 8, 256, iters, sink.data_ptr(), st.cuda_stream)
            if rc:
                raise RuntimeError("ntt_bench_butterflies: %d" % rc)
            b.record(st)
            b.synchronize()
            best = max(best, sms * 8 * 256 * iters * 8 / (a.elapsed_time(b) * 1e-3))
        out[kind] = best
    return out


def random_shapes(count, seed, max_log2_coef=27, sizes=(10, 11, 12, 13, 14, 15, 16)):
    """Shapes for the cost model's training sweep: N uniform over `sizes`,
    limbs log-uniform in 1..48, batch log-uniform in 1..4096, at most
    2^max_log2_coef coefficients (the batch is redrawn until it fits);
    N = 1024 shapes also use the 59- and 62-bit moduli."""
    import random
    rng = random.Random(seed)
    out = []
    while len(out) < count:
        log2n = rng.choice(sizes)
        limbs = max(1, min(48, int(round(math.exp(rng.uniform(0, math.log(48)))))))
        batch = max(1, min(4096, int(round(math.exp(rng.uniform(0, math.log(4096)))))))
        if (limbs * batch) << log2n > (1 << max_log2_coef):
            continue
        bits = 50 if log2n != 10 else rng.choice((50, 50, 59, 62))
        out.append((log2n, limbs, batch, bits))
    return out


MIN_SAMPLE_MS = 0.05


def _inner_count(torch, st, launch):
    """Back-to-back launches per timed sample so that a sample spans at least
    MIN_SAMPLE_MS: a single launch of a small shape lasts a few microseconds,
    close to the resolution of event timing."""
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(st)
    launch()
    b.record(st)
    b.synchronize()
    one = max(a.elapsed_time(b), 1e-3)
    return int(min(64, max(1, math.ceil(MIN_SAMPLE_MS / one))))


def sweep(shapes, db=DEFAULT_DB, reps=5, warmup=2, directions=(False,), skip_done=True, log=None):
    """Times every schedule of every shape with one plan per (N, limbs, bits)
    and shared buffers; appends to the DB.  Inputs are uniform below 2^49,
    canonical for every modulus of the pools."""
    import torch
    gpu, stamp = gpu_name(), build_stamp()
    done = {_key(r) for r in load_db(db)} if skip_done else set()
    max_coef = max((l * b) << n for n, l, b, _ in shapes)
    dev = torch.device("cuda", torch.cuda.current_device())
    g = torch.Generator(device=dev)
    g.manual_seed(1)
    x = torch.randint(0, 1 << 49, (max_coef,), dtype=torch.int64, device=dev, generator=g)
    y = torch.empty_like(x)
    flush = torch.empty(512 << 18, dtype=torch.int32, device=dev)
    st = torch.cuda.current_stream()
    plans = {}
    groups = {}
    for sh in shapes:
        groups.setdefault((sh[0], sh[1], sh[3]), []).append(sh)
    os.makedirs(os.path.dirname(db) or ".", exist_ok=True)
    n_rec = 0
    with open(db, "a") as f:
        for (log2n, limbs, bits), members in sorted(groups.items()):
            max_batch = max(m[2] for m in members)
            plan = _ntt.Plan(log2n, moduli_for(log2n, limbs, bits), max_batch)
            for _, _, batch, _ in members:
                rows = limbs * batch
                small = (rows << log2n) * 8 < (256 << 20)
                for inverse in directions:
                    fn = plan.inverse_rows if inverse else plan.forward_rows
                    for s in range(_ntt.schedule_count(log2n)):
                        rec = dict(gpu=gpu, build=stamp, sig=schedule_signature(log2n), log2n=log2n,
                                   limbs=limbs, batch=batch, bits=bits, inverse=bool(inverse), sched=s)
                        if _key(rec) in done:
                            continue
                        plan.schedule = s
                        for _ in range(warmup):
                            fn(x, y, 0, rows)
                        inner = _inner_count(torch, st, lambda: fn(x, y, 0, rows))
                        ms = []
                        for r in range(reps):
                            if small:
                                flush.fill_(r)
                            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                            a.record(st)
                            for _ in range(inner):
                                fn(x, y, 0, rows)
                            b.record(st)
                            b.synchronize()
                            ms.append(a.elapsed_time(b) / inner)
                        rec.update(ms=statistics.median(ms), ms_min=min(ms), ms_max=max(ms), inner=inner,
                                   t=time.time())
                        f.write(json.dumps(rec) + "\n")
                        done.add(_key(rec))
                        n_rec += 1
            plan.close()
            del plans
            plans = {}
            if log:
                log("group N=2^%d limbs=%d bits=%d done (%d records)" % (log2n, limbs, bits, n_rec))
    return n_rec


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--shape", action="append", default=[], help="log2n,limbs,batch[,bits]")
    ap.add_argument("--db", default=DEFAULT_DB)
    ap.add_argument("--reps", type=int, default=7)
    ap.add_argument("--redo", action="store_true")
    ap.add_argument("--sched", type=int, default=None, help="time only this schedule")
    ap.add_argument("--direction", choices=["fwd", "inv", "both"], default="both")
    ap.add_argument("--probe", action="store_true", help="print the butterfly probe rates")
    ap.add_argument("--sweep", type=int, default=0, help="time every schedule of this many random shapes")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--max-log2-coef", type=int, default=27)
    args = ap.parse_args()
    if args.sweep:
        shapes = random_shapes(args.sweep, args.seed, args.max_log2_coef)
        t0 = time.time()
        n = sweep(shapes, db=args.db, reps=args.reps, log=lambda m: print(m, flush=True))
        print("sweep: %d shapes, %d new records in %.1f s -> %s" % (len(shapes), n, time.time() - t0, args.db))
    if args.probe:
        names = {0: "CT exact", 1: "GS exact", 2: "CT small-modulus", 3: "GS small-modulus"}
        for k, v in probe_peaks().items():
            print("probe %-18s %.1f G butterflies/s" % (names[k], v / 1e9))
    dirs = {"fwd": (False,), "inv": (True,), "both": (False, True)}[args.direction]
    for sh in args.shape:
        v = [int(t) for t in sh.split(",")]
        log2n, limbs, batch = v[:3]
        bits = v[3] if len(v) > 3 else 50
        rows = limbs * batch
        if args.sched is not None:
            timer = Timer(log2n, limbs, batch, bits)
            for inv in dirs:
                med, lo, hi = timer.time(args.sched, inv, reps=args.reps)
                print("N=2^%d limbs=%d batch=%d %s sched %d: %.4f ms" % (
                    log2n, limbs, batch, "inv" if inv else "fwd", args.sched, med))
            timer.close()
            continue
        recs = tune_shape(log2n, limbs, batch, bits, db=args.db, reps=args.reps, skip_done=not args.redo,
                          directions=dirs)
        for r in recs:
            coef = rows * (1 << log2n)
            print("N=2^%d limbs=%d batch=%d %s sched %d: %.4f ms  (%.1f Gcoef/s)  %s" % (
                log2n, limbs, batch, "inv" if r["inverse"] else "fwd", r["sched"], r["ms"],
                coef / r["ms"] / 1e6, _ntt.schedule_name(log2n, r["sched"])))


if __name__ == "__main__":
    main()
