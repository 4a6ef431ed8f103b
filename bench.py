#!/usr/bin/env python3
"""Benchmark of the batched negacyclic NTT path on GB300.

Workload (one "step"): the CKKS-HMUL-shaped batch -- N = 65536, 24 RNS
limbs (the 24 largest 50-bit primes = 1 mod 2^17), 2 ciphertexts x 2
components = 96 rows -- forward NTT of all 96 rows, the 4 cross products
a_i (.) b_j per limb (96 product rows), inverse NTT of the 96 products
(Sec. II-D, Eq. 1).  Metric: coefficients pushed through the transforms per
second, counting both the forward and the inverse pass
(2 x 96 x 65536 = 12.58 M coefficient-transforms per step).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank runs its own independent batch (weak
scaling, no data-path collective); time is the max over ranks.
`--impl reference` times the CPU oracle (O(N^2) definitions) on a bounded
sample of the same workload on the host cores.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOAD = "ckks_hmul_n65536"
LOG2N, LIMBS, POLYS = 16, 24, 4
METRIC = "NTT coeffs/s (forward+inverse coefficient-transforms per second)"
UNIT = "coeffs/s"
L2_FLUSH_BYTES = 512 << 20     # > 2x the 129 MB L2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="default workload: skip the per-N sweep, mixed batch, TFHE batch and cost-model keys")
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="target CPU time of the oracle baseline sample")
    ap.add_argument("--schedule", type=int, default=None)
    ap.add_argument("--hybrid-min-log2-coef", type=int, default=22,
                    help="mixed batches: requests of at least 2^k coefficients run their own learned schedule")
    ap.add_argument("--workload", default=WORKLOAD,
                    choices=[WORKLOAD, "mixed_batch", "tfhe_blind_rotation", "plain_n1024", "cost_model",
                             "serving", "hmul_fused", "mixed_small", "tfhe_cmux", "ckks_bconv", "otf_twiddles", "n_sweep",
                             "ckks_rescale", "natural_order", "word32", "probe_pipes"],
                    help="the line the driver records is the default (CKKS-HMUL-shaped) workload")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ---------------------------------------------------------------- clocks --

class ClockSampler:
    """Samples nvidia-smi every 200 ms while the timed region runs."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (FileNotFoundError, OSError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------- CPU baseline --

def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the machine type)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.machine()


def oracle_sample(seconds_target, nthreads=None):
    """Times the C oracle (O(N^2) definitions) on a bounded sample of the
    workload: forward outputs and inverse outputs of rows of the same batch.
    Returns (coefficient-transforms/s, threads, description)."""
    from oracle import oracle as O
    from paper_2410_05934_gb300 import workloads as W
    n = 1 << LOG2N
    nthreads = nthreads or (os.cpu_count() or 1)
    w = W.ckks_hmul_n65536()
    x = w["x"].reshape(-1, n)
    mods = w["moduli"]
    # calibration: 1 row, 2*nthreads outputs each way
    def run(k):
        idx = np.arange(k, dtype=np.uint32)[None, :] * 7 % n
        t0 = time.perf_counter()
        O.transform_rows(x[:1], [mods[0]], idx=idx.astype(np.uint32), nthreads=1)
        return time.perf_counter() - t0
    t1 = run(4) / 4                      # seconds per output, one thread
    per_dir = max(2 * nthreads, int(seconds_target * nthreads / t1 / 2))
    rows = 2
    per_row = max(1, per_dir // rows)
    idx = np.stack([(np.arange(per_row, dtype=np.uint64) * 2654435761 + r) % n
                    for r in range(rows)]).astype(np.uint32)
    # split each row's outputs over threads: one "row" per chunk of outputs
    chunks = max(1, nthreads)
    sub = np.array_split(np.arange(per_row), chunks)
    xs, qs, ids = [], [], []
    for r in range(rows):
        for s in sub:
            if len(s) == 0:
                continue
            xs.append(x[r])
            qs.append(mods[r % LIMBS])
            ids.append(idx[r][s])
    m = min(len(i) for i in ids)
    ids = np.stack([i[:m] for i in ids])
    xs = np.stack(xs)
    t0 = time.perf_counter()
    O.transform_rows(xs, qs, idx=ids, nthreads=nthreads)
    O.transform_rows(xs, qs, idx=ids, inverse=True, nthreads=nthreads)
    dt = time.perf_counter() - t0
    count = 2 * ids.size
    desc = ("O(N^2) oracle (forward + inverse definitions, 128-bit products) at N=65536: "
            "%d output coefficients (%d forward + %d inverse, %d rows of the batch), %d threads"
            % (count, ids.size, ids.size, rows, nthreads))
    return count / dt, nthreads, desc, dt


def radix2_sample():
    """The second CPU baseline: the whole step's transforms (96 forward + 96
    inverse rows at N = 2^16) through the plain radix-2 O(N log N) transforms
    with Shoup twiddles, rows spread over all host cores."""
    from oracle import oracle as O
    from paper_2410_05934_gb300 import workloads as W
    n = 1 << LOG2N
    nthreads = os.cpu_count() or 1
    w = W.ckks_hmul_n65536()
    x = w["x"].reshape(-1, n)
    O.radix2_rows(x[:nthreads], w["moduli"], nthreads=nthreads)      # tables and pages warm
    t0 = time.perf_counter()
    f = O.radix2_rows(x, w["moduli"], nthreads=nthreads)
    O.radix2_rows(f, w["moduli"], inverse=True, nthreads=nthreads)
    dt = time.perf_counter() - t0
    return 2 * x.size / dt, nthreads, dt


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    from oracle import oracle as O
    from paper_2410_05934_gb300 import workloads as W
    n = 1 << LOG2N
    nthreads = os.cpu_count() or 1
    w = W.ckks_hmul_n65536()
    x = w["x"].reshape(-1, n)
    mods = w["moduli"]
    k = 32 * nthreads                    # outputs per direction per step
    per_thread = max(1, k // nthreads)

    def step(i):
        rows = [(i * nthreads + t) % (4 * LIMBS) for t in range(nthreads)]
        idx = np.stack([(np.arange(per_thread, dtype=np.uint64) * 40503 + 977 * i + t) % n
                        for t in range(nthreads)]).astype(np.uint32)
        xs = x[rows]
        qs = [mods[r % LIMBS] for r in rows]
        O.transform_rows(xs, qs, idx=idx, nthreads=nthreads)
        O.transform_rows(xs, qs, idx=idx, inverse=True, nthreads=nthreads)
        return 2 * idx.size

    for i in range(args.warmup):
        step(i)
    t0 = time.perf_counter()
    count = 0
    for i in range(args.steps):
        count += step(args.warmup + i)
    dt = time.perf_counter() - t0
    value = count / dt
    sample = ("per step: %d forward + %d inverse output coefficients of the O(N^2) definitions "
              "at N=65536 over %d rows of the CKKS-HMUL-shaped batch" % (count // args.steps // 2,
                                                                          count // args.steps // 2,
                                                                          nthreads))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "log2n": LOG2N, "limbs": LIMBS, "polys": POLYS},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": nthreads, "kind": "oracle",
                             "sample": sample, "cpu": cpu_model()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# --------------------------------------------------------------- GPU arm --

def flush_l2(torch, flush, sink, s):
    """Evicts L2 between timed steps: writes a buffer larger than L2, then
    reads it back, so that the lines the flush leaves behind are clean and the
    timed step does not pay for writing the flush buffer back to HBM."""
    flush.fill_(s)
    sink.copy_(flush.sum(dtype=torch.int64).view(1))


def probe_rate(torch, L, q, kind, sms, stream, reps=4, iters=4000):
    """Best of `reps` runs of the in-run integer-pipe probe (operations/s)."""
    sink = torch.empty(sms * 8 * 256, dtype=torch.int64, device="cuda")
    best = 0.0
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rc = L.ntt_bench_butterflies(q, kind, sms * 8, 256, iters, sink.data_ptr(), stream.cuda_stream)
        assert rc == 0, rc
        e1.record(stream)
        torch.cuda.synchronize()
        best = max(best, sms * 8 * 256 * iters * 8 / (e0.elapsed_time(e1) * 1e-3))
    return best


def committed_profile(name, stamp):
    """A committed ncu summary (profiles/<name>.json) when it was taken on
    these kernel sources, else None."""
    try:
        with open(os.path.join(ROOT, "profiles", name + ".json")) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    return d if d.get("kernel_stamp") == stamp else None


def metric_extras(torch, ntt, W, L, stream, sms, peak_fwd, flush, sink, hybrid_log2):
    """The other halves of the metric, measured in the same run: coefficients/s
    and roofline fraction for every N from 2^10 to 2^16, the 200-request mixed
    batch against plain per-request launches (with the ceiling the plain arm
    leaves: its time over the probe-rate time of the same butterflies), the
    TFHE-shaped batch, and the cost model's regret.  A few seconds each."""
    t0 = time.perf_counter()
    fl = lambda k: flush_l2(torch, flush, sink, k)
    out = {}
    sizes, _, total = measure_n_sweep(torch, ntt, W, stream, 3, 2, fl, W.DEFAULT_SEED)
    out["n_sweep"] = {
        "how": "forward + inverse of 2^%d coefficients (8 limbs of 50-bit primes) per N, default schedule, L2 "
               "flushed; frac against the forward probe" % (total.bit_length() - 1),
        "sizes": [{"log2n": z["log2n"], "rows": z["rows"], "schedule": z["schedule"], "ms": z["ms_per_step"],
                   "coeffs_per_s": z["coeffs_per_s"], "frac": z["butterflies_per_s"] / peak_fwd} for z in sizes]}
    spec = W.mixed_requests(seed=W.DEFAULT_SEED)
    res, coef, bfly, n_sched = measure_mixed(torch, ntt, W, stream, 3, 1, hybrid_log2, spec, W.DEFAULT_SEED)
    ms = {k: sum(v[0]) / len(v[0]) for k, v in res.items()}
    ideal_ms = bfly / peak_fwd * 1e3
    out["mixed_batch"] = {
        "requests": len(spec), "coefficients": coef, "scheduled_requests": n_sched, "ms": ms,
        "speedup_vs_plain": ms["plain_per_request"] / ms["batched"],
        "grouped_vs_plain": ms["plain_per_request"] / ms["grouped"],
        "persistent_only_vs_plain": ms["plain_per_request"] / ms["persistent_only"],
        "frac": {k: ideal_ms / v for k, v in ms.items()},
        "ceiling_vs_plain": ms["plain_per_request"] / ideal_ms,
        "how": "forward transforms of 200 uneven requests (inputs %.1f GB > L2); frac = probe-rate time of all "
               "butterflies / measured time; ceiling_vs_plain = the largest speedup any form could show over the "
               "plain arm" % (coef * 8 / 1e9)}
    res, coef, bfly, q = measure_tfhe_batch(torch, ntt, W, stream, 5, 2, fl)
    peak0 = probe_rate(torch, L, q, 0, sms, stream, reps=2)
    ms = {k: sum(v[0]) / len(v[0]) for k, v in res.items()}
    out["tfhe_batch"] = {
        "ms": ms, "speedup_vs_plain": ms["plain_per_request"] / ms["batched"],
        "grouped_vs_plain": ms["plain_per_request"] / ms["grouped"],
        "forward_inverse_vs_plain": ms["plain_per_request"] / ms["forward_inverse"],
        "persistent_only_vs_plain": ms["plain_per_request"] / ms["persistent_only"],
        "frac": {k: bfly / peak0 * 1e3 / v for k, v in ms.items()},
        "how": "3780 forward + 1260 inverse rows at N = 1024, 62-bit prime, L2 flushed; frac against the "
               "exact-class forward probe (kind 0)"}
    try:
        out["cost_model"] = cost_model_summary()
    except Exception as e:   # the committed model or DB is missing or does not match the schedule lists
        out["cost_model"] = {"unavailable": "%s: %s" % (type(e).__name__, e)}
    out["extras_seconds"] = time.perf_counter() - t0
    return out


def run_ours(args):
    import torch
    world, rank, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device for --impl ours")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    from paper_2410_05934_gb300 import build as B
    B.build_product()
    import paper_2410_05934_gb300 as ntt
    from paper_2410_05934_gb300 import _native, shard
    from paper_2410_05934_gb300 import workloads as W

    n = 1 << LOG2N
    rows = POLYS * LIMBS
    w = W.ckks_hmul_n65536(seed=W.DEFAULT_SEED + rank)
    mods = w["moduli"]
    x_host = w["x"].reshape(rows, n)
    stream = torch.cuda.current_stream()

    plan = ntt.Plan(LOG2N, mods, POLYS)
    if args.schedule is not None:
        plan.schedule = args.schedule
    x = torch.from_numpy(x_host.view(np.int64)).to(dev)
    A = torch.empty_like(x)
    P = torch.empty_like(x)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    flush_sink = torch.empty(1, dtype=torch.int64, device=dev)
    pairs = [(0, 0), (0, 1), (1, 0), (1, 1)]
    A_POLY, B_POLY = [i for i, _ in pairs], [2 + j for _, j in pairs]

    fwd_ev, inv_ev = [], []

    def step(x_in, record=False):
        launches = 0
        if record:
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record(stream)
        plan.forward(x_in, A)
        launches += plan.last_launches()
        if record:
            e1.record(stream)
        # the 4 cross products a_i (.) b_j, formed in the inverse's first kernel
        plan.inverse_mul(A, A, P, a_poly=A_POLY, b_poly=B_POLY)
        launches += plan.last_launches()
        if record:
            e2.record(stream)
            fwd_ev.append((e0, e1))
            inv_ev.append((e1, e2))
        return launches

    # ---- integer-pipe probes: the "alu" roofline denominators ----
    # the butterflies of the plan's modulus class (moduli below 2^57: the
    # approximate-quotient forward, kind 2; below 2^50 the inverse's lazy GS
    # butterfly, kind 7; else the exact-quotient kinds 0 and 1) and the
    # Montgomery product formed inside the inverse (kind 6)
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    L = _native.load()
    probe_kind = 2 if max(mods) < (1 << 57) else 0
    inv_kind = 7 if max(mods) < (1 << 50) else (3 if max(mods) < (1 << 57) else 1)
    probe_best = probe_rate(torch, L, mods[0], probe_kind, sms, stream)
    probe_inv = probe_rate(torch, L, mods[0], inv_kind, sms, stream)
    probe_mont = probe_rate(torch, L, mods[0], 6, sms, stream)

    # ---- warm-up ----
    for _ in range(max(3, args.warmup)):
        step(x)
    torch.cuda.synchronize()

    # ---- timed region: K steps, L2 flushed before each, events per step ----
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    shard.barrier()
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    launches = 0
    wall0 = time.perf_counter()
    for s in range(args.steps):
        flush_l2(torch, flush, flush_sink, s)
        starts[s].record(stream)
        launches += step(x, record=True)
        ends[s].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    shard.barrier()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in zip(starts, ends)]
    fwd_ms = [a.elapsed_time(b) for a, b in fwd_ev]
    inv_ms = [a.elapsed_time(b) for a, b in inv_ev]
    t_total = shard.max_over_ranks(sum(step_ms) * 1e-3)
    coeffs_step = 2 * rows * n
    value = world * args.steps * coeffs_step / t_total
    ms_per_step = 1e3 * t_total / args.steps

    # correctness guard on the measured output: INTT(NTT(a)) spot check via the oracle-free identity
    back = torch.empty_like(x)
    plan.forward(x, A)
    plan.inverse(A, back)
    torch.cuda.synchronize()
    if not torch.equal(back, x):
        raise SystemExit("round trip failed: results are wrong, refusing to report a number")

    # ---- e2e: host buffers, copies inside the timed region ----
    # Every step copies its 96 input rows from pinned host memory and reads
    # its 96 product rows back; steps are pipelined over two device buffers
    # and three streams (host->device copy of step s+1 and device->host copy
    # of step s-1 run while step s computes), as a streaming user would.
    h_in = torch.from_numpy(x_host.view(np.int64)).pin_memory()
    h_out = torch.empty_like(h_in).pin_memory()
    xs = [torch.empty_like(x) for _ in range(2)]
    ps = [torch.empty_like(x) for _ in range(2)]
    s_h2d, s_d2h = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)
    ev = {k: [torch.cuda.Event() for _ in range(2)] for k in ("h2d", "comp", "d2h")}
    for k in ev:
        for e in ev[k]:
            e.record(stream)

    def e2e_step(s_idx):
        b = s_idx % 2
        s_h2d.wait_event(ev["comp"][b])          # x buffer b free again
        with torch.cuda.stream(s_h2d):
            xs[b].copy_(h_in, non_blocking=True)
        ev["h2d"][b].record(s_h2d)
        stream.wait_event(ev["h2d"][b])
        stream.wait_event(ev["d2h"][b])          # product buffer b read back already
        step_into(xs[b], ps[b])
        ev["comp"][b].record(stream)
        s_d2h.wait_event(ev["comp"][b])
        with torch.cuda.stream(s_d2h):
            h_out.copy_(ps[b], non_blocking=True)
        ev["d2h"][b].record(s_d2h)

    def step_into(x_in, p_out):
        plan.forward(x_in, A)
        plan.inverse_mul(A, A, p_out, a_poly=A_POLY, b_poly=B_POLY)

    for s_idx in range(4):
        e2e_step(s_idx)
    torch.cuda.synchronize()
    shard.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s_h2d.wait_event(e0)
    s_d2h.wait_event(e0)
    for s_idx in range(args.steps):
        e2e_step(s_idx)
    stream.wait_stream(s_h2d)
    stream.wait_stream(s_d2h)
    e1.record(stream)
    torch.cuda.synchronize()
    t_e2e = shard.max_over_ranks(e0.elapsed_time(e1) * 1e-3)
    e2e_value = world * args.steps * coeffs_step / t_e2e
    if not torch.equal(h_out.to(dev), ps[(args.steps - 1) % 2]):
        raise SystemExit("e2e read-back differs from the device result")

    # ---- roofline of the dominant kernel: the forward transform ----
    fwd_s = statistics.mean(fwd_ms) * 1e-3
    bfly_fwd = rows * (n // 2) * LOG2N                       # N/2 log2 N per row
    bytes_fwd = rows * n * 16 + LIMBS * n * 16               # data in+out + one twiddle table pass
    achieved_bfly = bfly_fwd / fwd_s
    hbm_peak = None
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            hbm_peak = json.load(f).get("hbm_gbs")
    except (OSError, ValueError):
        pass
    hbm_src = "measured"
    if not hbm_peak:
        hbm_peak, hbm_src = 6800.0, "fallback"
    # DRAM bytes of one forward transform from the committed ncu capture, when
    # it was taken on these kernel sources and this schedule
    traffic = None
    tpath = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(tpath) as f:
            t = json.load(f)
        if t.get("kernel_stamp") == B.kernel_stamp() and t.get("schedule") == plan.schedule:
            traffic = t.get("fwd_bytes_per_transform")
    except (OSError, ValueError):
        pass
    # the inverse with its products: ideal time = its GS butterflies at the
    # inverse probe's rate + its Montgomery products at the product probe's rate
    inv_s = statistics.mean(inv_ms) * 1e-3
    bfly_inv = rows * (n // 2) * LOG2N
    prods = rows * n
    inv_ideal_s = bfly_inv / probe_inv + prods / probe_mont
    pipes = committed_profile("butterfly_probe_pipes", B.kernel_stamp())
    roofline = {
        "bound": "alu",
        "kernel": "ntt_forward (%s)" % ntt.schedule_name(LOG2N, plan.schedule),
        "achieved": achieved_bfly / 1e9, "peak": probe_best / 1e9, "unit": "Gbutterfly/s",
        "frac": achieved_bfly / probe_best,
        "peak_source": "in-run probe: %d SMs x 8 CTAs x 256 thr x 8 independent forward butterflies "
                       "with the kernels' arithmetic for these moduli (probe kind %d)" % (sms, probe_kind),
        "probe_pipes": pipes and pipes.get("summary"),
        "traffic": traffic,
        "hbm": {"achieved": bytes_fwd / fwd_s / 1e9, "peak": hbm_peak, "unit": "GB/s",
                "frac": bytes_fwd / fwd_s / 1e9 / hbm_peak, "peak_source": hbm_src,
                "algorithmic_bytes": bytes_fwd},
        "fwd_ms": statistics.mean(fwd_ms),
        "inverse": {
            "kernel": "ntt_inverse_mul (%s): 96 Montgomery cross products formed in its first kernel, then the "
                      "inverse of the 96 product rows" % ntt.schedule_name(LOG2N, plan.schedule),
            "achieved": bfly_inv / inv_s / 1e9, "unit": "Gbutterfly/s",
            "frac": inv_ideal_s / inv_s,
            "peak": probe_inv / 1e9, "peak_products": probe_mont / 1e9,
            "peak_source": "in-run probes: inverse butterfly (kind %d) and Montgomery product (kind 6); frac = "
                           "(butterflies / butterfly peak + products / product peak) / measured time" % inv_kind,
            "butterflies": bfly_inv, "products": prods, "inv_ms": statistics.mean(inv_ms)},
    }

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "log2n": LOG2N, "limbs": LIMBS, "polys": POLYS,
                   "rows": rows, "moduli": "24 largest primes < 2^50, = 1 mod 2^17",
                   "step": "NTT(96 rows) -> 4 cross products x 24 limbs formed inside the INTT's first kernel "
                           "-> INTT(96 rows)",
                   "schedule": plan.schedule,
                   "l2": "flushed before every timed step, outside the step events: 512 MiB written, then read "
                         "back so that the evicted L2 holds clean lines",
                   "timing": "CUDA events per step on the launching stream, summed; max over ranks",
                   "wall_s_timed_loop": wall},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(x.numel() * 8),
                "d2h_bytes_per_step": int(P.numel() * 8),
                "how": "per step: pinned host -> device copy of the 96 input rows, the step, device -> host "
                       "copy of the 96 product rows; steps pipelined over two device buffers and three "
                       "streams (copies of neighbouring steps overlap the compute), one event pair around "
                       "all steps"},
        "gpu_launches": launches,
        "clocks": clk,
        "roofline": roofline,
    }
    if world == 1 and not args.no_extras:
        line.update(metric_extras(torch, ntt, W, L, stream, sms, probe_best, flush, flush_sink,
                                  args.hybrid_min_log2_coef))
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, cores, desc, dt = oracle_sample(args.cpu_seconds)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": desc, "seconds": dt, "cpu": cpu_model()}
        v2, cores2, dt2 = radix2_sample()
        line["cpu_radix2"] = {"value": v2, "unit": UNIT, "cores": cores2,
                              "kind": "plain radix-2 O(N log N) transforms, Shoup twiddles (oracle/ntt_radix2.c)",
                              "sample": "the whole step's 96 forward + 96 inverse rows at N=65536 (tables "
                                        "built inside the timed call)", "seconds": dt2}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


# ------------------------------------------------- the other workloads --

def _events_loop(torch, stream, steps, fn, flush=None):
    """Per-step CUDA events on `stream`; L2 flushed before each step if given."""
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    launches = 0
    for s in range(steps):
        if flush is not None:
            flush.fill_(s)
        starts[s].record(stream)
        launches += fn()
        ends[s].record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in zip(starts, ends)], launches


def _probe(torch, L, q, kind, sms, stream):
    sink = torch.empty(sms * 8 * 256, dtype=torch.int64, device="cuda")
    best = 0.0
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        assert L.ntt_bench_butterflies(q, kind, sms * 8, 256, 4000, sink.data_ptr(), stream.cuda_stream) == 0
        e1.record(stream)
        torch.cuda.synchronize()
        best = max(best, sms * 8 * 256 * 4000 * 8 / (e0.elapsed_time(e1) * 1e-3))
    return best


def measure_mixed(torch, ntt, W, stream, steps, warmup, hybrid_log2, spec, seed):
    """Times one uneven request list four ways: the batched form (one CUDA
    graph: the persistent kernel beside the requests that fill the GPU by
    themselves, each on its learned schedule on a concurrent branch), the
    persistent kernel alone, plain per-request launches on each N's default
    schedule, and plain launches on learned schedules.  Returns per-arm
    (per-step ms, launches) and the list's coefficient and butterfly counts."""
    from paper_2410_05934_gb300.costmodel import choose_schedule, schedule_requests
    reqs, coef, bfly = [], 0, 0
    for i, (log2n, limbs, polys) in enumerate(spec):
        x = W.request_rows_torch(seed, i, log2n, limbs, polys)
        reqs.append(dict(log2n=log2n, n_moduli=limbs, n_polys=polys, moduli_offset=0, inverse=0,
                         **{"in": x, "out": torch.empty_like(x)}))
        coef += x.numel()
        bfly += x.shape[0] * (x.shape[1] // 2) * log2n
    sreqs = schedule_requests(reqs, W.POOL50, hybrid_log2)
    batch = ntt.Batch(sreqs, W.POOL50, flags=ntt.NTT_BATCH_GRAPH)
    persistent = ntt.Batch(reqs, W.POOL50, flags=ntt.NTT_BATCH_GRAPH)
    grouped = ntt.Batch(reqs, W.POOL50, flags=ntt.NTT_BATCH_GRAPH | ntt.NTT_BATCH_GROUPED)
    learned = [choose_schedule(r["log2n"], r["n_moduli"], r["n_polys"], 50)[0] for r in reqs]
    arms = [("batched", lambda: (batch.execute(), batch.info()["last_launches"])[1]),
            ("grouped", lambda: (grouped.execute(), grouped.info()["last_launches"])[1]),
            ("persistent_only", lambda: (persistent.execute(), 1)[1]),
            ("plain_per_request", lambda: (persistent.execute_plain(), persistent.info()["last_launches"])[1]),
            ("plain_learned_schedule",
             lambda: (persistent.execute_plain(learned), persistent.info()["last_launches"])[1])]
    for _ in range(max(1, warmup)):
        for _, fn in arms:
            fn()
    torch.cuda.synchronize()
    res = {name: _events_loop(torch, stream, steps, fn, None) for name, fn in arms}
    n_sched = sum(1 for r in sreqs if r["schedule"])
    batch.close()
    persistent.close()
    grouped.close()
    return res, coef, bfly, n_sched


def measure_tfhe_batch(torch, ntt, W, stream, steps, warmup, flush_fn):
    """The TFHE blind-rotation-shaped batch (3780 forward + 1260 inverse rows,
    N = 1024, 62-bit prime) three ways: one CUDA graph with both requests on
    their learned schedules on concurrent branches, one persistent launch,
    and the two plain launches."""
    from paper_2410_05934_gb300.costmodel import schedule_requests
    w = W.tfhe_blind_rotation()
    q = w["moduli"][0]
    xf, xi = to_dev_np(torch, w["fwd"]), to_dev_np(torch, w["inv"])
    reqs = [dict(log2n=10, n_moduli=1, n_polys=xf.shape[0], inverse=0, **{"in": xf, "out": torch.empty_like(xf)}),
            dict(log2n=10, n_moduli=1, n_polys=xi.shape[0], inverse=1, **{"in": xi, "out": torch.empty_like(xi)})]
    batch = ntt.Batch(schedule_requests(reqs, [q], 21), [q], flags=ntt.NTT_BATCH_GRAPH)
    persistent = ntt.Batch(reqs, [q], flags=ntt.NTT_BATCH_GRAPH)
    grouped = ntt.Batch(reqs, [q], flags=ntt.NTT_BATCH_GRAPH | ntt.NTT_BATCH_GROUPED)
    pf, pi = ntt.Plan(10, [q], xf.shape[0]), ntt.Plan(10, [q], xi.shape[0])
    of, oi = torch.empty_like(xf), torch.empty_like(xi)
    arms = [("batched", lambda: (batch.execute(), batch.info()["last_launches"])[1]),
            ("grouped", lambda: (grouped.execute(), grouped.info()["last_launches"])[1]),
            ("forward_inverse", lambda: (ntt.forward_inverse(pf, xf, xi, pi, of, oi), pf.last_launches())[1]),
            ("persistent_only", lambda: (persistent.execute(), 1)[1]),
            ("plain_per_request", lambda: (batch.execute_plain(), 2)[1])]
    for _ in range(max(1, warmup)):
        for _, fn in arms:
            fn()
    torch.cuda.synchronize()
    res = {}
    for name, fn in arms:
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        launches = 0
        for k in range(steps):
            flush_fn(k)
            starts[k].record(stream)
            launches += fn()
            ends[k].record(stream)
        torch.cuda.synchronize()
        res[name] = ([a.elapsed_time(b) for a, b in zip(starts, ends)], launches)
    coef = xf.numel() + xi.numel()
    bfly = (xf.shape[0] + xi.shape[0]) * 512 * 10
    batch.close()
    persistent.close()
    grouped.close()
    return res, coef, bfly, q


def measure_n_sweep(torch, ntt, W, stream, steps, warmup, flush_fn, seed, log2ns=range(10, 17)):
    """Forward + inverse of 2^25 coefficients (8 limbs of the 50-bit pool,
    256 MB per buffer, larger than L2) at each N on its default schedule."""
    mods = W.POOL50[:8]
    total = 1 << 25
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    x = torch.randint(0, 1 << 49, (total,), dtype=torch.int64, device="cuda", generator=g)   # < every q
    y = torch.empty_like(x)
    sizes, launches = [], 0
    for log2n in log2ns:
        n = 1 << log2n
        batch = total // (n * len(mods))
        plan = ntt.Plan(log2n, mods, batch)

        def step(p=plan):
            p.forward(x, y)
            k = p.last_launches()
            p.inverse(y, y)
            return k + p.last_launches()
        for _ in range(max(1, warmup)):
            step()
        torch.cuda.synchronize()
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        for k in range(steps):
            flush_fn(k)
            starts[k].record(stream)
            launches += step()
            ends[k].record(stream)
        torch.cuda.synchronize()
        t = sum(a.elapsed_time(b) for a, b in zip(starts, ends)) * 1e-3 / steps
        sizes.append({"log2n": log2n, "rows": batch * len(mods), "schedule": plan.schedule,
                      "ms_per_step": 1e3 * t, "coeffs_per_s": 2 * total / t,
                      "butterflies_per_s": 2 * (total // 2) * log2n / t})
        plan.close()
    del x, y
    return sizes, launches, total


def cost_model_summary():
    """Regret of the committed cost model on its held-out shapes of the
    committed timing DB (mean, p90, max), beside the paper's SM-count rule and
    the built-in default; decision time per shape."""
    from paper_2410_05934_gb300 import costmodel as CM
    from paper_2410_05934_gb300 import tune as T
    model = CM.CostModel.load()
    recs = T.load_db(CM.DEFAULT_DB, current=True)
    X, Tt, M, keys, times = CM.dataset(recs)
    _, ho = CM.split_heldout(keys, model.meta.get("heldout", 100), model.meta.get("split_seed", 7))
    rep = CM.evaluate(model, [keys[i] for i in ho], [times[i] for i in ho])
    stale = sorted(int(n) for n, sig in (model.meta.get("sigs") or {}).items() if sig != T.schedule_signature(int(n)))
    return {"mlp": rep["mlp"], "sm_rule_mean": rep["sm_rule"]["mean"], "default_mean": rep["default"]["mean"],
            "decision_us": rep["decision_us"], "heldout_shapes": len(ho), "db_records": len(recs),
            "model_stale_for_log2n": stale,
            "how": "committed model (trained on the GPU by the library's MLP kernels) on the held-out shapes of "
                   "the committed GB300 timing DB"}


def run_other(args):
    """Lines for the mixed batch, the TFHE-shaped batch and the plain N=1024
    workload (same schema; the default line is the default workload)."""
    import torch
    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    from paper_2410_05934_gb300 import build as B
    B.build_product()
    import paper_2410_05934_gb300 as ntt
    from paper_2410_05934_gb300 import _native
    from paper_2410_05934_gb300 import workloads as W
    L = _native.load()
    stream = torch.cuda.current_stream()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
    clocks = ClockSampler(local)
    extra = {}
    if args.workload in ("mixed_batch", "mixed_small"):
        if args.workload == "mixed_batch":
            spec = W.mixed_requests(seed=W.DEFAULT_SEED + rank)
            dist_note = "N in {2^10,2^12,2^14,2^16} (.5/.2/.2/.1), limbs U{1..32}, polys U{1..64}, forward"
        else:
            # many small independent transforms (the TFHE side of scheme switching)
            spec = W.mixed_requests(seed=W.DEFAULT_SEED + rank, n_requests=2000, max_limbs=4, max_polys=4,
                                    log2ns=(10, 11), weights=(0.7, 0.3))
            dist_note = "2000 requests, N in {2^10, 2^11} (.7/.3), limbs U{1..4}, polys U{1..4}, forward"
        q_probe, kind = W.POOL50[0], 2
        clocks.start()
        res, coef, bfly, n_sched = measure_mixed(torch, ntt, W, stream, args.steps, max(3, args.warmup),
                                                 args.hybrid_min_log2_coef, spec, W.DEFAULT_SEED + rank)
        clk = clocks.stop()
        ms, launches = res["batched"]
        for name, how in (("persistent_only", "every request as work items of the one persistent kernel (one "
                                               "launch under a CUDA graph)"),
                          ("plain_per_request", "one launch sequence per request, default schedule of its N, "
                                                "same tables"),
                          ("plain_learned_schedule", "one launch sequence per request, schedule from the "
                                                     "autotuner DB / cost model")):
            m, k = res[name]
            extra[name] = {"value": coef * args.steps / (sum(m) * 1e-3), "ms_per_step": sum(m) / args.steps,
                           "launches_per_step": k // args.steps, "how": how}
        extra["speedup_vs_plain"] = sum(res["plain_per_request"][0]) / sum(ms)
        extra["speedup_vs_plain_learned"] = sum(res["plain_learned_schedule"][0]) / sum(ms)
        config = {"workload": args.workload, "requests": len(spec), "coefficients": coef,
                  "distribution": dist_note,
                  "batched": ("one CUDA graph: persistent kernel over %d requests || %d requests of >= 2^%d "
                              "coefficients on their learned schedules" % (len(spec) - n_sched, n_sched,
                                                                         args.hybrid_min_log2_coef)),
                  "l2": ("inputs (%.1f GB) > L2" % (coef * 8 / 1e9)) if coef * 8 > (256 << 20)
                  else "inputs (%.0f MB) fit L2: timed warm" % (coef * 8 / 1e6)}
        unit_coef = coef
    elif args.workload == "tfhe_blind_rotation":
        sink = torch.empty(1, dtype=torch.int64, device="cuda")
        clocks.start()
        res, coef, bfly, q_probe = measure_tfhe_batch(torch, ntt, W, stream, args.steps, max(3, args.warmup),
                                                      lambda k: flush_l2(torch, flush, sink, k))
        clk = clocks.stop()
        kind = 0
        ms, launches = res["batched"]
        extra["plain_per_request"] = {"value": coef * args.steps / (sum(res["plain_per_request"][0]) * 1e-3),
                                      "ms_per_step": sum(res["plain_per_request"][0]) / args.steps,
                                      "how": "forward launch + inverse launch, default schedule"}
        extra["persistent_only"] = {"value": coef * args.steps / (sum(res["persistent_only"][0]) * 1e-3),
                                    "ms_per_step": sum(res["persistent_only"][0]) / args.steps,
                                    "how": "both requests as work items of one persistent kernel launch"}
        extra["forward_inverse"] = {"value": coef * args.steps / (sum(res["forward_inverse"][0]) * 1e-3),
                                    "ms_per_step": sum(res["forward_inverse"][0]) / args.steps,
                                    "how": "one ntt_forward_inverse call: both row sets in one grid"}
        extra["grouped"] = {"value": coef * args.steps / (sum(res["grouped"][0]) * 1e-3),
                            "ms_per_step": sum(res["grouped"][0]) / args.steps,
                            "how": "ntt_batch_execute with NTT_BATCH_GROUPED: one grid per kernel phase"}
        extra["speedup_vs_plain"] = sum(res["plain_per_request"][0]) / sum(ms)
        extra["forward_inverse_vs_plain"] = sum(res["plain_per_request"][0]) / sum(res["forward_inverse"][0])
        config = {"workload": "tfhe_blind_rotation", "log2n": 10, "modulus_bits": 62,
                  "rows": "3780 forward (signed digits) + 1260 inverse",
                  "batched": "one CUDA graph launch: the two requests on their learned schedules, concurrent branches",
                  "l2": "flushed before every step"}
    elif args.workload == "hmul_fused":
        w = W.ckks_hmul_n65536()
        mods = w["moduli"]
        Lm, n = len(mods), 1 << 16
        x = to_dev_np(torch, w["x"].reshape(4 * Lm, n))
        plan = ntt.Plan(16, mods, 4)
        limb_plan = ntt.Plan(16, mods, 1)
        A = torch.empty_like(x)
        D = torch.empty((3 * Lm, n), dtype=torch.int64, device="cuda")
        P = torch.empty_like(x)
        Av, Pv = A.view(4, Lm, n), P.view(4, Lm, n)

        def fused():
            plan.forward(x, A)
            n1 = plan.last_launches()
            plan.hmul_tensor(A[:2 * Lm], A[2 * Lm:], D)
            return n1 + plan.last_launches()

        def unfused():
            plan.forward(x, A)
            for k, (i, j) in enumerate([(0, 0), (0, 1), (1, 0), (1, 1)]):
                limb_plan.pointwise(Av[i], Av[2 + j], Pv[k])
            plan.inverse(P, P)
            return 8
        coef = (4 + 3) * Lm * n
        bfly = (4 + 3) * Lm * (n // 2) * 16
        q_probe, kind = mods[0], 2
        for _ in range(max(3, args.warmup)):
            fused()
            unfused()
        torch.cuda.synchronize()
        clocks.start()
        ms, launches = _events_loop(torch, stream, args.steps, fused, flush)
        clk = clocks.stop()
        ms_u, _ = _events_loop(torch, stream, args.steps, unfused, flush)
        extra["unfused"] = {"ms_per_step": sum(ms_u) / args.steps,
                            "how": "forward NTT, 4 cross products (4 launches), inverse NTT of 96 rows; "
                                   "d1 still needs one more addition"}
        extra["speedup_vs_unfused"] = sum(ms_u) / sum(ms)
        config = {"workload": "hmul_fused", "log2n": 16, "limbs": Lm,
                  "step": "NTT of a0,a1,b0,b1 (96 rows) -> tensor product fused into the inverse -> d0,d1,d2 (72 rows)",
                  "l2": "flushed before every step"}
    else:  # plain_n1024
        w = W.plain_n1024()
        q = w["moduli"][0]
        x = to_dev_np(torch, w["x"])
        plan64, plan32 = ntt.Plan(10, [q], 64), ntt.Plan(10, [q], 32)
        A = torch.empty_like(x)
        C = torch.empty_like(x[:32])

        def step():
            plan64.forward(x, A)
            plan32.pointwise(A[:32], A[32:], C)
            plan32.inverse(C, C)
            return 3
        coef = 64 * 1024 + 32 * 1024
        bfly = 96 * 512 * 10
        q_probe, kind = q, 0
        for _ in range(max(3, args.warmup)):
            step()
        torch.cuda.synchronize()
        clocks.start()
        ms, launches = _events_loop(torch, stream, args.steps, step, flush)
        clk = clocks.stop()
        config = {"workload": "plain_n1024", "log2n": 10, "rows": "64 forward, 32 products, 32 inverse",
                  "note": "launch-latency bound (1 MB per step); %HBM roofline not meaningful",
                  "l2": "flushed before every step"}
    t = sum(ms) * 1e-3
    peak = _probe(torch, L, q_probe, kind, sms, stream)
    achieved = bfly * args.steps / t
    line = {"metric": "NTT coeffs/s (coefficient-transforms per second)", "value": coef * args.steps / t,
            "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic", "config": config,
            "gpu_launches": launches, "clocks": clk,
            "roofline": {"bound": "alu", "achieved": achieved / 1e9, "peak": peak / 1e9,
                         "unit": "Gbutterfly/s", "frac": achieved / peak, "traffic": None,
                         "peak_source": "in-run butterfly probe (kind %d)" % kind}}
    line.update(extra)
    if rank == 0:
        print(json.dumps(line))
    return 0


def run_tfhe_cmux(args):
    """Blind rotation of 1024 TFHE accumulators (N = 1024, the 62-bit prime,
    gadget B = 2^8, l = 3): 630 batched CMux steps, each with its own RGSW
    key and one exponent per accumulator (Sec. IV-A: every CMux of an
    iteration shares the key), in place.  Beside it: the time of the
    transforms alone (6 forward + 2 inverse rows per ciphertext and step
    through the plain batched NTT), the least an unfused decompose / NTT /
    MAC / INTT pipeline would spend."""
    import torch
    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    from paper_2410_05934_gb300 import build as B
    B.build_product()
    import paper_2410_05934_gb300 as ntt
    from paper_2410_05934_gb300 import _native
    from paper_2410_05934_gb300 import workloads as W
    L = _native.load()
    stream = torch.cuda.current_stream()
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    n_slot, n_lwe, levels, log2_base, n = 1024, 630, 3, 8, 1024
    w = W.tfhe_cmux(seed=W.DEFAULT_SEED + rank, n_ct=n_slot, steps=n_lwe, levels=levels)
    q = w["moduli"][0]
    plan = ntt.Plan(10, [q])
    acc = to_dev_np(torch, w["acc"])
    raw = to_dev_np(torch, w["key"])
    keys = [plan.tfhe_key_prepare(raw[i], levels) for i in range(n_lwe)]     # once per key, outside timing
    del raw
    rots = torch.from_numpy(w["rot"].astype(np.int32)).cuda()

    def blind_rotation():
        for i in range(n_lwe):
            plan.tfhe_cmux_rotate(acc, rots[i], keys[i], levels, log2_base)
        return n_lwe
    blind_rotation()
    torch.cuda.synchronize()
    steps = max(1, args.steps // 10)
    clocks = ClockSampler(local)
    clocks.start()
    ms, launches = _events_loop(torch, stream, steps, blind_rotation)
    clk = clocks.stop()
    t = sum(ms) * 1e-3
    cmux = n_slot * n_lwe * steps
    # the transforms alone, per CMux step: 6 forward and 2 inverse rows per ciphertext
    fwd_plan, inv_plan = ntt.Plan(10, [q], 2 * levels * n_slot), ntt.Plan(10, [q], 2 * n_slot)
    xf = torch.empty((2 * levels * n_slot, n), dtype=torch.int64, device="cuda").fill_(1)
    xi = torch.empty((2 * n_slot, n), dtype=torch.int64, device="cuda").fill_(1)

    def transforms():
        fwd_plan.forward(xf)
        inv_plan.inverse(xi)
        return 2
    for _ in range(3):
        transforms()
    ms_t, _ = _events_loop(torch, stream, 50, transforms)
    per_step = t / (n_lwe * steps)
    bfly = cmux * 8 * (n // 2) * 10
    peak = _probe(torch, L, q, 0, sms, stream)
    line = {"metric": "NTT coeffs/s (coefficient-transforms per second)", "value": cmux * 8 * n / t,
            "unit": UNIT, "n_gpus": world, "steps": steps, "warmup": 1, "ms_per_step": 1e3 * t / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic", "gpu_launches": launches, "clocks": clk,
            "config": {"workload": "tfhe_cmux", "log2n": 10, "modulus_bits": 62, "slots": n_slot,
                       "cmux_steps": n_lwe, "gadget": "B = 2^8, l = 3",
                       "step": "one blind rotation: 630 batched CMux launches (decompose, 6 NTT, MAC with "
                               "the step's RGSW key, 2 INTT, add) over 1024 accumulators, in place",
                       "keys": "630 RGSW keys in Shoup pair form (124 MB), prepared once before timing",
                       "l2": "accumulators (16 MB) stay in L2 across steps, keys stream"},
            "cmux_per_s": cmux / t, "blind_rotations_per_s": n_slot * steps / t,
            "us_per_cmux_step": 1e6 * per_step,
            "transforms_only": {"us_per_cmux_step": 1e3 * sum(ms_t) / 50,
                                "how": "6144 forward + 2048 inverse N=1024 rows through ntt_forward / "
                                       "ntt_inverse (no decomposition, no MAC, digits in HBM)"},
            "roofline": {"bound": "alu", "achieved": bfly / t / 1e9, "peak": peak / 1e9, "unit": "Gbutterfly/s",
                         "frac": bfly / t / peak, "traffic": None,
                         "peak_source": "in-run butterfly probe (kind 0, exact class)",
                         "note": "butterflies of the 8 transforms per CMux; the MAC and the decomposition are "
                                 "extra work on the same pipes"}}
    if rank == 0 and not args.no_cpu_baseline:
        from oracle import tfhe_oracle as TO
        t0 = time.perf_counter()
        kc = TO.key_coefficients(w["key"][0], q)
        k = 0
        while k < 2 or time.perf_counter() - t0 < min(args.cpu_seconds, 10.0):
            TO.cmux_rotate(w["acc"][k], int(w["rot"][0][k]), w["key"][0], q, log2_base, levels, key_coef=kc)
            k += 1
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": k * 8 * n / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": "%d full CMux steps of step 0 (key brought to coefficients once, "
                                          "schoolbook ring products)" % k, "cmux_per_s": k / dt}
    if rank == 0:
        print(json.dumps(line))
    return 0


def run_ckks_bconv(args):
    """Key-switching basis conversion (ModUp of hybrid key switching with one
    digit): a ciphertext's 2 x 24 limbs at N = 2^16 converted to 24 special
    primes, one ntt_bconv launch per step, L2 flushed before every step."""
    import torch
    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    from paper_2410_05934_gb300 import build as B
    B.build_product()
    import paper_2410_05934_gb300 as ntt
    from paper_2410_05934_gb300 import _native
    from paper_2410_05934_gb300 import workloads as W
    L_ = _native.load()
    stream = torch.cuda.current_stream()
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    w = W.ckks_bconv(seed=W.DEFAULT_SEED + rank)
    Q, P, x = w["Q"], w["P"], w["x"]
    polys, L, K, n = x.shape[0], len(Q), len(P), x.shape[2]
    conv = ntt.BConv(Q, P)
    xd = to_dev_np(torch, x)
    out = torch.empty((polys, K, n), dtype=torch.int64, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")

    def step():
        conv(xd, out, 16)
        return 1
    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    ms, launches = _events_loop(torch, stream, args.steps, step, flush)
    clk = clocks.stop()
    t = sum(ms) * 1e-3
    coef = polys * n * args.steps
    macs = coef * L * K
    peak = _probe(torch, L_, Q[0], 4, sms, stream)
    hbm_bytes = coef * (L + K) * 8
    line = {"metric": "RNS basis conversion, coefficients/s (one coefficient = all its limbs)",
            "value": coef / t, "unit": "coeffs/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u64", "data": "synthetic", "gpu_launches": launches, "clocks": clk,
            "config": {"workload": "ckks_bconv", "log2n": 16, "polys": polys, "from_limbs": L, "to_limbs": K,
                       "moduli": "Q = 24 largest 50-bit primes = 1 mod 2^17, P = the next 24",
                       "l2": "flushed before every step (512 MiB write, outside the step events)"},
            "roofline": {"bound": "alu", "achieved": macs / t / 1e9, "peak": peak / 1e9, "unit": "GMAC/s",
                         "frac": macs / t / peak, "traffic": None,
                         "peak_source": "in-run probe (kind 4: 64x64->128-bit multiply-accumulate)",
                         "hbm": {"achieved_gbs": hbm_bytes / t / 1e9,
                                 "bytes_per_coefficient": (L + K) * 8}}}
    if rank == 0 and not args.no_cpu_baseline:
        from oracle import rns_oracle as RO
        t0 = time.perf_counter()
        k = 0
        while k < 64 or time.perf_counter() - t0 < min(args.cpu_seconds, 10.0):
            RO.bconv(x[0][:, k * 64:(k + 1) * 64], Q, P)
            k += 1
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": k * 64 / dt, "unit": "coeffs/s", "cores": 1, "kind": "oracle",
                                "sample": "%d coefficients of polynomial 0 (the definition in Python integers, "
                                          "one core)" % (k * 64)}
    if rank == 0:
        print(json.dumps(line))
    return 0


def run_ckks_rescale(args):
    """CKKS Rescale of a ciphertext in the NTT domain: 2 polynomials x 24
    limbs at N = 2^16 -> 23 limbs (strided copy of the dropped limb, its
    INTT, one forward NTT per remaining limb with the Rescale load and
    epilogue fused), L2 flushed before every step."""
    import torch
    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    from paper_2410_05934_gb300 import build as B
    B.build_product()
    import paper_2410_05934_gb300 as ntt
    from paper_2410_05934_gb300 import _native
    from paper_2410_05934_gb300 import workloads as W
    L_ = _native.load()
    stream = torch.cuda.current_stream()
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    w = W.ckks_hmul_n65536(seed=W.DEFAULT_SEED + rank, limbs=24, polys=2)
    Q, x = w["moduli"], w["x"]
    n, L = 1 << 16, len(Q)
    plan = ntt.Plan(16, Q, 2)
    xd = to_dev_np(torch, x)
    out = torch.empty((2, L - 1, n), dtype=torch.int64, device="cuda")
    work = torch.empty((2, n), dtype=torch.int64, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")

    def step():
        plan.rescale(xd, out, work)
        return plan.last_launches()
    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    ms, launches = _events_loop(torch, stream, args.steps, step, flush)
    clk = clocks.stop()
    t = sum(ms) * 1e-3
    rows = 2 + 2 * (L - 1)                           # INTT rows + forward rows
    coef = rows * n * args.steps
    bfly = rows * (n // 2) * 16 * args.steps
    peak = _probe(torch, L_, Q[0], 2, sms, stream)
    line = {"metric": "NTT coeffs/s (coefficient-transforms per second)", "value": coef / t, "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "gpu_launches": launches, "clocks": clk,
            "config": {"workload": "ckks_rescale", "log2n": 16, "polys": 2, "limbs": L,
                       "step": "Rescale by q_23: copy + INTT of 2 rows, fused NTT + epilogue of 46 rows",
                       "l2": "flushed before every step (512 MiB write, outside the step events)"},
            "rescales_per_s": 2 * args.steps / t,
            "roofline": {"bound": "alu", "achieved": bfly / t / 1e9, "peak": peak / 1e9, "unit": "Gbutterfly/s",
                         "frac": bfly / t / peak, "traffic": None,
                         "peak_source": "in-run butterfly probe (kind 2, small-modulus class)"}}
    if rank == 0:
        print(json.dumps(line))
    return 0


def run_natural_order(args):
    """Forward + inverse NTT of the CKKS-HMUL-shaped batch (96 rows at
    N = 2^16) with natural-order plans (NTT_FLAG_NATURAL_ORDER: one
    bit-reversal pass over HBM per transform for the two-kernel schedule),
    beside the same transforms in bit-reversed order; L2 flushed before every
    step."""
    import torch
    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    from paper_2410_05934_gb300 import build as B
    B.build_product()
    import paper_2410_05934_gb300 as ntt
    from paper_2410_05934_gb300 import workloads as W
    stream = torch.cuda.current_stream()
    w = W.ckks_hmul_n65536(seed=W.DEFAULT_SEED + rank)
    x = to_dev_np(torch, w["x"])
    y = torch.empty_like(x)
    nat = ntt.Plan(16, w["moduli"], 4, flags=ntt.NTT_FLAG_NATURAL_ORDER)
    brv = ntt.Plan(16, w["moduli"], 4)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")

    def step(p):
        p.forward(x, y)
        n1 = p.last_launches()
        p.inverse(y, y)
        return n1 + p.last_launches()
    for _ in range(max(3, args.warmup)):
        step(nat)
        step(brv)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    ms, launches = _events_loop(torch, stream, args.steps, lambda: step(nat), flush)
    clk = clocks.stop()
    ms_b, _ = _events_loop(torch, stream, args.steps, lambda: step(brv), flush)
    t = sum(ms) * 1e-3
    coef = 2 * 96 * 65536 * args.steps
    line = {"metric": "NTT coeffs/s (coefficient-transforms per second)", "value": coef / t, "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "gpu_launches": launches, "clocks": clk,
            "config": {"workload": "natural_order", "log2n": 16, "rows": 96,
                       "step": "forward (natural-order output) + inverse (natural-order input), 96 rows",
                       "l2": "flushed before every step (512 MiB write, outside the step events)"},
            "bit_reversed": {"ms_per_step": sum(ms_b) / args.steps, "value": coef / (sum(ms_b) * 1e-3)},
            "overhead": sum(ms) / sum(ms_b) - 1.0}
    if rank == 0:
        print(json.dumps(line))
    return 0


def run_otf_twiddles(args):
    """Forward + inverse NTT of the CKKS-HMUL-shaped batch (96 rows at
    N = 2^16) with on-the-fly twiddles (NTT_FLAG_OTF_TWIDDLES: every twiddle
    the product of two entries of 512-pair per-limb tables), beside the same
    transforms with the stored N-entry tables and the same kernel geometry;
    L2 flushed before every step."""
    import torch
    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    from paper_2410_05934_gb300 import build as B
    B.build_product()
    import paper_2410_05934_gb300 as ntt
    from paper_2410_05934_gb300 import _native
    from paper_2410_05934_gb300 import workloads as W
    L_ = _native.load()
    stream = torch.cuda.current_stream()
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    w = W.ckks_hmul_n65536(seed=W.DEFAULT_SEED + rank)
    x = to_dev_np(torch, w["x"])
    y = torch.empty_like(x)
    otf = ntt.Plan(16, w["moduli"], 4, flags=ntt.NTT_FLAG_OTF_TWIDDLES)
    tab = ntt.Plan(16, w["moduli"], 4)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")

    def step(p):
        p.forward(x, y)
        n1 = p.last_launches()
        p.inverse(y, y)
        return n1 + p.last_launches()
    for _ in range(max(3, args.warmup)):
        step(otf)
        step(tab)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    ms, launches = _events_loop(torch, stream, args.steps, lambda: step(otf), flush)
    clk = clocks.stop()
    ms_t, _ = _events_loop(torch, stream, args.steps, lambda: step(tab), flush)
    peak = _probe(torch, L_, w["moduli"][0], 2, sms, stream)
    t = sum(ms) * 1e-3
    coef = 2 * 96 * 65536 * args.steps
    bfly = 2 * 96 * 32768 * 16 * args.steps
    otf_entries = 2 ** 8 + 2 ** 8
    line = {"metric": "NTT coeffs/s (coefficient-transforms per second)", "value": coef / t, "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "gpu_launches": launches, "clocks": clk,
            "config": {"workload": "otf_twiddles", "log2n": 16, "rows": 96,
                       "step": "forward + inverse, 96 rows, twiddles generated on the fly",
                       "l2": "flushed before every step (512 MiB write, outside the step events)"},
            "roofline": {"bound": "alu", "achieved": bfly / t / 1e9, "peak": peak / 1e9, "unit": "Gbutterfly/s",
                         "frac": bfly / t / peak, "traffic": None,
                         "peak_source": "in-run butterfly probe (kind 2, small-modulus class)"},
            "twiddle_bytes_per_transform": {"otf": 24 * otf_entries * 16, "tables": 24 * 65536 * 16},
            "stored_tables": {"ms_per_step": sum(ms_t) / args.steps, "value": coef / (sum(ms_t) * 1e-3)},
            "overhead": sum(ms) / sum(ms_t) - 1.0}
    if rank == 0:
        print(json.dumps(line))
    return 0


def run_n_sweep(args):
    """Forward + inverse throughput for every N from 2^10 to 2^16 on a batch of
    2^25 coefficients (8 limbs of the 50-bit pool, 256 MB per buffer, larger
    than L2), each N on its default schedule; roofline fraction against the
    in-run butterfly probe.  One JSON line, the per-N results under "sizes"."""
    import torch
    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    from paper_2410_05934_gb300 import build as B
    B.build_product()
    import paper_2410_05934_gb300 as ntt
    from paper_2410_05934_gb300 import _native
    from paper_2410_05934_gb300 import workloads as W
    L_ = _native.load()
    stream = torch.cuda.current_stream()
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    peak = _probe(torch, L_, W.POOL50[0], 2, sms, stream)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
    sink = torch.empty(1, dtype=torch.int64, device="cuda")
    sizes, launches, total = measure_n_sweep(torch, ntt, W, stream, args.steps, max(3, args.warmup),
                                             lambda k: flush_l2(torch, flush, sink, k), W.DEFAULT_SEED + rank)
    mods = W.POOL50[:8]
    for sz in sizes:
        sz["frac"] = sz["butterflies_per_s"] / peak
    all_ms = [sz["ms_per_step"] * 1e-3 for sz in sizes]
    t_all = sum(all_ms)
    line = {"metric": "NTT coeffs/s (coefficient-transforms per second)", "value": 2 * total * len(sizes) / t_all,
            "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t_all, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u64", "data": "synthetic", "gpu_launches": launches,
            "config": {"workload": "n_sweep", "coefficients_per_size": total, "limbs": len(mods),
                       "step": "forward + inverse of 2^25 coefficients at each N = 2^10 .. 2^16",
                       "l2": "inputs (256 MB) > L2; flushed before every step"},
            "roofline": {"bound": "alu", "peak": peak / 1e9, "unit": "Gbutterfly/s",
                         "frac": min(sz["frac"] for sz in sizes), "traffic": None,
                         "peak_source": "in-run butterfly probe (kind 2); frac is the smallest over N"},
            "sizes": sizes}
    if rank == 0:
        print(json.dumps(line))
    return 0


def run_word32(args):
    """The TFHE blind-rotation-shaped batch (3780 forward + 1260 inverse rows
    at N = 1024) with a 30-bit prime on 32-bit words (NTT_FLAG_WORD32) as
    one ntt_forward_inverse launch, beside the same rows as two launches and
    the 62-bit batch on 64-bit words; L2 flushed before every step."""
    import torch
    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    from paper_2410_05934_gb300 import build as B
    B.build_product()
    import paper_2410_05934_gb300 as ntt
    from paper_2410_05934_gb300 import _native
    from paper_2410_05934_gb300 import workloads as W
    L_ = _native.load()
    stream = torch.cuda.current_stream()
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    q30, n = 1073692673, 1024
    xf = W.signed_digits_mod(W.DEFAULT_SEED + rank, 3, 3780 * n, q30).reshape(3780, n)
    xi = W.uniform_mod(W.DEFAULT_SEED + rank, 4, 1260 * n, q30).reshape(1260, n)
    f32 = torch.from_numpy(xf.astype(np.uint32).view(np.int32)).cuda()
    i32 = torch.from_numpy(xi.astype(np.uint32).view(np.int32)).cuda()
    pf = ntt.Plan(10, [q30], 3780, flags=ntt.NTT_FLAG_WORD32)
    pi = ntt.Plan(10, [q30], 1260, flags=ntt.NTT_FLAG_WORD32)
    w64 = W.tfhe_blind_rotation()
    f64, i64 = to_dev_np(torch, w64["fwd"]), to_dev_np(torch, w64["inv"])
    pf64, pi64 = ntt.Plan(10, w64["moduli"], 3780), ntt.Plan(10, w64["moduli"], 1260)
    of32, oi32, of64, oi64 = (torch.empty_like(t) for t in (f32, i32, f64, i64))
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")

    def step32():
        ntt.forward_inverse(pf, f32, i32, pi, of32, oi32)     # both directions in one launch
        return 1

    def step32_two():
        pf.forward(f32, of32)
        pi.inverse(i32, oi32)
        return 2

    def step64():
        pf64.forward(f64, of64)
        pi64.inverse(i64, oi64)
        return 2
    for _ in range(max(3, args.warmup)):
        step32()
        step32_two()
        step64()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    ms, launches = _events_loop(torch, stream, args.steps, step32, flush)
    clk = clocks.stop()
    ms_two, _ = _events_loop(torch, stream, args.steps, step32_two, flush)
    ms64, _ = _events_loop(torch, stream, args.steps, step64, flush)
    t = sum(ms) * 1e-3
    coef = (3780 + 1260) * n * args.steps
    bfly = (3780 + 1260) * (n // 2) * 10 * args.steps
    # the 32-bit butterfly in both conditional-subtraction forms: the faster is the peak
    peak5, peak8 = _probe(torch, L_, q30, 5, sms, stream), _probe(torch, L_, q30, 8, sms, stream)
    peak = max(peak5, peak8)
    line = {"metric": "NTT coeffs/s (coefficient-transforms per second)", "value": coef / t, "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "gpu_launches": launches, "clocks": clk,
            "config": {"workload": "word32", "log2n": 10, "modulus_bits": 30,
                       "rows": "3780 forward (signed digits) + 1260 inverse, one ntt_forward_inverse launch",
                       "l2": "flushed before every step"},
            "two_launches": {"ms_per_step": sum(ms_two) / args.steps,
                             "how": "ntt_forward then ntt_inverse on the same stream"},
            "word64_62bit": {"ms_per_step": sum(ms64) / args.steps, "value": coef / (sum(ms64) * 1e-3)},
            "speedup_vs_word64": sum(ms64) / sum(ms),
            "roofline": {"bound": "alu", "achieved": bfly / t / 1e9, "peak": peak / 1e9, "unit": "Gbutterfly/s",
                         "frac": bfly / t / peak, "traffic": None,
                         "peak_source": "in-run butterfly probes, the faster of kind 5 (the kernels' 32-bit "
                                        "forward butterfly, %.0f G/s) and kind 8 (the same with compare-and-select "
                                        "subtractions, %.0f G/s)" % (peak5 / 1e9, peak8 / 1e9),
                         "hbm": {"achieved_gbs": coef * 8 / t / 1e9, "bytes_per_coefficient": 8}}}
    if rank == 0:
        print(json.dumps(line))
    return 0


def run_cost_model(args):
    """Schedule cost model: train on the committed GB300 timing sweep with the
    library's GPU kernels; regret on 100 held-out shapes vs exhaustive tuning."""
    from paper_2410_05934_gb300 import costmodel as CM
    import torch
    torch.cuda.set_device(dist_env()[2])
    model, rep = CM.train_and_evaluate(steps=16000)
    # what the model replaces: exhaustive autotuning of a shape (every candidate
    # schedule timed, as the sweep does), on three held-out-sized shapes
    import tempfile
    from paper_2410_05934_gb300 import tune as T
    shapes = [(16, 24, 4, 50), (14, 8, 32, 50), (10, 1, 3780, 62)]
    with tempfile.TemporaryDirectory() as tmp:
        t0 = time.perf_counter()
        T.sweep(shapes, db=os.path.join(tmp, "t.jsonl"), reps=5, skip_done=False)
        exhaustive_ms = 1e3 * (time.perf_counter() - t0) / len(shapes)
    line = {"metric": "schedule regret vs exhaustive autotuning (mean over held-out shapes)",
            "value": rep["mlp"]["mean"], "unit": "fraction", "n_gpus": 1, "steps": rep["train"]["train_steps"],
            "warmup": 0, "ms_per_step": 1e3 * rep["train"]["train_seconds"] / rep["train"]["train_steps"],
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "autotuner timings measured on GB300 (%d)" % rep["timings"],
            "config": {"workload": "cost_model", "mlp": "4-64-64-12 ReLU, FP32, Adam, cosine lr",
                       "train_shapes": rep["train"]["train_shapes"], "heldout_shapes": rep["mlp"]["n"]},
            "regret": {"mlp": rep["mlp"], "sm_rule": rep["sm_rule"], "default": rep["default"]},
            "decision_us": rep["decision_us"], "train_seconds_gpu": rep["train"]["train_seconds"],
            "exhaustive_tuning_ms_per_shape": exhaustive_ms,
            "exhaustive_shapes": ["N=2^%d limbs=%d batch=%d %d-bit" % sh for sh in shapes]}
    print(json.dumps(line))
    return 0


def run_serving(args):
    """Poisson stream of mixed-batch-distributed requests at 5k req/s."""
    import torch
    torch.cuda.set_device(dist_env()[2])
    from paper_2410_05934_gb300 import build as B
    B.build_product()
    from paper_2410_05934_gb300 import serve
    pool = serve.RequestPool()
    n = max(500, args.steps * 200)
    serve.serve(pool, 5000.0, 200, "per_request", seed=99)        # warm-up
    clocks = ClockSampler(dist_env()[2])
    clocks.start()
    per = serve.serve(pool, 5000.0, n, "per_request", seed=1)
    clk = clocks.stop()
    mb = serve.serve(pool, 5000.0, n, "microbatch", window_us=500.0, seed=1)
    mb2 = serve.serve(pool, 5000.0, n, "microbatch", window_us=2000.0, seed=1)
    line = {"metric": "p99 latency at 5k req/s (mixed-batch request distribution)", "value": per["p99_ms"],
            "unit": "ms", "n_gpus": 1, "steps": n, "warmup": 200, "ms_per_step": per["mean_ms"],
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic", "config": {"workload": "serving", "rate_req_s": 5000, "requests": n,
                                            "policy": "per-request launches, cost-model schedules"},
            "p50_ms": per["p50_ms"], "throughput_coef_s": per["throughput_coef_s"],
            "offered_coef_s": per["offered_coef_s"], "clocks": clk,
            "policies": {"per_request": per, "microbatch_500us": mb, "microbatch_2ms": mb2}}
    print(json.dumps(line))
    return 0


def run_probe_pipes(args):
    """The workload of the integer-pipe counter capture (profiles/butterfly_probe_pipes.md):
    one launch of each butterfly probe kind (2, 7, 6, 3 with a 50-bit prime, 0 with a 62-bit
    one; SMs x 8 CTAs x 256 threads x 400 iterations x 8 operations), then one forward and one
    ntt_inverse_mul of 16 rows (4 polynomials x 4 limbs of 50-bit primes) at N = 2^16 on the
    plan's default schedule.  Prints a JSON line with the timings; meant to run under ncu."""
    import torch
    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    from paper_2410_05934_gb300 import build as B
    B.build_product()
    import paper_2410_05934_gb300 as ntt
    from paper_2410_05934_gb300 import _native
    from paper_2410_05934_gb300 import workloads as W
    L_ = _native.load()
    stream = torch.cuda.current_stream()
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    sink = torch.empty(sms * 8 * 256, dtype=torch.int64, device="cuda")
    out = {}
    for kind in (2, 7, 6, 3, 0):
        q = W.Q62_N1024 if kind == 0 else W.POOL50[0]
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        assert L_.ntt_bench_butterflies(q, kind, sms * 8, 256, 400, sink.data_ptr(), stream.cuda_stream) == 0
        e1.record(stream)
        torch.cuda.synchronize()
        out["probe_%d_ms" % kind] = e0.elapsed_time(e1)
    mods = W.POOL50[:4]
    x = to_dev_np(torch, W.rows_uniform(3, 16, [m for _ in range(4) for m in mods], 1 << 16))
    A, P = torch.empty_like(x), torch.empty_like(x)
    plan = ntt.Plan(16, mods, 4)
    plan.forward(x, A)
    plan.inverse_mul(A, A, P, a_poly=[0, 0, 1, 1], b_poly=[2, 3, 2, 3])
    torch.cuda.synchronize()
    out.update(workload="probe_pipes", schedule=plan.schedule)
    if rank == 0:
        print(json.dumps(out))
    return 0


def to_dev_np(torch, x):
    return torch.from_numpy(np.ascontiguousarray(x).view(np.int64)).cuda()


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "cost_model":
        return run_cost_model(args)
    if args.workload == "serving":
        return run_serving(args)
    if args.workload == "tfhe_cmux":
        return run_tfhe_cmux(args)
    if args.workload == "otf_twiddles":
        return run_otf_twiddles(args)
    if args.workload == "n_sweep":
        return run_n_sweep(args)
    if args.workload == "ckks_bconv":
        return run_ckks_bconv(args)
    if args.workload == "ckks_rescale":
        return run_ckks_rescale(args)
    if args.workload == "natural_order":
        return run_natural_order(args)
    if args.workload == "word32":
        return run_word32(args)
    if args.workload == "probe_pipes":
        return run_probe_pipes(args)
    if args.workload != WORKLOAD:
        return run_other(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
