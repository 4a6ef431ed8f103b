"""Learned schedule cost model (the schedule-choice row of the hot path).

The paper picks its switch point with a closed-form rule (data chunks closest
to the SM count, Sec. V-D).  Here a small FP32 MLP predicts the log-time of
every candidate schedule of a shape from (log2 N, limbs, batch, modulus
bits); the schedule with the smallest prediction is chosen.  It is trained on
timings the autotuner measures, on the GPU, by the library's own forward,
backward and Adam kernels (C ABI ``ntt_mlp_*``); exhaustive autotuning stays
the fallback for shapes in the timing DB and the yardstick of the model's regret.

Features (all in [0, 1] over the supported range):
  (log2 N - 10) / 6,  log2(limbs) / 6,  log2(batch) / 12,  (bits - 50) / 12
Targets: ln(milliseconds) of each schedule id (slot k = schedule id k);
slots a shape's N does not have are masked out of the loss and the argmin.
"""
import ctypes
import json
import math
import os
import time

import numpy as np

from . import ntt as _ntt
from ._native import check, load

IN, H, OUT = 4, 64, 12
N_PARAMS = H * IN + H + H * H + H + OUT * H + OUT
N_ACT = 2 * H + OUT
DATA_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data")
DEFAULT_DB = os.path.join(DATA_DIR, "tune_gb300.jsonl")
DEFAULT_PARAMS = os.path.join(DATA_DIR, "costmodel_gb300.npz")


def features(log2n, limbs, batch, bits=50):
    return np.array([(log2n - 10) / 6.0, math.log2(max(1, limbs)) / 6.0,
                     math.log2(max(1, batch)) / 12.0, (bits - 50) / 12.0], dtype=np.float32)


def n_schedules(log2n):
    return min(OUT, _ntt.schedule_count(log2n))


def init_params(seed=0):
    """He-style initialisation, float32, layout of ntt_mlp_*."""
    rng = np.random.default_rng(seed)
    parts = [rng.normal(0, math.sqrt(2.0 / IN), H * IN), np.zeros(H),
             rng.normal(0, math.sqrt(2.0 / H), H * H), np.zeros(H),
             rng.normal(0, math.sqrt(1.0 / H), OUT * H), np.zeros(OUT)]
    return np.concatenate(parts).astype(np.float32)


# ---- the timing DB -> a supervised dataset ----------------------------------

def shape_key(r):
    return (int(r["log2n"]), int(r["limbs"]), int(r["batch"]), int(r.get("bits", 50)))


def dataset(records, inverse=False):
    """Groups DB records by shape: X [S, IN], T [S, OUT] (ln ms), M [S, OUT], keys, times."""
    by = {}
    for r in records:
        if bool(r.get("inverse", False)) != inverse or r["sched"] >= OUT:
            continue
        by.setdefault(shape_key(r), {})[int(r["sched"])] = float(r["ms"])
    keys = sorted(k for k, v in by.items() if len(v) == n_schedules(k[0]))
    X = np.stack([features(*k) for k in keys]) if keys else np.zeros((0, IN), np.float32)
    T = np.zeros((len(keys), OUT), np.float32)
    M = np.zeros((len(keys), OUT), np.float32)
    times = []
    for i, k in enumerate(keys):
        ms = by[k]
        for s, v in ms.items():
            T[i, s] = math.log(v)
            M[i, s] = 1.0
        times.append(ms)
    return X, T, M, keys, times


def split_heldout(keys, n_heldout=100, seed=7):
    rng = np.random.default_rng(seed)
    idx = rng.permutation(len(keys))
    return np.sort(idx[n_heldout:]), np.sort(idx[:n_heldout])


# ---- GPU training through the C ABI ----------------------------------------

def _dev(a, torch):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _vp(t):
    return ctypes.c_void_p(t.data_ptr())


def gpu_forward_backward(p, x, t, m):
    """One forward + backward through the CUDA kernels (for parity tests)."""
    import torch
    L = load()
    st = torch.cuda.current_stream()
    sp = ctypes.c_void_p(st.cuda_stream)
    P, X, T, M = _dev(p, torch), _dev(x, torch), _dev(t, torch), _dev(m, torch)
    b = X.shape[0]
    act = torch.empty((b, N_ACT), dtype=torch.float32, device="cuda")
    grad = torch.empty(N_PARAMS, dtype=torch.float32, device="cuda")
    work = torch.empty(b * (N_ACT + 1), dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    check(L.ntt_mlp_forward(_vp(P), _vp(X), b, _vp(act), sp), "ntt_mlp_forward")
    check(L.ntt_mlp_backward(_vp(P), _vp(X), _vp(act), _vp(T), _vp(M), b, float(np.sum(m)), _vp(grad),
                             _vp(work), _vp(loss), sp), "ntt_mlp_backward")
    torch.cuda.synchronize()
    return (act[:, 2 * H:].cpu().numpy().astype(np.float64), grad.cpu().numpy().astype(np.float64),
            float(loss.item()))


def gpu_adam(p, g, m, v, lr, step, beta1=0.9, beta2=0.999, eps=1e-8):
    import torch
    L = load()
    P, G, Mm, V = _dev(p, torch), _dev(g, torch), _dev(m, torch), _dev(v, torch)
    check(L.ntt_mlp_adam(_vp(P), _vp(G), _vp(Mm), _vp(V), P.numel(), lr, beta1, beta2, eps, step,
                         ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)), "ntt_mlp_adam")
    torch.cuda.synchronize()
    return (P.cpu().numpy().astype(np.float64), Mm.cpu().numpy().astype(np.float64),
            V.cpu().numpy().astype(np.float64))


class CostModel:
    def __init__(self, params=None, meta=None):
        self.params = init_params() if params is None else np.asarray(params, dtype=np.float32)
        self.meta = dict(meta or {})

    # -- training (GPU, library kernels) --
    def fit(self, X, T, M, steps=3000, lr=3e-3, seed=0, log_every=0):
        import torch
        L = load()
        sp = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        self.params = init_params(seed)
        P = _dev(self.params, torch)
        Xd, Td, Md = _dev(X, torch), _dev(T, torch), _dev(M, torch)
        b = Xd.shape[0]
        act = torch.empty((b, N_ACT), dtype=torch.float32, device="cuda")
        grad = torch.empty(N_PARAMS, dtype=torch.float32, device="cuda")
        mom = torch.zeros(N_PARAMS, dtype=torch.float32, device="cuda")
        vel = torch.zeros(N_PARAMS, dtype=torch.float32, device="cuda")
        work = torch.empty(b * (N_ACT + 1), dtype=torch.float32, device="cuda")
        loss = torch.empty(1, dtype=torch.float32, device="cuda")
        count = float(M.sum())
        history = []
        t0 = time.perf_counter()
        for step in range(1, steps + 1):
            check(L.ntt_mlp_forward(_vp(P), _vp(Xd), b, _vp(act), sp), "ntt_mlp_forward")
            check(L.ntt_mlp_backward(_vp(P), _vp(Xd), _vp(act), _vp(Td), _vp(Md), b, count, _vp(grad),
                                     _vp(work), _vp(loss), sp), "ntt_mlp_backward")
            # cosine decay of the learning rate
            lr_t = lr * 0.5 * (1 + math.cos(math.pi * step / steps))
            check(L.ntt_mlp_adam(_vp(P), _vp(grad), _vp(mom), _vp(vel), N_PARAMS, lr_t, 0.9, 0.999, 1e-8, step,
                                 sp), "ntt_mlp_adam")
            if log_every and (step % log_every == 0 or step == steps):
                history.append((step, float(loss.item())))
        torch.cuda.synchronize()
        self.params = P.cpu().numpy()
        self.meta.update(train_steps=steps, lr=lr, train_shapes=int(b), train_seconds=time.perf_counter() - t0,
                         final_loss=float(loss.item()))
        return history

    # -- prediction (host, float32: a 4-64-64-12 forward is a few microseconds) --
    def predict(self, X):
        p = self.params
        o = 0
        W1 = p[o:o + H * IN].reshape(H, IN); o += H * IN
        b1 = p[o:o + H]; o += H
        W2 = p[o:o + H * H].reshape(H, H); o += H * H
        b2 = p[o:o + H]; o += H
        W3 = p[o:o + OUT * H].reshape(OUT, H); o += OUT * H
        b3 = p[o:o + OUT]
        h1 = np.maximum(np.asarray(X, np.float32) @ W1.T + b1, 0)
        h2 = np.maximum(h1 @ W2.T + b2, 0)
        return h2 @ W3.T + b3

    def choose(self, log2n, limbs, batch, bits=50):
        y = self.predict(features(log2n, limbs, batch, bits)[None, :])[0]
        k = n_schedules(log2n)
        return int(np.argmin(y[:k]))

    # -- persistence --
    def save(self, path=DEFAULT_PARAMS):
        os.makedirs(os.path.dirname(path), exist_ok=True)
        np.savez(path, params=self.params, meta=json.dumps(self.meta))

    @classmethod
    def load(cls, path=DEFAULT_PARAMS):
        z = np.load(path, allow_pickle=False)
        return cls(z["params"], json.loads(str(z["meta"])))


# ---- evaluation --------------------------------------------------------------

def heuristic_choice(log2n, limbs, batch, sms=152):
    """The paper's SM-aware rule (Sec. V-D) restated for these schedules: the
    first kernel's number of independent chunks (CTAs, or tile groups of a
    persistent kernel) closest to the SM count; fewer kernels on ties."""
    rows = limbs * batch
    best, best_score = 0, None
    for s in range(n_schedules(log2n)):
        p = _ntt.schedule_params(log2n, s)
        if p["kernels"] == 1:
            chunks = math.ceil(rows / p["tpc"])
        else:
            cols = 1 << p["logp"]
            tiles = rows * (1 << (log2n - p["split"])) // cols
            chunks = math.ceil(tiles / p["tpc_col"])
        score = (abs(math.log2(max(chunks, 1) / sms)), p["kernels"])
        if best_score is None or score < best_score:
            best, best_score = s, score
    return best


def default_choice(log2n, limbs, batch):
    """The library's built-in default (ntt_plan's choice before any tuning)."""
    return int(load().ntt_default_schedule(log2n, limbs * batch))


def regret(times, choice):
    """t(chosen) / t(best) - 1 for one shape's measured times {sched: ms}."""
    best = min(times.values())
    return times[choice] / best - 1.0


def regret_report(keys, times, chooser):
    r = np.array([regret(t, chooser(*k)) for k, t in zip(keys, times)])
    return {"mean": float(r.mean()), "p90": float(np.percentile(r, 90)), "max": float(r.max()),
            "exact": float((r == 0).mean()), "n": int(r.size)}


_CACHE = {}


def choose_schedule(log2n, limbs, batch, bits=50, inverse=False, db=DEFAULT_DB, params=DEFAULT_PARAMS):
    """Schedule for a shape: the exhaustive autotuner result when the timing DB
    holds this exact shape, else the cost model's prediction, else the
    library default.  Returns (schedule id, source)."""
    from .tune import load_db, schedule_signature
    if "db" not in _CACHE:
        _CACHE["db"] = {}
        for r in load_db(db, current=True):
            k = shape_key(r) + (bool(r.get("inverse", False)),)
            best = _CACHE["db"].get(k)
            if best is None or r["ms"] < best[1]:
                _CACHE["db"][k] = (int(r["sched"]), float(r["ms"]))
    hit = _CACHE["db"].get((log2n, limbs, batch, bits, bool(inverse)))
    if hit is not None:
        return hit[0], "autotuner"
    if "model" not in _CACHE:
        m = CostModel.load(params) if os.path.exists(params) else None
        _CACHE["model"] = m if m is not None and m.params.size == N_PARAMS else None   # another layer width
    model = _CACHE["model"]
    if model is not None and not inverse and model.meta.get("sigs", {}).get(str(log2n)) == schedule_signature(log2n):
        return model.choose(log2n, limbs, batch, bits), "cost_model"
    return default_choice(log2n, limbs, batch), "default"


def schedule_requests(requests, moduli_pool, min_log2_coef=22):
    """Mixed-batch requests with their `schedule` field set: requests of at
    least 2^min_log2_coef coefficients fill the GPU by themselves and run as
    their own launches with the schedule chosen here (autotuner hit, else the
    cost model, else the default) + 1; the rest stay work items (0) of the
    persistent kernel."""
    out = []
    for r in requests:
        r = dict(r)
        rows = int(r["n_polys"]) * int(r["n_moduli"])
        if rows << int(r["log2n"]) >= 1 << min_log2_coef:
            off = int(r.get("moduli_offset", 0))
            bits = max(int(q).bit_length() for q in moduli_pool[off:off + int(r["n_moduli"])])
            sid, _ = choose_schedule(int(r["log2n"]), int(r["n_moduli"]), int(r["n_polys"]), bits,
                                     inverse=bool(r.get("inverse", 0)))
            r["schedule"] = sid + 1
        else:
            r["schedule"] = 0
        out.append(r)
    return out


def evaluate(model, keys, times):
    """Regret of the model, the paper's SM-aware rule and the built-in default."""
    t0 = time.perf_counter()
    for k in keys:
        model.choose(*k)
    decide_us = (time.perf_counter() - t0) / max(1, len(keys)) * 1e6
    return {
        "mlp": regret_report(keys, times, model.choose),
        "sm_rule": regret_report(keys, times, lambda n, l, b, bits: heuristic_choice(n, l, b)),
        "default": regret_report(keys, times, lambda n, l, b, bits: default_choice(n, l, b)),
        "decision_us": decide_us,
    }


def load_db_default():
    from .tune import load_db
    return load_db(DEFAULT_DB, current=True)


def train_and_evaluate(db=DEFAULT_DB, n_heldout=100, steps=16000, lr=3e-3, seed=0, split_seed=7):
    from .tune import load_db, schedule_signature
    recs = load_db(db, current=True)
    X, T, M, keys, times = dataset(recs)
    tr, ho = split_heldout(keys, n_heldout, split_seed)
    model = CostModel(meta={"db": os.path.basename(db), "records": len(recs), "shapes": len(keys),
                            "heldout": int(len(ho)), "split_seed": split_seed,
                            "gpu": recs[0]["gpu"] if recs else None, "build": recs[0]["build"] if recs else None,
                            "sigs": {str(n): schedule_signature(n) for n in sorted({int(r["log2n"]) for r in recs})}})
    model.fit(X[tr], T[tr], M[tr], steps=steps, lr=lr, seed=seed)
    report = evaluate(model, [keys[i] for i in ho], [times[i] for i in ho])
    report["train"] = {k: model.meta[k] for k in ("train_steps", "train_shapes", "train_seconds", "final_loss")}
    report["timings"] = len(recs)
    return model, report


def main():
    import argparse
    ap = argparse.ArgumentParser(description="train the schedule cost model on the GPU and report regret")
    ap.add_argument("--db", default=DEFAULT_DB)
    ap.add_argument("--out", default=DEFAULT_PARAMS)
    ap.add_argument("--steps", type=int, default=16000)
    ap.add_argument("--heldout", type=int, default=100)
    args = ap.parse_args()
    model, report = train_and_evaluate(args.db, args.heldout, args.steps)
    model.meta["report"] = report
    model.save(args.out)
    print(json.dumps(report))


if __name__ == "__main__":
    main()
