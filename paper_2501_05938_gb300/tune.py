"""Launch-parameter tuning: timing sweeps, predictor training, regret.

  collect  time the solver on this GPU over the parameter grid: block size m
           for device-resident single and batched solves, stream count S and
           chunk size for the host-resident pipeline, fp64 (double-float) and
           fp32, n = 2^10 .. 2^28 and 3 * 2^k; writes a CSV
  train    per point the fastest configuration (exhaustive search) is the
           target; the MLP (4 -> 64 -> 64 -> 3, ReLU) is trained on the
           GPU with libtps's CUDA kernels (tps_mlp_loss_backward,
           tps_mlp_adam_step) on the training points; writes weights.bin
  evaluate regret T(choice)/T(best) - 1 on held-out points (odd exponents,
           3 * 2^k sizes, an unseen batch count) for the MLP, for the paper's
           stream rule (Eq. 4, 6, 7) refit on this GPU's timings, and for the
           fixed defaults
  paper    the paper's own modelling pipeline on this GPU's host-pipeline
           timings: sum model, both overhead models, their R-squared / MSE /
           RMSE on a shuffled 3:1 split, and the rule's stream counts against
           the measured optimum per size; writes paper_models_gb300.json

  solve    repeated solves of one synthetic system with given parameters
           (for a profiler to capture, or a quick timing of one setting):
           solve [--n N] [--dtype f64_df] [--m M] [--m-reduced H]
                 [--truncate] [--no-onchip] [--repeat K]

Usage: python -m paper_2501_05938_gb300.tune collect|train|evaluate|paper|all [dir]
       python -m paper_2501_05938_gb300.tune solve [options]
"""
from __future__ import annotations

import csv
import ctypes
import json
import math
import os
import struct
import sys
import time

import numpy as np

from . import binding

HERE = os.path.dirname(os.path.abspath(__file__))
PRED_DIR = os.path.join(HERE, "predictor")

M_GRID = (8, 16, 32, 64, 128, 256, 512, 1024)
S_GRID = (1, 2, 4, 8, 16, 32)
CHUNK_GRID = (0, 1 << 18, 1 << 20, 1 << 22, 1 << 24)  # 0: n/S rows per chunk
M_HOST = 128
BATCHES = (16, 256, 1024, 4096)
HELD_OUT_BATCH = 1024
DTYPES = {"f64_df": 0, "f32": 1}
FIELDS = ("kind", "n", "batch", "dtype", "residency", "m", "S", "chunk", "ms", "s13_ms")


def sizes():
    out = [1 << k for k in range(10, 29)]
    out += [3 << k for k in (12, 16, 20, 24)]
    return sorted(out)


def held_out(rec):
    n, batch = int(rec["n"]), int(rec["batch"])
    if batch == HELD_OUT_BATCH:
        return True
    if batch > 1:
        return False
    k = math.log2(n)
    return (k != int(k)) or (int(k) % 2 == 1)


# ---------------------------------------------------------------------------
# collect
# ---------------------------------------------------------------------------
def _time(fn, stream, budget_ms=30.0, min_reps=3, max_reps=50, rounds=2):
    """Mean time of `reps` back-to-back calls, the best of `rounds` rounds."""
    import torch

    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    fn()
    e1.record(stream)
    torch.cuda.synchronize()
    est = max(e0.elapsed_time(e1), 1e-3)
    reps = int(min(max_reps, max(min_reps, budget_ms / est)))
    best = None
    for _ in range(rounds):
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / reps
        best = t if best is None else min(best, t)
    return best


def collect(path, log=print):
    import torch

    from . import synth

    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    nmax = max(sizes())
    g = synth.system_device(2024, nmax)
    dev = {"f64_df": {k: g[k] for k in "abcd"}}
    dev["f32"] = {k: g[k].float() for k in "abcd"}
    xs = {"f64_df": torch.empty(nmax, dtype=torch.float64, device="cuda"),
          "f32": torch.empty(nmax, dtype=torch.float32, device="cuda")}
    rows = []
    t0 = time.time()
    # device-resident single systems: block size
    for dt in DTYPES:
        for n in sizes():
            a, b, c, d = (dev[dt][k][:n] for k in "abcd")
            x = xs[dt][:n]
            for m in M_GRID:
                plan = binding.Plan(n, dtype=dt, m=m, m_reduced=32,
                                    flags=binding.TRACE | binding.GRAPH)
                ms = _time(lambda: plan.solve(a, b, c, d, x, stream=stream), stream)
                st = plan.query()["stage_ms"]
                rows.append(dict(kind="device", n=n, batch=1, dtype=DTYPES[dt], residency=0,
                                 m=m, S=1, chunk=0, ms=ms, s13_ms=st[0] + st[2]))
                plan.close()
        log(f"device {dt} done {time.time() - t0:.0f}s")
    # device-resident batches: block size
    for dt in DTYPES:
        for batch in BATCHES:
            sz = synth.batch_sizes(3000 + batch, batch, 8, 20)
            off = synth.offsets_from_sizes(sz)
            n = int(off[-1])
            gb = synth.system_device(3000 + batch, n, offsets=off)
            tdt = torch.float32 if dt == "f32" else torch.float64
            a, b, c, d = (gb[k].to(tdt) for k in "abcd")
            del gb
            x = torch.empty(n, dtype=tdt, device="cuda")
            offs = torch.as_tensor(off, device="cuda")
            for m in M_GRID:
                plan = binding.Plan(n, dtype=dt, m=m, m_reduced=32, batch_max=batch,
                                    flags=binding.GRAPH)
                ms = _time(lambda: plan.solve_batched(offs, a, b, c, d, x, host_offsets=off,
                                                      stream=stream), stream)
                rows.append(dict(kind="batched", n=n, batch=batch, dtype=DTYPES[dt],
                                 residency=0, m=m, S=1, chunk=0, ms=ms, s13_ms=0.0))
                plan.close()
            del a, b, c, d, x
        log(f"batched {dt} done {time.time() - t0:.0f}s")
    # host-resident pipeline: streams and chunk size
    for dt in DTYPES:
        hk = {k: dev[dt][k].cpu().pin_memory() for k in "abcd"}
        hx = torch.empty(nmax, dtype=hk["b"].dtype).pin_memory()
        for n in sizes():
            a, b, c, d = (hk[k][:n] for k in "abcd")
            x = hx[:n]
            for S in S_GRID:
                for chunk in CHUNK_GRID:
                    if chunk and chunk * 2 > n:
                        continue
                    plan = binding.Plan(n, dtype=dt, residency="host", m=M_HOST, streams=S,
                                        chunk=chunk)
                    ms = _time(lambda: plan.solve_host_async(a, b, c, d, x, stream=stream),
                               stream, budget_ms=20.0, max_reps=20)
                    rows.append(dict(kind="host", n=n, batch=1, dtype=DTYPES[dt], residency=1,
                                     m=M_HOST, S=S, chunk=chunk, ms=ms, s13_ms=0.0))
                    plan.close()
        del hk, hx
        log(f"host {dt} done {time.time() - t0:.0f}s")
    with open(path, "w", newline="") as f:
        w = csv.DictWriter(f, fieldnames=FIELDS)
        w.writeheader()
        for r in rows:
            w.writerow(r)
    return rows


def load(path):
    with open(path) as f:
        return [{k: (float(v) if k in ("ms", "s13_ms") else (v if k == "kind" else int(v)))
                 for k, v in r.items()} for r in csv.DictReader(f)]


# ---------------------------------------------------------------------------
# dataset
# ---------------------------------------------------------------------------
def points(rows):
    """Group timings by point (kind, n, batch, dtype, residency)."""
    pts = {}
    for r in rows:
        key = (r["kind"], r["n"], r["batch"], r["dtype"], r["residency"])
        pts.setdefault(key, []).append(r)
    return pts


def chunk_eff(n, S, chunk):
    return chunk if chunk > 0 else -(-n // S)


def features(n, batch, dtype, residency):
    return [math.log2(max(n, 2)), math.log2(max(batch, 1)), float(dtype), float(residency)]


def target(best):
    n = best["n"]
    return [math.log2(best["m"]), math.log2(best["S"]),
            math.log2(chunk_eff(n, best["S"], best["chunk"]))]


def dataset(rows, train=True):
    X, T, keys = [], [], []
    for key, recs in sorted(points(rows).items()):
        if held_out(recs[0]) == train:
            continue
        best = min(recs, key=lambda r: r["ms"])
        X.append(features(key[1], key[2], key[3], key[4]))
        T.append(target(best))
        keys.append(key)
    return np.array(X, dtype=np.float64), np.array(T, dtype=np.float64), keys


# ---------------------------------------------------------------------------
# train (on the GPU, with libtps's kernels)
# ---------------------------------------------------------------------------
def _mlp_lib():
    L = binding.lib()
    P, I32 = ctypes.c_void_p, ctypes.c_int32
    L.tps_mlp_workspace_floats.argtypes = [I32]
    L.tps_mlp_workspace_floats.restype = ctypes.c_size_t
    L.tps_mlp_forward.argtypes = [P, I32, P, P, P, P]
    L.tps_mlp_loss_backward.argtypes = [P, I32, P, P, P, P, P, P]
    L.tps_mlp_adam_step.argtypes = [P, P, P, P, I32, ctypes.c_float, ctypes.c_float,
                                    ctypes.c_float, ctypes.c_float, P]
    for f in ("tps_mlp_forward", "tps_mlp_loss_backward", "tps_mlp_adam_step"):
        getattr(L, f).restype = ctypes.c_int
    return L


def init_params(seed=0):
    rng = np.random.default_rng(seed)
    dims = (4, 64, 64, 3)
    parts = []
    for i in range(3):
        lim = math.sqrt(6.0 / dims[i])
        parts.append(rng.uniform(-lim, lim, size=(dims[i + 1], dims[i])).ravel())
        parts.append(np.zeros(dims[i + 1]))
    return np.concatenate(parts).astype(np.float32)


def train(rows, out_path, steps=4000, lr=3e-3, seed=0, log=print):
    import torch

    X, T, _ = dataset(rows, train=True)
    fmean = X.mean(axis=0)
    fstd = X.std(axis=0)
    fscale = np.where(fstd > 0, 1.0 / np.where(fstd > 0, fstd, 1.0), 1.0)
    oscale = np.array([10.0, 5.0, 28.0])
    Xn = ((X - fmean) * fscale).astype(np.float32)
    Tn = (T / oscale).astype(np.float32)
    L = _mlp_lib()
    dev = torch.device("cuda")
    p = torch.as_tensor(init_params(seed), device=dev)
    g = torch.zeros_like(p)
    m1 = torch.zeros_like(p)
    v1 = torch.zeros_like(p)
    x = torch.as_tensor(Xn, device=dev)
    t = torch.as_tensor(Tn, device=dev)
    B = x.shape[0]
    work = torch.empty(int(L.tps_mlp_workspace_floats(B)), dtype=torch.float32, device=dev)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    ptr = lambda z: ctypes.c_void_p(z.data_ptr())
    hist = []
    for it in range(1, steps + 1):
        binding.check(L.tps_mlp_loss_backward(ptr(p), B, ptr(x), ptr(t), ptr(g), ptr(loss),
                                              ptr(work), st), "tps_mlp_loss_backward")
        lr_t = 0.5 * lr * (1.0 + math.cos(math.pi * (it - 1) / steps))  # cosine decay
        binding.check(L.tps_mlp_adam_step(ptr(p), ptr(g), ptr(m1), ptr(v1), it, lr_t, 0.9,
                                          0.999, 1e-8, st), "tps_mlp_adam_step")
        if it % 500 == 0 or it == 1:
            hist.append((it, float(loss.item())))
            log(f"step {it} loss {hist[-1][1]:.3e}")
    params = p.cpu().numpy()
    os.makedirs(os.path.dirname(out_path) or ".", exist_ok=True)
    with open(out_path, "wb") as f:
        f.write(b"TPSMLP1\0")
        f.write(struct.pack("<i", params.size))
        f.write(fmean.astype("<f4").tobytes())
        f.write(fscale.astype("<f4").tobytes())
        f.write(oscale.astype("<f4").tobytes())
        f.write(params.astype("<f4").tobytes())
    return hist


# ---------------------------------------------------------------------------
# evaluate
# ---------------------------------------------------------------------------
def _predict(desc_kw):
    d = binding.PlanDesc(**desc_kw)
    m, S, c = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
    L = binding.lib()
    L.tps_predict_params.argtypes = [ctypes.POINTER(binding.PlanDesc), ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_void_p]
    L.tps_predict_params.restype = ctypes.c_int
    rc = L.tps_predict_params(ctypes.byref(d), ctypes.byref(m), ctypes.byref(S),
                              ctypes.byref(c))
    if rc != 0:
        raise RuntimeError("predictor weights not loaded")
    return m.value, S.value, c.value


def _lookup(recs, m=None, S=None, chunk=None):
    """Time of the grid configuration nearest the requested one; records
    that describe the same configuration (a chunk of n/S rows given as 0 or
    explicitly) count as one, at their best time."""
    def cfg(r):
        return (r["m"], r["S"], chunk_eff(r["n"], r["S"], r["chunk"]))

    def dist(r):
        dm, dS, dc = cfg(r)
        v = 0.0
        if m is not None:
            v += abs(math.log2(dm) - math.log2(m))
        if S is not None:
            v += abs(math.log2(dS) - math.log2(S))
        if chunk is not None:
            v += 1e-3 * abs(math.log2(dc) - math.log2(chunk_eff(r["n"], S or dS, chunk)))
        return v

    dmin = min(dist(r) for r in recs)
    near = [r for r in recs if dist(r) == dmin]
    c0 = cfg(near[0])
    return min(r["ms"] for r in recs if cfg(r) == c0)


def paper_rule_coeffs(rows):
    """Eq. 4 and Eq. 7 refit on this GPU's training timings (fp64, host
    pipeline, one chunk per stream): sum = the Stage-1 + Stage-3 kernel time
    at m = 128 (the work the streams overlap), T_overhead from Eq. 5."""
    sums = {}
    for r in rows:
        if r["kind"] == "device" and r["m"] == M_HOST and not held_out(r):
            sums[(r["n"], r["dtype"])] = r["s13_ms"]
    xs, ys = [], []
    for (n, dt), s in sums.items():
        if dt == 0:
            xs.append(n)
            ys.append(s)
    A = np.stack([np.array(xs, float), np.ones(len(xs))], axis=1)
    k_sum, q_sum = np.linalg.lstsq(A, np.array(ys), rcond=None)[0]
    small, big = [], []
    for key, recs in points(rows).items():
        kind, n, batch, dt, res = key
        if kind != "host" or dt != 0 or held_out(recs[0]):
            continue
        t1 = [r["ms"] for r in recs if r["S"] == 1 and r["chunk"] == 0]
        if not t1:
            continue
        s = k_sum * n + q_sum
        for r in recs:
            if r["chunk"] == 0 and r["S"] > 1:
                ov = (r["ms"] - t1[0]) + (r["S"] - 1) / r["S"] * s  # Eq. 5
                (small if n <= 1e6 else big).append((n, r["S"], ov))
    def lsq(cols, y):
        return np.linalg.lstsq(np.stack(cols, axis=1), np.array(y), rcond=None)[0]
    sm = np.array([x[0] for x in small], float)
    ss = np.array([x[1] for x in small], float)
    co_small = lsq([sm, np.log10(ss), np.ones_like(sm)], [x[2] for x in small])
    bn = np.array([x[0] for x in big], float)
    bs = (4.0 / 3.0) * np.log2(np.array([x[1] for x in big], float))
    co_big = lsq([bn * bs, bs, np.ones_like(bn)], [x[2] for x in big])
    return np.array([k_sum, q_sum]), co_small, co_big


def paper_rule_streams(n, coeffs):
    """The rule of Eq. 6 with the models of Eq. 4 and Eq. 7, evaluated in
    libtps; coeffs None: the paper's RTX 2080 Ti coefficients."""
    L = binding.lib()
    L.tps_paper_predict_streams.argtypes = [ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_void_p, ctypes.c_double]
    L.tps_paper_predict_streams.restype = ctypes.c_int32
    if coeffs is None:
        return int(L.tps_paper_predict_streams(float(n), None, None, None, 1e6))
    s, sm, bg = (np.ascontiguousarray(c, dtype=np.float64) for c in coeffs)
    return int(L.tps_paper_predict_streams(float(n), s.ctypes.data, sm.ctypes.data,
                                           bg.ctypes.data, 1e6))


def default_params(n, residency):
    """The library's defaults (tps_plan with zero parameters, no predictor)."""
    m = 128
    while m > 8 and n // m < 152 * 32 * 4:
        m //= 2
    return m, (4 if residency else 1), 0


def evaluate(rows, weights_path):
    L = binding.lib()
    L.tps_predict_load.argtypes = [ctypes.c_char_p]
    if L.tps_predict_load(weights_path.encode()) != 0:
        raise RuntimeError(f"cannot load {weights_path}")
    coeffs = paper_rule_coeffs(rows)
    res = {"mlp": [], "paper_rule": [], "defaults": []}
    detail = []
    for key, recs in sorted(points(rows).items()):
        if not held_out(recs[0]):
            continue
        kind, n, batch, dt, resid = key
        tbest = min(r["ms"] for r in recs)
        pm, pS, pc = _predict(dict(n_max=n, batch_max=batch if batch > 1 else 0,
                                   dtype=(1 if dt == 1 else 3), residency=resid))
        dm, dS, dc = default_params(n, resid)
        if kind == "host":
            t_mlp = _lookup(recs, S=pS, chunk=pc)
            t_def = _lookup(recs, S=dS, chunk=dc)
            t_pap = _lookup(recs, S=paper_rule_streams(n, coeffs), chunk=0)
        else:
            t_mlp = _lookup(recs, m=pm)
            t_def = _lookup(recs, m=dm)
            t_pap = t_def  # the paper's rule chooses only S
        res["mlp"].append(t_mlp / tbest - 1)
        res["defaults"].append(t_def / tbest - 1)
        res["paper_rule"].append(t_pap / tbest - 1)
        detail.append(dict(kind=kind, n=n, batch=batch, dtype=dt, best_ms=tbest,
                           mlp=t_mlp / tbest - 1, defaults=t_def / tbest - 1,
                           paper_rule=t_pap / tbest - 1, pred=(pm, pS, pc)))
    summary = {k: {"mean": float(np.mean(v)), "max": float(np.max(v)), "points": len(v)}
               for k, v in res.items()}
    return summary, detail, coeffs


# ---------------------------------------------------------------------------
# the paper's modelling pipeline (Sec. 2.4, Tables 4 and 6) on this GPU
# ---------------------------------------------------------------------------
SPLIT_SEED = 2025


def _split(count, seed):
    """Shuffled 3:1 train/test split of `count` samples (indices)."""
    perm = np.random.RandomState(seed).permutation(count)
    cut = (3 * count + 3) // 4
    return perm[:cut], perm[cut:]


def _metrics(y, yhat):
    y, yhat = np.asarray(y, float), np.asarray(yhat, float)
    mse = float(np.mean((y - yhat) ** 2))
    tot = float(np.sum((y - y.mean()) ** 2))
    r2 = 1.0 - float(np.sum((y - yhat) ** 2)) / tot if tot > 0 else 0.0
    return {"r2": r2, "mse": mse, "rmse": math.sqrt(mse), "samples": int(len(y))}


def _lsq(cols, y):
    return np.linalg.lstsq(np.stack(cols, axis=1), np.asarray(y, float), rcond=None)[0]


def paper_samples(rows, dtype=0):
    """Per size: the overlapped sum (Eq. 3: the Stage-1 and Stage-3 kernel
    time; the reduced transfers of the paper's CPU Stage 2 do not exist
    here), T_non_str (one stream, one chunk) and T_str(S) (S streams, one
    chunk per stream), from the host-pipeline sweep."""
    sums = {r["n"]: r["s13_ms"] for r in rows
            if r["kind"] == "device" and r["m"] == M_HOST and r["dtype"] == dtype}
    t = {}
    for r in rows:
        if r["kind"] == "host" and r["dtype"] == dtype and r["chunk"] == 0 and r["n"] in sums:
            t.setdefault(r["n"], {})[r["S"]] = r["ms"]
    return {n: {"sum": sums[n], "t": t[n]} for n in sorted(t) if 1 in t[n]}


def paper_models(rows, dtype=0, seed=SPLIT_SEED, split=1e6):
    """Eq. 4 (linear sum model) and the two Eq. 7 forms (T_overhead of Eq. 5,
    small for size <= 1e6, big above) fitted on a shuffled 3:1 split, their
    R-squared / MSE / RMSE on both sets, and the rule of Eq. 6 with the
    fitted models against the measured optimum stream count per size.  The
    preset forms are linear in their coefficients, so least squares gives
    the coefficients a curve fit converges to."""
    smp = paper_samples(rows, dtype)
    ns = np.array(sorted(smp), float)
    sums = np.array([smp[int(n)]["sum"] for n in ns])
    tr, te = _split(len(ns), seed)
    k, q = _lsq([ns[tr], np.ones(len(tr))], sums[tr])
    sum_fit = {"coeffs": [float(k), float(q)],
               "train": _metrics(sums[tr], k * ns[tr] + q),
               "test": _metrics(sums[te], k * ns[te] + q)}
    # Eq. 5 per (size, S > 1), with the measured sum
    ov = {"small": [], "big": []}
    for n in sorted(smp):
        t1, sm = smp[n]["t"][1], smp[n]["sum"]
        for S, ts in sorted(smp[n]["t"].items()):
            if S > 1:
                ov["small" if n <= split else "big"].append(
                    (float(n), float(S), (ts - t1) + (S - 1) / S * sm))
    forms = {
        "small": lambda n, S: [n, np.log10(S), np.ones_like(n)],
        "big": lambda n, S: [n * (4.0 / 3.0) * np.log2(S), (4.0 / 3.0) * np.log2(S),
                             np.ones_like(n)],
    }
    ov_fit = {}
    for name, pts in ov.items():
        a = np.array(pts, float)
        tr2, te2 = _split(len(a), seed + (1 if name == "big" else 0))
        co = _lsq(forms[name](a[tr2, 0], a[tr2, 1]), a[tr2, 2])
        pred = lambda idx: np.stack(forms[name](a[idx, 0], a[idx, 1]), axis=1) @ co
        ov_fit[name] = {"coeffs": [float(c) for c in co], "train": _metrics(a[tr2, 2], pred(tr2)),
                        "test": _metrics(a[te2, 2], pred(te2))}
    coeffs = (np.array(sum_fit["coeffs"]), np.array(ov_fit["small"]["coeffs"]),
              np.array(ov_fit["big"]["coeffs"]))
    table = []
    for n in sorted(smp):
        t = smp[n]["t"]
        act = min(t, key=t.get)
        pre = paper_rule_streams(n, coeffs)
        pre_2080 = paper_rule_streams(n, None)
        table.append({"n": n, "N_act": act, "N_pre": pre, "N_pre_2080ti": pre_2080,
                      "T1_ms": t[1], "T_act_ms": t[act], "T_pre_ms": t.get(pre, float("nan")),
                      "speedup_act": t[1] / t[act], "regret_pre": t.get(pre, float("nan")) / t[act] - 1,
                      "regret_pre_2080ti": t.get(pre_2080, float("nan")) / t[act] - 1})
    return {"dtype": dtype, "seed": seed, "split": split, "sum_model": sum_fit,
            "overhead_small": ov_fit["small"], "overhead_big": ov_fit["big"], "table": table}


def solve_cmd(args):
    """K solves of one paper system (device generator) with the given plan
    parameters; prints the last solve's mean time and the plan's report."""
    import argparse

    import torch

    from . import binding, synth

    ap = argparse.ArgumentParser(prog="tune solve")
    ap.add_argument("--n", type=int, default=1 << 24)
    ap.add_argument("--dtype", default="f64_df", choices=list(binding.DTYPES))
    ap.add_argument("--m", type=int, default=0)
    ap.add_argument("--m-reduced", type=int, default=0)
    ap.add_argument("--truncate", action="store_true")
    ap.add_argument("--no-onchip", action="store_true")
    ap.add_argument("--repeat", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=0)
    ap.add_argument("--trace", action="store_true",
                    help="per-stage event times (mean over the timed solves)")
    a = ap.parse_args(args)
    g = synth.system_device(1002, a.n)
    tdt = torch.float32 if a.dtype == "f32" else torch.float64
    arrs = [g[k].to(tdt) for k in "abcd"]
    x = torch.empty_like(arrs[1])
    flags = (binding.TRUNCATE if a.truncate else 0) | (binding.NO_ONCHIP if a.no_onchip else 0)
    flags |= binding.TRACE if a.trace else 0
    plan = binding.Plan(a.n, dtype=a.dtype, m=a.m, m_reduced=a.m_reduced, flags=flags)
    for _ in range(a.warmup):
        plan.solve(*arrs, x)
    if a.warmup:
        plan.query()  # the trace averages over the timed solves only
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(a.repeat):
        plan.solve(*arrs, x)
    e1.record()
    torch.cuda.synchronize()
    info = plan.query()
    print(json.dumps({"n": a.n, "dtype": a.dtype, "ms_per_solve": e0.elapsed_time(e1) / a.repeat,
                      "status": info["status_name"], "m": info["m"],
                      "m_reduced": info["m_reduced"], "bound": info["last_correction"],
                      **({"stage_ms": info["stage_ms"]} if a.trace else {})}))
    return 0 if info["status"] == 0 else 1


def main(argv):
    cmd = argv[1] if len(argv) > 1 else "all"
    if cmd == "solve":
        sys.exit(solve_cmd(argv[2:]))
    out = argv[2] if len(argv) > 2 else PRED_DIR
    os.makedirs(out, exist_ok=True)
    csv_path = os.path.join(out, "timings_gb300.csv")
    w_path = os.path.join(out, "weights.bin")
    if cmd in ("collect", "all"):
        collect(csv_path)
    rows = load(csv_path)
    if cmd in ("train", "all"):
        hist = train(rows, w_path)
        with open(os.path.join(out, "train_log.json"), "w") as f:
            json.dump(hist, f)
    if cmd in ("evaluate", "all"):
        summary, detail, coeffs = evaluate(rows, w_path)
        with open(os.path.join(out, "regret.json"), "w") as f:
            json.dump({"summary": summary, "detail": detail,
                       "paper_rule_coeffs": [list(map(float, c)) for c in coeffs]}, f, indent=1)
        print(json.dumps(summary))
    if cmd in ("paper", "all"):
        res = paper_models(rows)
        with open(os.path.join(out, "paper_models_gb300.json"), "w") as f:
            json.dump(res, f, indent=1)
        for k in ("sum_model", "overhead_small", "overhead_big"):
            print(k, json.dumps({s: res[k][s] for s in ("coeffs", "train", "test")}))
        for r in res["table"]:
            print(r["n"], r["N_act"], r["N_pre"], r["N_pre_2080ti"], round(r["speedup_act"], 3),
                  round(r["regret_pre"], 4))


if __name__ == "__main__":
    main(sys.argv)
