"""Learned planner: train the plan cost model on timings the planner
measures, and score its choices against exhaustive empirical search.

The paper ranks fusion implementations with an additive predictor of
benchmarked routine times and can search them empirically (Section 3.2; the
predictor's accuracy is tabulated in Section 4.3).  Here a 3-layer
perceptron (16 plan features -> 64 -> 64 -> 1, ReLU) predicts log plan time;
its forward, backward and Adam steps are libkf kernels (kf_mlp_*), and
kf_plan_select uses it to rank every enumerated plan and re-time only the
best-ranked few.

Data.  Random scripts (synth.scripts) of 6-10 calls over shared vectors and
matrices, n = 2^k with k drawn per script in [kmin, kmax].  For a training
script up to `per_script` plans are timed (kf_plan_time on the bound data):
all of them when there are that few, else the best-predicted half by the
analytic model, the fewest-kernel plan, the one-kernel-per-call plan and a
seeded uniform sample of the rest.

Scoring.  For a held-out script every enumerated plan is timed
(kf_plan_time_all); each method's choice is scored by t(choice) / t(best)
on that table: the MLP's first choice (no timing), the MLP's top-k re-timed
(kf_plan_select, KF_SELECT_MLP), the analytic model, the fewest-kernel plan
and the unfused chain.

    python -m paper_1305_1183_gb300.learn --scripts 500 --train 400 --out learned.json
"""

from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import synth  # noqa: E402
from synth import scripts as sscripts  # noqa: E402

from . import kf  # noqa: E402


def to_script(sd):
    s = kf.Script()
    for name, spec in sd["vars"].items():
        if spec[0] == "v":
            s.vector(name, spec[1])
        elif spec[0] == "m":
            s.matrix(name, spec[1], spec[2])
        else:
            s.scalar(name)
    s.input(*sd["inputs"])
    s.output(*sd["outputs"])
    for op, outs, ins, sc in sd["calls"]:
        s.call(op, outs, ins, sc)
    return s


def bindings(sd, seed, device):
    out = {}
    for i, (name, spec) in enumerate(sorted(sd["vars"].items())):
        shape = (spec[1],) if spec[0] == "v" else ((spec[1], spec[2]) if spec[0] == "m" else (1,))
        out[name] = synth.uniform(shape, seed, 300 + i, device=device)
    return out


def script_size(seed, index, kmin, kmax):
    u = synth.uniform_scalar(seed, synth.TID["sizes"], index) * 0.5 + 0.5
    return 1 << (kmin + min(int(u * (kmax - kmin + 1)), kmax - kmin))


def make(seed, i, kmin, kmax):
    n = script_size(seed, i, kmin, kmax)
    sd = sscripts.random_script(seed, i, n)
    return n, sd, to_script(sd)


def training_subset(seed, i, pred, nk, ncalls, per_script):
    count = len(pred)
    if count <= per_script:
        return list(range(count))
    chosen = [int(j) for j in np.argsort(pred, kind="stable")[: per_script // 2]]
    greedy = int(np.argmin(nk))
    unfused = [j for j in range(count) if nk[j] == ncalls]
    for j in [greedy] + unfused[:1]:
        if j not in chosen:
            chosen.append(j)
    rest = [j for j in range(count) if j not in chosen]
    k = 0
    while len(chosen) < per_script and rest:
        u = synth.uniform_scalar(seed + 1, synth.TID["script"], i * 1000 + k) * 0.5 + 0.5
        chosen.append(rest.pop(min(int(u * len(rest)), len(rest) - 1)))
        k += 1
    return sorted(chosen)


def collect(seed, indices, kmin, kmax, per_script, reps, cap=2000, device="cuda"):
    """Training data: features and measured ms of a subset of each script's plans."""
    X, y, pu, sid, meta = [], [], [], [], []
    for i in indices:
        n, sd, s = make(seed, i, kmin, kmax)
        feats, pred, nk = s.enumerate_info(cap)
        chosen = training_subset(seed, i, pred, nk, len(sd["calls"]), per_script)
        bind = bindings(sd, i, device)
        ws = None
        for j in chosen:
            p = s.plan(kf.KF_PLAN_INDEX, index=j, max_plans=cap)
            need = max(p.workspace_size(), 256)
            if ws is None or ws.numel() < need:
                ws = torch.zeros(need, dtype=torch.uint8, device=device)
            X.append(feats[j])
            pu.append(pred[j])
            sid.append(int(i))
            y.append(p.time(bind, ws, reps=reps))
        meta.append({"index": int(i), "n": n, "calls": len(sd["calls"]), "plans": len(pred), "timed": len(chosen)})
        del bind, ws
    return (np.array(X, dtype=np.float64), np.array(y, dtype=np.float64), np.array(pu, dtype=np.float64),
            np.array(sid, dtype=np.int64), meta)


def timing_key(seed, indices, kmin, kmax, per_script, reps, device):
    """What a plan-timing table was measured on.  A stored table is reused
    only under the same key: timings belong to one device and one workload."""
    if torch.cuda.is_available() and str(device).startswith("cuda"):
        dev = torch.cuda.get_device_name(torch.device(device))
    else:
        dev = str(device)
    return {"seed": int(seed), "indices": [int(i) for i in indices], "kmin": int(kmin), "kmax": int(kmax),
            "per_script": int(per_script), "reps": int(reps), "device": dev}


def save_timings(path, key, X, ms, pu, sid, meta):
    """Write a plan-timing table (features, measured ms, analytic prediction,
    script ids, per-script notes) with its key, as one .npz file at ``path``."""
    with open(path, "wb") as fh:
        np.savez(fh, X=X, ms=ms, pu=pu, sid=sid, meta=json.dumps(meta), key=json.dumps(key, sort_keys=True))


def load_timings(path, key):
    """The table stored at ``path`` if it was measured under ``key``, else None."""
    if not path or not os.path.exists(path):
        return None
    with np.load(path, allow_pickle=False) as z:
        if str(z["key"]) != json.dumps(key, sort_keys=True):
            return None
        return (z["X"].copy(), z["ms"].copy(), z["pu"].copy(), z["sid"].copy(), json.loads(str(z["meta"])))


def he_uniform_params(d_in, seed, device):
    """He-uniform weights from the seeded generator, zero biases (kf_mlp
    layout): the initial weights kf_planner_train draws itself when given
    none, here for tests that train step by step."""
    H = kf.MLP_HIDDEN
    count = kf.kf_mlp_param_count(d_in)
    u = synth.uniform((count,), seed, synth.TID["mlp"]).double()
    out = torch.zeros(count, dtype=torch.float64)
    k = 0
    for rows, cols, is_w in [(H, d_in, True), (H, 0, False), (H, H, True), (H, 0, False), (1, H, True), (1, 0, False)]:
        c = rows * cols if is_w else rows
        if is_w:
            out[k:k + c] = u[k:k + c] * math.sqrt(6.0 / cols)
        k += c
    return out.float().to(device)


def train(X, ms, pred_us, script_ids=None, analytic_weight=1.0, epochs=3000, lr=3e-3, seed=0, device="cuda"):
    """Train the cost model with the library's kf_planner_train: it
    standardises the features, forms the targets ln(ms) - analytic_weight *
    ln(analytic ms) (centred per script when script ids are given: only
    differences between one script's plans decide a choice), draws the
    initial weights and runs full-batch Adam, all in libkf.  With weight 1
    the network learns the analytic model's error and the score
    ln(analytic ms) + f(x) ranks plans.  Returns (CostModel, loss history)."""
    return kf.kf_planner_train(X, ms, pred_us, script_ids, epochs=epochs, lr=lr, analytic_weight=analytic_weight,
                               centre=script_ids is not None, loss_every=500, seed=seed, device=device)


def evaluate(seed, indices, kmin, kmax, model, reps, top_k=3, cap=2000, margin=0.1, device="cuda"):
    """Per held-out script: exhaustive timings, and each method's choice."""
    rows = []
    for i in indices:
        n, sd, s = make(seed, i, kmin, kmax)
        bind = bindings(sd, i, device)
        unf = s.plan(kf.KF_PLAN_UNFUSED)
        ws = torch.zeros(max(s.select_workspace_size(cap), unf.workspace_size(), 256), dtype=torch.uint8,
                         device=device)
        t = s.time_all(bind, ws, reps=reps, max_plans=cap)
        nk = s.enumerate_info(cap)[2]
        _, ia = s.select(kf.KF_SELECT_ANALYTIC, max_plans=cap)
        _, i1 = s.select(kf.KF_SELECT_MLP, bind, ws, model, top_k=1, max_plans=cap)
        _, ik = s.select(kf.KF_SELECT_MLP, bind, ws, model, top_k=top_k, reps=reps, max_plans=cap)
        _, i5 = s.select(kf.KF_SELECT_MLP, bind, ws, model, top_k=2 * top_k, reps=reps, max_plans=cap)
        _, im = s.select(kf.KF_SELECT_MLP, bind, ws, model, top_k=top_k, reps=reps, max_plans=cap, margin=margin)
        t_unf = unf.time(bind, ws, reps=reps)
        best = float(t.min())
        rows.append({"index": int(i), "n": n, "calls": len(sd["calls"]), "plans": len(t), "best_ms": best,
                     "mlp": float(t[i1["index"]]) / best, "mlp_topk": float(t[ik["index"]]) / best,
                     "mlp_top2k": float(t[i5["index"]]) / best,
                     "mlp_margin": float(t[im["index"]]) / best, "timed_margin": im["timed"],
                     "analytic": float(t[ia["index"]]) / best, "greedy": float(t[int(np.argmin(nk))]) / best,
                     "unfused": t_unf / best, "timed_topk": ik["timed"]})
        del bind, ws
    return rows


def summary(rows, key):
    r = np.array([row[key] for row in rows])
    return {"mean_ratio": round(float(r.mean()), 4), "geomean_ratio": round(float(np.exp(np.log(r).mean())), 4),
            "within_5pct": round(float((r <= 1.05).mean()), 4), "worst": round(float(r.max()), 4)}


def run(seed=0, scripts=500, ntrain=400, kmin=10, kmax=14, per_script=64, reps=5, epochs=3000, top_k=3,
        analytic_weight=1.0, centre=True, margin=0.1, device="cuda", log=print, timings=""):
    """Collect (or load from ``timings``) the training table, train, and
    score the held-out scripts.  With a ``timings`` path, a table measured
    under the same key is reused and a freshly collected one is saved."""
    t0 = time.time()
    key = timing_key(seed, range(ntrain), kmin, kmax, per_script, reps, device)
    got = load_timings(timings, key)
    if got is None:
        X, ms, pu, sid, meta = collect(seed, range(ntrain), kmin, kmax, per_script, reps, device=device)
        if timings:
            save_timings(timings, key, X, ms, pu, sid, meta)
    else:
        X, ms, pu, sid, meta = got
    t1 = time.time()
    model, hist = train(X, ms, pu, sid if centre else None, analytic_weight, epochs=epochs, seed=seed,
                        device=device)
    t2 = time.time()
    rows = evaluate(seed, range(ntrain, scripts), kmin, kmax, model, reps, top_k=top_k, margin=margin,
                    device=device)
    t3 = time.time()
    plans = np.array([r["plans"] for r in rows])
    out = {
        "config": {"seed": seed, "scripts": scripts, "train": ntrain, "test": scripts - ntrain,
                   "n": f"2^{kmin}..2^{kmax}", "per_script": per_script, "reps": reps, "epochs": epochs,
                   "top_k": top_k, "margin": margin, "analytic_weight": analytic_weight,
                   "centred_per_script": centre,
                   "features": kf.NFEATURES,
                   "hidden": kf.MLP_HIDDEN},
        "train_timings": "loaded" if got is not None else "measured",
        "train_plans_timed": int(len(ms)), "test_plans_timed": int(plans.sum()),
        "test_plans_per_script": {"mean": float(plans.mean()), "max": int(plans.max())},
        "seconds": {"collect": round(t1 - t0, 1), "train": round(t2 - t1, 2), "evaluate": round(t3 - t2, 1)},
        "loss": hist,
        "test": {k: summary(rows, k) for k in ("mlp", "mlp_topk", "mlp_top2k", "mlp_margin", "analytic", "greedy",
                                                "unfused")},
        "timed_per_script": {"topk": float(np.mean([r["timed_topk"] for r in rows])),
                             "margin": float(np.mean([r["timed_margin"] for r in rows]))},
        "rows": rows,
    }
    if log:
        for k, v in out["test"].items():
            log(f"{k:10s} mean {v['mean_ratio']:.4f}  geomean {v['geomean_ratio']:.4f}  "
                f"within 5%: {v['within_5pct']:.3f}  worst {v['worst']:.3f}")
    return out, model


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--scripts", type=int, default=500)
    ap.add_argument("--train", type=int, default=400)
    ap.add_argument("--kmin", type=int, default=10)
    ap.add_argument("--kmax", type=int, default=14)
    ap.add_argument("--per-script", type=int, default=64)
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--epochs", type=int, default=3000)
    ap.add_argument("--top-k", type=int, default=3)
    ap.add_argument("--analytic-weight", type=float, default=1.0)
    ap.add_argument("--no-centre", action="store_true", help="absolute targets instead of per-script centred")
    ap.add_argument("--margin", type=float, default=0.1, help="score margin (ln ms) of plans also re-timed")
    ap.add_argument("--out", default="")
    ap.add_argument("--save-model", default="")
    ap.add_argument("--timings", default="",
                    help="plan-timing table (.npz): reused if measured with the same seed, scripts, sizes, "
                         "plans per script, repetitions and device; written after a fresh collection")
    a = ap.parse_args(argv)
    kf.lib()
    res, model = run(a.seed, a.scripts, a.train, a.kmin, a.kmax, a.per_script, a.reps, a.epochs, a.top_k,
                     a.analytic_weight, centre=not a.no_centre, margin=a.margin, timings=a.timings)
    if a.out:
        with open(a.out, "w") as fh:
            json.dump(res, fh, indent=1)
    if a.save_model:
        model.save(a.save_model)
    print(json.dumps({k: v for k, v in res.items() if k != "rows"}))


if __name__ == "__main__":
    main()
