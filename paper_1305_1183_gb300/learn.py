"""Learned planner: measure plan timings on random scripts, train the MLP cost
model with the library's own kernels, and compare its choices.

The paper ranks fusion implementations with an additive predictor of
pre-benchmarked routine times and falls back on empirical search
(Section 3.2; its accuracy in the table of Section 4.3).  Here a 3-layer
perceptron (16 plan features -> 64 -> 64 -> 1, ReLU) learns log plan time
from timings the planner itself measures; forward, backward and Adam run in
libkf (kf_mlp_*).  Per script, up to `per_script` plans are timed: every plan
when there are that few, else the best predicted half by the analytic model,
the fewest-kernel plan, the one-kernel-per-call plan and a seeded uniform
sample of the rest.  The best measured plan of that set is the judge; the
MLP's first choice, the analytic choice and the fewest-kernel choice are
scored by t(choice) / t(best).

    python -m paper_1305_1183_gb300.learn --scripts 500 --train 400 --out results.json
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


def collect(seed, indices, kmin, kmax, per_script, reps, cap=2000, device="cuda", log=None):
    records = []
    for i in indices:
        n = script_size(seed, i, kmin, kmax)
        sd = sscripts.random_script(seed, i, n)
        s = to_script(sd)
        feats, pred, nk = s.enumerate_info(cap)
        count = len(pred)
        ncalls = len(sd["calls"])
        order = np.argsort(pred, kind="stable")
        chosen = []
        if count <= per_script:
            chosen = list(range(count))
        else:
            chosen = list(order[: per_script // 2])
            greedy = int(np.lexsort((pred, nk))[0])
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
        bind = bindings(sd, i, device)
        timed = []
        ws = None
        for j in sorted(int(x) for x in chosen):
            p = s.plan(kf.KF_PLAN_INDEX, index=j, max_plans=cap)
            need = max(p.workspace_size(), 256)
            if ws is None or ws.numel() < need:
                ws = torch.zeros(need, dtype=torch.uint8, device=device)
            ms = p.time(bind, ws, reps=reps)
            timed.append({"plan": j, "ms": ms, "pred_us": float(pred[j]), "kernels": int(nk[j]),
                          "feats": [float(x) for x in feats[j]]})
        del bind, ws
        records.append({"index": int(i), "n": n, "calls": ncalls, "plans": count,
                        "exhaustive": count <= per_script, "timed": timed})
        if log:
            log(f"script {i}: n={n} calls={ncalls} plans={count} timed={len(timed)}")
    return records


def he_uniform_params(d_in, seed, device):
    """He-uniform weights from the seeded generator, zero biases (flat libkf layout)."""
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


def train(X, y, epochs=3000, lr=3e-3, seed=0, device="cuda"):
    """Full-batch Adam on standardised features; returns (params, mu, sd, losses)."""
    mu = X.mean(axis=0)
    sd = X.std(axis=0) + 1e-6
    Xs = torch.tensor((X - mu) / sd, dtype=torch.float32, device=device)
    yt = torch.tensor(y, dtype=torch.float32, device=device)
    d = X.shape[1]
    p = he_uniform_params(d, seed, device)
    g = torch.empty_like(p)
    m = torch.zeros_like(p)
    v = torch.zeros_like(p)
    loss = torch.empty(1, device=device)
    ws = torch.zeros(kf.kf_mlp_workspace_size(d, X.shape[0]), dtype=torch.uint8, device=device)
    losses = []
    for t in range(1, epochs + 1):
        kf.kf_mlp_loss_grad(p, Xs, yt, g, loss, ws)
        kf.kf_mlp_adam(p, g, m, v, t, lr=lr)
        if t == 1 or t % 250 == 0:
            losses.append((t, float(loss)))
    kf.kf_mlp_loss_grad(p, Xs, yt, g, loss, ws)
    losses.append((epochs, float(loss)))
    return p, mu, sd, losses


def predict(p, mu, sd, X, device="cuda"):
    Xs = torch.tensor((X - mu) / sd, dtype=torch.float32, device=device)
    out = torch.empty(X.shape[0], device=device)
    kf.kf_mlp_forward(p, Xs, out)
    return out.double().cpu().numpy()


def score(records, choose):
    """Ratios t(choice)/t(best) over the records, with choose(record) -> timed index."""
    r = []
    for rec in records:
        ts = np.array([t["ms"] for t in rec["timed"]])
        j = choose(rec)
        r.append(float(ts[j] / ts.min()))
    r = np.array(r)
    return {"mean_ratio": float(r.mean()), "geomean_ratio": float(np.exp(np.log(r).mean())),
            "within_5pct": float((r <= 1.05).mean()), "worst": float(r.max()), "ratios": [round(x, 4) for x in r]}


def run(seed=0, scripts=500, ntrain=400, kmin=10, kmax=14, per_script=24, reps=3, epochs=3000, device="cuda",
        log=print):
    t0 = time.time()
    recs = collect(seed, range(scripts), kmin, kmax, per_script, reps, device=device, log=None)
    t1 = time.time()
    train_recs, test_recs = recs[:ntrain], recs[ntrain:]
    X = np.array([t["feats"] for r in train_recs for t in r["timed"]], dtype=np.float64)
    y = np.log(np.array([t["ms"] for r in train_recs for t in r["timed"]], dtype=np.float64))
    p, mu, sd, losses = train(X, y, epochs=epochs, seed=seed, device=device)
    t2 = time.time()

    def mlp_choice(rec):
        F = np.array([t["feats"] for t in rec["timed"]])
        return int(np.argmin(predict(p, mu, sd, F, device)))

    def mlp_top3(rec):
        F = np.array([t["feats"] for t in rec["timed"]])
        top = np.argsort(predict(p, mu, sd, F, device))[:3]
        ts = np.array([rec["timed"][j]["ms"] for j in top])
        return int(top[int(np.argmin(ts))])

    def analytic_choice(rec):
        return int(np.argmin([t["pred_us"] for t in rec["timed"]]))

    def greedy_choice(rec):
        return int(np.lexsort(([t["pred_us"] for t in rec["timed"]], [t["kernels"] for t in rec["timed"]]))[0])

    def unfused_choice(rec):
        k = [t["kernels"] for t in rec["timed"]]
        return int(np.argmax(k))

    out = {
        "config": {"seed": seed, "scripts": scripts, "train": ntrain, "test": scripts - ntrain,
                   "n": f"2^{kmin}..2^{kmax}", "per_script": per_script, "reps": reps, "epochs": epochs,
                   "features": 16, "hidden": kf.MLP_HIDDEN},
        "timed_plans": int(sum(len(r["timed"]) for r in recs)),
        "fully_enumerated_scripts": int(sum(r["exhaustive"] for r in recs)),
        "collect_s": round(t1 - t0, 1), "train_s": round(t2 - t1, 1),
        "losses": losses,
        "test": {"mlp": score(test_recs, mlp_choice), "mlp_top3_retimed": score(test_recs, mlp_top3),
                 "analytic": score(test_recs, analytic_choice), "greedy": score(test_recs, greedy_choice),
                 "unfused": score(test_recs, unfused_choice)},
        "train_fit": {"mlp": score(train_recs, mlp_choice), "analytic": score(train_recs, analytic_choice)},
    }
    if log:
        for k, v in out["test"].items():
            log(f"{k:18s} mean {v['mean_ratio']:.4f}  geomean {v['geomean_ratio']:.4f}  "
                f"within 5%: {v['within_5pct']:.3f}  worst {v['worst']:.3f}")
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--scripts", type=int, default=500)
    ap.add_argument("--train", type=int, default=400)
    ap.add_argument("--kmin", type=int, default=10)
    ap.add_argument("--kmax", type=int, default=14)
    ap.add_argument("--per-script", type=int, default=24)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--epochs", type=int, default=3000)
    ap.add_argument("--out", default="")
    a = ap.parse_args(argv)
    from . import _build
    _build.build()
    kf.lib()
    res = run(a.seed, a.scripts, a.train, a.kmin, a.kmax, a.per_script, a.reps, a.epochs)
    if a.out:
        with open(a.out, "w") as fh:
            json.dump(res, fh, indent=1)
    print(json.dumps({k: v for k, v in res.items() if k != "train_fit"} | {
        "test": {k: {kk: vv for kk, vv in v.items() if kk != "ratios"} for k, v in res["test"].items()}}))


if __name__ == "__main__":
    main()
