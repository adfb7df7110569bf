"""The learned planner's workload and its host-side selection logic (no GPU).

Random scripts of 6-10 elementary calls (AXPY, SCAL, DOT, GEMV, GEMVT, GER)
over shared vectors and matrices, n = 2^k with k in [10, 14], are the
training and test data of the plan cost model.  These tests check the
generator's stated rule on the full 500-script set, that the planner accepts
every generated script, and the subset of plans timed per training script.
"""

from collections import Counter

import numpy as np
import pytest

from synth import scripts as sscripts

OPS = {"AXPBY", "SCAL", "DOT", "GEMV", "GEMVT", "GER"}


@pytest.fixture(scope="module")
def learn():
    from paper_1305_1183_gb300 import _build
    _build.build()
    from paper_1305_1183_gb300 import learn as L
    return L


def _shape_ok(sd, name, kind):
    return sd["vars"][name][0] == kind


def test_random_scripts_follow_the_generation_rule():
    n = 64
    ops = Counter()
    shared = 0
    for i in range(500):
        sd = sscripts.random_script(0, i, n)
        calls = sd["calls"]
        assert 6 <= len(calls) <= 10
        for op, outs, ins, sc in calls:
            assert op in OPS
            ops[op] += 1
            if op in ("GEMV", "GEMVT"):
                assert _shape_ok(sd, ins[0], "m") and _shape_ok(sd, ins[1], "v") and _shape_ok(sd, outs[0], "v")
                assert outs[0] != ins[1]                       # never overwrites its own input
            elif op == "GER":
                assert _shape_ok(sd, ins[0], "m") and _shape_ok(sd, outs[0], "m")
            elif op == "DOT":
                assert _shape_ok(sd, outs[0], "s")
            else:
                assert all(_shape_ok(sd, v, "v") for v in ins + outs)
            assert all(-1.0 <= a < 1.0 or a in (0.0, 1.0) for a in sc)
        reads = Counter(v for _, _, ins, _ in calls for v in ins)
        shared += any(c >= 2 for c in reads.values())
        assert all(spec[1] == n for spec in sd["vars"].values() if spec[0] in "vm")
        assert set(sd["outputs"]) == {c[1][0] for c in calls}
    # every op of the vocabulary is drawn about one time in six
    total = sum(ops.values())
    for op in OPS:
        assert 0.12 < ops[op] / total < 0.22, (op, ops[op] / total)
    # operands are shared: nearly every script reads some variable twice
    assert shared >= 450


def test_every_generated_script_is_accepted_by_the_planner(learn):
    for i in range(100):
        sd = sscripts.random_script(0, i, 1024)
        s = learn.to_script(sd)
        s.validate()
        count, _ = s.count_plans(cap=64)
        assert count >= 1


def test_script_sizes_are_powers_of_two_in_range(learn):
    sizes = Counter(learn.script_size(0, i, 10, 14) for i in range(500))
    assert set(sizes) == {1 << k for k in range(10, 15)}
    assert min(sizes.values()) >= 60                   # each of the five about 100 times


def test_training_subset(learn):
    """Up to per_script plans: all of them when there are that few, else the
    best-predicted half, the fewest-kernel plan, the unfused plan and a
    seeded sample of the rest; deterministic for a seed."""
    pred = np.array([5.0, 1.0, 3.0, 2.0, 4.0])
    nk = np.array([2, 3, 1, 4, 2])
    assert learn.training_subset(0, 0, pred, nk, 4, per_script=8) == [0, 1, 2, 3, 4]
    count, per = 300, 40
    pred = np.linspace(1.0, 2.0, count)[::-1].copy()   # the last plans are predicted best
    nk = np.full(count, 3)
    nk[7] = 1                                          # fewest kernels
    nk[11] = 6                                         # the unfused plan (one kernel per call)
    sub = learn.training_subset(0, 5, pred, nk, 6, per_script=per)
    assert len(sub) == per and len(set(sub)) == per and sub == sorted(sub)
    assert set(range(count - per // 2, count)) <= set(sub)
    assert 7 in sub and 11 in sub
    assert sub == learn.training_subset(0, 5, pred, nk, 6, per_script=per)
    assert sub != learn.training_subset(1, 5, pred, nk, 6, per_script=per)


def test_summary_of_ratios(learn):
    rows = [{"r": 1.0}, {"r": 1.04}, {"r": 1.21}, {"r": 1.0}]
    s = learn.summary(rows, "r")
    assert s["within_5pct"] == 0.75
    assert s["worst"] == 1.21
    assert s["mean_ratio"] == pytest.approx(1.0625, abs=1e-4)
    assert s["geomean_ratio"] == pytest.approx(float(np.exp(np.mean(np.log([1.0, 1.04, 1.21, 1.0])))), abs=1e-4)


def test_timing_table_round_trip_and_key(learn, tmp_path):
    """A stored plan-timing table comes back unchanged under its own key and
    is refused under any other (another seed, size range or device)."""
    key = learn.timing_key(0, range(4), 10, 14, 64, 5, "cpu")
    X = np.arange(48, dtype=np.float64).reshape(3, 16)
    ms, pu, sid = np.array([0.5, 0.25, 1.0]), np.array([400.0, 200.0, 900.0]), np.array([0, 0, 3])
    meta = [{"index": 0, "n": 1024, "calls": 7, "plans": 12, "timed": 2}]
    path = str(tmp_path / "timings.npz")
    learn.save_timings(path, key, X, ms, pu, sid, meta)
    got = learn.load_timings(path, key)
    assert got is not None
    for a, b in zip(got[:4], (X, ms, pu, sid)):
        assert np.array_equal(a, b) and a.dtype == b.dtype
    assert got[4] == meta
    for other in (learn.timing_key(1, range(4), 10, 14, 64, 5, "cpu"),
                  learn.timing_key(0, range(4), 10, 13, 64, 5, "cpu"),
                  learn.timing_key(0, range(4), 10, 14, 64, 5, "another-device")):
        assert learn.load_timings(path, other) is None
    assert learn.load_timings(str(tmp_path / "none.npz"), key) is None
    assert learn.load_timings("", key) is None


def test_run_resumes_from_a_stored_timing_table(learn, tmp_path, monkeypatch):
    """With a timings path, the first run collects and stores the training
    table and a second run with the same key loads it instead of timing
    plans again (the GPU stages are replaced by fakes here)."""
    collected = []

    def fake_collect(seed, indices, kmin, kmax, per_script, reps, cap=2000, device="cuda"):
        collected.append(list(indices))
        X = np.arange(32, dtype=np.float64).reshape(2, 16)
        return X, np.array([0.5, 0.7]), np.array([400.0, 600.0]), np.array([0, 1]), [{"index": 0}]

    seen = []

    def fake_train(X, ms, pu, sid, analytic_weight, epochs=0, seed=0, device="cpu"):
        seen.append((X.copy(), ms.copy()))
        return None, [(1, 0.5)]

    row = {"plans": 3, "timed_topk": 3, "timed_margin": 5}
    row.update({k: 1.0 for k in ("mlp", "mlp_topk", "mlp_top2k", "mlp_margin", "analytic", "greedy", "unfused")})
    monkeypatch.setattr(learn, "collect", fake_collect)
    monkeypatch.setattr(learn, "train", fake_train)
    monkeypatch.setattr(learn, "evaluate", lambda *a, **k: [dict(row)])
    path = str(tmp_path / "t.npz")
    out1, _ = learn.run(seed=3, scripts=4, ntrain=2, device="cpu", log=None, timings=path)
    out2, _ = learn.run(seed=3, scripts=4, ntrain=2, device="cpu", log=None, timings=path)
    assert (out1["train_timings"], out2["train_timings"]) == ("measured", "loaded")
    assert collected == [[0, 1]]
    assert np.array_equal(seen[0][0], seen[1][0]) and np.array_equal(seen[0][1], seen[1][1])
    out3, _ = learn.run(seed=4, scripts=4, ntrain=2, device="cpu", log=None, timings=path)
    assert out3["train_timings"] == "measured" and len(collected) == 2     # another seed: timed again
