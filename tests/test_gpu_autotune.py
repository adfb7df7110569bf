"""Autotuner: empirical search over compiled implementations, tuning cache,
its persistence, and tuned launches keeping parity with the oracle."""

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import built, dev, host  # noqa: F401
from tolerance import check_reduce
from test_planner_cpu import bicgk, gemver

pytestmark = pytest.mark.gpu


def bind_bicgk(m, n):
    A = synth.uniform((m, n), 0, 1, device=dev())
    p = synth.uniform((n,), 0, 3, device=dev())
    r = synth.uniform((m,), 0, 4, device=dev())
    return {"A": A, "p": p, "r": r, "q": torch.empty(m, device=dev()), "s": torch.empty(n, device=dev())}


def test_autotune_plan_and_cache(built, tmp_path):
    kf = built
    kf.kf_tune_cache_clear()
    m = n = 4096
    s = bicgk(kf, m, n)
    p = s.plan(kf.KF_PLAN_ANALYTIC)
    b = bind_bicgk(m, n)
    ws = torch.zeros(p.workspace_size(), dtype=torch.uint8, device=dev())
    tuned, before = p.autotune(b, ws, reps=3)
    # the default is among the candidates; medians of separate runs differ
    # by a few percent at this size
    assert 0 < tuned <= before * 1.05
    assert kf.kf_tune_cache_entries() >= 1
    # the fixed entry point of the same size class now runs the tuned kernel
    q = torch.empty(m, device=dev()); sv = torch.empty(n, device=dev())
    kf.kf_bicgk(b["A"], b["p"], b["r"], q, sv, kf.workspace(kf.KF_SEQ_BICGK, m, n))
    Ah, ph, rh = host(b["A"]), host(b["p"]), host(b["r"])
    qo, so = oracle.bicgk(Ah, ph, rh)
    check_reduce(host(q), qo, oracle.abs_gemv(Ah, ph), n, "q tuned")
    check_reduce(host(sv), so, oracle.abs_gemvt(Ah, rh), m, "s tuned")
    # persistence
    path = tmp_path / "tune.txt"
    kf.kf_tune_cache_save(path)
    entries = kf.kf_tune_cache_entries()
    kf.kf_tune_cache_clear()
    assert kf.kf_tune_cache_entries() == 0
    assert kf.kf_tune_cache_load(path) == entries
    # a cache written on another device is ignored; a malformed one is an error
    other = tmp_path / "other.txt"
    other.write_text(open(path).read().replace("device ", "device SomeOtherGPU_", 1))
    kf.kf_tune_cache_clear()
    assert kf.kf_tune_cache_load(other) == 0
    bad = tmp_path / "bad.txt"
    bad.write_text(open(path).read() + "mat 1 2 3 : nonsense\n")
    with pytest.raises(kf.KFError):
        kf.kf_tune_cache_load(bad)
    kf.kf_tune_cache_clear()


def test_autotune_gemver_plan(built):
    kf = built
    n = 4096
    s = gemver(kf, n)
    p = s.plan(kf.KF_PLAN_ANALYTIC)
    names = ["A", "B", "u1", "v1", "u2", "v2", "y", "z", "x", "w", "t"]
    b = {k: (synth.uniform((n, n) if k in ("A", "B") else (n,), 0, 20 + i, device=dev())) for i, k in enumerate(names)}
    ws = torch.zeros(p.workspace_size(), dtype=torch.uint8, device=dev())
    tuned, before = p.autotune(b, ws, reps=5)
    # the previous choice is among the candidates; medians of separate runs
    # differ by a few percent at this size
    assert 0 < tuned <= before * 1.05
    kf.kf_tune_cache_clear()


def test_batched_autotune(built):
    kf = built
    ms = synth.log_uniform_int(32, 1024, 5, synth.TID["sizes"], 128).tolist()
    ns = synth.log_uniform_int(32, 1024, 6, synth.TID["sizes"], 128).tolist()
    descs, keep = [], []
    for i, (m, n) in enumerate(zip(ms, ns)):
        A = synth.uniform((m, n), i, 1, device=dev())
        x = synth.uniform((n,), i, 3, device=dev()); r = synth.uniform((m,), i, 4, device=dev())
        y = torch.empty(m, device=dev()); s = torch.empty(n, device=dev())
        keep += [A, x, r, y, s]
        descs.append({"m": m, "n": n, "lda": n, "A": A, "x": x, "r": r, "y": y, "s": s})
    br, t = kf.kf_batched_autotune(kf.KF_SEQ_BICGK, descs, reps=3)
    assert br in (32, 64, 128, 256, 512) and t > 0


def test_tune_on_first_use(built):
    """kf_set_autotune: the first automatic launch of a key runs the search
    and fills the cache (matrix and vector passes); results keep parity; a
    second launch of the key adds no entry; capture does not search."""
    kf = built
    kf.kf_tune_cache_clear()
    kf.kf_set_autotune(2)
    try:
        m, n = 3000, 2048
        b = bind_bicgk(m, n)
        W = kf.workspace(kf.KF_SEQ_BICGK, m, n)
        kf.kf_bicgk(b["A"], b["p"], b["r"], b["q"], b["s"], W)
        e1 = kf.kf_tune_cache_entries()
        assert e1 == 1
        kf.kf_bicgk(b["A"], b["p"], b["r"], b["q"], b["s"], W)
        assert kf.kf_tune_cache_entries() == e1
        Ah, ph, rh = host(b["A"]), host(b["p"]), host(b["r"])
        qo, so = oracle.bicgk(Ah, ph, rh)
        check_reduce(host(b["q"]), qo, oracle.abs_gemv(Ah, ph), n, "q")
        check_reduce(host(b["s"]), so, oracle.abs_gemvt(Ah, rh), m, "s")
        # a vector pass: AXPYDOT
        k = 1 << 20
        w, v, u = (synth.uniform((k,), 0, t, device=dev()) for t in (10, 11, 12))
        z = torch.empty(k, device=dev()); r = torch.empty(1, device=dev())
        kf.kf_axpydot(w, v, u, 1.5, z, r, kf.workspace(kf.KF_SEQ_AXPYDOT, 1, k))
        assert kf.kf_tune_cache_entries() == e1 + 1
        zo, ro = oracle.axpydot(host(w), host(v), host(u), 1.5)
        assert abs(float(r[0]) - ro) <= 1e-5 * np.sqrt(k) * float(np.sum(np.abs(zo) * np.abs(host(u))))
        # capture: a new key is not searched (and the launch is recorded)
        b2 = bind_bicgk(700, 900)
        W2 = kf.workspace(kf.KF_SEQ_BICGK, 700, 900)
        st = torch.cuda.Stream()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=st):
            kf.kf_bicgk(b2["A"], b2["p"], b2["r"], b2["q"], b2["s"], W2)
        assert kf.kf_tune_cache_entries() == e1 + 1
        g.replay()
        torch.cuda.synchronize()
        Ah, ph = host(b2["A"]), host(b2["p"])
        check_reduce(host(b2["q"]), oracle.gemv(Ah, ph), oracle.abs_gemv(Ah, ph), 900, "q captured")
    finally:
        kf.kf_set_autotune(0)


def test_tune_on_first_use_atax(built, tmp_path):
    """ATAX's ring depth and blocks per SM go through the same first-use
    search and cache (saved and loaded with the rest); results keep parity."""
    kf = built
    kf.kf_tune_cache_clear()
    kf.kf_set_autotune(2)
    try:
        m, n = 3000, 4096
        A = synth.uniform((m, n), 0, 1, device=dev())
        x = synth.uniform((n,), 0, 3, device=dev())
        y = torch.empty(n, device=dev())
        kf.kf_atax(A, x, y, kf.workspace(kf.KF_SEQ_ATAX, m, n))
        assert kf.kf_tune_cache_entries() == 1
        Ah, xh = host(A), host(x)
        yo, _ = oracle.atax(Ah, xh)
        check_reduce(host(y), yo, oracle.abs_gemvt(Ah, oracle.abs_gemv(Ah, xh)), m, "atax tuned")
        path = tmp_path / "tune.txt"
        kf.kf_tune_cache_save(path)
        assert "atax " in open(path).read()
        kf.kf_tune_cache_clear()
        assert kf.kf_tune_cache_load(path) == 1
    finally:
        kf.kf_set_autotune(0)
        kf.kf_tune_cache_clear()


def _force_atax_form(kf, tmp_path, m, n, vec, rp):
    """Put one ATAX tuning for the size class of (m, n) into the cache: vec
    1 = cluster reduction, 2 = per-block partials for the finishing kernel."""
    kf.kf_tune_cache_clear()
    base = tmp_path / "dev.txt"
    kf.kf_tune_cache_save(base)
    dev_line = [ln for ln in open(base) if ln.startswith("device ")][0]
    f = tmp_path / "atax.txt"
    f.write_text(dev_line + f"atax {m.bit_length() - 1} {n.bit_length() - 1} : 1 {vec} {rp} 0 0\n")
    assert kf.kf_tune_cache_load(f) == 1


@pytest.mark.parametrize("vec", [1, 2])
@pytest.mark.parametrize("rp", [1, 2])
def test_atax_every_form(built, tmp_path, vec, rp):
    """Each way of adding ATAX's column partials (clusters first, or every
    block's partial to the finishing kernel) and rows per barrier, fixed
    through the tuning cache: kf_atax matches the oracle twice in a row on
    one workspace, and a planner pair with scale 1.5 * -0.5 matches too."""
    kf = built
    try:
        for m, n in [(3000, 4096), (5, 16384), (2000, 1028), (9, 8), (1031, 8192)]:
            _force_atax_form(kf, tmp_path, m, n, vec, rp)
            A = synth.uniform((m, n), m, 1, device=dev())
            x = synth.uniform((n,), m, 3, device=dev())
            W = kf.workspace(kf.KF_SEQ_ATAX, m, n)
            Ah, xh = host(A), host(x)
            yo, _ = oracle.atax(Ah, xh)
            sy = oracle.abs_gemvt(Ah, oracle.abs_gemv(Ah, xh))
            for call in range(2):
                y = torch.full((n,), float("nan"), device=dev())
                kf.kf_atax(A, x, y, W)
                check_reduce(host(y), yo, sy, max(m, n), f"atax form {vec}/{rp}, call {call}")
            kf.kf_workspace_status(W)
            s = kf.Script()
            s.matrix("A", m, n); s.vector("x", n); s.vector("t", m); s.vector("y", n)
            s.input("A", "x"); s.output("y")
            s.call("GEMV", ["t"], ["A", "x"], [1.5, 0.0])
            s.call("GEMVT", ["y"], ["A", "t"], [-0.5, 0.0])
            p = s.plan(kf.KF_PLAN_ANALYTIC)
            assert [k["kind"] for k in p.describe()["kernels"]] == ["atax"]
            ws = torch.zeros(max(p.workspace_size(), 256), dtype=torch.uint8, device=dev())
            bind = {"A": A, "x": x, "t": torch.empty(m, device=dev()), "y": torch.empty(n, device=dev())}
            p.execute(bind, ws)
            check_reduce(host(bind["y"]), -0.75 * yo, 0.75 * sy, max(m, n), f"planner atax form {vec}/{rp}")
    finally:
        kf.kf_tune_cache_clear()
