"""Every enumerated plan of a script computes what the script computes.

For the canonical scripts of Table 1 and for random scripts of AXPY, SCAL,
DOT, GEMV, GEMVT and GER calls, each legal plan (up to a cap) is executed
through kf_plan_execute and compared with the FP64 oracle's call-by-call
evaluation of the same script (oracle.script.run):
  * integer inputs and scalars in {-1, 1, 2}: bitwise, when the same script
    evaluated on absolute values stays below 2^24 (then every partial sum of
    every call is an integer that FP32 holds exactly, whatever the order);
  * uniform inputs: |yhat - y| <= 1e-5 sqrt(n) * calls * |script|(|inputs|),
    the absolute-value evaluation giving the backward-error scale.
This pins the legality rules: a fusion that consumed a reduction result in
its own kernel, stored the wrong version of a variable or broke a
dependency would show up here.
"""

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import built, dev, host  # noqa: F401
from oracle import script as oscript
from tolerance import check_reduce
from synth import scripts as sscripts
from test_planner_cpu import atax, axpydot, bicgk, gemver, gesummv, waxpby

pytestmark = pytest.mark.gpu


def to_kf(kf, sd):
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


def inputs_for(sd, seed, integer):
    vals = {}
    for i, (name, spec) in enumerate(sorted(sd["vars"].items())):
        shape = (spec[1],) if spec[0] == "v" else ((spec[1], spec[2]) if spec[0] == "m" else (1,))
        tid = 200 + i
        vals[name] = (synth.integers(shape, seed, tid) if integer else synth.uniform(shape, seed, tid))
    return vals


def run_plans(kf, sd, integer, cap=64, seed=0):
    s = to_kf(kf, sd)
    vals = inputs_for(sd, seed, integer)
    env = {k: (v.numpy().astype(np.float64) if sd["vars"][k][0] != "s" else 0.0) for k, v in vals.items()}
    ref = oscript.run(sd["calls"], env)
    absenv = {k: (np.abs(v) if not np.isscalar(v) else 0.0) for k, v in env.items()}
    abscalls = [(op, o, i, [abs(x) for x in sc]) for op, o, i, sc in sd["calls"]]
    scale = oscript.run(abscalls, absenv)
    int_scalars = all(float(x).is_integer() for _, _, _, sc in sd["calls"] for x in sc)
    exact = integer and int_scalars and all(np.max(np.abs(np.atleast_1d(scale[k]))) < 2 ** 24 for k in scale)
    count, _ = s.count_plans(cap=cap)
    assert count >= 1
    n = sd["n"]
    tol = 1e-5 * np.sqrt(n) * len(sd["calls"])
    nplans = 0
    for idx in range(count):
        p = s.plan(kf.KF_PLAN_INDEX, index=idx, max_plans=cap)
        ws = torch.zeros(max(p.workspace_size(), 256), dtype=torch.uint8, device=dev())
        bind = {k: v.clone().to(dev()) for k, v in vals.items()}
        p.execute(bind, ws)
        torch.cuda.synchronize()
        for k in sd["outputs"]:
            got = bind[k].double().cpu().numpy().reshape(np.shape(ref[k])) if np.ndim(ref[k]) else float(bind[k][0])
            want = ref[k]
            if exact:
                assert np.array_equal(np.asarray(got), np.asarray(want)), (idx, k, p.describe())
            else:
                err = np.abs(np.asarray(got) - np.asarray(want))
                bound = tol * np.asarray(scale[k]) + 1e-30
                assert np.all(err <= bound), (idx, k, float(np.max(err / bound)), p.describe())
        nplans += 1
    return nplans


@pytest.mark.parametrize("builder", [bicgk, gemver, gesummv, atax, axpydot, waxpby])
def test_canonical_scripts_every_plan(built, builder):
    kf = built
    s = builder(kf)
    # rebuild the script as a dict for the oracle
    import inspect  # noqa: F401
    sd = canonical_dict(builder)
    assert run_plans(kf, sd, integer=False) >= 1
    assert run_plans(kf, sd, integer=True) >= 1
    del s


def canonical_dict(builder):
    """The canonical scripts of test_planner_cpu as generator dicts."""
    A, B = 1.5, 1.2
    n = 40
    if builder is bicgk:
        return {"n": 64, "vars": {"A": ("m", 64, 64), "p": ("v", 64), "r": ("v", 64), "q": ("v", 64), "s": ("v", 64)},
                "inputs": ["A", "p", "r"], "outputs": ["q", "s"],
                "calls": [("GEMV", ["q"], ["A", "p"], [1.0, 0.0]), ("GEMVT", ["s"], ["A", "r"], [1.0, 0.0])]}
    if builder is gemver:
        v = {k: ("v", n) for k in ("u1", "v1", "u2", "v2", "y", "z", "x", "w", "t")}
        v.update({"A": ("m", n, n), "B": ("m", n, n)})
        return {"n": n, "vars": v, "inputs": ["A", "u1", "v1", "u2", "v2", "y", "z"], "outputs": ["B", "x", "w"],
                "calls": [("GER", ["B"], ["A", "u1", "v1"], [1.0]), ("GER", ["B"], ["B", "u2", "v2"], [1.0]),
                          ("GEMVT", ["t"], ["B", "y"], [1.0, 0.0]), ("AXPBY", ["x"], ["t", "z"], [B, 1.0]),
                          ("GEMV", ["w"], ["B", "x"], [A, 0.0])]}
    if builder is gesummv:
        v = {k: ("v", n) for k in ("x", "y", "t1", "t2")}
        v.update({"A": ("m", n, n), "B": ("m", n, n)})
        return {"n": n, "vars": v, "inputs": ["A", "B", "x"], "outputs": ["y"],
                "calls": [("GEMV", ["t1"], ["A", "x"], [A, 0.0]), ("GEMV", ["t2"], ["B", "x"], [B, 0.0]),
                          ("AXPBY", ["y"], ["t1", "t2"], [1.0, 1.0])]}
    if builder is atax:
        return {"n": n, "vars": {"A": ("m", n, n), "x": ("v", n), "t": ("v", n), "y": ("v", n)},
                "inputs": ["A", "x"], "outputs": ["y"],
                "calls": [("GEMV", ["t"], ["A", "x"], [1.0, 0.0]), ("GEMVT", ["y"], ["A", "t"], [1.0, 0.0])]}
    if builder is axpydot:
        v = {k: ("v", 1000) for k in ("w", "v", "u", "z")}
        v["r"] = ("s",)
        return {"n": 1000, "vars": v, "inputs": ["w", "v", "u"], "outputs": ["z", "r"],
                "calls": [("AXPBY", ["z"], ["w", "v"], [1.0, -A]), ("DOT", ["r"], ["z", "u"], [])]}
    v = {k: ("v", 1000) for k in ("x", "y", "t", "w")}
    return {"n": 1000, "vars": v, "inputs": ["x", "y"], "outputs": ["w"],
            "calls": [("SCAL", ["t"], ["x"], [A]), ("AXPBY", ["w"], ["y", "t"], [B, 1.0])]}


@pytest.mark.parametrize("index", range(12))
def test_random_scripts_integer_exact(built, index):
    kf = built
    sd = sscripts.random_script(seed=1, index=index, n=16, integer=True)
    run_plans(kf, sd, integer=True, cap=48, seed=index)


@pytest.mark.parametrize("index", range(12))
def test_random_scripts_float(built, index):
    kf = built
    sd = sscripts.random_script(seed=2, index=index, n=100 + 4 * index)
    run_plans(kf, sd, integer=False, cap=32, seed=index)


def test_random_scripts_aligned_sizes(built):
    """A few scripts at sizes that take the vectorised and specialised paths."""
    kf = built
    for index in range(4):
        sd = sscripts.random_script(seed=3, index=index, n=1024)
        run_plans(kf, sd, integer=False, cap=8, seed=index)


def test_planner_gemver_matches_fixed_entry_point(built):
    """The analytic plan of the GEMVER script and kf_gemver run the same
    kernels: identical bits."""
    kf = built
    sd = canonical_dict(gemver)
    s = to_kf(kf, sd)
    p = s.plan(kf.KF_PLAN_ANALYTIC)
    assert p.kernel_count() == 2
    vals = {k: v.to(dev()) for k, v in inputs_for(sd, 0, False).items()}
    ws = torch.zeros(max(p.workspace_size(), 256), dtype=torch.uint8, device=dev())
    bind = {k: v.clone() for k, v in vals.items()}
    p.execute(bind, ws)
    n = sd["n"]
    B = torch.empty(n, n, device=dev()); x = torch.empty(n, device=dev()); w = torch.empty(n, device=dev())
    kf.kf_gemver(vals["A"], vals["u1"], vals["v1"], vals["u2"], vals["v2"], vals["y"], vals["z"], 1.5, 1.2,
                 B, x, w, kf.workspace(kf.KF_SEQ_GEMVER, n, n))
    torch.cuda.synchronize()
    assert torch.equal(bind["B"], B) and torch.equal(bind["x"], x) and torch.equal(bind["w"], w)


@pytest.mark.parametrize("m,n", [(3000, 2048), (40, 16384), (777, 1000)])
def test_planner_single_pass_atax(built, m, n):
    """{t = 1.5 A x; y = -0.5 A^T t}: the planner's choice is the single-pass
    ATAX kernel (one read of A), and it and the two-kernel plan both match
    the oracle's call-by-call evaluation."""
    kf = built
    sd = {"n": max(m, n), "vars": {"A": ("m", m, n), "x": ("v", n), "t": ("v", m), "y": ("v", n)},
          "inputs": ["A", "x"], "outputs": ["y"],
          "calls": [("GEMV", ["t"], ["A", "x"], [1.5, 0.0]), ("GEMVT", ["y"], ["A", "t"], [-0.5, 0.0])]}
    s = to_kf(kf, sd)
    assert [k["kind"] for k in s.plan(kf.KF_PLAN_ANALYTIC).describe()["kernels"]] == ["atax"]
    assert run_plans(kf, sd, integer=False) == 2
    assert run_plans(kf, sd, integer=True) == 2


@pytest.mark.parametrize("m,n", [(3000, 2048), (1000, 1003)])
def test_call_order_search_runs_the_specialised_kernel(built, m, n):
    """BiCGK written with s = A^T r before q = A p: the call-order search
    runs the two calls in the specialised BiCGK order, so the plan computes
    exactly kf_bicgk's bits, and both match the oracle."""
    kf = built
    s = kf.Script()
    s.matrix("A", m, n); s.vector("p", n); s.vector("r", m); s.vector("q", m); s.vector("s", n)
    s.input("A", "p", "r"); s.output("q", "s")
    s.call("GEMVT", ["s"], ["A", "r"], [1.0, 0.0])
    s.call("GEMV", ["q"], ["A", "p"], [1.0, 0.0])
    p = s.plan(kf.KF_PLAN_ANALYTIC)
    (k,) = p.describe()["kernels"]
    assert k["order"] == [1, 0] and k["specialised"] is True
    A = synth.uniform((m, n), 7, synth.TID["A"], device=dev())
    pv = synth.uniform((n,), 7, synth.TID["p"], device=dev())
    rv = synth.uniform((m,), 7, synth.TID["r"], device=dev())
    bind = {"A": A, "p": pv, "r": rv, "q": torch.empty(m, device=dev()), "s": torch.empty(n, device=dev())}
    ws = torch.zeros(max(p.workspace_size(), 256), dtype=torch.uint8, device=dev())
    p.execute(bind, ws)
    q = torch.empty(m, device=dev()); sv = torch.empty(n, device=dev())
    kf.kf_bicgk(A, pv, rv, q, sv, kf.workspace(kf.KF_SEQ_BICGK, m, n))
    torch.cuda.synchronize()
    assert torch.equal(bind["q"], q) and torch.equal(bind["s"], sv)
    Ah, ph, rh = host(A), host(pv), host(rv)
    qo, so = oracle.bicgk(Ah, ph, rh)
    check_reduce(host(q), qo, oracle.abs_gemv(Ah, ph), n, "q")
    check_reduce(host(sv), so, oracle.abs_gemvt(Ah, rh), m, "s")


def _padded(m, n, ld, seed, tid, fill=12345.0):
    """An m x n view with row stride ld of a sentinel-filled buffer."""
    buf = torch.full((m * ld + 8,), fill, device=dev())
    v = buf[:m * ld].view(m, ld)[:, :n]
    v.copy_(synth.uniform((m, n), seed, tid, device=dev()))
    return buf, v


@pytest.mark.parametrize("ld_pad", [4, 5])
def test_strided_matrices_in_plans(built, ld_pad):
    """Scripts over views of wider arrays (kf_script_matrix_ld; rows 16-byte
    aligned with a pad of 4 floats, not with 5): BiCGK computes kf_bicgk's
    bits on the same view; GEMVER writes B inside its view only and matches
    the oracle; the ATAX pair (single pass when aligned, two passes when not)
    matches the oracle."""
    kf = built
    m, n = 1500, 1028
    ld = n + ld_pad
    # BiCGK
    _, A = _padded(m, n, ld, 3, synth.TID["A"])
    p = synth.uniform((n,), 3, synth.TID["p"], device=dev()); r = synth.uniform((m,), 3, synth.TID["r"], device=dev())
    s = kf.Script()
    s.matrix("A", m, n, ld=ld); s.vector("p", n); s.vector("r", m); s.vector("q", m); s.vector("s", n)
    s.input("A", "p", "r"); s.output("q", "s")
    s.call("GEMV", ["q"], ["A", "p"], [1.0, 0.0])
    s.call("GEMVT", ["s"], ["A", "r"], [1.0, 0.0])
    pl = s.plan(kf.KF_PLAN_ANALYTIC)
    bind = {"A": A, "p": p, "r": r, "q": torch.empty(m, device=dev()), "s": torch.empty(n, device=dev())}
    pl.execute(bind, torch.zeros(max(pl.workspace_size(), 256), dtype=torch.uint8, device=dev()))
    q = torch.empty(m, device=dev()); sv = torch.empty(n, device=dev())
    kf.kf_bicgk(A, p, r, q, sv, kf.workspace(kf.KF_SEQ_BICGK, m, n))
    torch.cuda.synchronize()
    assert torch.equal(bind["q"], q) and torch.equal(bind["s"], sv)
    Ah = host(A)
    check_reduce(host(q), oracle.gemv(Ah, host(p)), oracle.abs_gemv(Ah, host(p)), n, "q")
    # GEMVER (square) with A and B both strided
    nn = 1028
    _, A2 = _padded(nn, nn, nn + ld_pad, 4, synth.TID["A"])
    bufB, B2 = _padded(nn, nn, nn + ld_pad, 4, synth.TID["B"])
    sc = kf.Script()
    sc.matrix("A", nn, nn, ld=nn + ld_pad); sc.matrix("B", nn, nn, ld=nn + ld_pad)
    for v in ("u1", "v1", "u2", "v2", "y", "z", "x", "w", "t"):
        sc.vector(v, nn)
    sc.input("A", "u1", "v1", "u2", "v2", "y", "z"); sc.output("B", "x", "w")
    sc.call("GER", ["B"], ["A", "u1", "v1"], [1.0])
    sc.call("GER", ["B"], ["B", "u2", "v2"], [1.0])
    sc.call("GEMVT", ["t"], ["B", "y"], [1.0, 0.0])
    sc.call("AXPBY", ["x"], ["t", "z"], [1.2, 1.0])
    sc.call("GEMV", ["w"], ["B", "x"], [1.5, 0.0])
    vs = {v: synth.uniform((nn,), 4, synth.TID[v], device=dev()) for v in ("u1", "v1", "u2", "v2", "y", "z")}
    pg = sc.plan(kf.KF_PLAN_ANALYTIC)
    bg = dict(vs, A=A2, B=B2, x=torch.empty(nn, device=dev()), w=torch.empty(nn, device=dev()),
              t=torch.empty(nn, device=dev()))
    pg.execute(bg, torch.zeros(max(pg.workspace_size(), 256), dtype=torch.uint8, device=dev()))
    torch.cuda.synchronize()
    Bo, xo, wo = oracle.gemver(host(A2), *[host(vs[k]) for k in ("u1", "v1", "u2", "v2", "y", "z")], 1.5, 1.2)
    assert np.max(np.abs(host(B2) - Bo)) <= 4 * 2.0 ** -24 * 4.0 * (1 + np.max(np.abs(Bo)))
    pad = bufB[:nn * (nn + ld_pad)].view(nn, nn + ld_pad)[:, nn:]
    assert torch.all(pad == 12345.0) and torch.all(bufB[nn * (nn + ld_pad):] == 12345.0)
    sx = 1.2 * oracle.abs_gemvt(Bo, host(vs["y"])) + np.abs(host(vs["z"]))
    check_reduce(host(bg["x"]), xo, sx, nn, "x")
    check_reduce(host(bg["w"]), wo, 1.5 * oracle.abs_gemv(Bo, np.abs(xo) + sx), nn, "w")
    # ATAX pair on the strided A of the BiCGK case
    sa = kf.Script()
    sa.matrix("A", m, n, ld=ld); sa.vector("x", n); sa.vector("t", m); sa.vector("y", n)
    sa.input("A", "x"); sa.output("y")
    sa.call("GEMV", ["t"], ["A", "x"], [1.5, 0.0])
    sa.call("GEMVT", ["y"], ["A", "t"], [-0.5, 0.0])
    pa = sa.plan(kf.KF_PLAN_ANALYTIC)
    ba = {"A": A, "x": p, "t": torch.empty(m, device=dev()), "y": torch.empty(n, device=dev())}
    pa.execute(ba, torch.zeros(max(pa.workspace_size(), 256), dtype=torch.uint8, device=dev()))
    yo, _ = oracle.atax(Ah, host(p))
    check_reduce(host(ba["y"]), -0.75 * yo, 0.75 * oracle.abs_gemvt(Ah, oracle.abs_gemv(Ah, host(p))), max(m, n),
                 "atax strided")
    with pytest.raises(ValueError):
        pa.execute(dict(ba, A=A.contiguous()), torch.zeros(max(pa.workspace_size(), 256), dtype=torch.uint8,
                                                           device=dev()))
