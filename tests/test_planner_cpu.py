"""Planner host logic (no GPU): dependency analysis, fusion legality, plan
enumeration and the analytic choice, on the canonical scripts of Table 1.

The expected fusions follow from the rules of Section 3.2: calls that share
data and have the same nesting depth fuse; a reduction result (DOT, GEMV,
GEMVT) is never consumed in the kernel that computes it, except by a linear
epilogue map after the last-block barrier.
"""

import pytest

ALPHA, BETA = 1.5, 1.2


@pytest.fixture(scope="module")
def kf():
    from paper_1305_1183_gb300 import _build, kf as K
    _build.build()
    K.lib()
    return K


def bicgk(kf, m=64, n=48):
    s = kf.Script()
    s.matrix("A", m, n); s.vector("p", n); s.vector("r", m); s.vector("q", m); s.vector("s", n)
    s.input("A", "p", "r"); s.output("q", "s")
    s.call("GEMV", ["q"], ["A", "p"], [1.0, 0.0])
    s.call("GEMVT", ["s"], ["A", "r"], [1.0, 0.0])
    return s


def gemver(kf, n=40):
    s = kf.Script()
    s.matrix("A", n, n); s.matrix("B", n, n)
    for v in ("u1", "v1", "u2", "v2", "y", "z", "x", "w", "t"):
        s.vector(v, n)
    s.input("A", "u1", "v1", "u2", "v2", "y", "z"); s.output("B", "x", "w")
    s.call("GER", ["B"], ["A", "u1", "v1"], [1.0])
    s.call("GER", ["B"], ["B", "u2", "v2"], [1.0])
    s.call("GEMVT", ["t"], ["B", "y"], [1.0, 0.0])
    s.call("AXPBY", ["x"], ["t", "z"], [BETA, 1.0])
    s.call("GEMV", ["w"], ["B", "x"], [ALPHA, 0.0])
    return s


def gesummv(kf, n=40):
    s = kf.Script()
    s.matrix("A", n, n); s.matrix("B", n, n)
    for v in ("x", "y", "t1", "t2"):
        s.vector(v, n)
    s.input("A", "B", "x"); s.output("y")
    s.call("GEMV", ["t1"], ["A", "x"], [ALPHA, 0.0])
    s.call("GEMV", ["t2"], ["B", "x"], [BETA, 0.0])
    s.call("AXPBY", ["y"], ["t1", "t2"], [1.0, 1.0])
    return s


def atax(kf, n=40):
    s = kf.Script()
    s.matrix("A", n, n); s.vector("x", n); s.vector("t", n); s.vector("y", n)
    s.input("A", "x"); s.output("y")
    s.call("GEMV", ["t"], ["A", "x"], [1.0, 0.0])
    s.call("GEMVT", ["y"], ["A", "t"], [1.0, 0.0])
    return s


def axpydot(kf, n=1000):
    s = kf.Script()
    for v in ("w", "v", "u", "z"):
        s.vector(v, n)
    s.scalar("r")
    s.input("w", "v", "u"); s.output("z", "r")
    s.call("AXPBY", ["z"], ["w", "v"], [1.0, -ALPHA])
    s.call("DOT", ["r"], ["z", "u"])
    return s


def waxpby(kf, n=1000):
    s = kf.Script()
    for v in ("x", "y", "t", "w"):
        s.vector(v, n)
    s.input("x", "y"); s.output("w")
    s.call("SCAL", ["t"], ["x"], [ALPHA])
    s.call("AXPBY", ["w"], ["y", "t"], [BETA, 1.0])
    return s


@pytest.mark.parametrize("name,nplans,fused_kernels", [
    ("bicgk", 2, 1), ("gemver", None, 2), ("gesummv", None, 1), ("atax", 2, 1),
    ("axpydot", 2, 1), ("waxpby", 2, 1)])
def test_canonical_scripts(kf, name, nplans, fused_kernels):
    s = globals()[name](kf)
    s.validate()
    count, trunc = s.count_plans()
    assert not trunc
    if nplans is not None:
        assert count == nplans
    ncalls = len(s.shapes) and None
    unf = s.plan(kf.KF_PLAN_UNFUSED)
    p = s.plan(kf.KF_PLAN_ANALYTIC)
    assert p.kernel_count() == fused_kernels
    assert p.predicted_us() <= unf.predicted_us() + 1e-9
    g = s.plan(kf.KF_PLAN_GREEDY)
    assert g.kernel_count() <= p.kernel_count()
    d = p.describe()
    assert len(d["kernels"]) == fused_kernels
    assert sum(len(k["calls"]) for k in d["kernels"]) == unf.kernel_count()
    assert len(p.features()) == 16
    assert ncalls is None


def _atax_script(kf, m, n, t_out=False, beta=0.0, a1=1.0, a2=1.0):
    s = kf.Script()
    s.matrix("A", m, n); s.vector("x", n); s.vector("t", m); s.vector("y", n); s.vector("y0", m)
    s.input("A", "x", "y0"); s.output("y")
    if t_out:
        s.output("t")
    s.call("GEMV", ["t"], ["A", "x", "y0"] if beta else ["A", "x"], [a1, beta])
    s.call("GEMVT", ["y"], ["A", "t"], [a2, 0.0])
    return s


def test_atax_single_pass_fusion(kf):
    """{t = a1 A x; y = a2 A^T t}: the GEMV result is consumed in the same
    kernel, which is legal only for the row-owning single pass (one read of
    A, Section 4.2's persistent row reuse): one "atax" kernel moving
    4 (m n + 2 n) bytes, scale a1 a2."""
    m, n = 300, 512
    s = _atax_script(kf, m, n, a1=1.5, a2=-0.5)
    assert s.count_plans()[0] == 2
    d = s.plan(kf.KF_PLAN_ANALYTIC).describe()
    assert [k["kind"] for k in d["kernels"]] == ["atax"]
    assert d["bytes"] == 4 * (m * n + 2 * n)
    assert [b[0] for b in d["kernels"][0]["bind"]] == ["A", "x", "y"]
    assert s.plan(kf.KF_PLAN_GREEDY).kernel_count() == 1


@pytest.mark.parametrize("case", ["t_is_output", "gemv_accumulates", "row_too_long", "row_not_float4"])
def test_atax_fusion_refused(kf, case):
    """No single pass when t is needed after the kernel, when the GEMV adds a
    term the rows pass does not compute, or when a row does not fit the
    ring's 16-byte chunks (n > 16384 or n not a multiple of 4): the paper's
    two kernels remain."""
    m, n = 100, 512
    kw = {}
    if case == "t_is_output":
        kw["t_out"] = True
    elif case == "gemv_accumulates":
        kw["beta"] = 1.0
    elif case == "row_too_long":
        n = 16388
    else:
        n = 514
    s = _atax_script(kf, m, n, **kw)
    assert s.count_plans()[0] == 1
    assert s.plan(kf.KF_PLAN_ANALYTIC).kernel_count() == 2


def test_gemver_fusion_shape(kf):
    """GEMVER: {GER, GER, GEMVT, AXPBY epilogue} then {GEMV} (w needs all of x)."""
    d = gemver(kf).plan(kf.KF_PLAN_ANALYTIC).describe()
    assert [k["calls"] for k in d["kernels"]] == [[0, 1, 2, 3], [4]]
    assert [k["kind"] for k in d["kernels"]] == ["matrix", "matrix"]
    # bytes: A read, B written; then B read (vectors small)
    n = 40
    assert abs(d["bytes"] - (3 * 4 * n * n + 4 * n * 9)) < 4 * n * 2


def test_gesummv_epilogue_and_bytes(kf):
    d = gesummv(kf).plan(kf.KF_PLAN_ANALYTIC).describe()
    assert [k["calls"] for k in d["kernels"]] == [[0, 1, 2]]
    n = 40
    assert d["bytes"] == 4 * (2 * n * n + 2 * n)


def test_errors(kf):
    s = kf.Script()
    s.vector("x", 10); s.vector("y", 10); s.vector("z", 11)
    s.input("x")
    s.call("AXPBY", ["z"], ["x", "y"])
    with pytest.raises(kf.KFError) as e:
        s.validate()
    assert e.value.status == -2                 # shape
    s = kf.Script()
    s.vector("x", 10); s.vector("y", 10); s.vector("z", 10)
    s.input("x")
    s.call("AXPBY", ["z"], ["x", "y"])
    with pytest.raises(kf.KFError) as e:
        s.validate()
    assert e.value.status == -6                 # y read before written
    s = kf.Script()
    s.matrix("A", 8, 8); s.vector("x", 8)
    s.input("A", "x")
    s.call("GEMV", ["x"], ["A", "x"])
    with pytest.raises(kf.KFError):
        s.validate()                            # GEMV may not overwrite its x


def test_dependencies_respected(kf):
    """AXPY in place then DOT of the old value: the DOT must run first
    (write-after-read edge); in one vector pass both see per-element order."""
    s = kf.Script()
    for v in ("x", "y"):
        s.vector(v, 100)
    s.scalar("d1"); s.scalar("d2")
    s.input("x", "y"); s.output("y", "d1", "d2")
    s.call("DOT", ["d1"], ["x", "y"])
    s.call("AXPBY", ["y"], ["x", "y"], [2.0, 1.0])
    s.call("DOT", ["d2"], ["x", "y"])
    count, _ = s.count_plans()
    assert count >= 2
    p = s.plan(kf.KF_PLAN_ANALYTIC)
    assert p.kernel_count() == 1


def test_reduction_results_not_consumed_in_kernel(kf):
    """A GEMV result feeding a GEMVT (ATAX) or a DOT of a map of it never
    shares a kernel with its producer."""
    s = kf.Script()
    s.matrix("A", 16, 16)
    for v in ("x", "t", "u"):
        s.vector(v, 16)
    s.scalar("d")
    s.input("A", "x"); s.output("d")
    s.call("GEMV", ["t"], ["A", "x"])
    s.call("SCAL", ["u"], ["t"], [3.0])
    s.call("DOT", ["d"], ["u", "x"])
    for i in range(s.count_plans()[0]):
        d = s.plan(kf.KF_PLAN_INDEX, index=i).describe()
        for k in d["kernels"]:
            assert not (0 in k["calls"] and 2 in k["calls"])


def test_enumeration_cap(kf):
    s = kf.Script()
    for v in range(8):
        s.vector(f"v{v}", 64)
    s.input("v0", "v1")
    for i in range(2, 8):
        s.call("AXPBY", [f"v{i}"], [f"v{i - 1}", f"v{i - 2}"], [0.5, 0.25])
    s.output("v7")
    c, t = s.count_plans(cap=10)
    assert c == 10 and t


def _groupings(kf, s):
    """The kernels (lists of call indices) of every enumerated plan."""
    c, _ = s.count_plans()
    return [[k["calls"] for k in s.plan(kf.KF_PLAN_INDEX, index=i).describe()["kernels"]] for i in range(c)]


def test_fusion_refused_across_lengths_and_shapes(kf):
    """Vector calls of different lengths, and GEMVs on matrices of different
    shapes, never share a kernel (Section 3.2: fused calls iterate over the
    same index space)."""
    s = kf.Script()
    s.vector("x", 100); s.vector("y", 100); s.vector("a", 50); s.vector("b", 50)
    s.input("x", "a"); s.output("y", "b")
    s.call("SCAL", ["y"], ["x"], [2.0]); s.call("SCAL", ["b"], ["a"], [2.0])
    assert _groupings(kf, s) == [[[0], [1]]]
    s = kf.Script()
    s.matrix("A", 64, 32); s.matrix("B", 48, 32)
    s.vector("x", 32); s.vector("y", 64); s.vector("z", 48)
    s.input("A", "B", "x"); s.output("y", "z")
    s.call("GEMV", ["y"], ["A", "x"]); s.call("GEMV", ["z"], ["B", "x"])
    assert _groupings(kf, s) == [[[0], [1]]]


def test_at_most_two_matrices_per_kernel(kf):
    """GEMVs of three matrices sharing x: every pair may fuse (GESUMMV's
    shape), the three together may not."""
    s = kf.Script()
    for M in "ABC":
        s.matrix(M, 32, 32)
    for v in ("x", "y1", "y2", "y3"):
        s.vector(v, 32)
    s.input("A", "B", "C", "x"); s.output("y1", "y2", "y3")
    for i, M in enumerate("ABC"):
        s.call("GEMV", [f"y{i + 1}"], [M, "x"])
    g = _groupings(kf, s)
    assert all(len(k) <= 2 for plan in g for k in plan)
    pairs = {tuple(k) for plan in g for k in plan if len(k) == 2}
    assert pairs == {(0, 1), (0, 2), (1, 2)}


def test_epilogue_never_mixes_row_and_column_results(kf):
    """u = q + s with q = A p (row-indexed) and s = A^T r (column-indexed):
    the map may join the kernel of one of them once the other is complete,
    never the kernel that produces both."""
    s = kf.Script()
    s.matrix("A", 32, 32)
    for v in ("p", "r", "q", "s", "u"):
        s.vector(v, 32)
    s.input("A", "p", "r"); s.output("u")
    s.call("GEMV", ["q"], ["A", "p"]); s.call("GEMVT", ["s"], ["A", "r"])
    s.call("AXPBY", ["u"], ["q", "s"], [1.0, 1.0])
    g = _groupings(kf, s)
    assert not any(sorted(k) == [0, 1, 2] for plan in g for k in plan)
    assert any([0, 1] in plan for plan in g)            # the BiCGK core still fuses
    assert any(sorted(k) == [0, 2] for plan in g for k in plan)
    assert any(sorted(k) == [1, 2] for plan in g for k in plan)


def test_analytic_predictor_is_max_of_transfer_and_compute_plus_launch(kf):
    """Per kernel: max(bytes / bandwidth, flops / FP32 rate) + launch cost
    (Section 3.2's max(t_t, t_c), plus the per-kernel cost), summed over
    kernels.  BiCGK 16384^2: 4mn flops (2 per multiply-add) at 80 TFLOP/s."""
    m = n = 16384
    try:
        kf.kf_planner_set_model(1000.0, 3.0)            # 1 TB/s: transfer bound
        s = bicgk(kf, m, n)
        for mode in (kf.KF_PLAN_ANALYTIC, kf.KF_PLAN_UNFUSED):
            p = s.plan(mode)
            d = p.describe()
            want = sum(k["bytes"] / 1e12 * 1e6 + 3.0 for k in d["kernels"])
            assert p.predicted_us() == pytest.approx(want, rel=1e-5)
        kf.kf_planner_set_model(1e9, 3.0)               # bandwidth out of the way: compute bound
        p = bicgk(kf, m, n).plan(kf.KF_PLAN_ANALYTIC)
        assert p.predicted_us() == pytest.approx(4.0 * m * n / 80e12 * 1e6 + 3.0, rel=1e-3)
        with pytest.raises(kf.KFError):
            kf.kf_planner_set_model(0.0, 3.0)
        with pytest.raises(kf.KFError):
            kf.kf_planner_set_model(1000.0, -1.0)
    finally:
        kf.kf_planner_set_model(6500.0, 2.0)            # the built-in model


def test_plan_features_describe_the_plan(kf):
    """The 16 features of the learned cost model match what the plan is:
    kernel counts by kind, log2 of bytes (total, matrix, vector), log2 n,
    calls per kernel, matrix ops per kernel, dependent finishing phases,
    epilogue outputs, matrix stores, log2 of the analytic prediction."""
    import math
    n = 4096
    s = gemver(kf, n)
    fused, unf = s.plan(kf.KF_PLAN_ANALYTIC), s.plan(kf.KF_PLAN_UNFUSED)
    for p in (fused, unf):
        f, d = p.features(), p.describe()
        assert f[0] == p.kernel_count() == f[1] + f[2]
        assert f[3] == pytest.approx(math.log2(1 + d["bytes"]), abs=1e-4)
        assert f[6] == pytest.approx(math.log2(n))
        assert f[7] == pytest.approx(5 / p.kernel_count())          # GEMVER's 5 calls
        assert f[13] == pytest.approx(math.log2(1 + p.predicted_us()), abs=1e-4)
    f, fu = fused.features(), unf.features()
    assert (f[1], f[2]) == (2, 0)                       # {GER, GER, GEMVT, AXPBY} and {GEMV}
    assert f[8] == 3                                     # GER, GER, GEMVT in one pass
    assert f[15] == 1 and fu[15] == 2                    # B stored once; twice by the GER chain
    assert f[4] == pytest.approx(math.log2(1 + 2 * 4.0 * n * n), abs=1e-3)   # matrix reads: A, then B
    assert f[5] == pytest.approx(math.log2(1 + fused.describe()["bytes"] - 2 * 4.0 * n * n), abs=1e-3)
    assert fu[3] > f[3] + 0.9                            # the chain moves about twice the bytes
    g = bicgk(kf, 2048, 2048).plan(kf.KF_PLAN_ANALYTIC).features()
    assert (g[0], g[1], g[8], g[9], g[10]) == (1, 1, 2, 1, 1)   # row and column results: two finishes


def _random_valid_script(rng, n, m):
    """A valid script over vectors of length n ("x") and m ("y") and m x n
    matrices, every operand written or declared input before it is read."""
    kinds, inputs, calls = {}, [], []

    def new(kind):
        nm = f"{kind}{len(kinds)}"
        kinds[nm] = kind
        return nm

    def pick(kind):
        pool = sorted(k for k, v in kinds.items() if v == kind)
        if pool and rng.random() < 0.7:
            return rng.choice(pool)
        nm = new(kind)
        inputs.append(nm)
        return nm

    for _ in range(rng.randint(1, 9)):
        op = rng.choice(["AXPBY", "SCAL", "DOT", "VADD", "GEMV", "GEMVT", "GER"])
        vk = rng.choice("xy")
        a, b = rng.uniform(-1, 1), rng.uniform(-1, 1)
        if op == "AXPBY":
            ins = [pick(vk), pick(vk)]
            out, sc = (ins[1] if rng.random() < 0.5 else pick(vk)), [a, b]
        elif op == "SCAL":
            ins = [pick(vk)]
            out, sc = (ins[0] if rng.random() < 0.5 else pick(vk)), [a]
        elif op == "VADD":
            ins, out, sc = [pick(vk), pick(vk), pick(vk)], pick(vk), []
        elif op == "DOT":
            ins, out, sc = [pick(vk), pick(vk)], new("s"), []
        elif op in ("GEMV", "GEMVT"):
            src, dst = ("x", "y") if op == "GEMV" else ("y", "x")
            ins = [pick("A"), pick(src)] + ([pick(dst)] if rng.random() < 0.3 else [])
            out = pick(dst)
            if out in ins[1:]:
                out = new(dst)
            sc = [a, b]
        else:
            ins = [pick("A"), pick("y"), pick("x")]
            out, sc = (ins[0] if rng.random() < 0.6 else new("A")), [a]
        calls.append((op, [out], ins, sc))
    return kinds, sorted(set(inputs)), calls


def test_random_scripts_every_plan_is_well_formed(kf):
    """Every enumerated plan of 300 random valid scripts (sizes 1 to 64,
    square and not) covers each call once, orders its kernels so that every
    read-after-write, write-after-read and write-after-write dependency
    points forward, and never feeds a GEMV / GEMVT result to a matrix op of
    the kernel that computes it."""
    import random
    rng = random.Random(1305)
    nplans = 0
    for _ in range(300):
        n = rng.choice([1, 2, 7, 33, 64])
        m = rng.choice([n, 5])
        kinds, inputs, calls = _random_valid_script(rng, n, m)
        s = kf.Script()
        for nm, kd in kinds.items():
            if kd == "x":
                s.vector(nm, n)
            elif kd == "y":
                s.vector(nm, m)
            elif kd == "A":
                s.matrix(nm, m, n)
            else:
                s.scalar(nm)
        s.input(*inputs)
        written = sorted({c[1][0] for c in calls})
        s.output(*rng.sample(written, rng.randint(1, len(written))))
        for op, outs, ins, sc in calls:
            s.call(op, outs, ins, sc)
        s.validate()
        # dependencies: (earlier call, later call, reduction result consumed by a matrix op)
        deps, last_w, readers = [], {}, {}
        for j, (op, outs, ins, _) in enumerate(calls):
            for pos, v in enumerate(ins):
                if v in last_w:
                    i = last_w[v]
                    deep = calls[i][0] in ("GEMV", "GEMVT") and op in ("GEMV", "GEMVT", "GER") and pos > 0
                    deps.append((i, j, deep))
                readers.setdefault(v, []).append(j)
            o = outs[0]
            deps += [(i, j, False) for i in readers.get(o, []) if i != j]
            if o in last_w:
                deps.append((last_w[o], j, False))
            last_w[o], readers[o] = j, []
        count, _ = s.count_plans(cap=100)
        assert count >= 1
        for idx in range(count):
            p = s.plan(kf.KF_PLAN_INDEX, index=idx, max_plans=100)
            kernels = [k["calls"] for k in p.describe()["kernels"]]
            assert sorted(c for k in kernels for c in k) == list(range(len(calls))), kernels
            where = {c: ki for ki, k in enumerate(kernels) for c in k}
            for i, j, deep in deps:
                assert where[i] <= where[j], (calls, kernels, i, j)
                assert not (deep and where[i] == where[j]), (calls, kernels, i, j)
            assert p.predicted_us() > 0 and p.workspace_size() >= 0 and len(p.features()) == 16
            nplans += 1
    assert nplans > 1000


# ------------------------------------------------------------ call-order search (Section 3.2, variant (i))

def bicgk_reversed(kf, m=64, n=48):
    """BiCGK with its two calls in the other order: s = A^T r first."""
    s = kf.Script()
    s.matrix("A", m, n); s.vector("p", n); s.vector("r", m); s.vector("q", m); s.vector("s", n)
    s.input("A", "p", "r"); s.output("q", "s")
    s.call("GEMVT", ["s"], ["A", "r"], [1.0, 0.0])
    s.call("GEMV", ["q"], ["A", "p"], [1.0, 0.0])
    return s


def _matrix_kernels(d):
    return [k for k in d["kernels"] if k["kind"] == "matrix"]


def test_call_order_keeps_a_specialised_script_order(kf):
    """The canonical scripts already list their calls in the order of a
    specialised instance: the search keeps script order."""
    for builder, n_calls in ((bicgk, 2), (gesummv, 3)):
        (k,) = _matrix_kernels(builder(kf).plan(kf.KF_PLAN_ANALYTIC).describe())
        assert k["specialised"] is True
        assert k["order"] == sorted(k["order"]) and len(k["order"]) == n_calls
    ks = _matrix_kernels(gemver(kf).plan(kf.KF_PLAN_ANALYTIC).describe())
    assert [k["specialised"] for k in ks] == [True, True]
    assert ks[0]["order"] == [0, 1, 2, 3] and ks[1]["order"] == [4]


def test_call_order_search_reorders_independent_calls(kf):
    """s = A^T r listed before q = A p: no variable is written by one call
    and used by the other, so they may swap; the swapped order is the
    specialised BiCGK signature, which the search picks."""
    (k,) = _matrix_kernels(bicgk_reversed(kf).plan(kf.KF_PLAN_ANALYTIC).describe())
    assert k["calls"] == [0, 1]
    assert k["order"] == [1, 0]
    assert k["specialised"] is True


def test_call_order_search_keeps_ger_fences(kf):
    """A GEMV of A listed before the GER that rewrites A (in place in the
    kernel's rows) and a GEMVT of the new version after it: every pair
    shares A with one writer, so only script order is legal, and no
    instance is specialised for it."""
    n = 40
    s = kf.Script()
    s.matrix("A", n, n)
    for v in ("u", "v", "x", "r", "q", "t"):
        s.vector(v, n)
    s.input("A", "u", "v", "x", "r"); s.output("A", "q", "t")
    s.call("GEMV", ["q"], ["A", "x"], [1.0, 0.0])
    s.call("GER", ["A"], ["A", "u", "v"], [1.0])
    s.call("GEMVT", ["t"], ["A", "r"], [1.0, 0.0])
    fused = 0
    for i in range(s.count_plans()[0]):
        for k in _matrix_kernels(s.plan(kf.KF_PLAN_INDEX, index=i).describe()):
            fused += len(k["order"]) > 1
            pos = {c: j for j, c in enumerate(k["order"])}
            for a, b in ((0, 1), (1, 2), (0, 2)):
                if a in pos and b in pos:
                    assert pos[a] < pos[b], (i, k)
    assert fused > 0  # some plan fuses the GER with a reader


def test_call_order_search_never_crosses_a_fence_for_a_specialised_order(kf):
    """t = A^T y on the old A, then two GERs rewriting A.  The kinds of
    (GER, GER, GEMVT) are those of the specialised GEMVER pass 1, but there
    the GEMVT reads the rewritten rows; here it reads the old version, which
    after the GERs would be a second matrix (another signature), so no
    reordering matches an instance: the search keeps script order and
    reports none.  (The conflict rule also forbids the move: the GERs write
    the variable the GEMVT reads.)"""
    n = 40
    s = kf.Script()
    s.matrix("A", n, n)
    for v in ("u1", "v1", "u2", "v2", "y", "t"):
        s.vector(v, n)
    s.input("A", "u1", "v1", "u2", "v2", "y"); s.output("A", "t")
    s.call("GEMVT", ["t"], ["A", "y"], [1.0, 0.0])
    s.call("GER", ["A"], ["A", "u1", "v1"], [1.0])
    s.call("GER", ["A"], ["A", "u2", "v2"], [1.0])
    seen = 0
    for i in range(s.count_plans()[0]):
        for k in _matrix_kernels(s.plan(kf.KF_PLAN_INDEX, index=i).describe()):
            if k["order"] == [0, 1, 2] or sorted(k["order"]) == [0, 1, 2]:
                assert k["order"] == [0, 1, 2] and k["specialised"] is False, (i, k)
                seen += 1
    assert seen > 0  # some plan fuses all three


def test_strided_script_matrix(kf):
    """kf_script_matrix_ld: a row stride below n is refused; a strided
    matrix plans exactly like a packed one (the stride only changes the
    kernels' addressing)."""
    s = kf.Script()
    with pytest.raises(kf.KFError) as e:
        s.matrix("A", 8, 16, ld=15)
    assert e.value.status == kf.KF_ERR_SHAPE

    def build(ld):
        s = kf.Script()
        s.matrix("A", 64, 48, ld=ld); s.vector("p", 48); s.vector("r", 64); s.vector("q", 64); s.vector("s", 48)
        s.input("A", "p", "r"); s.output("q", "s")
        s.call("GEMV", ["q"], ["A", "p"], [1.0, 0.0])
        s.call("GEMVT", ["s"], ["A", "r"], [1.0, 0.0])
        return s.plan(kf.KF_PLAN_ANALYTIC).describe()

    a, b = build(None), build(53)
    assert [(k["kind"], k["calls"], k["order"]) for k in a["kernels"]] == \
           [(k["kind"], k["calls"], k["order"]) for k in b["kernels"]]
    assert a["bytes"] == b["bytes"]
