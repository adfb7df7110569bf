"""Each entry point returns the status its declaration in include/kf.h
documents, for each kind of bad argument (no GPU).

Every call below breaks at least one rule, so it returns from argument
checking before any device work: stand-in addresses are never dereferenced.
"""

import ctypes

import pytest

P = 1 << 16                # stand-in device address (16-byte aligned, never dereferenced)
Q = 1 << 20                # a second one
F32, BF16, E4M3 = 0, 1, 2


@pytest.fixture(scope="module")
def L():
    from paper_1305_1183_gb300 import _build, kf
    _build.build()
    return kf.lib()


@pytest.fixture(scope="module")
def K():
    from paper_1305_1183_gb300 import kf
    return kf


def _ws_size(L, seq, m, n, fmt=F32):
    b = ctypes.c_size_t(0)
    assert L.kf_workspace_size(seq, m, n, fmt, ctypes.byref(b)) == 0
    return b.value


def test_gemver_errors(L, K):
    n = 8
    ok = dict(n=n, A=P, lda=n, u1=P, v1=P, u2=P, v2=P, y=P, z=P, alpha=1.5, beta=1.2, B=Q, ldb=n, x=P, w=P)

    def call(**kw):
        a = dict(ok, **kw)
        return L.kf_gemver(a["n"], a["A"], a["lda"], a["u1"], a["v1"], a["u2"], a["v2"], a["y"], a["z"],
                           a["alpha"], a["beta"], a["B"], a["ldb"], a["x"], a["w"], None, 0, None)
    assert call(n=-1) == K.KF_ERR_INVALID_ARG
    assert call(A=None) == K.KF_ERR_INVALID_ARG
    assert call(lda=n - 1) == K.KF_ERR_SHAPE
    assert call(ldb=n - 1) == K.KF_ERR_SHAPE
    for v in ("u1", "v1", "u2", "v2", "y", "z", "x", "w"):
        assert call(**{v: None}) == K.KF_ERR_INVALID_ARG, v
        assert v.encode() in L.kf_last_error()
    assert call(B=P, lda=2 * n, ldb=n) == K.KF_ERR_SHAPE          # in place with ldb != lda
    assert call() == K.KF_ERR_WORKSPACE                             # no workspace


def test_gemver_q_errors(L, K):
    n = 8

    def call(fmt=BF16, sA=P, QB=Q, sB=P, ws=None, wsb=0, lda=n):
        return L.kf_gemver_q(n, P, lda, fmt, sA, P, P, P, P, P, P, 1.5, 1.2, QB, n, sB, P, P, ws, wsb, None)
    assert call(fmt=F32) == K.KF_ERR_DTYPE
    assert call(fmt=7) == K.KF_ERR_DTYPE
    assert call(sA=None) == K.KF_ERR_INVALID_ARG
    assert call(sB=None) == K.KF_ERR_INVALID_ARG
    assert call(QB=P) == K.KF_ERR_SHAPE                             # QB aliases QA
    assert call(lda=n - 1) == K.KF_ERR_SHAPE
    assert call(fmt=E4M3) == K.KF_ERR_WORKSPACE
    assert call(fmt=E4M3, ws=Q, wsb=16) == K.KF_ERR_WORKSPACE        # below the header
    # above the header but short of the passes' partial sums: refused before
    # the norm pre-pass is enqueued
    assert call(fmt=E4M3, ws=Q, wsb=4096) == K.KF_ERR_WORKSPACE
    assert b"kf_workspace_size" in L.kf_last_error()


def test_gesummv_atax_errors(L, K):
    m, n = 8, 12
    g = lambda A=P, B=Q, lda=n, x=P, y=P, ws=None, wsb=0: L.kf_gesummv(  # noqa: E731
        m, n, A, B, lda, x, 1.5, 1.2, y, ws, wsb, None)
    assert g(B=None) == K.KF_ERR_INVALID_ARG
    assert g(lda=n - 1) == K.KF_ERR_SHAPE
    assert g(x=None) == K.KF_ERR_INVALID_ARG and g(y=None) == K.KF_ERR_INVALID_ARG
    assert g() == K.KF_ERR_WORKSPACE
    assert g(ws=Q, wsb=_ws_size(L, K.KF_SEQ_GESUMMV, m, n) - 1) == K.KF_ERR_WORKSPACE
    a = lambda lda=n, x=P, y=Q, ws=None: L.kf_atax(m, n, P, lda, x, y, ws, 0, None)  # noqa: E731
    assert a(x=None) == K.KF_ERR_INVALID_ARG and a(y=None) == K.KF_ERR_INVALID_ARG
    assert a(lda=n - 1) == K.KF_ERR_SHAPE
    assert a() == K.KF_ERR_WORKSPACE
    assert a(x=P + 4) == K.KF_ERR_WORKSPACE                         # unaligned: two-pass form, same rule


def test_bicgk_and_elementary_matrix_errors(L, K):
    m, n = 8, 12
    b = lambda fmt=F32, rs=None, ws=None, wsb=0: L.kf_bicgk(  # noqa: E731
        m, n, P, n, fmt, rs, P, P, Q, Q, ws, wsb, None)
    assert b(fmt=BF16) == K.KF_ERR_INVALID_ARG                      # row scales required
    assert b() == K.KF_ERR_WORKSPACE
    assert b(ws=Q, wsb=_ws_size(L, K.KF_SEQ_BICGK, m, n) - 1) == K.KF_ERR_WORKSPACE
    gv = lambda fmt=F32, beta=0.0, y0=None, ws=None: L.kf_gemv(  # noqa: E731
        m, n, P, n, fmt, None, 1.0, P, beta, y0, Q, ws, 0, None)
    assert gv(fmt=5) == K.KF_ERR_DTYPE
    assert gv(fmt=E4M3) == K.KF_ERR_INVALID_ARG
    assert gv(beta=1.0) == K.KF_ERR_INVALID_ARG                     # y0 needed when beta != 0
    assert gv() == K.KF_ERR_WORKSPACE
    gt = lambda beta=0.0, x0=None, lda=n: L.kf_gemvt(  # noqa: E731
        m, n, P, lda, F32, None, 1.0, P, beta, x0, Q, None, 0, None)
    assert gt(beta=2.0) == K.KF_ERR_INVALID_ARG
    assert gt(lda=n - 1) == K.KF_ERR_SHAPE
    assert gt() == K.KF_ERR_WORKSPACE
    gr = lambda u=P, v=P, B=Q, ldb=n: L.kf_ger(m, n, P, n, 1.0, u, v, B, ldb, None)  # noqa: E731
    assert gr(u=None) == K.KF_ERR_INVALID_ARG and gr(v=None) == K.KF_ERR_INVALID_ARG
    assert gr(B=None) == K.KF_ERR_INVALID_ARG
    assert gr(ldb=n - 1) == K.KF_ERR_SHAPE
    md = lambda A=P, lda=n, ldb=n, ldc=n: L.kf_madd(m, n, A, lda, Q, ldb, Q, ldc, None)  # noqa: E731
    assert md(A=None) == K.KF_ERR_INVALID_ARG
    assert md(lda=n - 1) == K.KF_ERR_SHAPE and md(ldb=n - 1) == K.KF_ERR_SHAPE and md(ldc=n - 1) == K.KF_ERR_SHAPE
    qr = lambda fmt=BF16, Qp=Q, rs=P: L.kf_quantize_rows(m, n, P, n, fmt, Qp, rs, None)  # noqa: E731
    assert qr(fmt=F32) == K.KF_ERR_DTYPE
    assert qr(Qp=None) == K.KF_ERR_INVALID_ARG and qr(rs=None) == K.KF_ERR_INVALID_ARG


def test_vector_errors(L, K):
    n = 100
    assert L.kf_waxpby(-1, 1.0, P, 1.0, P, Q, None) == K.KF_ERR_INVALID_ARG
    assert L.kf_waxpby(n, 1.0, None, 1.0, P, Q, None) == K.KF_ERR_INVALID_ARG
    assert L.kf_waxpby(n, 1.0, P, 1.0, P, None, None) == K.KF_ERR_INVALID_ARG
    assert L.kf_axpydot(n, P, P, P, 1.5, Q, None, None, 0, None) == K.KF_ERR_INVALID_ARG       # null r
    assert L.kf_axpydot(n, P, None, P, 1.5, Q, Q, None, 0, None) == K.KF_ERR_INVALID_ARG
    assert L.kf_axpydot(n, P, P, P, 1.5, Q, Q, None, 0, None) == K.KF_ERR_WORKSPACE
    assert L.kf_axpby(n, 1.0, P, 1.0, None, Q, None) == K.KF_ERR_INVALID_ARG                  # y with beta != 0
    assert L.kf_axpby(-3, 1.0, P, 0.0, None, Q, None) == K.KF_ERR_INVALID_ARG
    assert L.kf_scal(n, 2.0, None, Q, None) == K.KF_ERR_INVALID_ARG
    assert L.kf_vadd3(n, P, P, None, Q, None) == K.KF_ERR_INVALID_ARG
    assert L.kf_dot(n, P, P, None, Q, 4096, None) == K.KF_ERR_INVALID_ARG
    assert L.kf_dot(n, P, P, Q, None, 0, None) == K.KF_ERR_WORKSPACE
    assert L.kf_dot(n, P, P, Q, Q, 8, None) == K.KF_ERR_WORKSPACE


def test_empty_problems_return_before_any_launch(L, K):
    """Empty sizes are valid and need no pointers or workspace."""
    assert L.kf_bicgk(0, 0, None, 0, F32, None, None, None, None, None, None, 0, None) == K.KF_OK
    assert L.kf_gemver(0, None, 0, None, None, None, None, None, None, 1.0, 1.0, None, 0, None, None,
                       None, 0, None) == K.KF_OK
    assert L.kf_gesummv(0, 5, None, None, 5, P, 1.0, 1.0, None, None, 0, None) == K.KF_OK
    assert L.kf_atax(5, 0, None, 0, None, None, None, 0, None) == K.KF_OK
    assert L.kf_waxpby(0, 1.0, None, 1.0, None, None, None) == K.KF_OK
    assert L.kf_ger(0, 4, None, 4, 1.0, None, P, None, 4, None) == K.KF_OK
    assert L.kf_madd(3, 0, None, 0, None, 0, None, 0, None) == K.KF_OK


def _exec(L, plan, binds, ws, ws_bytes):
    arr = (ctypes.c_void_p * len(binds))(*binds)
    return L.kf_plan_execute(plan.h, arr, len(binds), ws, ws_bytes, None)


def test_plan_execute_checks_every_kernel_before_launching(L, K):
    """A binding missing only from a later kernel, or a workspace that only a
    later kernel needs, is refused before the first kernel launches."""
    import torch
    from test_planner_cpu import gemver
    s = gemver(K, 40)
    p = s.plan(K.KF_PLAN_ANALYTIC)
    assert p.kernel_count() == 2                     # {GER, GER, GEMVT, AXPBY}, then {GEMV}
    binds = [P] * len(s.ids)
    binds[s.ids["w"]] = None                         # read only by the second kernel
    assert _exec(L, p, binds, Q, p.workspace_size()) == K.KF_ERR_INVALID_ARG
    assert b"not bound" in L.kf_last_error()
    g = K.Script()                                   # GER (no workspace), then GEMV (needs one)
    g.matrix("A", 32, 32); g.matrix("B", 32, 32)
    for v in ("u", "v", "x", "y"):
        g.vector(v, 32)
    g.input("A", "u", "v", "x"); g.output("B", "y")
    g.call("GER", ["B"], ["A", "u", "v"], [1.0])
    g.call("GEMV", ["y"], ["B", "x"], [1.0, 0.0])
    up = g.plan(K.KF_PLAN_UNFUSED)
    assert up.kernel_count() == 2
    binds = [P] * len(g.ids)
    assert _exec(L, up, binds, None, 0) == K.KF_ERR_WORKSPACE
    assert _exec(L, up, binds, Q, 1024) == K.KF_ERR_WORKSPACE        # below the matrix pass's region
    if torch.cuda.is_available():
        return                                       # below, the checks pass and a launch would follow
    # with everything bound and the plan's workspace, every plan passes the
    # checks (here the launch itself then fails: there is no device)
    for sc in (s, g):
        for i in range(sc.count_plans()[0]):
            pl = sc.plan(K.KF_PLAN_INDEX, index=i)
            st = _exec(L, pl, [P] * len(sc.ids), Q, pl.workspace_size())
            assert st not in (K.KF_ERR_INVALID_ARG, K.KF_ERR_WORKSPACE), (i, st, L.kf_last_error())


def test_plan_checks_accept_every_valid_plan(L, K):
    """Every plan of 150 random valid scripts, fully bound and given its
    reported workspace, passes the up-front checks (the launch that follows
    fails here, with no device)."""
    import random

    import torch
    if torch.cuda.is_available():
        pytest.skip("the checks pass, so a launch on stand-in addresses would follow")
    from test_planner_cpu import _random_valid_script
    rng = random.Random(77)
    checked = 0
    for _ in range(150):
        n = rng.choice([1, 7, 64])
        m = rng.choice([n, 5])
        kinds, inputs, calls = _random_valid_script(rng, n, m)
        s = K.Script()
        for nm, kd in kinds.items():
            (s.vector(nm, n) if kd == "x" else s.vector(nm, m) if kd == "y" else
             s.matrix(nm, m, n) if kd == "A" else s.scalar(nm))
        s.input(*inputs)
        s.output(*sorted({c[1][0] for c in calls}))
        for op, outs, ins, sc in calls:
            s.call(op, outs, ins, sc)
        for i in range(min(s.count_plans(cap=50)[0], 50)):
            pl = s.plan(K.KF_PLAN_INDEX, index=i, max_plans=50)
            st = _exec(L, pl, [P] * len(s.ids), Q, pl.workspace_size())
            assert st not in (K.KF_ERR_INVALID_ARG, K.KF_ERR_WORKSPACE), (calls, i, L.kf_last_error())
            checked += 1
    assert checked > 500


def test_last_error_is_per_thread(L, K):
    """Each thread reads the message of its own last failed call."""
    import threading
    results = {}
    barrier = threading.Barrier(2)

    def worker(name, call, expect):
        barrier.wait()
        for _ in range(200):
            assert call() != K.KF_OK
            msg = L.kf_last_error()
            if expect not in msg:
                results[name] = msg
                return
        results[name] = "ok"

    a = threading.Thread(target=worker, args=("a", lambda: L.kf_waxpby(-1, 1.0, P, 1.0, P, Q, None),
                                               b"negative size"))
    b = threading.Thread(target=worker, args=("b", lambda: L.kf_waxpby(8, 1.0, None, 1.0, P, Q, None),
                                               b"null vector x"))
    a.start(); b.start(); a.join(); b.join()
    assert results == {"a": "ok", "b": "ok"}, results


def test_mlp_entry_point_errors(L, K):
    """The cost model's network: 64 hidden units, 1..32 inputs; parameter
    count H d + H + H H + H + H + 1; bad sizes, missing operands and a short
    workspace are refused before any launch."""
    c = ctypes.c_int(0)
    assert L.kf_mlp_param_count(16, 64, ctypes.byref(c)) == K.KF_OK
    assert c.value == 64 * 16 + 64 + 64 * 64 + 64 + 64 + 1
    for d, h in ((16, 32), (0, 64), (33, 64)):
        assert L.kf_mlp_param_count(d, h, ctypes.byref(c)) == K.KF_ERR_INVALID_ARG
    b = ctypes.c_size_t(0)
    assert L.kf_mlp_workspace_size(16, 64, -1, ctypes.byref(b)) == K.KF_ERR_INVALID_ARG
    assert L.kf_mlp_workspace_size(16, 64, 1000, ctypes.byref(b)) == K.KF_OK and b.value > 0
    assert L.kf_mlp_forward(P, 16, 64, P, 10, None, None) == K.KF_ERR_INVALID_ARG
    assert L.kf_mlp_forward(P, 16, 64, P, 0, None, None) == K.KF_OK            # empty batch
    assert L.kf_mlp_loss_grad(P, 16, 64, P, P, 0, Q, None, None, 0, None) == K.KF_ERR_INVALID_ARG
    assert L.kf_mlp_loss_grad(P, 16, 64, P, P, 10, None, None, None, 0, None) == K.KF_ERR_INVALID_ARG
    assert L.kf_mlp_loss_grad(P, 16, 64, P, P, 10, Q, None, None, 0, None) == K.KF_ERR_WORKSPACE
    assert L.kf_mlp_loss_grad(P, 16, 64, P, P, 10, Q, None, Q, b.value // 1000, None) == K.KF_ERR_WORKSPACE
    assert L.kf_mlp_adam(P, P, Q, Q, 100, 0, 1e-3, 0.9, 0.999, 1e-8, None) == K.KF_ERR_INVALID_ARG
    assert L.kf_mlp_adam(P, P, Q, Q, 0, 1, 1e-3, 0.9, 0.999, 1e-8, None) == K.KF_ERR_INVALID_ARG
    assert L.kf_mlp_adam(P, None, Q, Q, 100, 1, 1e-3, 0.9, 0.999, 1e-8, None) == K.KF_ERR_INVALID_ARG


def test_script_and_plan_api_errors(L, K):
    """Bad variable ids and operand counts are refused when the script is
    validated (KF_ERR_SHAPE); null handles are KF_ERR_INVALID_ARG; a short
    description buffer gets a truncated, terminated string and the size
    needed."""
    def script():
        h = ctypes.c_void_p()
        assert L.kf_script_create(ctypes.byref(h)) == K.KF_OK
        i = ctypes.c_int()
        for nm in (b"x", b"y"):
            assert L.kf_script_vector(h, nm, 8, ctypes.byref(i)) == K.KF_OK
        assert L.kf_script_input(h, 0) == K.KF_OK
        return h

    for outs, ins, msg in (([99], [0, 1], b"out of range"), ([1], [-3, 0], b"out of range"),
                           ([1], [0], b"AXPBY"), ([1], [0, 0, 0, 0], b"AXPBY"), ([], [0, 1], b"exactly one output")):
        h = script()
        o = (ctypes.c_int * max(1, len(outs)))(*outs)
        n = (ctypes.c_int * len(ins))(*ins)
        assert L.kf_script_call(h, K.KF_OP_AXPBY, o, len(outs), n, len(ins), None, 0) == K.KF_OK
        assert L.kf_script_validate(h) == K.KF_ERR_SHAPE
        assert msg in L.kf_last_error(), (outs, ins, L.kf_last_error())
        L.kf_script_destroy(h)
    h = script()
    i = ctypes.c_int()
    assert L.kf_script_call(h, 7, (ctypes.c_int * 1)(1), 1, (ctypes.c_int * 2)(0, 1), 2, None, 0) \
        == K.KF_ERR_INVALID_ARG                                              # unknown op
    assert L.kf_script_call(h, K.KF_OP_AXPBY, (ctypes.c_int * 1)(1), 1, (ctypes.c_int * 2)(0, 1), 2,
                            (ctypes.c_double * 3)(1, 2, 3), 3) == K.KF_ERR_INVALID_ARG   # three scalars
    assert L.kf_script_vector(h, b"z", -1, ctypes.byref(i)) == K.KF_ERR_INVALID_ARG
    assert L.kf_script_input(h, 42) == K.KF_ERR_INVALID_ARG
    assert L.kf_script_output(h, -1) == K.KF_ERR_INVALID_ARG
    L.kf_script_destroy(h)
    assert L.kf_script_vector(None, b"x", 8, ctypes.byref(i)) == K.KF_ERR_INVALID_ARG
    assert L.kf_script_validate(None) == K.KF_ERR_INVALID_ARG
    need = ctypes.c_size_t(0)
    assert L.kf_plan_describe(None, None, 0, ctypes.byref(need)) == K.KF_ERR_INVALID_ARG
    assert L.kf_plan_execute(None, None, 0, None, 0, None) == K.KF_ERR_INVALID_ARG
    from test_planner_cpu import bicgk
    p = bicgk(K).plan(K.KF_PLAN_ANALYTIC)
    assert L.kf_plan_describe(p.h, None, 0, ctypes.byref(need)) == K.KF_OK and need.value > 20
    buf = ctypes.create_string_buffer(b"#" * 16, 16)
    assert L.kf_plan_describe(p.h, buf, 16, ctypes.byref(need)) == K.KF_OK
    assert len(buf.value) == 15 and buf.raw[15] == 0
    full = ctypes.create_string_buffer(need.value)
    assert L.kf_plan_describe(p.h, full, need.value, ctypes.byref(need)) == K.KF_OK
    assert full.value.startswith(buf.value) and len(full.value) == need.value - 1


def test_wait_limit_and_probe_errors(L, K):
    """The wait limit is range checked and unchanged by a refused value; the
    probe needs a workspace for its error word and a limit in range."""
    old = K.kf_get_wait_limit_ns()
    assert old == 1_000_000_000
    assert L.kf_set_wait_limit_ns(999) == K.KF_ERR_INVALID_ARG
    assert L.kf_set_wait_limit_ns(60_000_000_001) == K.KF_ERR_INVALID_ARG
    assert K.kf_get_wait_limit_ns() == old
    assert L.kf_get_wait_limit_ns(None) == K.KF_ERR_INVALID_ARG
    assert L.kf_set_wait_limit_ns(1000) == 0 and K.kf_get_wait_limit_ns() == 1000
    assert L.kf_set_wait_limit_ns(old) == 0
    assert L.kf_wait_probe(5000, None, 0, None, None) == K.KF_ERR_WORKSPACE
    assert L.kf_wait_probe(5000, P, 255, None, None) == K.KF_ERR_WORKSPACE
    assert L.kf_wait_probe(10, P, 256, None, None) == K.KF_ERR_INVALID_ARG


def test_planner_train_errors(L, K):
    """kf_planner_train checks its sizes, options and times before any
    device work."""
    import numpy as np
    n, d = 8, 16
    X = np.zeros((n, d), np.float32)
    ms = np.ones(n)
    pu = np.ones(n)
    fp, dp = ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_double)
    cm = K._CostModel()

    def call(opt, d_in=d, count=n, ms_=ms, sid=None, ws=P, wsb=1 << 30):
        return L.kf_planner_train(X.ctypes.data_as(fp), ms_.ctypes.data_as(dp), pu.ctypes.data_as(dp), sid,
                                  count, d_in, ctypes.byref(opt), None, P, ws, wsb, None, ctypes.byref(cm), None,
                                  0, None)
    good = K._TrainOptions(10, 1e-3, 0.9, 0.999, 1e-8, 1.0, 0, 0, 0)
    assert call(good, d_in=15) == K.KF_ERR_INVALID_ARG
    assert call(good, count=0) == K.KF_ERR_INVALID_ARG
    assert call(K._TrainOptions(0, 1e-3, 0.9, 0.999, 1e-8, 1.0, 0, 0, 0)) == K.KF_ERR_INVALID_ARG   # no epochs
    assert call(K._TrainOptions(10, 1e-3, 1.0, 0.999, 1e-8, 1.0, 0, 0, 0)) == K.KF_ERR_INVALID_ARG  # beta1
    assert call(K._TrainOptions(10, 1e-3, 0.9, 0.999, 1e-8, 1.0, 1, 0, 0)) == K.KF_ERR_INVALID_ARG  # centring, no ids
    bad = ms.copy(); bad[3] = 0.0
    assert call(good, ms_=bad) == K.KF_ERR_INVALID_ARG                                                 # time 0
    assert call(good, ws=None, wsb=0) == K.KF_ERR_WORKSPACE
    b = ctypes.c_size_t(0)
    assert L.kf_planner_train_workspace_size(n, d, ctypes.byref(b)) == 0 and b.value > n * d * 4
    assert L.kf_planner_train_workspace_size(n, 12, ctypes.byref(b)) == K.KF_ERR_INVALID_ARG
