"""The byte model behind every GB/s the bench reports (no GPU).

bench.py counts the bytes a sequence must move at least once (each matrix
and vector crossing HBM once), and the bytes of its one-kernel-per-call
chain.  The planner counts the bytes of each plan from the script on its
own.  The two models must agree at the benchmarked sizes.  The counts must
also equal the closed forms of the byte table (A read once: 4mn bytes plus
the vectors).
"""

import pytest

import bench
from test_planner_cpu import atax, axpydot, bicgk, gemver, gesummv, waxpby

BUILDERS = {
    "bicgk": lambda kf: bicgk(kf, 16384, 16384),
    "gemver": lambda kf: gemver(kf, 8192),
    "gesummv": lambda kf: gesummv(kf, 8192),
    "atax": lambda kf: atax(kf, 8192),
    "axpydot": lambda kf: axpydot(kf, 1 << 26),
    "waxpby": lambda kf: waxpby(kf, 1 << 26),
}


@pytest.fixture(scope="module")
def kf():
    from paper_1305_1183_gb300 import _build, kf as K
    _build.build()
    K.lib()
    return K


def test_closed_forms_at_the_benchmarked_sizes():
    F = bench.FULL
    n = 8192
    assert bench.algorithmic_bytes("bicgk", F["bicgk"]) == 4 * 16384 * 16384 + 8 * (2 * 16384)
    assert bench.algorithmic_bytes("gemver", F["gemver"]) == 12 * n * n + 36 * n
    assert bench.algorithmic_bytes("gesummv", F["gesummv"]) == 8 * n * n + 8 * n
    assert bench.algorithmic_bytes("atax", F["atax"]) == 4 * n * n + 8 * n
    assert bench.algorithmic_bytes("axpydot", F["axpydot"]) == 16 * (1 << 26) + 4
    assert bench.algorithmic_bytes("waxpby", F["waxpby"]) == 12 * (1 << 26)
    # the matrix passes are matrix bound: vectors add under 0.1 %
    for s in ("bicgk", "gemver", "gesummv", "atax"):
        b = bench.algorithmic_bytes(s, F[s])
        mat = {"bicgk": 4 * 16384 ** 2, "gemver": 12 * n * n, "gesummv": 8 * n * n, "atax": 4 * n * n}[s]
        assert 0 <= b - mat < 1e-3 * mat


@pytest.mark.parametrize("seq,ideal", [("bicgk", 2.0), ("gemver", 2.0), ("gesummv", 1.0), ("atax", 2.0),
                                       ("axpydot", 1.25), ("waxpby", 5 / 3)])
def test_ideal_speedups(seq, ideal):
    s = bench.FULL[seq]
    assert bench.unfused_bytes(seq, s) / bench.algorithmic_bytes(seq, s) == pytest.approx(ideal, rel=2e-3)


@pytest.mark.parametrize("seq", sorted(BUILDERS))
def test_planner_byte_counts_agree_with_the_bench(kf, seq):
    """The planner's fused and unfused plans move exactly the bench's bytes
    (ATAX included: the planner emits the single pass that reads A once)."""
    s = BUILDERS[seq](kf)
    size = bench.FULL[seq]
    fused = s.plan(kf.KF_PLAN_ANALYTIC).describe()["bytes"]
    unfused = s.plan(kf.KF_PLAN_UNFUSED).describe()["bytes"]
    assert unfused == bench.unfused_bytes(seq, size)
    assert fused == bench.algorithmic_bytes(seq, size)


def _sgemv(kf, n):
    s = kf.Script()
    s.matrix("A", n, n)
    for v in ("x", "y", "t", "z"):
        s.vector(v, n)
    s.input("A", "x", "y"); s.output("z")
    s.call("GEMV", ["t"], ["A", "x"], [1.5, 0.0])
    s.call("AXPBY", ["z"], ["t", "y"], [1.0, 1.2])
    return s


def _sgemvt(kf, n):
    s = kf.Script()
    s.matrix("A", n, n)
    for v in ("y", "z", "t", "x", "w"):
        s.vector(v, n)
    s.input("A", "y", "z"); s.output("x", "w")
    s.call("GEMVT", ["t"], ["A", "y"], [1.0, 0.0])
    s.call("AXPBY", ["x"], ["t", "z"], [1.2, 1.0])
    s.call("GEMV", ["w"], ["A", "x"], [1.5, 0.0])
    return s


def _vadd(kf, n):
    s = kf.Script()
    for v in ("w", "y", "z", "t", "x"):
        s.vector(v, n)
    s.input("w", "y", "z"); s.output("x")
    s.call("AXPBY", ["t"], ["w", "y"], [1.0, 1.0])
    s.call("AXPBY", ["x"], ["t", "z"], [1.0, 1.0])
    return s


@pytest.mark.parametrize("seq,build,size", [("sgemv", _sgemv, 8192), ("sgemvt", _sgemvt, 8192),
                                            ("vadd", _vadd, 1 << 26)])
def test_table1_byte_counts_agree_with_the_planner(kf, seq, build, size):
    """SGEMV, SGEMVT and VADD: the bench's fused and unfused byte counts are
    the planner's for the same scripts (SGEMVT fused: two passes over A,
    since w needs all of x)."""
    s = build(kf, size)
    alg, unf = bench.table1_bytes(seq, size)
    assert s.plan(kf.KF_PLAN_ANALYTIC).describe()["bytes"] == alg
    assert s.plan(kf.KF_PLAN_UNFUSED).describe()["bytes"] == unf


def test_read_probe_section(monkeypatch):
    """The read-only probe times kf_dot over the AXPYDOT vectors and reports
    (8n + 4) bytes per launch; an error becomes an entry, not a crash."""
    calls = []

    class FakeKF:
        @staticmethod
        def kf_dot(x, y, out, ws, stream=None):
            calls.append((x, y, out, ws, stream))

    def fake_time(fn, steps, warmup, st):
        fn(st)
        return 0.25                                     # ms

    class FakeSuite:
        axpydot = {"w": "W", "v": "V", "r": "R", "ws": "WS", "u": "U", "z": "Z"}

    monkeypatch.setattr(bench, "time_calls", fake_time)
    n = 1 << 26
    r = bench.read_probe_section(FakeKF, FakeSuite, {"axpydot": n}, 5, 3, "ST")
    assert calls == [("W", "V", "R", "WS", "ST")]
    assert r["bytes_per_launch"] == 8 * n + 4 and r["ms"] == 0.25
    assert r["gbs"] == pytest.approx((8 * n + 4) / 0.25e-3 / 1e9)

    def failing_time(fn, steps, warmup, st):
        raise RuntimeError("no device")

    monkeypatch.setattr(bench, "time_calls", failing_time)
    assert bench.read_probe_section(FakeKF, FakeSuite, {"axpydot": n}, 5, 3, "ST") == {"error": "no device"}
