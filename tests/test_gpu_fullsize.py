"""Parity at the benchmarked sizes, in the launch configuration bench.py times.

The fused suite is built and launched through bench.Suite (the same inputs,
calls, workspaces and automatic tuning the benchmark times) and checked
against the FP64 oracle:
  * BiCGK 16384 x 16384: on sampled rows (q) and columns (s), each computed
    one by one by the oracle from the regenerated rows / columns of A;
  * GEMVER, GESUMMV, ATAX at n = 8192, AXPYDOT and WAXPBY at n = 2^26: the
    oracle on the whole problem;
  * the row-scaled forms at n = 16384 (BiCGK and GEMVER, BF16 and E4M3):
    codes bitwise, results against the oracle on the stored matrices and,
    with the format's bound, against the FP64 results of the FP32 problem
    (the errors are printed);
  * the batched form, 4096 instances: a sample of instances one by one.
"""

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import ALPHA, BETA, built, dev, host  # noqa: F401
from tolerance import check_map, check_reduce

pytestmark = pytest.mark.gpu

SAMPLE = 48


def suite_for(kf, seqs):
    import bench
    s = bench.Suite(kf, bench.FULL, dev(), seqs=seqs)
    st = torch.cuda.Stream()
    torch.cuda.synchronize()  # the inputs are generated on the default stream
    with torch.cuda.stream(st):
        for q in seqs:
            s.fused(q, st)
    st.synchronize()
    return s


def sample_idx(n, seed):
    idx = synth.integers((SAMPLE,), seed, synth.TID["sizes"], lo=0, hi=n - 1).numpy().astype(np.int64)
    return np.unique(np.concatenate([idx, [0, n - 1]]))


def test_bicgk_16384_sampled(built):
    kf = built
    s = suite_for(kf, ["bicgk"])
    b = s.bicgk
    m, n = b["A"].shape
    p, r = host(b["p"]), host(b["r"])
    rows = sample_idx(m, 1)
    Ar = synth.matrix_rows(m, n, rows, 0, synth.TID["A"]).numpy()
    assert np.array_equal(Ar, b["A"][torch.from_numpy(rows).to(dev())].cpu().numpy())
    q = host(b["q"])[rows]
    check_reduce(q, oracle.gemv(Ar, p), oracle.abs_gemv(Ar, p), n, "q sampled")
    cols = sample_idx(n, 2)
    Ac = synth.matrix_cols(m, n, cols, 0, synth.TID["A"]).numpy()  # (len(cols), m)
    sv = host(b["s"])[cols]
    check_reduce(sv, oracle.gemv(Ac, r), oracle.abs_gemv(Ac, r), m, "s sampled")


def test_gemver_gesummv_atax_8192(built):
    kf = built
    s = suite_for(kf, ["gemver", "gesummv", "atax"])
    g = s.gemver
    H = [host(g[k]) for k in ("A", "u1", "v1", "u2", "v2", "y", "z")]
    Bo, xo, wo = oracle.gemver(*H, ALPHA, BETA)
    Ah, u1, v1, u2, v2, y, z = H
    n = Ah.shape[0]
    rows = sample_idx(n, 3)
    scaleB = np.abs(Ah[rows]) + np.abs(np.outer(u1[rows], v1)) + np.abs(np.outer(u2[rows], v2))
    check_map(g["B"][torch.from_numpy(rows).to(dev())].double().cpu().numpy(), Bo[rows], scaleB, "B rows")
    sx = BETA * oracle.abs_gemvt(Bo, y) + np.abs(z)
    check_reduce(host(g["x"]), xo, sx, n, "x")
    check_reduce(host(g["w"]), wo, ALPHA * oracle.abs_gemv(Bo, np.abs(xo) + sx), n, "w")
    del Bo, H
    e = s.gesummv
    A2, B2, x2 = host(e["A"]), host(e["B"]), host(e["x"])
    yo = oracle.gesummv(A2, B2, x2, ALPHA, BETA)
    sy = ALPHA * oracle.abs_gemv(A2, x2) + BETA * oracle.abs_gemv(B2, x2)
    check_reduce(host(e["y"]), yo, sy, n, "gesummv y")
    del A2, B2
    a = s.atax
    A3, x3 = host(a["A"]), host(a["x"])
    ya, ta = oracle.atax(A3, x3)
    check_reduce(host(a["y"]), ya, oracle.abs_gemvt(A3, oracle.abs_gemv(A3, x3)), n, "atax y")


def test_axpydot_waxpby_2pow26(built):
    kf = built
    s = suite_for(kf, ["axpydot", "waxpby"])
    a = s.axpydot
    w, v, u = host(a["w"]), host(a["v"]), host(a["u"])
    zo, ro = oracle.axpydot(w, v, u, ALPHA)
    check_map(host(a["z"]), zo, np.abs(w) + ALPHA * np.abs(v), "z")
    scale = float(np.sum((np.abs(w) + ALPHA * np.abs(v)) * np.abs(u)))
    check_reduce(host(a["r"]), np.array([ro]), np.array([scale]), w.shape[0], "r")
    x = s.waxpby
    xh, yh = host(x["x"]), host(x["y"])
    check_map(host(x["w"]), oracle.waxpby(ALPHA, xh, BETA, yh), ALPHA * np.abs(xh) + BETA * np.abs(yh), "w")


LOWP = [("bf16", 1, oracle.FMT_BF16, torch.int16, 2.0 ** -8), ("e4m3", 2, oracle.FMT_E4M3, torch.uint8, 2.0 ** -4)]


def codes_of(Q):
    c = Q.cpu().numpy()
    return c.view(np.uint16) if c.dtype == np.int16 else c


def upload(Qo):
    c = Qo.view(np.int16) if Qo.dtype == np.uint16 else Qo
    return torch.from_numpy(np.ascontiguousarray(c)).to(dev())


@pytest.mark.parametrize("name,kfmt,ofmt,tdt,rel", LOWP)
def test_lowp_bicgk_16384(built, name, kfmt, ofmt, tdt, rel):
    """Quantiser bitwise on the whole matrix; q and s against the oracle on
    Ahat (FP32 tolerance) and against the FP32 problem's FP64 results within
    half a unit of the format (sampled rows and columns)."""
    kf = built
    n = 16384
    A = synth.uniform((n, n), 0, synth.TID["A"], device=dev())
    p = synth.uniform((n,), 0, synth.TID["p"], device=dev())
    r = synth.uniform((n,), 0, synth.TID["r"], device=dev())
    Q = torch.empty((n, n), dtype=tdt, device=dev())
    sA = torch.empty(n, device=dev())
    kf.kf_quantize_rows(A, kfmt, Q, sA)
    q, sv = torch.empty(n, device=dev()), torch.empty(n, device=dev())
    kf.kf_bicgk(Q, p, r, q, sv, kf.workspace(kf.KF_SEQ_BICGK, n, n, kfmt), fmt=kfmt, row_scale=sA, n=n)
    Ah = A.cpu().numpy()
    Qo, so = oracle.quantize_rows(Ah, ofmt)
    assert np.array_equal(sA.cpu().numpy(), so)
    assert np.array_equal(codes_of(Q), Qo)
    ph, rh = host(p), host(r)
    rows, cols = sample_idx(n, 4), sample_idx(n, 5)
    Ahat_r = oracle.dequantize_rows(Qo[rows], so[rows], ofmt)
    Ahat_c = (so.astype(np.float64)[:, None] * oracle.dequantize_rows(Qo[:, cols].copy(), np.ones(n, np.float32),
                                                                      ofmt)).T
    qh, sh = host(q), host(sv)
    check_reduce(qh[rows], oracle.gemv(Ahat_r, ph), oracle.abs_gemv(Ahat_r, ph), n, "q vs O_q")
    check_reduce(sh[cols], oracle.gemv(Ahat_c, rh), oracle.abs_gemv(Ahat_c, rh), n, "s vs O_q")
    Ar = Ah[rows].astype(np.float64)
    Ac = Ah[:, cols].astype(np.float64).T
    qt, st_ = oracle.gemv(Ar, ph), oracle.gemv(Ac, rh)
    floor = 2.0 ** -10 if ofmt == oracle.FMT_E4M3 else 0.0
    bq = (rel * 1.01 + 2e-5) * oracle.abs_gemv(Ar, ph) + floor * so[rows].astype(np.float64) * np.abs(ph).sum()
    bs = (rel * 1.01 + 2e-5) * oracle.abs_gemv(Ac, rh) + floor * float((so.astype(np.float64) * np.abs(rh)).sum())
    eq, es = np.abs(qh[rows] - qt), np.abs(sh[cols] - st_)
    assert np.all(eq <= bq) and np.all(es <= bs)
    print(f"\n{name} BiCGK n={n}: q max err {eq.max():.3e} (rel {eq.max() / np.abs(qt).max():.3e}), "
          f"s max err {es.max():.3e} (rel {es.max() / np.abs(st_).max():.3e}) vs FP64 of the FP32 problem")


@pytest.mark.parametrize("name,kfmt,ofmt,tdt,rel", LOWP)
def test_lowp_gemver_16384(built, name, kfmt, ofmt, tdt, rel):
    """B's codes and scales bitwise on the whole matrix; x and w against the
    oracle on the stored B, and against the FP32 problem within the bound of
    two roundings into the format."""
    kf = built
    n = 16384
    A = synth.uniform((n, n), 0, synth.TID["A"], device=dev())
    vs = {k: synth.uniform((n,), 0, synth.TID[k], device=dev()) for k in ("u1", "v1", "u2", "v2", "y", "z")}
    Ah = A.cpu().numpy()
    QAo, sAo = oracle.quantize_rows(Ah, ofmt)
    QA, sA = upload(QAo), torch.from_numpy(sAo).to(dev())
    QB, sB = torch.empty_like(QA), torch.empty(n, device=dev())
    x, w = torch.empty(n, device=dev()), torch.empty(n, device=dev())
    kf.kf_gemver_q(QA, kfmt, sA, vs["u1"], vs["v1"], vs["u2"], vs["v2"], vs["y"], vs["z"], ALPHA, BETA,
                   QB, sB, x, w, kf.workspace(kf.KF_SEQ_GEMVER, n, n, kfmt))
    h = {k: t.cpu().numpy() for k, t in vs.items()}
    QBo, sBo, Bhat, xo, wo = oracle.gemver_rowscaled(QAo, sAo, ofmt, h["u1"], h["v1"], h["u2"], h["v2"], h["y"],
                                                     h["z"], ALPHA, BETA)
    assert np.array_equal(sB.cpu().numpy(), sBo)
    assert np.array_equal(codes_of(QB), QBo)
    sx = BETA * oracle.abs_gemvt(Bhat, h["y"]) + np.abs(h["z"])
    check_reduce(host(x), xo, sx, n, "x vs stored B")
    check_reduce(host(w), wo, ALPHA * oracle.abs_gemv(Bhat, np.abs(xo) + sx), n, "w vs stored B")
    del Bhat, QBo
    B, xt, wt = oracle.gemver(Ah, h["u1"], h["v1"], h["u2"], h["v2"], h["y"], h["z"], ALPHA, BETA)
    floor = 2.0 ** -10 if ofmt == oracle.FMT_E4M3 else 0.0
    Eb = (2 * rel * 1.01 + 2e-5) * np.abs(B) + floor * (sAo.astype(np.float64) + sBo.astype(np.float64))[:, None]
    tol = 1e-5 * np.sqrt(n)
    bx = BETA * (Eb.T @ np.abs(h["y"])) + tol * (BETA * oracle.abs_gemvt(B, h["y"]) + np.abs(h["z"]))
    ex = np.abs(host(x) - xt)
    assert np.all(ex <= bx)
    bw = ALPHA * (Eb @ (np.abs(xt) + bx) + np.abs(B) @ bx) + tol * ALPHA * oracle.abs_gemv(B, np.abs(xt) + bx)
    ew = np.abs(host(w) - wt)
    assert np.all(ew <= bw)
    print(f"\n{name} GEMVER n={n}: x max err {ex.max():.3e} (rel {ex.max() / np.abs(xt).max():.3e}), "
          f"w max err {ew.max():.3e} (rel {ew.max() / np.abs(wt).max():.3e}) vs FP64 of the FP32 problem")


@pytest.mark.parametrize("kind", ["bicgk", "gesummv"])
def test_batched_4096_sampled(built, kind):
    """The benchmarked batch (4096 instances, tile height from the
    autotuner, graph replay): a sample of instances against the oracle."""
    import bench
    kf = built
    shapes = bench.batched_shapes()
    descs, views, bufs, _ = bench.make_batched(kind, dev(), shapes)
    seq = kf.KF_SEQ_BICGK if kind == "bicgk" else kf.KF_SEQ_GESUMMV
    band, _ = kf.kf_batched_autotune(seq, descs, reps=1)
    for v in views:
        v[4].fill_(float("nan"))
        v[5].fill_(float("nan"))
    b = kf.Batched(seq, descs, band)
    ws = torch.zeros(max(b.workspace_size(), 256), dtype=torch.uint8, device=dev())
    b.upload(ws)
    b.capture(ws)
    b.replay()
    torch.cuda.synchronize()
    pick = sorted(set(synth.integers((40,), 9, synth.TID["sizes"], lo=0, hi=len(shapes) - 1).numpy().astype(int)
                      .tolist()) | {0, len(shapes) - 1})
    for i in pick:
        a, bm, x, r, y, sv = views[i]
        Ah, xh, rh = host(a), host(x), host(r)
        n = Ah.shape[1]
        if kind == "bicgk":
            qo, so_ = oracle.bicgk(Ah, xh, rh)
            check_reduce(host(y), qo, oracle.abs_gemv(Ah, xh), n, f"q #{i}")
            check_reduce(host(sv), so_, oracle.abs_gemvt(Ah, rh), Ah.shape[0], f"s #{i}")
        else:
            Bh = host(bm)
            yo = oracle.gesummv(Ah, Bh, xh, ALPHA, BETA)
            sc = ALPHA * oracle.abs_gemv(Ah, xh) + BETA * oracle.abs_gemv(Bh, xh)
            check_reduce(host(y), yo, sc, n, f"y #{i}")
