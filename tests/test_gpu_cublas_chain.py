"""The cuBLAS chains bench.py reports as context (the paper's comparison
system, Section 5) compute the same sequences: each chain's results are
checked against the FP64 oracle with the same tolerance as the fused
kernels, at the small suite sizes."""

import numpy as np
import pytest
import torch

import oracle
from gpu_util import ALPHA, BETA, built, dev, host  # noqa: F401
from tolerance import check_map, check_reduce

pytestmark = pytest.mark.gpu


def test_cublas_chains_match_oracle(built):
    import bench
    kf = built
    s = bench.Suite(kf, bench.SMALL, dev())
    st = torch.cuda.Stream()
    torch.cuda.synchronize()
    cb = bench.CublasChain(s, st)
    try:
        with torch.cuda.stream(st):
            for q in bench.SEQS:
                cb.run(q)
        st.synchronize()

        b = s.bicgk
        A, p, r = host(b["A"]), host(b["p"]), host(b["r"])
        qo, so = oracle.bicgk(A, p, r)
        qc, sc = (host(t) for t in cb.outputs("bicgk"))
        check_reduce(qc, qo, oracle.abs_gemv(A, p), A.shape[1], "cuBLAS q")
        check_reduce(sc, so, oracle.abs_gemvt(A, r), A.shape[0], "cuBLAS s")

        g = s.gemver
        A, u1, v1, u2, v2, y, z = (host(g[k]) for k in ("A", "u1", "v1", "u2", "v2", "y", "z"))
        Bo, xo, wo = oracle.gemver(A, u1, v1, u2, v2, y, z, ALPHA, BETA)
        Bc, xc, wc = (host(t) for t in cb.outputs("gemver"))
        n = A.shape[0]
        check_map(Bc, Bo, np.abs(A) + np.abs(np.outer(u1, v1)) + np.abs(np.outer(u2, v2)), "cuBLAS B")
        sx = BETA * oracle.abs_gemvt(Bo, y) + np.abs(z)
        check_reduce(xc, xo, sx, n, "cuBLAS x")
        check_reduce(wc, wo, ALPHA * oracle.abs_gemv(Bo, np.abs(xo) + sx), n, "cuBLAS w")

        e = s.gesummv
        A, B, x = host(e["A"]), host(e["B"]), host(e["x"])
        yo = oracle.gesummv(A, B, x, ALPHA, BETA)
        check_reduce(host(cb.outputs("gesummv")[0]), yo,
                     ALPHA * oracle.abs_gemv(A, x) + BETA * oracle.abs_gemv(B, x), A.shape[1], "cuBLAS GESUMMV")

        a = s.atax
        A, x = host(a["A"]), host(a["x"])
        yo, _ = oracle.atax(A, x)
        check_reduce(host(cb.outputs("atax")[0]), yo, oracle.abs_gemvt(A, oracle.abs_gemv(A, x)),
                     max(A.shape), "cuBLAS ATAX")

        d = s.axpydot
        w, v, u = host(d["w"]), host(d["v"]), host(d["u"])
        zo, ro = oracle.axpydot(w, v, u, ALPHA)
        zc, rc = (host(t) for t in cb.outputs("axpydot"))
        check_map(zc, zo, np.abs(w) + ALPHA * np.abs(v), "cuBLAS z")
        scale = float(np.sum((np.abs(w) + ALPHA * np.abs(v)) * np.abs(u)))
        check_reduce(rc, np.array([ro]), np.array([scale]), w.size, "cuBLAS r")

        wx = s.waxpby
        x, y = host(wx["x"]), host(wx["y"])
        check_map(host(cb.outputs("waxpby")[0]), oracle.waxpby(ALPHA, x, BETA, y),
                  ALPHA * np.abs(x) + BETA * np.abs(y), "cuBLAS WAXPBY")
    finally:
        cb.close()


def test_cublas_section_reports_every_sequence(built):
    import bench
    kf = built
    s = bench.Suite(kf, bench.SMALL, dev())
    st = torch.cuda.Stream()
    _, per = bench.time_suite(s, "fused", 3, 1, st, bench.SEQS)
    sec = bench.cublas_section(s, st, 3, 1, bench.SEQS, per)
    assert "unavailable" not in sec, sec
    for q in bench.SEQS:
        assert sec[q]["ms"] > 0 and sec[q]["fused_speedup"] > 0
        # both paths compute the same FP32 results up to rounding order
        assert sec[q]["max_rel_diff_vs_fused"] < 1e-4, (q, sec[q])
