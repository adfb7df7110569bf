"""Row-scaled BF16 / FP8-E4M3 storage of A: quantiser parity and low-precision
BiCGK, GEMV and GEMVT against the FP64 oracle.

Two references (the low-precision forms are not in the paper, which is FP32
only):
  O_q -- the oracle on the dequantised matrix Ahat_ij = s_i Q_ij (exact in
         double): pins the arithmetic, FP32 tolerance 1e-5 sqrt(n);
  O   -- the oracle on the original FP32 A: the total error, bounded by the
         format's half-unit rounding (2^-9 BF16, 2^-4 E4M3, plus the E4M3
         subnormal floor s_i 2^-10) times the |A||p| scale.
The GPU's codes are first checked bitwise against the oracle's, so both
sides then work on the same Ahat.
"""

import numpy as np
import pytest
import torch

import oracle
from gpu_util import U, built, dev, host  # noqa: F401
from tolerance import check_reduce

pytestmark = pytest.mark.gpu

FMTS = [(1, oracle.FMT_BF16, torch.int16, 2.0 ** -9), (2, oracle.FMT_E4M3, torch.uint8, 2.0 ** -4)]


def gpu_quantize(kf, A, kfmt, tdt):
    m, n = A.shape
    Q = torch.empty((m, n), dtype=tdt, device=dev())
    s = torch.empty(m, dtype=torch.float32, device=dev())
    kf.kf_quantize_rows(A, kfmt, Q, s)
    torch.cuda.synchronize()
    return Q, s


def codes_np(Q):
    c = Q.cpu().numpy()
    return c.view(np.uint16) if c.dtype == np.int16 else c


@pytest.mark.parametrize("kfmt,ofmt,tdt,half_ulp", FMTS)
@pytest.mark.parametrize("m,n", [(1, 1), (37, 1003), (512, 2048), (300, 4096)])
def test_quantizer_bitwise(built, kfmt, ofmt, tdt, half_ulp, m, n):
    kf = built
    A = U((m, n), 1)
    A[min(5, m - 1), :] = 0.0                 # an all-zero row
    A[0, 0] = 0.75                            # exact values and a tie-prone row
    Q, s = gpu_quantize(kf, A, kfmt, tdt)
    Qo, so = oracle.quantize_rows(A.cpu().numpy(), ofmt)
    assert np.array_equal(s.cpu().numpy(), so)
    assert np.array_equal(codes_np(Q), Qo)


@pytest.mark.parametrize("kfmt,ofmt,tdt,half_ulp", FMTS)
@pytest.mark.parametrize("m,n", [(33, 31), (1000, 1024), (2048, 2048), (777, 4096)])
def test_lowp_bicgk_gemv_gemvt(built, kfmt, ofmt, tdt, half_ulp, m, n):
    kf = built
    A, p, r = U((m, n), 1), U((n,), 3), U((m,), 4)
    Q, s = gpu_quantize(kf, A, kfmt, tdt)
    Qo, so = oracle.quantize_rows(A.cpu().numpy(), ofmt)
    assert np.array_equal(codes_np(Q), Qo)
    Ahat = oracle.dequantize_rows(Qo, so, ofmt)
    ph, rh = host(p), host(r)
    q = torch.empty(m, device=dev()); sv = torch.empty(n, device=dev())
    W = kf.workspace(kf.KF_SEQ_BICGK, m, n, kfmt)
    kf.kf_bicgk(Q, p, r, q, sv, W, fmt=kfmt, row_scale=s, n=n)
    qo, so_ = oracle.bicgk(Ahat, ph, rh)
    check_reduce(host(q), qo, oracle.abs_gemv(Ahat, ph), n, "q vs O_q")
    check_reduce(host(sv), so_, oracle.abs_gemvt(Ahat, rh), m, "s vs O_q")
    # total error against the original FP32 matrix, within the format's bound
    Ah = host(A)
    qt, st = oracle.bicgk(Ah, ph, rh)
    floor = (2.0 ** -10 if ofmt == oracle.FMT_E4M3 else 0.0)
    bq = (half_ulp * 1.01 + 2e-5) * oracle.abs_gemv(Ah, ph) + floor * so.astype(np.float64) * np.abs(ph).sum()
    bs = (half_ulp * 1.01 + 2e-5) * oracle.abs_gemvt(Ah, rh) + floor * (so.astype(np.float64) * np.abs(rh)).sum()
    assert np.all(np.abs(host(q) - qt) <= bq)
    assert np.all(np.abs(host(sv) - st) <= bs)
    # the elementaries on the same storage
    y = torch.empty(m, device=dev())
    kf.kf_gemv(Q, p, y, W, alpha=1.5, fmt=kfmt, row_scale=s, n=n)
    check_reduce(host(y), 1.5 * qo, 1.5 * oracle.abs_gemv(Ahat, ph), n, "gemv lowp")
    x = torch.empty(n, device=dev())
    kf.kf_gemvt(Q, r, x, W, alpha=1.5, fmt=kfmt, row_scale=s, n=n)
    check_reduce(host(x), 1.5 * so_, 1.5 * oracle.abs_gemvt(Ahat, rh), m, "gemvt lowp")


def upload_codes(Qo, tdt):
    c = Qo.view(np.int16) if Qo.dtype == np.uint16 else Qo
    return torch.from_numpy(np.ascontiguousarray(c)).to(dev())


def run_gemver_q(kf, n, kfmt, ofmt, tdt, seed=0):
    A = U((n, n), 1, seed)
    vs = {k: U((n,), t, seed) for k, t in (("u1", 5), ("v1", 6), ("u2", 7), ("v2", 8), ("y", 4), ("z", 9))}
    QAo, sAo = oracle.quantize_rows(A.cpu().numpy(), ofmt)
    QA = upload_codes(QAo, tdt)
    sA = torch.from_numpy(sAo).to(dev())
    QB = torch.empty_like(QA)
    sB = torch.empty(n, device=dev())
    x = torch.empty(n, device=dev()); w = torch.empty(n, device=dev())
    W = kf.workspace(kf.KF_SEQ_GEMVER, n, n, kfmt)
    kf.kf_gemver_q(QA, kfmt, sA, vs["u1"], vs["v1"], vs["u2"], vs["v2"], vs["y"], vs["z"], 1.5, 1.2,
                   QB, sB, x, w, W)
    torch.cuda.synchronize()
    h = {k: t.cpu().numpy() for k, t in vs.items()}
    ref = oracle.gemver_rowscaled(QAo, sAo, ofmt, h["u1"], h["v1"], h["u2"], h["v2"], h["y"], h["z"], 1.5, 1.2)
    return A, h, QAo, sAo, (QB, sB, x, w), ref


@pytest.mark.parametrize("kfmt,ofmt,tdt,half_ulp", FMTS)
@pytest.mark.parametrize("n", [1, 33, 777, 1000, 2048])
def test_lowp_gemver_codes_bitwise_and_results(built, kfmt, ofmt, tdt, half_ulp, n):
    """kf_gemver_q against the oracle's storage rule: B's codes and row
    scales bit for bit (the rule's decisions are FP32 on both sides), x and
    w within the FP32 tolerance of the FP64 results on the stored matrix.
    777 and 1000 take the unaligned (element-interleaved) path for E4M3."""
    kf = built
    A, h, QAo, sAo, (QB, sB, x, w), (QBo, sBo, Bhat, xo, wo) = run_gemver_q(kf, n, kfmt, ofmt, tdt)
    assert np.array_equal(sB.cpu().numpy(), sBo)
    assert np.array_equal(codes_np(QB), QBo)
    sx = 1.2 * oracle.abs_gemvt(Bhat, h["y"]) + np.abs(h["z"])
    check_reduce(host(x), xo, sx, n, "x vs stored B")
    sw = 1.5 * oracle.abs_gemv(Bhat, np.abs(xo) + sx)
    check_reduce(host(w), wo, sw, n, "w vs stored B")


@pytest.mark.parametrize("kfmt,ofmt,tdt,half_ulp", FMTS)
def test_lowp_gemver_error_vs_fp32_problem(built, kfmt, ofmt, tdt, half_ulp):
    """Total error of x and w against the FP64 GEMVER of the original FP32
    A: within the bound from two roundings into the format (A, then B) per
    element, half a unit each (plus the E4M3 subnormal floor), propagated
    through B^T y and B x, plus the FP32 tolerance."""
    kf = built
    n = 1024
    A, h, QAo, sAo, (QB, sB, x, w), _ = run_gemver_q(kf, n, kfmt, ofmt, tdt, seed=2)
    Ah = host(A)
    B, xt, wt = oracle.gemver(Ah, h["u1"], h["v1"], h["u2"], h["v2"], h["y"], h["z"], 1.5, 1.2)
    floor = 2.0 ** -10 if ofmt == oracle.FMT_E4M3 else 0.0
    rel = 2.0 ** -4 if ofmt == oracle.FMT_E4M3 else 2.0 ** -8   # worst-case half unit, relative
    sBh = sB.cpu().numpy().astype(np.float64)
    Eb = (2 * rel * 1.01 + 2e-5) * np.abs(B) + floor * (sAo.astype(np.float64) + sBh)[:, None]
    tol = 1e-5 * np.sqrt(n)
    bx = 1.2 * (Eb.T @ np.abs(h["y"])) + tol * (1.2 * oracle.abs_gemvt(B, h["y"]) + np.abs(h["z"]))
    assert np.all(np.abs(host(x) - xt) <= bx)
    bw = 1.5 * (Eb @ (np.abs(xt) + bx) + np.abs(B) @ bx) + tol * 1.5 * oracle.abs_gemv(B, np.abs(xt) + bx)
    assert np.all(np.abs(host(w) - wt) <= bw)


def test_lowp_gemver_rejects_f32(built):
    kf = built
    n = 16
    Q = torch.zeros((n, n), dtype=torch.int16, device=dev())
    s = torch.ones(n, device=dev())
    v = torch.zeros(n, device=dev())
    with pytest.raises(kf.KFError):
        kf.kf_gemver_q(Q, kf.KF_F32, s, v, v, v, v, v, v, 1.0, 1.0, Q.clone(), s.clone(), v.clone(), v.clone(),
                       kf.workspace(kf.KF_SEQ_GEMVER, n, n))
