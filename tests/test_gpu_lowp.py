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
