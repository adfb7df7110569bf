"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Sizes span several column strips and row groups and end in ragged tails;
exact cases (identity, one-hot, integer inputs) are compared bitwise.
"""

import numpy as np
import pytest
import torch

import oracle
from gpu_util import ALPHA, BETA, I, U, built, dev, host  # noqa: F401
from tolerance import check_map, check_reduce

pytestmark = pytest.mark.gpu

SHAPES = [(1, 1), (4, 4), (31, 33), (33, 31), (257, 1031), (1000, 1003), (1024, 2048),
          (2048, 2048), (3001, 700), (64, 8192), (5000, 96)]


def ws(kf, seq, m, n, fmt=0):
    return kf.workspace(seq, m, n, fmt)


# ------------------------------------------------------------------ BiCGK

@pytest.mark.parametrize("m,n", SHAPES)
def test_bicgk_parity(built, m, n):
    kf = built
    A, p, r = U((m, n), 1), U((n,), 3), U((m,), 4)
    q = torch.empty(m, device=dev()); s = torch.empty(n, device=dev())
    W = ws(kf, kf.KF_SEQ_BICGK, m, n)
    kf.kf_bicgk(A, p, r, q, s, W)
    Ah, ph, rh = host(A), host(p), host(r)
    qo, so = oracle.bicgk(Ah, ph, rh)
    check_reduce(host(q), qo, oracle.abs_gemv(Ah, ph), n, "q")
    check_reduce(host(s), so, oracle.abs_gemvt(Ah, rh), m, "s")
    # the workspace counters are left zeroed: a second call gives identical bits
    q2 = torch.empty_like(q); s2 = torch.empty_like(s)
    kf.kf_bicgk(A, p, r, q2, s2, W)
    torch.cuda.synchronize()
    assert torch.equal(q, q2) and torch.equal(s, s2)


@pytest.mark.parametrize("m,n", [(5, 7), (300, 517), (2048, 2048), (2047, 1999)])
def test_bicgk_integer_exact(built, m, n):
    kf = built
    A, p, r = I((m, n), 1), I((n,), 3), I((m,), 4)
    q = torch.empty(m, device=dev()); s = torch.empty(n, device=dev())
    kf.kf_bicgk(A, p, r, q, s, ws(kf, kf.KF_SEQ_BICGK, m, n))
    qo, so = oracle.bicgk(host(A), host(p), host(r))
    assert np.array_equal(host(q), qo) and np.array_equal(host(s), so)


def test_bicgk_identity_and_one_hot(built):
    kf = built
    n = 600
    p, r = U((n,), 3), U((n,), 4)
    q = torch.empty(n, device=dev()); s = torch.empty(n, device=dev())
    W = ws(kf, kf.KF_SEQ_BICGK, n, n)
    kf.kf_bicgk(torch.eye(n, device=dev()), p, r, q, s, W)
    assert torch.equal(q, p) and torch.equal(s, r)
    m, n = 37, 1100
    A = torch.zeros(m, n, device=dev()); A[19, 1037] = 1.0
    p, r = U((n,), 3), U((m,), 4)
    q = torch.empty(m, device=dev()); s = torch.empty(n, device=dev())
    kf.kf_bicgk(A, p, r, q, s, ws(kf, kf.KF_SEQ_BICGK, m, n))
    qe = torch.zeros(m, device=dev()); qe[19] = p[1037]
    se = torch.zeros(n, device=dev()); se[1037] = r[19]
    assert torch.equal(q, qe) and torch.equal(s, se)


def test_bicgk_padded_and_misaligned(built):
    """lda > n (padded rows) and a matrix starting one float past an aligned
    address (element-wise path) give the oracle's result."""
    kf = built
    m, n = 300, 500
    base = U((m, 512), 1)
    A = base[:, :n]                        # lda = 512
    p, r = U((n,), 3), U((m,), 4)
    q = torch.empty(m, device=dev()); s = torch.empty(n, device=dev())
    W = ws(kf, kf.KF_SEQ_BICGK, m, n)
    kf.kf_bicgk(A, p, r, q, s, W)
    qo, so = oracle.bicgk(host(A), host(p), host(r))
    check_reduce(host(q), qo, oracle.abs_gemv(host(A), host(p)), n, "q padded")
    check_reduce(host(s), so, oracle.abs_gemvt(host(A), host(r)), m, "s padded")
    flat = U((m * n + 1,), 1)
    A2 = flat[1:].view(m, n)               # 4-byte aligned only
    kf.kf_bicgk(A2, p, r, q, s, W)
    qo, so = oracle.bicgk(host(A2), host(p), host(r))
    check_reduce(host(q), qo, oracle.abs_gemv(host(A2), host(p)), n, "q misaligned")
    check_reduce(host(s), so, oracle.abs_gemvt(host(A2), host(r)), m, "s misaligned")


def test_bicgk_empty_dimensions(built):
    kf = built
    W = ws(kf, kf.KF_SEQ_BICGK, 16, 16)
    A = torch.empty(0, 16, device=dev())
    s = torch.full((16,), 7.0, device=dev())
    kf.kf_bicgk(A, U((16,), 3), torch.empty(0, device=dev()), torch.empty(0, device=dev()), s, W)
    torch.cuda.synchronize()
    assert torch.equal(s, torch.zeros(16, device=dev()))     # sum over no rows
    A = torch.empty(16, 0, device=dev())
    q = torch.full((16,), 7.0, device=dev())
    kf.kf_bicgk(A, torch.empty(0, device=dev()), U((16,), 4), q, torch.empty(0, device=dev()), W)
    torch.cuda.synchronize()
    assert torch.equal(q, torch.zeros(16, device=dev()))


def test_errors_are_reported_not_launched(built):
    kf = built
    A = U((8, 8), 1)
    q = torch.empty(8, device=dev())
    with pytest.raises(kf.KFError) as e:
        kf.kf_bicgk(A, U((8,), 3), U((8,), 4), q, q, torch.zeros(16, dtype=torch.uint8, device=dev()))
    assert e.value.status == -11                                # workspace too small
    st = kf.lib().kf_bicgk(8, 8, A.data_ptr(), 4, 0, None, None, None, None, None, None, 0, None)
    assert st == -2                                             # lda < n


# ------------------------------------------------------------------ GEMVER

@pytest.mark.parametrize("n", [1, 7, 33, 515, 1024, 2500])
def test_gemver_parity(built, n):
    kf = built
    A = U((n, n), 1)
    u1, v1, u2, v2, y, z = (U((n,), t) for t in (5, 6, 7, 8, 4, 9))
    B = torch.empty_like(A); x = torch.empty(n, device=dev()); w = torch.empty(n, device=dev())
    kf.kf_gemver(A, u1, v1, u2, v2, y, z, ALPHA, BETA, B, x, w, ws(kf, kf.KF_SEQ_GEMVER, n, n))
    H = [host(t) for t in (A, u1, v1, u2, v2, y, z)]
    Bo, xo, wo = oracle.gemver(*H, ALPHA, BETA)
    Ah, u1h, v1h, u2h, v2h, yh, zh = H
    scaleB = np.abs(Ah) + np.abs(np.outer(u1h, v1h)) + np.abs(np.outer(u2h, v2h))
    check_map(host(B), Bo, scaleB, "B")
    sx = BETA * oracle.abs_gemvt(Bo, yh) + np.abs(zh)
    check_reduce(host(x), xo, sx, n, "x")
    sw = ALPHA * oracle.abs_gemv(Bo, np.abs(xo) + sx)
    check_reduce(host(w), wo, sw, n, "w")


def test_gemver_in_place(built):
    """B may overwrite A (the map reads each element before writing it)."""
    kf = built
    n = 700
    A = U((n, n), 1)
    Ah = host(A)
    vs = [U((n,), t) for t in (5, 6, 7, 8, 4, 9)]
    x = torch.empty(n, device=dev()); w = torch.empty(n, device=dev())
    kf.kf_gemver(A, *vs, ALPHA, BETA, A, x, w, ws(kf, kf.KF_SEQ_GEMVER, n, n))
    Bo, xo, wo = oracle.gemver(Ah, *[host(v) for v in vs], ALPHA, BETA)
    scaleB = np.abs(Ah) + 2.0
    check_map(host(A), Bo, scaleB, "B in place")
    sx = BETA * oracle.abs_gemvt(Bo, host(vs[4])) + np.abs(host(vs[5]))
    check_reduce(host(x), xo, sx, n, "x")


def test_gemver_rank_one_closed_form(built):
    """A = 0, u2 = v2 = 0 with integer vectors: B = u1 v1^T and x exactly."""
    kf = built
    n = 900
    A = torch.zeros(n, n, device=dev())
    u1, v1, y, z = I((n,), 5), I((n,), 6), I((n,), 4), I((n,), 9)
    zero = torch.zeros(n, device=dev())
    B = torch.empty_like(A); x = torch.empty(n, device=dev()); w = torch.empty(n, device=dev())
    kf.kf_gemver(A, u1, v1, zero, zero, y, z, 1.0, 2.0, B, x, w, ws(kf, kf.KF_SEQ_GEMVER, n, n))
    assert torch.equal(B, torch.outer(u1, v1))
    xe = 2.0 * host(v1) * float(host(u1) @ host(y)) + host(z)
    assert np.array_equal(host(x), xe)


# ------------------------------------------------------------------ GEMVER, one launch

@pytest.mark.parametrize("n", [8, 516, 1024, 2500, 4100])
def test_gemver_single_launch(built, n):
    """kf_gemver_single (grid-wide barriers instead of a kernel boundary):
    B bit for bit the two-pass form's, x and w within the oracle tolerance;
    twice in a row and after a two-pass call on the same workspace (its
    barrier words and the passes' counters are left at zero)."""
    kf = built
    A = U((n, n), 1)
    u1, v1, u2, v2, y, z = (U((n,), t) for t in (5, 6, 7, 8, 4, 9))
    W = ws(kf, kf.KF_SEQ_GEMVER, n, n)
    B2 = torch.empty_like(A); x2 = torch.empty(n, device=dev()); w2 = torch.empty(n, device=dev())
    H = [host(t) for t in (A, u1, v1, u2, v2, y, z)]
    Bo, xo, wo = oracle.gemver(*H, ALPHA, BETA)
    Ah, u1h, v1h, u2h, v2h, yh, zh = H
    sx = BETA * oracle.abs_gemvt(Bo, yh) + np.abs(zh)
    sw = ALPHA * oracle.abs_gemv(Bo, np.abs(xo) + sx)
    for call in range(3):
        B = torch.full_like(A, float("nan")); x = torch.full((n,), float("nan"), device=dev())
        w = torch.full((n,), float("nan"), device=dev())
        kf.kf_gemver_single(A, u1, v1, u2, v2, y, z, ALPHA, BETA, B, x, w, W)
        check_reduce(host(x), xo, sx, n, f"x, call {call}")
        check_reduce(host(w), wo, sw, n, f"w, call {call}")
        kf.kf_gemver(A, u1, v1, u2, v2, y, z, ALPHA, BETA, B2, x2, w2, W)   # the two-pass form, same workspace
        torch.cuda.synchronize()
        assert torch.equal(B, B2)
        check_reduce(host(x2), xo, sx, n, "x two-pass")
        check_reduce(host(w2), wo, sw, n, "w two-pass")
    kf.kf_workspace_status(W)


def test_gemver_single_launch_refusals(built):
    kf = built
    n = 514
    A = U((n, n), 1)
    vs = [U((n,), t) for t in (5, 6, 7, 8, 4, 9)]
    x = torch.empty(n, device=dev()); w = torch.empty(n, device=dev())
    W = ws(kf, kf.KF_SEQ_GEMVER, n, n)
    with pytest.raises(kf.KFError) as e:
        kf.kf_gemver_single(A, *vs, ALPHA, BETA, torch.empty_like(A), x, w, W)   # n not a multiple of 4
    assert e.value.status == kf.KF_ERR_UNSUPPORTED
    n = 512
    A = U((n, n), 1)
    vs = [U((n,), t) for t in (5, 6, 7, 8, 4, 9)]
    x = torch.empty(n, device=dev()); w = torch.empty(n, device=dev())
    with pytest.raises(kf.KFError) as e:
        kf.kf_gemver_single(A, *vs, ALPHA, BETA, A, x, w, ws(kf, kf.KF_SEQ_GEMVER, n, n))   # in place
    assert e.value.status == kf.KF_ERR_UNSUPPORTED


# ------------------------------------------------------------------ SGEMVT

@pytest.mark.parametrize("m,n", [(1, 1), (31, 33), (1000, 1003), (2048, 2048), (513, 4096), (4100, 700)])
def test_sgemvt_parity(built, m, n):
    """x = beta A^T y + z, w = alpha A x (Table 1), against the FP64 oracle;
    w's tolerance takes the longer of its two reduction stages."""
    kf = built
    A, y, z = U((m, n), 1), U((m,), 4), U((n,), 9)
    x = torch.empty(n, device=dev()); w = torch.empty(m, device=dev())
    kf.kf_sgemvt(A, y, z, ALPHA, BETA, x, w, ws(kf, kf.KF_SEQ_SGEMVT, m, n))
    Ah, yh, zh = host(A), host(y), host(z)
    xo, wo = oracle.sgemvt(Ah, yh, zh, ALPHA, BETA)
    sx = BETA * oracle.abs_gemvt(Ah, yh) + np.abs(zh)
    check_reduce(host(x), xo, sx, m, "x")
    sw = ALPHA * oracle.abs_gemv(Ah, np.abs(xo) + sx)
    check_reduce(host(w), wo, sw, max(m, n), "w")


def test_sgemvt_identity_and_empty(built):
    """A = I: x = beta y + z and w = alpha x exactly for integer inputs with
    beta = alpha = 2; an empty A gives x = z and w = 0."""
    kf = built
    n = 777
    A = torch.eye(n, device=dev())
    y, z = I((n,), 4), I((n,), 9)
    x = torch.empty(n, device=dev()); w = torch.empty(n, device=dev())
    kf.kf_sgemvt(A, y, z, 2.0, 2.0, x, w, ws(kf, kf.KF_SEQ_SGEMVT, n, n))
    assert torch.equal(x, 2 * y + z) and torch.equal(w, 2 * x)
    m, n = 0, 300
    A = torch.zeros((1, n), device=dev())[:0]
    z = U((n,), 9)
    x = torch.full((n,), float("nan"), device=dev())
    kf.kf_sgemvt(A, None, z, ALPHA, BETA, x, None, ws(kf, kf.KF_SEQ_SGEMVT, 1, n))
    assert torch.equal(x, z)


@pytest.mark.parametrize("m,n", [(8, 4), (31, 36), (513, 4096), (2048, 2048), (4100, 700), (3001, 516),
                                 (64, 8192)])
def test_sgemvt_single_launch(built, m, n):
    """kf_sgemvt_single (grid-wide barriers instead of a kernel boundary,
    rectangular A): x and w within the oracle tolerance; three calls in a
    row, each followed by the two-launch form on the same workspace."""
    kf = built
    A, y, z = U((m, n), 1), U((m,), 4), U((n,), 9)
    W = ws(kf, kf.KF_SEQ_SGEMVT, m, n)
    Ah, yh, zh = host(A), host(y), host(z)
    xo, wo = oracle.sgemvt(Ah, yh, zh, ALPHA, BETA)
    sx = BETA * oracle.abs_gemvt(Ah, yh) + np.abs(zh)
    sw = ALPHA * oracle.abs_gemv(Ah, np.abs(xo) + sx)
    for call in range(3):
        x = torch.full((n,), float("nan"), device=dev()); w = torch.full((m,), float("nan"), device=dev())
        kf.kf_sgemvt_single(A, y, z, ALPHA, BETA, x, w, W)
        check_reduce(host(x), xo, sx, m, f"x, call {call}")
        check_reduce(host(w), wo, sw, max(m, n), f"w, call {call}")
        x2 = torch.empty(n, device=dev()); w2 = torch.empty(m, device=dev())
        kf.kf_sgemvt(A, y, z, ALPHA, BETA, x2, w2, W)
        check_reduce(host(x2), xo, sx, m, "x two-pass")
        check_reduce(host(w2), wo, sw, max(m, n), "w two-pass")
    kf.kf_workspace_status(W)


def test_sgemvt_single_launch_exact_and_refusals(built):
    """A = I with integer inputs: x = 2 y + z and w = 2 x bit for bit in one
    launch; shapes outside the single launch's rule are refused."""
    kf = built
    n = 776
    A = torch.eye(n, device=dev())
    y, z = I((n,), 4), I((n,), 9)
    x = torch.empty(n, device=dev()); w = torch.empty(n, device=dev())
    kf.kf_sgemvt_single(A, y, z, 2.0, 2.0, x, w, ws(kf, kf.KF_SEQ_SGEMVT, n, n))
    assert torch.equal(x, 2 * y + z) and torch.equal(w, 2 * x)
    for m, n in [(100, 514), (7, 64)]:   # n not a multiple of 4; m < 8
        A, y, z = U((m, n), 1), U((m,), 4), U((n,), 9)
        x = torch.empty(n, device=dev()); w = torch.empty(m, device=dev())
        with pytest.raises(kf.KFError) as e:
            kf.kf_sgemvt_single(A, y, z, ALPHA, BETA, x, w, ws(kf, kf.KF_SEQ_SGEMVT, m, n))
        assert e.value.status == kf.KF_ERR_UNSUPPORTED


# ------------------------------------------------------------------ GESUMMV

@pytest.mark.parametrize("m,n", [(1, 1), (31, 33), (1000, 1003), (2048, 2048), (513, 4096)])
def test_gesummv_parity(built, m, n):
    kf = built
    A, B, x = U((m, n), 1), U((m, n), 2), U((n,), 3)
    y = torch.empty(m, device=dev())
    kf.kf_gesummv(A, B, x, ALPHA, BETA, y, ws(kf, kf.KF_SEQ_GESUMMV, m, n))
    Ah, Bh, xh = host(A), host(B), host(x)
    yo = oracle.gesummv(Ah, Bh, xh, ALPHA, BETA)
    scale = ALPHA * oracle.abs_gemv(Ah, xh) + BETA * oracle.abs_gemv(Bh, xh)
    check_reduce(host(y), yo, scale, n, "y")


def test_gesummv_cancels_exactly(built):
    kf = built
    m, n = 300, 1000
    A, x = I((m, n), 1), I((n,), 3)
    y = torch.empty(m, device=dev())
    kf.kf_gesummv(A, -A, x, 2.0, 2.0, y, ws(kf, kf.KF_SEQ_GESUMMV, m, n))
    assert torch.equal(y, torch.zeros(m, device=dev()))


# ------------------------------------------------------------------ ATAX

@pytest.mark.parametrize("m,n", [(1, 4), (3, 8), (31, 36), (1000, 1004), (2048, 2048),
                                 (4100, 8192), (777, 16384), (33, 31), (500, 1001)])
def test_atax_parity(built, m, n):
    kf = built
    A, x = U((m, n), 1), U((n,), 3)
    y = torch.empty(n, device=dev())
    W = ws(kf, kf.KF_SEQ_ATAX, m, n)
    kf.kf_atax(A, x, y, W)
    kf.kf_workspace_status(W)
    Ah, xh = host(A), host(x)
    yo, to = oracle.atax(Ah, xh)
    scale = oracle.abs_gemvt(Ah, oracle.abs_gemv(Ah, xh))
    check_reduce(host(y), yo, scale, max(m, n), "y")


def test_atax_permutation_exact(built):
    kf = built
    n = 1024
    perm = torch.roll(torch.arange(n), 77)
    P = torch.eye(n, device=dev())[perm]
    x = I((n,), 3)
    y = torch.empty(n, device=dev())
    kf.kf_atax(P, x, y, ws(kf, kf.KF_SEQ_ATAX, n, n))
    assert torch.equal(y, x)


def test_atax_hadamard_exact(built):
    kf = built
    n = 256
    H = torch.ones(1, 1)
    while H.shape[0] < n:
        H = torch.cat([torch.cat([H, H], 1), torch.cat([H, -H], 1)], 0)
    x = I((n,), 3)
    y = torch.empty(n, device=dev())
    kf.kf_atax(H.to(dev()), x, y, ws(kf, kf.KF_SEQ_ATAX, n, n))
    assert torch.equal(y, n * x)


# ------------------------------------------------------------------ BLAS-1

@pytest.mark.parametrize("n", [1, 3, 4, 5, 1000, 4097, 1 << 20, (1 << 20) + 3])
def test_axpydot_parity(built, n):
    kf = built
    w, v, u = U((n,), 10), U((n,), 11), U((n,), 12)
    z = torch.empty(n, device=dev()); r = torch.empty(1, device=dev())
    kf.kf_axpydot(w, v, u, ALPHA, z, r, ws(kf, kf.KF_SEQ_AXPYDOT, 1, n))
    wh, vh, uh = host(w), host(v), host(u)
    zo, ro = oracle.axpydot(wh, vh, uh, ALPHA)
    check_map(host(z), zo, np.abs(wh) + ALPHA * np.abs(vh), "z")
    scale = float(np.sum((np.abs(wh) + ALPHA * np.abs(vh)) * np.abs(uh)))
    check_reduce(host(r), np.array([ro]), np.array([scale]), n, "r")


def test_axpydot_special_cases(built):
    kf = built
    n = 100003
    w, u = U((n,), 10), U((n,), 12)
    z = torch.empty(n, device=dev()); r = torch.empty(1, device=dev())
    W = ws(kf, kf.KF_SEQ_AXPYDOT, 1, n)
    kf.kf_axpydot(w, torch.zeros(n, device=dev()), u, ALPHA, z, r, W)
    torch.cuda.synchronize()
    assert torch.equal(z, w)
    e = torch.zeros(n, device=dev()); e[77777] = 1.0
    kf.kf_axpydot(w, U((n,), 11), e, ALPHA, z, r, W)
    torch.cuda.synchronize()
    assert float(r[0]) == float(z[77777])


@pytest.mark.parametrize("n", [1, 2, 7, 1000, 1 << 20, (1 << 20) + 1])
def test_waxpby_parity(built, n):
    kf = built
    x, y = U((n,), 3), U((n,), 4)
    w = torch.empty(n, device=dev())
    kf.kf_waxpby(ALPHA, x, BETA, y, w)
    xh, yh = host(x), host(y)
    check_map(host(w), oracle.waxpby(ALPHA, xh, BETA, yh), ALPHA * np.abs(xh) + BETA * np.abs(yh), "w")
    kf.kf_waxpby(1.0, x, 0.0, y, w)
    torch.cuda.synchronize()
    assert torch.equal(w, x)
    kf.kf_waxpby(ALPHA, x, ALPHA, -x, w)
    torch.cuda.synchronize()
    assert torch.equal(w, torch.zeros(n, device=dev()))


# ------------------------------------------------------------------ elementaries

@pytest.mark.parametrize("m,n", [(1, 1), (45, 77), (1000, 1003), (2048, 2048)])
def test_elementaries_parity(built, m, n):
    kf = built
    A, x, y, y0, x0 = U((m, n), 1), U((n,), 3), U((m,), 4), U((m,), 9), U((n,), 10)
    Ah, xh, yh = host(A), host(x), host(y)
    W = ws(kf, kf.KF_SEQ_BICGK, m, n)
    out = torch.empty(m, device=dev())
    kf.kf_gemv(A, x, out, W, alpha=ALPHA, beta=BETA, y0=y0)
    check_reduce(host(out), oracle.gemv(Ah, xh, ALPHA, BETA, host(y0)),
                 ALPHA * oracle.abs_gemv(Ah, xh) + BETA * np.abs(host(y0)), n, "gemv")
    outt = torch.empty(n, device=dev())
    kf.kf_gemvt(A, y, outt, W, alpha=ALPHA, beta=BETA, x0=x0)
    check_reduce(host(outt), oracle.gemvt(Ah, yh, ALPHA, BETA, host(x0)),
                 ALPHA * oracle.abs_gemvt(Ah, yh) + BETA * np.abs(host(x0)), m, "gemvt")
    u, v = U((m,), 5), U((n,), 6)
    B = torch.empty_like(A)
    kf.kf_ger(A, u, v, B, alpha=ALPHA)
    check_map(host(B), oracle.ger(Ah, host(u), host(v), ALPHA),
              np.abs(Ah) + ALPHA * np.abs(np.outer(host(u), host(v))), "ger")
    kf.kf_ger(A, u, v, A, alpha=ALPHA)                       # in place
    check_map(host(A), oracle.ger(Ah, host(u), host(v), ALPHA),
              np.abs(Ah) + ALPHA * np.abs(np.outer(host(u), host(v))), "ger in place")


@pytest.mark.parametrize("n", [1, 6, 1001, 1 << 18])
def test_blas1_elementaries(built, n):
    kf = built
    x, y, z = U((n,), 3), U((n,), 4), U((n,), 9)
    xh, yh, zh = host(x), host(y), host(z)
    out = torch.empty(n, device=dev())
    kf.kf_axpby(ALPHA, x, BETA, y, out)
    check_map(host(out), oracle.axpby(ALPHA, xh, BETA, yh), ALPHA * np.abs(xh) + BETA * np.abs(yh), "axpby")
    kf.kf_scal(ALPHA, x, out)
    check_map(host(out), ALPHA * xh, ALPHA * np.abs(xh), "scal")
    kf.kf_vadd3(x, y, z, out)
    check_map(host(out), oracle.vadd3(xh, yh, zh), np.abs(xh) + np.abs(yh) + np.abs(zh), "vadd3")
    d = torch.empty(1, device=dev())
    kf.kf_dot(x, y, d, ws(kf, kf.KF_SEQ_DOT, 1, n))
    check_reduce(host(d), np.array([oracle.dot(xh, yh)]), np.array([float(np.abs(xh * yh).sum())]), n, "dot")
    yy = y.clone()
    kf.kf_axpby(0.5, x, 1.0, yy, yy)                          # AXPY in place
    check_map(host(yy), oracle.axpby(0.5, xh, 1.0, yh), 0.5 * np.abs(xh) + np.abs(yh), "axpy in place")


# ------------------------------------------------------------------ MADD

@pytest.mark.parametrize("m,n,pad", [(1, 1, 0), (37, 1001, 0), (1024, 1024, 0), (300, 517, 3), (2048, 96, 32)])
def test_madd_parity(built, m, n, pad):
    """C = A + B (Table 1's MADD): contiguous operands (one vector pass) and
    padded leading dimensions (the strided map); one rounding per element,
    so the result is the correctly rounded sum."""
    kf = built
    A = U((m, n + pad), 1)[:, :n]
    B = U((m, n + 2 * pad), 2)[:, :n]
    C = torch.full((m, n + pad), float("nan"), device=dev())[:, :n]
    kf.kf_madd(A, B, C)
    Ah, Bh = host(A), host(B)
    want = (Ah + Bh).astype(np.float32).astype(np.float64)   # the correctly rounded FP32 sum
    assert np.array_equal(host(C), want)
    check_map(host(C), oracle.madd(Ah, Bh), np.abs(Ah) + np.abs(Bh), "C")
    # in place
    kf.kf_madd(A, B, A)
    assert np.array_equal(host(A), want)
